// Body values through the Schur complement of the body unknowns (an algebraically
// equivalent form of the multi-point-constraint system of section "Matrix-Free
// Conjugate Gradient with Multiple Constraint Enforcement").
//
// Split the reduced unknowns into free (F) and body (B) ones.  With the body values
// held as data, psi_0 solves the free rows with every C_k = 0 and the Dirichlet data,
// and phi_k solves them with C_k = 1, the other bodies 0 and no Dirichlet data.  The
// collapsed body rows of K phi_k form the Schur matrix S[:, k] and those of K psi_0 give
// the right-hand side: S C = -(body rows of K psi_0).  Then psi = psi_0 + sum_k C_k phi_k.
//
// The N_b + 1 fixed-body solves of every variant run as one batch (one persistent
// launch per CG iteration over all right-hand sides); S is factorised in FP64 on the
// host (N_b <= 64).  A final warm-started MPC solve on the original handle checks the
// combined solution's true residual (zero iterations when it already meets tol).
//
// Kutta condition (section "Boundary Conditions"): for a body with a trailing-edge wake
// node W, the row "collapsed body row = 0" (zero circulation) is replaced by
// psi(W) = C_k, i.e. psi_0(W) + sum_j C_j phi_j(W) - C_k = 0, with the values at W read
// from the same fixed-body solves.  The small system is then not symmetric and is solved
// by Gaussian elimination with partial pivoting, and the MPC check is skipped (its
// iteration would return to zero circulation): the reported residual is the largest of
// the fixed-body solves'.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "batch.h"

namespace pfq4 {

namespace {

// psi of variant v = sum_k coef[k] * x64 of copy k (same grid, same pitch)
__global__ void k_schur_combine(const DevVariant* var, const int* tile_var, const int2* tile_ij, const uint8_t* tag,
                                const DevVariant* svar, const int* copy0, const double* coef, const int* coef0,
                                const double* sx64, double* x64) {
  const long long t = blockIdx.x;
  const int v = tile_var[t];
  const DevVariant& V = var[v];
  const int2 ij = tile_ij[t];
  const int i = ij.x + threadIdx.x, j = ij.y + threadIdx.y;
  if (i > V.nx || j > V.ny) return;
  const long long off = (long long)j * V.P + i;
  const int kind = tag[V.base + off] & KIND_MASK;
  if (kind != K_FREE) return;
  double u = 0.0;
  for (int k = 0; k <= V.nb; ++k) {
    const DevVariant& W = svar[copy0[v] + k];
    u += coef[coef0[v] + k] * sx64[W.base + off];
  }
  x64[V.base + off] = u;
}

void cholesky_solve(int n, std::vector<double>& A, std::vector<double>& b) {
  for (int j = 0; j < n; ++j) {
    double s = A[j * n + j];
    for (int k = 0; k < j; ++k) s -= A[j * n + k] * A[j * n + k];
    if (!(s > 0)) throw Error{PF_EBREAKDOWN, "Schur matrix is not positive definite"};
    const double d = std::sqrt(s);
    A[j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double t = A[i * n + j];
      for (int k = 0; k < j; ++k) t -= A[i * n + k] * A[j * n + k];
      A[i * n + j] = t / d;
    }
  }
  for (int i = 0; i < n; ++i) {
    double t = b[i];
    for (int k = 0; k < i; ++k) t -= A[i * n + k] * b[k];
    b[i] = t / A[i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = b[i];
    for (int k = i + 1; k < n; ++k) t -= A[k * n + i] * b[k];
    b[i] = t / A[i * n + i];
  }
}

void lu_solve(int n, std::vector<double>& A, std::vector<double>& b) {
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (std::fabs(A[r * n + c]) > std::fabs(A[piv * n + c])) piv = r;
    if (!(std::fabs(A[piv * n + c]) > 0)) throw Error{PF_EBREAKDOWN, "singular body system"};
    if (piv != c) {
      for (int k = 0; k < n; ++k) std::swap(A[c * n + k], A[piv * n + k]);
      std::swap(b[c], b[piv]);
    }
    for (int r = c + 1; r < n; ++r) {
      const double f = A[r * n + c] / A[c * n + c];
      for (int k = c; k < n; ++k) A[r * n + k] -= f * A[c * n + k];
      b[r] -= f * b[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double t = b[r];
    for (int k = r + 1; k < n; ++k) t -= A[r * n + k] * b[k];
    b[r] = t / A[r * n + r];
  }
}

struct BatchGuard {
  Batch* p;
  ~BatchGuard() {
    if (p) {
      for (int k = 0; k < 2; ++k)
        if (p->graph[k]) cudaGraphExecDestroy(p->graph[k]);
      if (p->graph_pcg) cudaGraphExecDestroy(p->graph_pcg);
      for (int k = 0; k < Batch::N_EV; ++k)
        if (p->ev[k]) cudaEventDestroy(p->ev[k]);
      if (p->h_poll) cudaFreeHost(p->h_poll);
      if (p->h_vs) cudaFreeHost(p->h_vs);
      dev_free_all(*p);
      delete p;
    }
  }
};

}  // namespace

pf_status schur_solve(Batch& b, double U, const pf_solve_opts& o, double* dev_psi, double* body_psi,
                      pf_solve_info* info) {
  if (!b.valid) throw Error{PF_EMESH_INVALID, "mesh has det J <= 0 at a Gauss point; solve refused"};
  if (o.k_max < 1) throw Error{PF_EINVAL, "k_max must be >= 1"};
  b.rhs_active = false;
  b.fixed_bodies = false;
  b.Uv_active = false;
  // ---- internal batch: for every variant its N_b + 1 fixed-body problems
  std::vector<pf_grid> grids;
  std::vector<int> offs{0}, copy0(b.nv), coef0(b.nv);
  std::vector<pf_body> bodies;
  std::vector<double> Uv, fixedC;
  ShapeInput shp;                       // the body shapes of every copy (polygons, Kutta)
  shp.off.push_back(0);
  int ncoef = 0;
  for (int v = 0; v < b.nv; ++v) {
    const HostVariant& H = b.hv[v];
    copy0[v] = (int)grids.size();
    coef0[v] = ncoef;
    ncoef += H.nb + 1;
    for (int k = 0; k <= H.nb; ++k) {
      grids.push_back(H.g);
      for (int m = 0; m < H.nb; ++m) {
        const int gm = H.body0 + m;
        bodies.push_back(b.bodies[gm]);
        fixedC.push_back((k > 0 && m == k - 1) ? 1.0 : 0.0);
        shp.kind.push_back(b.shape_kind[gm]);
        shp.kutta.push_back(b.kutta[gm]);
        shp.xy.insert(shp.xy.end(), b.poly_xy.begin() + 2 * b.poly_off[gm], b.poly_xy.begin() + 2 * b.poly_off[gm + 1]);
        shp.off.push_back((int)(shp.xy.size() / 2));
      }
      offs.push_back((int)bodies.size());
      Uv.push_back(k == 0 ? U : 0.0);
    }
  }
  BatchGuard g{new Batch()};
  Batch& S = *g.p;
  S.device = b.device;
  S.stream = b.stream;
  S.alloc_fn = b.alloc_fn;
  S.free_fn = b.free_fn;
  S.alloc_ctx = b.alloc_ctx;
  S.cut = b.cut;                        // the copies are meshed as the handle was
  S.cut_sigma = b.cut_sigma;
  build_batch(S, grids.data(), offs.data(), bodies.data(), (int)grids.size(), b.sweeps, b.bc,
              b.has_polygons ? &shp : nullptr);
  if (!S.valid) throw Error{PF_EMESH_INVALID, "Schur sub-problem mesh invalid"};
  ensure_solver_memory(S, o.precision);
  cudaStream_t s = b.stream;
  if (S.B > 0)
    PF_CUDA(cudaMemcpyAsync(S.sol64, fixedC.data(), S.B * sizeof(double), cudaMemcpyHostToDevice, s));
  S.d_Uv = (double*)dev_alloc(S, Uv.size() * sizeof(double));
  PF_CUDA(cudaMemcpyAsync(S.d_Uv, Uv.data(), Uv.size() * sizeof(double), cudaMemcpyHostToDevice, s));
  S.Uv_active = true;
  S.fixed_bodies = true;
  std::vector<pf_solve_info> sinfo(S.nv);
  pf_solve_opts so = o;
  so.warm_start = 0;
  const pf_status st = solve_core(S, U, so, nullptr, nullptr, sinfo.data(), false);
  if (st != PF_OK) throw Error{st, "a fixed-body Schur sub-solve failed"};
  // ---- Schur systems (FP64, host)
  std::vector<double> rows(std::max(1, S.B));
  if (S.B > 0) {
    PF_CUDA(cudaMemcpyAsync(rows.data(), S.sbr64, S.B * sizeof(double), cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaStreamSynchronize(s));
  }
  std::vector<double> coef(std::max(1, ncoef)), C(std::max(1, b.B), 0.0);
  // Kutta rows need the fixed-body solutions at each wake node: psi_0(W) and phi_k(W)
  auto wake_value = [&](int copy, int body) -> double {
    const long long n = S.h_wake[S.hv[copy].body0 + body];
    if (n < 0) throw Error{PF_EINVAL, "internal: Kutta body without a wake node"};
    double x = 0.0;
    PF_CUDA(cudaMemcpyAsync(&x, S.x64 + n, sizeof(double), cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaStreamSynchronize(s));
    return x;
  };
  for (int v = 0; v < b.nv; ++v) {
    const int nb = b.hv[v].nb;
    const int sb0 = S.hv[copy0[v]].body0;   // body rows of copy k start at sb0 + k * nb
    std::vector<double> A(nb * nb), rhs(nb);
    for (int j = 0; j < nb; ++j) {
      rhs[j] = rows[sb0 + j];                                   // = -(row j of K psi_0)
      for (int k = 0; k < nb; ++k) A[j * nb + k] = -rows[sb0 + (k + 1) * nb + j];   // row j of K phi_k
    }
    bool kutta = false;
    for (int j = 0; j < nb; ++j) kutta |= b.kutta[b.hv[v].body0 + j] >= 0;
    if (kutta) {
      for (int j = 0; j < nb; ++j) {
        if (b.kutta[b.hv[v].body0 + j] < 0) continue;
        rhs[j] = -wake_value(copy0[v], j);                     // psi_0(W_j) + sum_k C_k phi_k(W_j) = C_j
        for (int k = 0; k < nb; ++k) A[j * nb + k] = wake_value(copy0[v] + 1 + k, j) - (k == j ? 1.0 : 0.0);
      }
      lu_solve(nb, A, rhs);
    } else {
      // symmetrise (S is symmetric up to the sub-solve tolerance)
      for (int j = 0; j < nb; ++j)
        for (int k = 0; k < j; ++k) A[j * nb + k] = A[k * nb + j] = 0.5 * (A[j * nb + k] + A[k * nb + j]);
      if (nb > 0) cholesky_solve(nb, A, rhs);
    }
    coef[coef0[v]] = 1.0;
    for (int k = 0; k < nb; ++k) {
      coef[coef0[v] + 1 + k] = rhs[k];
      C[b.hv[v].body0 + k] = rhs[k];
    }
  }
  // ---- psi = psi_0 + sum_k C_k phi_k into the original handle, then verify
  ensure_solver_memory(b, o.precision);
  int *d_copy0 = (int*)dev_alloc(S, b.nv * sizeof(int)), *d_coef0 = (int*)dev_alloc(S, b.nv * sizeof(int));
  double* d_coef = (double*)dev_alloc(S, std::max(1, ncoef) * sizeof(double));
  PF_CUDA(cudaMemcpyAsync(d_copy0, copy0.data(), b.nv * sizeof(int), cudaMemcpyHostToDevice, s));
  PF_CUDA(cudaMemcpyAsync(d_coef0, coef0.data(), b.nv * sizeof(int), cudaMemcpyHostToDevice, s));
  PF_CUDA(cudaMemcpyAsync(d_coef, coef.data(), ncoef * sizeof(double), cudaMemcpyHostToDevice, s));
  if (b.B > 0) PF_CUDA(cudaMemcpyAsync(b.sol64, C.data(), b.B * sizeof(double), cudaMemcpyHostToDevice, s));
  k_schur_combine<<<(unsigned)b.T, dim3(TX, TY), 0, s>>>(b.d_var, b.tile_var, b.tile_ij, b.tag, S.d_var, d_copy0,
                                                         d_coef, d_coef0, S.x64, b.x64);
  PF_CUDA(cudaGetLastError());
  PF_CUDA(cudaStreamSynchronize(s));
  b.launches += S.launches + 1;
  // the MPC solve warm-started from the combined solution reports the true residual
  // (and continues CG only if the Schur solution misses tol)
  bool need_bnorm = b.bnorm2_unit.empty() || U == 0.0 || b.has_kutta;
  for (double x : b.bnorm2_unit) need_bnorm |= x < 0;
  if (need_bnorm) {
    // ||b|| has not been measured on this handle yet: one residual evaluation at x = 0
    pf_solve_opts r0 = o;
    r0.warm_start = 0;
    r0.k_max = 0;
    std::vector<double> keepC(C);
    solve_core(b, U, r0, nullptr, nullptr, nullptr, true);
    if (b.B > 0) PF_CUDA(cudaMemcpyAsync(b.sol64, keepC.data(), b.B * sizeof(double), cudaMemcpyHostToDevice, s));
    k_schur_combine<<<(unsigned)b.T, dim3(TX, TY), 0, s>>>(b.d_var, b.tile_var, b.tile_ij, b.tag, S.d_var, d_copy0,
                                                           d_coef, d_coef0, S.x64, b.x64);
    PF_CUDA(cudaGetLastError());
  }
  b.solved = true;
  if (b.has_kutta) {
    // the combined solution with the Kutta rows is the answer (an MPC iteration from it
    // would return to zero circulation); its accuracy is that of the fixed-body solves
    PF_CUDA(cudaStreamSynchronize(s));
    b.lastU = U;
    b.last_precision = o.precision;
    if (dev_psi) export_psi(b, dev_psi);
    if (body_psi && b.B) {
      PF_CUDA(cudaMemcpyAsync(body_psi, C.data(), b.B * sizeof(double), cudaMemcpyHostToHost, s));
    }
    PF_CUDA(cudaStreamSynchronize(s));
    if (info) {
      for (int v = 0; v < b.nv; ++v) {
        info[v] = pf_solve_info{};
        for (int k = 0; k <= b.hv[v].nb; ++k) {
          const pf_solve_info& si = sinfo[copy0[v] + k];
          info[v].iters += si.iters;
          info[v].refinements = std::max(info[v].refinements, si.refinements);
          info[v].rel_true_residual = std::max(info[v].rel_true_residual, si.rel_true_residual);
        }
        info[v].status = PF_OK;
        info[v].n_dof = b.hv[v].stats.n_dof;
      }
    }
    return PF_OK;
  }
  pf_solve_opts vo = o;
  vo.warm_start = 1;
  const pf_status st2 = solve_core(b, U, vo, dev_psi, body_psi, info, true);
  if (info) {
    for (int v = 0; v < b.nv; ++v)
      for (int k = 0; k <= b.hv[v].nb; ++k) info[v].iters += sinfo[copy0[v] + k].iters;
  }
  return st2;
}

}  // namespace pfq4
