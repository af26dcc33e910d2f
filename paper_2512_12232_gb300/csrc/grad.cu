// Adjoint shape gradients of J = C_hi - C_lo (transverse-gap flow) or
// J = (C_hi - C_lo) / (U (cy_hi - cy_lo)) (CoPFI, section "Effect of Gap Ratio") with
// respect to the smoothed node coordinates X and the body centres c.  The paper has
// no gradient; its conclusions name shape optimisation and sensitivity analysis.
//
// With the reduced residual R(u, X) = P^T K(X) psi(u, X) (P collapses body rows, psi
// carries the Dirichlet data g = U y) and the adjoint A lambda = dJ/du,
//   dJ/dX = - sum_e Lambda_e^T (dK_e/dX) psi_e - U (K Lambda)_n  [y of Dirichlet nodes]
// The element term is the shape derivative of the 2x2-Gauss form: for a corner a and
// a component c, d/dx_{a,c} [det J grad(lambda).grad(psi)] at a Gauss point equals
//   det J [ (grad lambda . grad psi) dN_a/dx_c - d_c lambda (grad N_a . grad psi)
//                                             - d_c psi (grad N_a . grad lambda) ],
// exact for the quadrature sum because the Gauss points move with the element.
// The mesh is linear in the projection displacement d0 (X = X_grid + M^S d0), so
// dJ/dd0 = (M^T)^S dJ/dX, and d0 of a body node depends on the centre through the
// radial projection: dx_b/dc = I - (r/rho)(I - u u^T).  Topology is held fixed.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "batch.h"

namespace pfq4 {

namespace {

__device__ __forceinline__ double node_value(int kind, long long n, int bidn, int body0, const double* nodal,
                                             const double* bodyv) {
  if (kind == K_BODY) return bodyv[body0 + bidn];
  if (kind == K_INACT) return 0.0;
  return nodal[n];
}

// Per active cell: G[a][c] = Lambda_e^T (dK_e/dx_{a,c}) psi_e for its four corners.
__global__ void k_shape_cells(const DevVariant* var, const int* tile_var, const int2* tile_ij, const uint8_t* tag,
                              const int* bid, const double* X, long long Vtot, const double* psi,
                              const double* psib, const double* lam, const double* lamb, double* G) {
  const long long t = blockIdx.x;
  const int v = tile_var[t];
  const DevVariant& V = var[v];
  const int2 ij = tile_ij[t];
  const int i = ij.x + threadIdx.x, j = ij.y + threadIdx.y;
  if (i >= V.nx || j >= V.ny) return;
  const long long n = V.base + (long long)j * V.P + i;
  if (!(tag[n] & CELL_ACTIVE)) return;
  const long long idx[4] = {n, n + 1, n + 1 + V.P, n + V.P};
  double x[4], y[4], ps[4], lm[4];
  for (int a = 0; a < 4; ++a) {
    const int kind = tag[idx[a]] & KIND_MASK;
    const int bn = bid[idx[a]];
    x[a] = X[idx[a]];
    y[a] = X[Vtot + idx[a]];
    ps[a] = node_value(kind, idx[a], bn, V.body0, psi, psib);
    lm[a] = node_value(kind, idx[a], bn, V.body0, lam, lamb);
  }
  const double g = 0.57735026918962576451;   // 1/sqrt(3)
  const double xi_a[4] = {-1, 1, 1, -1}, eta_a[4] = {-1, -1, 1, 1};
  const double gx[4] = {-g, g, g, -g}, gy[4] = {-g, -g, g, g};
  double out[4][2] = {};
  for (int q = 0; q < 4; ++q) {
    double dxi[4], deta[4];
    for (int a = 0; a < 4; ++a) {
      dxi[a] = 0.25 * xi_a[a] * (1.0 + eta_a[a] * gy[q]);
      deta[a] = 0.25 * eta_a[a] * (1.0 + xi_a[a] * gx[q]);
    }
    double j00 = 0, j01 = 0, j10 = 0, j11 = 0;
    for (int a = 0; a < 4; ++a) {
      j00 += dxi[a] * x[a]; j01 += dxi[a] * y[a];
      j10 += deta[a] * x[a]; j11 += deta[a] * y[a];
    }
    const double det = j00 * j11 - j01 * j10;
    const double inv = 1.0 / det;
    double bx[4], by[4];
    double gl[2] = {0, 0}, gp[2] = {0, 0};
    for (int a = 0; a < 4; ++a) {
      bx[a] = (j11 * dxi[a] - j01 * deta[a]) * inv;
      by[a] = (-j10 * dxi[a] + j00 * deta[a]) * inv;
      gl[0] += bx[a] * lm[a]; gl[1] += by[a] * lm[a];
      gp[0] += bx[a] * ps[a]; gp[1] += by[a] * ps[a];
    }
    const double lp = gl[0] * gp[0] + gl[1] * gp[1];
    for (int a = 0; a < 4; ++a) {
      const double na_p = bx[a] * gp[0] + by[a] * gp[1];
      const double na_l = bx[a] * gl[0] + by[a] * gl[1];
      const double b2[2] = {bx[a], by[a]};
      for (int c = 0; c < 2; ++c) out[a][c] += det * (lp * b2[c] - gl[c] * na_p - gp[c] * na_l);
    }
  }
  for (int a = 0; a < 4; ++a)
    for (int c = 0; c < 2; ++c) G[(a * 2 + c) * Vtot + n] = out[a][c];
}

// Per node: dJ/dX_n = - sum of the corner entries of its active cells, and for Dirichlet
// nodes the data term - U (K Lambda)_n on the y component.
__global__ void k_shape_nodes(const DevVariant* var, const int* tile_var, const int2* tile_ij, const uint8_t* tag,
                              const int* bid, long long Vtot, const double* G, const double* K64,
                              const double* lam, const double* lamb, double U, double* dX) {
  const long long t = blockIdx.x;
  const int v = tile_var[t];
  const DevVariant& V = var[v];
  const int2 ij = tile_ij[t];
  const int i = ij.x + threadIdx.x, j = ij.y + threadIdx.y;
  if (i > V.nx || j > V.ny) return;
  const long long n = V.base + (long long)j * V.P + i;
  double gx = 0.0, gy = 0.0;
  // cells around the node and the node's corner number in each
  const int ci[4] = {i, i - 1, i - 1, i};
  const int cj[4] = {j, j, j - 1, j - 1};
  const int corner[4] = {0, 1, 2, 3};
  for (int k = 0; k < 4; ++k) {
    if (ci[k] < 0 || cj[k] < 0 || ci[k] >= V.nx || cj[k] >= V.ny) continue;
    const long long c = V.base + (long long)cj[k] * V.P + ci[k];
    if (!(tag[c] & CELL_ACTIVE)) continue;
    gx += G[(corner[k] * 2 + 0) * Vtot + c];
    gy += G[(corner[k] * 2 + 1) * Vtot + c];
  }
  gx = -gx;
  gy = -gy;
  if ((tag[n] & KIND_MASK) == K_DIR && U != 0.0) {
    // (K Lambda)_n = sum over cells of sum_{b != a} K_ab (Lambda_b - Lambda_a), Lambda_a = 0 here
    auto lv = [&](long long m) -> double {
      const int kind = tag[m] & KIND_MASK;
      return node_value(kind, m, bid[m], V.body0, lam, lamb);
    };
    auto kc = [&](int m, long long c, bool gen) -> double { return gen ? K64[m * Vtot + c] : V.kr64[m]; };
    double kl = 0.0;
    const long long P = V.P;
    // cell (i, j), corner 0: K01 E, K02 NE, K03 N
    if (i < V.nx && j < V.ny && (tag[n] & CELL_ACTIVE)) {
      const bool gen = tag[n] & CELL_GENERAL;
      kl += kc(0, n, gen) * lv(n + 1) + kc(1, n, gen) * lv(n + 1 + P) + kc(2, n, gen) * lv(n + P);
    }
    // cell (i-1, j), corner 1: K01 W, K12 N, K13 NW
    if (i > 0 && j < V.ny && (tag[n - 1] & CELL_ACTIVE)) {
      const long long c = n - 1;
      const bool gen = tag[c] & CELL_GENERAL;
      kl += kc(0, c, gen) * lv(n - 1) + kc(3, c, gen) * lv(n + P) + kc(4, c, gen) * lv(n - 1 + P);
    }
    // cell (i-1, j-1), corner 2: K02 SW, K12 S, K23 W
    if (i > 0 && j > 0 && (tag[n - P - 1] & CELL_ACTIVE)) {
      const long long c = n - P - 1;
      const bool gen = tag[c] & CELL_GENERAL;
      kl += kc(1, c, gen) * lv(n - P - 1) + kc(3, c, gen) * lv(n - P) + kc(5, c, gen) * lv(n - 1);
    }
    // cell (i, j-1), corner 3: K03 S, K13 SE, K23 E
    if (j > 0 && i < V.nx && (tag[n - P] & CELL_ACTIVE)) {
      const long long c = n - P;
      const bool gen = tag[c] & CELL_GENERAL;
      kl += kc(2, c, gen) * lv(n - P) + kc(4, c, gen) * lv(n - P + 1) + kc(5, c, gen) * lv(n + 1);
    }
    gy -= U * kl;
  }
  dX[n] = gx;
  dX[Vtot + n] = gy;
}

// Transposed Jacobi sweeps, JKT per launch: out_m = [m fixed] in_m + sum over the updated
// neighbours n of in_n / 4 (W, E, S, N), on a fused-CG tile's window with a JKT-node halo
// swept in shared memory (sweep s of the launch covers the nodes at distance >= s + 1 from
// the window edge, the only ones read again), the tile written back.  Only the body nodes'
// values are read after the last sweep, and a sweep moves a value one node, so after this
// launch only nodes within `reach` (the sweeps still to come) of a body node matter.  A
// tile whose L1 distance from every body's node box exceeds that is skipped: its stale
// values are only ever read by nodes that are themselves too far to matter.
constexpr int JKT = 4;
constexpr int JTW = CTX + 2 * JKT, JTH = CTY + 2 * JKT;    // window 72 x 24
constexpr int JT_SMEM = 2 * JTW * JTH * (int)sizeof(double2) + JTW * JTH;

__global__ void __launch_bounds__(NT) k_jacobi_T(const DevVariant* var, const int* tile_var, const int2* tile_ij,
                                                 const uint8_t* tag, const int* bid, const int4* bbox, int reach,
                                                 int nsw, long long Vtot, const double* in, double* out) {
  extern __shared__ __align__(16) unsigned char jts[];
  double2* w0 = reinterpret_cast<double2*>(jts);
  double2* w1 = w0 + JTW * JTH;
  uint8_t* upd = reinterpret_cast<uint8_t*>(w1 + JTW * JTH);
  const int t = blockIdx.x;
  const DevVariant& V = var[tile_var[t]];
  const int2 ij = tile_ij[t];
  {
    bool near = false;
    for (int k = 0; k < V.nb && !near; ++k) {
      const int4 bx = bbox[V.body0 + k];
      const int gx = max(0, max(bx.x - (ij.x + CTX - 1), ij.x - bx.y));
      const int gy = max(0, max(bx.z - (ij.y + CTY - 1), ij.y - bx.w));
      near = gx + gy <= reach;
    }
    if (!near) return;
  }
  const int tid = linear_tid();
  for (int q = tid; q < JTW * JTH; q += NT) {
    const int i = ij.x - JKT + q % JTW, j = ij.y - JKT + q / JTW;
    double2 v = make_double2(0.0, 0.0);
    uint8_t u = 0;
    if (i >= 0 && j >= 0 && i <= V.nx && j <= V.ny) {
      const long long n = V.base + (long long)j * V.P + i;
      v = make_double2(in[n], in[Vtot + n]);
      u = bid[n] < 0 && !(tag[n] & (RING | WAKE));
    }
    w0[q] = v;
    upd[q] = u;
  }
  __syncthreads();
  double2* a = w0;
  double2* b = w1;
  for (int sw = 0; sw < nsw; ++sw) {
    const int rw = JTW - 2 * (sw + 1), rh = JTH - 2 * (sw + 1);
    for (int k = tid; k < rw * rh; k += NT) {
      const int ri = sw + 1 + k % rw, rj = sw + 1 + k / rw;
      const int q = rj * JTW + ri;
      double ox = 0.0, oy = 0.0;
      if (!upd[q]) {
        ox = a[q].x;
        oy = a[q].y;
      }
      // neighbours outside the grid carry upd = 0 and add nothing
      const int nq[4] = {q - 1, q + 1, q - JTW, q + JTW};
#pragma unroll
      for (int e = 0; e < 4; ++e)
        if (upd[nq[e]]) {
          ox += 0.25 * a[nq[e]].x;
          oy += 0.25 * a[nq[e]].y;
        }
      b[q] = make_double2(ox, oy);
    }
    __syncthreads();
    double2* tmp = a;
    a = b;
    b = tmp;
  }
  for (int q = tid; q < CTX * CTY; q += NT) {
    const int i = ij.x + q % CTX, j = ij.y + q / CTX;
    if (i <= V.nx && j <= V.ny) {
      const long long n = V.base + (long long)j * V.P + i;
      const double2 r = a[(JKT + q / CTX) * JTW + JKT + q % CTX];
      out[n] = r.x;
      out[Vtot + n] = r.y;
    }
  }
}

// dJ/dc_k = sum over the body's nodes of Jp^T (dJ/dd0)_n, Jp = I - (r/rho)(I - u u^T) at
// the node's background-grid position.  One CTA per global body, fixed-order sum.
__global__ void k_centre_grad(const DevVariant* var, const int* body_var, const pf_body* bodies, const int* body_ptr,
                              const long long* body_nodes, long long Vtot, const double* gd, double* out) {
  __shared__ double scratch[NT / 32 + 1];
  const int gb = blockIdx.x;
  const DevVariant& V = var[body_var[gb]];
  const pf_body Bd = bodies[gb];
  double sx = 0.0, sy = 0.0;
  for (int e = body_ptr[gb] + linear_tid(); e < body_ptr[gb + 1]; e += NT) {
    const long long n = body_nodes[e];
    const long long rem = n - V.base;
    const int i = (int)(rem % V.P), j = (int)(rem / V.P);
    const double xg = V.x0 + (double)i * V.hx, yg = V.y0 + (double)j * V.hy;
    const double ex = xg - Bd.cx, ey = yg - Bd.cy;
    const double rho = sqrt(ex * ex + ey * ey);
    const double ux = ex / rho, uy = ey / rho, s = Bd.r / rho;
    const double j00 = 1.0 - s * (1.0 - ux * ux), j01 = s * ux * uy, j11 = 1.0 - s * (1.0 - uy * uy);
    const double gx = gd[n], gy = gd[Vtot + n];
    sx += j00 * gx + j01 * gy;
    sy += j01 * gx + j11 * gy;
  }
  sx = block_sum(sx, scratch);
  sy = block_sum(sy, scratch);
  if (linear_tid() == 0) {
    out[2 * gb] = sx;
    out[2 * gb + 1] = sy;
  }
}

__global__ void k_export_grad(const DevVariant* var, const long long* lbase, long long Vtot, const double* dX,
                              double* out) {
  const int v = blockIdx.y;
  const DevVariant& V = var[v];
  const long long N = (long long)(V.nx + 1) * (V.ny + 1);
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(m % (V.nx + 1)), j = (int)(m / (V.nx + 1));
    const long long n = V.base + (long long)j * V.P + i;
    out[2 * (lbase[v] + m)] = dX[n];
    out[2 * (lbase[v] + m) + 1] = dX[Vtot + n];
  }
}

// Inverse of k_export_grad: a logical [nodes][2] cotangent into the padded planes.
__global__ void k_import_grad(const DevVariant* var, const long long* lbase, long long Vtot, const double* in,
                              double* g) {
  const int v = blockIdx.y;
  const DevVariant& V = var[v];
  const long long N = (long long)(V.nx + 1) * (V.ny + 1);
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(m % (V.nx + 1)), j = (int)(m / (V.nx + 1));
    const long long n = V.base + (long long)j * V.P + i;
    g[n] = in[2 * (lbase[v] + m)];
    g[Vtot + n] = in[2 * (lbase[v] + m) + 1];
  }
}

}  // namespace

static void ensure_grad_memory(Batch& b) {
  if (b.psi_save) return;
  const long long Vt = b.Vtot;
  const int B = std::max(1, b.B);
  b.psi_save = (double*)dev_alloc(b, Vt * sizeof(double));
  b.sol_save = (double*)dev_alloc(b, B * sizeof(double));
  b.d_rhsb = (double*)dev_alloc(b, B * sizeof(double));
  b.gradX = (double*)dev_alloc(b, 2 * Vt * sizeof(double));
  b.gradT = (double*)dev_alloc(b, 2 * Vt * sizeof(double));
  b.cellG = (double*)dev_alloc(b, 8 * Vt * sizeof(double));
}

// Centre cotangent of the coordinate cotangent held in b.gradX (padded planes, consumed):
// the S transposed smoothing sweeps, then the projection Jacobian summed over each body's
// nodes.  Host output [B][2].
static void centre_chain(Batch& b, double* gc) {
  cudaStream_t s = b.stream;
  const long long Vt = b.Vtot;
  const dim3 blk(TX, TY);
  double* a = b.gradX;
  double* c = b.gradT;
  PF_CUDA(cudaMemsetAsync(c, 0, 2 * Vt * sizeof(double), s));
  if (b.sweeps > 0) PF_CUDA(cudaFuncSetAttribute(k_jacobi_T, cudaFuncAttributeMaxDynamicSharedMemorySize, JT_SMEM));
  int launches = 0;
  for (int k = 0; k < b.sweeps; k += JKT, ++launches) {
    const int nsw = std::min(JKT, b.sweeps - k);
    k_jacobi_T<<<(unsigned)b.Tcg, NT, JT_SMEM, s>>>(b.d_var, b.tile_cg_var, b.tile_cg_ij, b.tag, b.bid, b.d_bbox,
                                                    b.sweeps - k - nsw, nsw, Vt, a, c);
    std::swap(a, c);
  }
  PF_CUDA(cudaGetLastError());
  double* out = b.cellG;   // reuse as a [B][2] result buffer
  if (b.B > 0) {
    k_centre_grad<<<b.B, blk, 0, s>>>(b.d_var, b.d_body_var, b.d_bodies, b.body_ptr, b.body_nodes, Vt, a, out);
    PF_CUDA(cudaGetLastError());
    PF_CUDA(cudaMemcpyAsync(gc, out, 2 * b.B * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  PF_CUDA(cudaStreamSynchronize(s));
  b.launches += launches + (b.B > 0 ? 1 : 0);
}

void coords_vjp(Batch& b, const double* dev_gX, double* gc) {
  if (b.cut) throw Error{PF_EINVAL, "pf_coords_vjp: the mesh generator's Jacobian is that of the Q4 mesh"};
  if (b.has_polygons)
    throw Error{PF_EINVAL, "pf_coords_vjp: the projection Jacobian is that of circular bodies"};
  ensure_grad_memory(b);
  PF_CUDA(cudaMemsetAsync(b.gradX, 0, 2 * b.Vtot * sizeof(double), b.stream));
  k_import_grad<<<dim3(256, b.nv), 256, 0, b.stream>>>(b.d_var, lbase_cached(b), b.Vtot, dev_gX, b.gradX);
  PF_CUDA(cudaGetLastError());
  b.launches += 1;
  centre_chain(b, gc);
}

pf_status shape_gradient(Batch& b, int obj, int lo, int hi, double U, double tol, double* dev_dJdX, double* dJdc,
                         double* J) {
  if (!b.solved) throw Error{PF_EINVAL, "pf_grad needs a solve on this handle first"};
  if (b.cut) throw Error{PF_EINVAL, "pf_grad: the shape derivative is written for the Q4 mesh"};
  if (b.has_polygons)
    throw Error{PF_EINVAL, "pf_grad: the centre chain rule is that of circular bodies (radial projection)"};
  if (U != b.lastU) throw Error{PF_EINVAL, "pf_grad must use the U of the last solve"};
  if (!(tol > 0)) throw Error{PF_EINVAL, "invalid tol"};
  cudaStream_t s = b.stream;
  const long long Vt = b.Vtot;
  const int B = std::max(1, b.B);
  // objective values and adjoint right-hand sides (host)
  std::vector<double> C;
  body_values(b, C);
  std::vector<double> Jv(b.nv), w(b.nv), dy(b.nv), rhs(B, 0.0);
  for (int v = 0; v < b.nv; ++v) {
    const int g0 = b.hv[v].body0;
    const double q = C[g0 + hi] - C[g0 + lo];
    dy[v] = b.bodies[g0 + hi].cy - b.bodies[g0 + lo].cy;
    if (obj == PF_OBJ_COPFI) {
      if (U == 0.0 || dy[v] == 0.0) throw Error{PF_EINVAL, "CoPFI needs U != 0 and distinct body heights"};
      Jv[v] = q / (U * dy[v]);
      w[v] = 1.0 / (U * dy[v]);
    } else {
      Jv[v] = q;
      w[v] = 1.0;
    }
    rhs[g0 + hi] += w[v];
    rhs[g0 + lo] -= w[v];
  }
  ensure_grad_memory(b);
  PF_CUDA(cudaMemcpyAsync(b.psi_save, b.x64, Vt * sizeof(double), cudaMemcpyDeviceToDevice, s));
  PF_CUDA(cudaMemcpyAsync(b.sol_save, b.sol64, B * sizeof(double), cudaMemcpyDeviceToDevice, s));
  PF_CUDA(cudaMemcpyAsync(b.d_rhsb, rhs.data(), B * sizeof(double), cudaMemcpyHostToDevice, s));
  // adjoint solve: same operator (self-adjoint), no Dirichlet data, body-row right-hand side
  pf_solve_opts o{};
  o.tol = tol;
  o.k_max = 100000000;
  o.precision = PF_MIXED;
  o.inner_tol = PF_DEFAULT_INNER_TOL;
  o.preconditioner = b.last_precond;   // the forward solve's choice (both run in PF_MIXED)
  b.rhs_active = true;
  pf_status st = PF_OK;
  try {
    st = solve_core(b, 0.0, o, nullptr, nullptr, nullptr, false);
  } catch (...) {
    b.rhs_active = false;
    throw;
  }
  b.rhs_active = false;
  // element shape derivatives and node gradient
  const dim3 blk(TX, TY);
  PF_CUDA(cudaMemsetAsync(b.cellG, 0, 8 * Vt * sizeof(double), s));
  k_shape_cells<<<(unsigned)b.T, blk, 0, s>>>(b.d_var, b.tile_var, b.tile_ij, b.tag, b.bid, b.X, Vt, b.psi_save,
                                              b.sol_save, b.x64, b.sol64, b.cellG);
  PF_CUDA(cudaMemsetAsync(b.gradX, 0, 2 * Vt * sizeof(double), s));
  k_shape_nodes<<<(unsigned)b.T, blk, 0, s>>>(b.d_var, b.tile_var, b.tile_ij, b.tag, b.bid, Vt, b.cellG, b.K64,
                                              b.x64, b.sol64, U, b.gradX);
  PF_CUDA(cudaGetLastError());
  if (dev_dJdX) {
    k_export_grad<<<dim3(256, b.nv), 256, 0, s>>>(b.d_var, lbase_cached(b), Vt, b.gradX, dev_dJdX);
    PF_CUDA(cudaGetLastError());
  }
  if (dJdc) {
    centre_chain(b, dJdc);
    if (obj == PF_OBJ_COPFI) {
      for (int v = 0; v < b.nv; ++v) {
        const int g0 = b.hv[v].body0;
        dJdc[2 * (g0 + hi) + 1] += -Jv[v] / dy[v];
        dJdc[2 * (g0 + lo) + 1] += Jv[v] / dy[v];
      }
    }
  }
  // restore the forward solution
  PF_CUDA(cudaMemcpyAsync(b.x64, b.psi_save, Vt * sizeof(double), cudaMemcpyDeviceToDevice, s));
  PF_CUDA(cudaMemcpyAsync(b.sol64, b.sol_save, B * sizeof(double), cudaMemcpyDeviceToDevice, s));
  PF_CUDA(cudaStreamSynchronize(s));
  b.lastU = U;
  b.launches += 2 + (dev_dJdX ? 1 : 0);
  if (J)
    for (int v = 0; v < b.nv; ++v) J[v] = Jv[v];
  return st;
}

}  // namespace pfq4
