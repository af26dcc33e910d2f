// Multigrid-preconditioned Conjugate Gradient for the stream-function system (an
// extension beyond the paper, whose Appendix A CG is unpreconditioned; its iteration
// count grows with the grid, about 2,100 iterations on a 1024x512 grid).
//
// Preconditioner M^-1 (symmetric positive definite, the same every iteration):
//   * free unknowns: one V(1,1)-cycle of geometric multigrid on the logical node grid of
//     each variant.  Level 0 is the mesh itself with its Q4 element matrices (the FP32
//     operator of the CG); level l+1 has ceil(n_l / 2) cells per direction, coarse node I
//     sitting on fine node min(2I, n_l).  Interpolation P is bilinear along the index
//     lines (an odd fine node takes half of each coarse neighbour, the last node of an odd
//     line copies its coarse node).  A coarse node carries an unknown only if the fine node
//     under it does (constraints are injected), and P has no entries for constrained
//     nodes.  Coarse operators are Galerkin products A_{l+1} = P^T A_l P (9-point
//     stencils, formed once in FP32, the precision the cycle applies them in).  Smoother: damped Jacobi (omega = 0.85), one sweep
//     before (from zero) and one after the coarse correction on every level (two each way
//     took more time per solve: fewer iterations did not pay for the extra passes); the
//     coarsest level (at most 17 x 17 nodes) takes 100 Jacobi sweeps from zero.  Jacobi with a fixed sweep
//     count is a fixed symmetric operator, so the cycle is a valid CG preconditioner.
//   * body unknowns (one per body, the multi-point constraint) and their coupling to the
//     free unknowns: a symmetric block Gauss-Seidel sweep body, free, body.  Forward:
//     y_b = r_b / D (D: the collapsed body row's diagonal, sum over the body's nodes n, m
//     of A(n, m)); the V-cycle then runs on r_f - A_fb y_b (the sweeps hold y_b at the
//     BODY nodes); backward: z_b = (r_b - A_bf z_f) / D.  A_fb and A_bf go through the
//     list of free nodes next to each body with their summed couplings.  The result is
//     [I, 0; -D^-1 A_bf, I] [B, 0; 0, D^-1] [I, -A_fb D^-1; 0, I] with B the V-cycle:
//     symmetric positive definite.  (The body-diagonal preconditioner alone, without the
//     coupling, took 21-31 iterations instead of 15-22 on the 256-variant sweep.)
//
// The CG iteration itself is the paper's with the preconditioner inserted:
//   x += alpha p, r -= alpha q; z = M^-1 r; beta = (r.z) / (r.z)_old; p = z + beta p;
//   q = A p; alpha = (r.z) / (p.q),
// one kernel per step over all variants of the batch, with per-variant scalars formed
// by small finaliser kernels (one CTA per variant, partial sums added in a fixed order,
// so repeated solves are bitwise identical).  The vectors are FP32 planes in the padded
// node layout; the FP64 true residual and the iterative refinement are the kernels of
// the unpreconditioned solve (k_fold, k_resid), which restart this CG from the FP64
// residual until the outer tolerance is met.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "batch.h"

namespace pfq4 {

namespace {

constexpr float MG_OMEGA = 0.85f;        // Jacobi damping (smoothing factor ~1/3 for Q4 Laplace stencils)
constexpr int MG_CMAX = 16;              // coarsen while a level has more than this many cells per direction
constexpr int MG_COARSE_SWEEPS = 100;    // Jacobi sweeps of the coarsest solve
constexpr int MG_MAXC = 17 * 17;         // nodes of a coarsest level at most

// ---------------------------------------------------------------- index rules
// Weight of coarse index I in the interpolation of fine index i on a line of n cells.
__device__ __forceinline__ double pw(int i, int n, int I) {
  if ((i & 1) == 0) return I == (i >> 1) ? 1.0 : 0.0;
  if (i == n) return I == ((i + 1) >> 1) ? 1.0 : 0.0;
  return (I == ((i - 1) >> 1) || I == ((i + 1) >> 1)) ? 0.5 : 0.0;
}
// Coarse parents of fine index i: count, indices and weights.
__device__ __forceinline__ int parents(int i, int n, int* I, double* w) {
  if ((i & 1) == 0) { I[0] = i >> 1; w[0] = 1.0; return 1; }
  if (i == n) { I[0] = (i + 1) >> 1; w[0] = 1.0; return 1; }
  I[0] = (i - 1) >> 1; I[1] = (i + 1) >> 1; w[0] = w[1] = 0.5;
  return 2;
}
__device__ __forceinline__ int fine_of(int I, int n) { return min(2 * I, n); }
// The same rules in FP32 for the cycle (the weights 1 and 1/2 are exact in FP32).
__device__ __forceinline__ float pwf(int i, int n, int I) {
  if ((i & 1) == 0) return I == (i >> 1) ? 1.0f : 0.0f;
  if (i == n) return I == ((i + 1) >> 1) ? 1.0f : 0.0f;
  return (I == ((i - 1) >> 1) || I == ((i + 1) >> 1)) ? 0.5f : 0.0f;
}
__device__ __forceinline__ int parentsf(int i, int n, int* I, float* w) {
  if ((i & 1) == 0) { I[0] = i >> 1; w[0] = 1.0f; return 1; }
  if (i == n) { I[0] = (i + 1) >> 1; w[0] = 1.0f; return 1; }
  I[0] = (i - 1) >> 1; I[1] = (i + 1) >> 1; w[0] = w[1] = 0.5f;
  return 2;
}

// Row of the fine (level-0) operator at node n = (i, j) as a 9-point stencil in FP64,
// slot (dy + 1) * 3 + (dx + 1): off-diagonal entries summed over the active cells that
// contain both nodes, the diagonal minus their sum (every element row sums to zero).
__device__ void fine_stencil(const MeshDev& m, const DevVariant& V, long long n, int i, int j, double st[9]) {
  for (int k = 0; k < 9; ++k) st[k] = 0.0;
  const long long plane = m.Vtot;
  const long long P = V.P;
  auto coef = [&](long long c, int mm, bool gen) { return gen ? m.K64[mm * plane + c] : V.kr64[mm]; };
  // cell (i, j): node is corner 0: K01 -> E, K02 -> NE, K03 -> N
  if (i < V.nx && j < V.ny && (m.tag[n] & CELL_ACTIVE)) {
    const bool g = m.tag[n] & CELL_GENERAL;
    st[5] += coef(n, 0, g); st[8] += coef(n, 1, g); st[7] += coef(n, 2, g);
  }
  // cell (i-1, j): corner 1: K01 -> W, K12 -> N, K13 -> NW
  if (i > 0 && j < V.ny && (m.tag[n - 1] & CELL_ACTIVE)) {
    const long long c = n - 1;
    const bool g = m.tag[c] & CELL_GENERAL;
    st[3] += coef(c, 0, g); st[7] += coef(c, 3, g); st[6] += coef(c, 4, g);
  }
  // cell (i-1, j-1): corner 2: K02 -> SW, K12 -> S, K23 -> W
  if (i > 0 && j > 0 && (m.tag[n - P - 1] & CELL_ACTIVE)) {
    const long long c = n - P - 1;
    const bool g = m.tag[c] & CELL_GENERAL;
    st[0] += coef(c, 1, g); st[1] += coef(c, 3, g); st[3] += coef(c, 5, g);
  }
  // cell (i, j-1): corner 3: K03 -> S, K13 -> SE, K23 -> E
  if (j > 0 && i < V.nx && (m.tag[n - P] & CELL_ACTIVE)) {
    const long long c = n - P;
    const bool g = m.tag[c] & CELL_GENERAL;
    st[1] += coef(c, 2, g); st[2] += coef(c, 4, g); st[5] += coef(c, 5, g);
  }
  double s = 0.0;
  for (int k = 0; k < 9; ++k)
    if (k != 4) s += st[k];
  st[4] = -s;
}

// The same row from the FP32 coefficients, summed in FP32 (the multigrid set-up: the
// preconditioner's operators are FP32, and FP64 arithmetic runs at a small fraction of
// the FP32 rate on this GPU).  Stored coefficients are read only where their FP32 values
// differ from the rectangle's (CELL_GEN32); elsewhere they equal kr32 exactly.
__device__ void fine_stencil32(const MeshDev& m, const DevVariant& V, long long n, int i, int j, float st[9]) {
  for (int k = 0; k < 9; ++k) st[k] = 0.0f;
  const long long plane = m.Vtot;
  const long long P = V.P;
  auto coef = [&](long long c, int mm, bool gen) { return gen ? m.K32[mm * plane + c] : V.kr32[mm]; };
  if (i < V.nx && j < V.ny && (m.tag[n] & CELL_ACTIVE)) {
    const bool g = m.tag[n] & CELL_GEN32;
    st[5] += coef(n, 0, g); st[8] += coef(n, 1, g); st[7] += coef(n, 2, g);
  }
  if (i > 0 && j < V.ny && (m.tag[n - 1] & CELL_ACTIVE)) {
    const long long c = n - 1;
    const bool g = m.tag[c] & CELL_GEN32;
    st[3] += coef(c, 0, g); st[7] += coef(c, 3, g); st[6] += coef(c, 4, g);
  }
  if (i > 0 && j > 0 && (m.tag[n - P - 1] & CELL_ACTIVE)) {
    const long long c = n - P - 1;
    const bool g = m.tag[c] & CELL_GEN32;
    st[0] += coef(c, 1, g); st[1] += coef(c, 3, g); st[3] += coef(c, 5, g);
  }
  if (j > 0 && i < V.nx && (m.tag[n - P] & CELL_ACTIVE)) {
    const long long c = n - P;
    const bool g = m.tag[c] & CELL_GEN32;
    st[1] += coef(c, 2, g); st[2] += coef(c, 4, g); st[5] += coef(c, 5, g);
  }
  float s = 0.0f;
  for (int k = 0; k < 9; ++k)
    if (k != 4) s += st[k];
  st[4] = -s;
}

// Node of a packed coarse level handled by this thread: variant, (i, j) and the index,
// or false for padding / variants without the level.
struct LvNode {
  int v, i, j, nx, ny;
  long long k;
};
__device__ __forceinline__ bool lv_node(const long long* off, const int2* dims, const int* blkvar, LvNode& q) {
  const int v = blkvar[blockIdx.x];
  if (v < 0) return false;
  const long long o = off[v];
  if (o < 0) return false;
  const int2 d = dims[v];
  const long long loc = (long long)blockIdx.x * blockDim.x + threadIdx.x - o;
  if (loc >= (long long)(d.x + 1) * (d.y + 1)) return false;
  q.v = v;
  q.nx = d.x;
  q.ny = d.y;
  q.i = (int)(loc % (d.x + 1));
  q.j = (int)(loc / (d.x + 1));
  q.k = o + loc;
  return true;
}

struct LvArgs {              // one coarse level, device view
  const long long* off;
  const int2* dims;
  const int* blkvar;
  long long n;
  const uint8_t* act;
  const float* A;            // [9][n]
  const float* dinv;
  float *r, *za, *zb, *res;
};

// ---------------------------------------------------------------- setup kernels
// Activity of level l+1 from level l (l = 0: FREE nodes of the mesh).
__global__ void k_mg_act(LvArgs c, const uint8_t* act_f, const long long* off_f, const int2* dims_f,
                         const DevVariant* var, const uint8_t* tag, uint8_t* act_c) {
  LvNode q;
  if (!lv_node(c.off, c.dims, c.blkvar, q)) return;
  const int2 df = off_f ? dims_f[q.v] : make_int2(var[q.v].nx, var[q.v].ny);
  const int fi = fine_of(q.i, df.x), fj = fine_of(q.j, df.y);
  uint8_t a;
  if (off_f) a = act_f[off_f[q.v] + (long long)fj * (df.x + 1) + fi];
  else a = (tag[var[q.v].base + (long long)fj * var[q.v].P + fi] & KIND_MASK) == K_FREE;
  act_c[q.k] = a;
}

// Galerkin stencil of coarse node I = sum_{a, b} P(a, I) A_f(a, b) P(b, J) over active
// fine nodes a, b, in FP32 (the precision the cycle applies it in), and the Jacobi factor.
__global__ void k_mg_rap(LvArgs c, float* A32c, float* dinvc, MeshDev m, const uint8_t* act_f, const float* A32f,
                         const long long* off_f, const int2* dims_f, long long nf) {
  LvNode q;
  if (!lv_node(c.off, c.dims, c.blkvar, q)) return;
  float acc[9];
  for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
  const DevVariant& V = m.var[q.v];
  const bool fine0 = off_f == nullptr;
  const int2 df = fine0 ? make_int2(V.nx, V.ny) : dims_f[q.v];
  const long long of = fine0 ? 0 : off_f[q.v];
  auto fidx = [&](int i, int j) -> long long {
    return fine0 ? V.base + (long long)j * V.P + i : of + (long long)j * (df.x + 1) + i;
  };
  auto factive = [&](int i, int j) -> bool {
    const long long n = fidx(i, j);
    return fine0 ? ((m.tag[n] & KIND_MASK) == K_FREE) : act_f[n] != 0;
  };
  if (c.act[q.k]) {
    const int fx = fine_of(q.i, df.x), fy = fine_of(q.j, df.y);
    // every interpolation weight is 1 or 1/2, so each product weight x stencil entry is
    // the entry scaled by 2^-h (h halves): exact, one FP32 multiply by that power of two
    for (int ay = fy - 1; ay <= fy + 1; ++ay) {
      if (ay < 0 || ay > df.y) continue;
      const double wy = pw(ay, df.y, q.j);
      if (wy == 0.0) continue;
      for (int ax = fx - 1; ax <= fx + 1; ++ax) {
        if (ax < 0 || ax > df.x) continue;
        const double wxa = pw(ax, df.x, q.i);
        const int ha = (wxa == 0.5) + (wy == 0.5);       // halves of wa = wxa * wy
        if (wxa == 0.0 || !factive(ax, ay)) continue;
        float st[9];
        const long long na = fidx(ax, ay);
        if (fine0) fine_stencil32(m, V, na, ax, ay, st);
        else
          for (int k = 0; k < 9; ++k) st[k] = A32f[k * nf + na];
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const float sv = st[(dy + 1) * 3 + dx + 1];
            const int bx = ax + dx, by = ay + dy;
            if (sv == 0.0f || bx < 0 || by < 0 || bx > df.x || by > df.y || !factive(bx, by)) continue;
            int Ix[2], Iy[2];
            double wx[2], wyb[2];
            const int nxp = parents(bx, df.x, Ix, wx), nyp = parents(by, df.y, Iy, wyb);
            for (int u = 0; u < nyp; ++u)
              for (int t = 0; t < nxp; ++t) {
                const int ddx = Ix[t] - q.i, ddy = Iy[u] - q.j;
                if (ddx < -1 || ddx > 1 || ddy < -1 || ddy > 1) continue;
                if (!c.act[q.k + (long long)ddy * (q.nx + 1) + ddx]) continue;
                const int h = ha + (wx[t] == 0.5) + (wyb[u] == 0.5);
                acc[(ddy + 1) * 3 + ddx + 1] += sv * __int_as_float((127 - h) << 23);   // sv * 2^-h
              }
          }
      }
    }
  }
  for (int k = 0; k < 9; ++k) A32c[k * c.n + q.k] = acc[k];
  dinvc[q.k] = (c.act[q.k] && acc[4] > 0.0f) ? (float)MG_OMEGA / acc[4] : 0.0f;
}

// Jacobi factor of the fine level: omega / diagonal at FREE nodes.
__global__ void k_mg_dinv0(MeshDev m, const int* tile_var, const int2* tile_ij, float* dinv0) {
  const DevVariant& V = m.var[tile_var[blockIdx.x]];
  const int2 ij = tile_ij[blockIdx.x];
  const int i = ij.x + threadIdx.x, j = ij.y + threadIdx.y;
  if (i > V.nx || j > V.ny) return;
  const long long n = V.base + (long long)j * V.P + i;
  float d = 0.0f;
  if ((m.tag[n] & KIND_MASK) == K_FREE) {
    float st[9];
    fine_stencil32(m, V, n, i, j, st);
    d = st[4] > 0.0f ? (float)MG_OMEGA / st[4] : 0.0f;
  }
  dinv0[n] = d;
}

// Diagonal of each collapsed body row: sum over the body's nodes n of the stencil
// entries A(n, m) towards nodes m of the same body (one CTA per body, fixed order).
__global__ void __launch_bounds__(NT) k_mg_body_diag(MeshDev m, const int* body_var, double* Abb) {
  __shared__ double scratch[NT / 32 + 1];
  const int gb = blockIdx.x;
  const DevVariant& V = m.var[body_var[gb]];
  const int kb = gb - V.body0;
  double s = 0.0;
  for (int e = m.body_ptr[gb] + linear_tid(); e < m.body_ptr[gb + 1]; e += NT) {
    const long long n = m.body_nodes[e];
    const long long rem = n - V.base;
    const int i = (int)(rem % V.P), j = (int)(rem / V.P);
    double st[9];
    fine_stencil(m, V, n, i, j, st);
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        const int bi = i + dx, bj = j + dy;
        if (bi < 0 || bj < 0 || bi > V.nx || bj > V.ny) continue;
        const long long nb = n + (long long)dy * V.P + dx;
        if ((m.tag[nb] & KIND_MASK) == K_BODY && m.bid[nb] == kb) s += st[(dy + 1) * 3 + dx + 1];
      }
  }
  s = block_sum(s, scratch);
  if (linear_tid() == 0) Abb[gb] = s;
}

// ---------------------------------------------------------------- cycle kernels, fine level
// The fine-level kernels run on the 64 x 16 tiles of the fused CG step, 256 threads per
// tile, each thread a vertical strip of 4 nodes (column tid % 64, rows 4 (tid / 64) ..
// + 3), with the tile's one-node halo in shared memory.  Every FP32 plane of the cycle
// is zero at nodes without an unknown (only FREE nodes are ever written), so values and
// tags are loaded together, without a tag-dependent second load.
constexpr int FW = CTX + 2;                 // shared tile width (66)
constexpr int FH = CTY + 2;                 // shared tile height (18)
constexpr int FS = CTY * CTX / NT;          // nodes per thread (4)
constexpr int FNH = 2 * FW + 2 * CTY;       // halo positions (164)
static_assert(FS * NT == CTX * CTY && FNH <= NT, "fine-level tile mapping");

struct FineArgs {
  MeshDev m;
  const int* tile_var;       // fused-CG tile list (64 x 16)
  const int2* tile_ij;
  const VarState* st;
  const float* dinv0;
  float *x, *r, *z, *t, *res, *q;
  float* p[2];
  const float* sb;           // [4][B] body CG values x, r, p, q
  const float* yb;           // [B] body values of the forward body step (held at BODY nodes by the sweeps)
  int B;
  double* part;              // [tiles] partial sums of the kernel's dot product
  const long long* c_off;    // level 1 (the prolongation folded into the first post-sweep)
  const int2* c_dims;
  const float* c_zb;
};

__device__ __forceinline__ void halo_pos66(int h, int& li, int& lj) {
  if (h < FW) { li = h; lj = 0; }
  else if (h < 2 * FW) { li = h - FW; lj = CTY + 1; }
  else if (h < 2 * FW + CTY) { li = 0; lj = 1 + (h - 2 * FW); }
  else { li = CTX + 1; lj = 1 + (h - 2 * FW - CTY); }
}

// P e at fine node (i, j) of variant v: the bilinear interpolation from level 1.
__device__ __forceinline__ float coarse_interp(const FineArgs& a, int v, const DevVariant& V, int i, int j) {
  const int2 dc = a.c_dims[v];
  const long long oc = a.c_off[v];
  int Ix[2], Iy[2];
  float wx[2], wy[2];
  const int nxp = parentsf(i, V.nx, Ix, wx), nyp = parentsf(j, V.ny, Iy, wy);
  float e = 0.0f;
  for (int u = 0; u < nyp; ++u)
    for (int t = 0; t < nxp; ++t) e += wx[t] * wy[u] * a.c_zb[oc + (long long)Iy[u] * (dc.x + 1) + Ix[t]];
  return e;
}

// Value of a level-0 vector of the cycle at node n with tag tg: the plane f at FREE nodes
// (0 where f is NULL: the first sweep starts from zero), the forward body step's value
// of the node's body at BODY nodes (the sweeps hold the body unknowns there, so every
// application of A includes A_fb y_b), 0 elsewhere.
__device__ __forceinline__ float cycle_value(const FineArgs& a, const DevVariant& V, const float* f, long long n,
                                             uint8_t tg) {
  const int kind = tg & KIND_MASK;
  if (kind == K_FREE) return f ? f[n] : 0.0f;
  if (kind == K_BODY) return a.yb[V.body0 + a.m.bid[n]];
  return 0.0f;
}

// Tile (with halo) of a cycle vector (cycle_value of the plane f) into ps and the tags
// into ts; PROL: plus P e at FREE nodes (coarse values are zero at inactive coarse nodes).
template <bool PROL>
__device__ __forceinline__ void load_tile66(const FineArgs& a, int v, const DevVariant& V, int2 ij, const float* f,
                                            float (*ps)[FW], uint8_t (*ts)[FW]) {
  const int tid = linear_tid(), col = tid % CTX, r0 = (tid / CTX) * FS;
  const int i = ij.x + col;
#pragma unroll
  for (int u = 0; u < FS; ++u) {
    const int j = ij.y + r0 + u;
    const bool in = i <= V.nx && j <= V.ny;
    const long long n = V.base + (long long)j * V.P + i;
    const uint8_t tg = in ? a.m.tag[n] : K_INACT;
    float val = in ? cycle_value(a, V, f, n, tg) : 0.0f;
    if (PROL && in) {
      const float e = coarse_interp(a, v, V, i, j);
      if ((tg & KIND_MASK) == K_FREE) val += e;
    }
    ps[1 + r0 + u][1 + col] = val;
    ts[1 + r0 + u][1 + col] = tg;
  }
  if (tid < FNH) {
    int li, lj;
    halo_pos66(tid, li, lj);
    const int hi = ij.x - 1 + li, hj = ij.y - 1 + lj;
    uint8_t ht = K_INACT;
    float hv = 0.0f;
    if (hi >= 0 && hj >= 0 && hi <= V.nx && hj <= V.ny) {
      const long long hn = V.base + (long long)hj * V.P + hi;
      ht = a.m.tag[hn];
      hv = cycle_value(a, V, f, hn, ht);
      if (PROL) {
        const float e = coarse_interp(a, v, V, hi, hj);
        if ((ht & KIND_MASK) == K_FREE) hv += e;
      }
    }
    ps[lj][li] = hv;
    ts[lj][li] = ht;
  }
}

// Block sum of the threads' two-float dot accumulators (FP64 across warps, fixed order)
// into part[blockIdx.x].
__device__ __forceinline__ void block_dot_acc(Acc<float>& acc, double* part, double* sh) {
  double w[4];
  acc.warp_reduce(w);
  const int tid = linear_tid(), lane = tid & 31, wp = tid >> 5;
  if (lane == 0) sh[wp] = w[0];
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int k = 0; k < NT / 32; ++k) s += sh[k];
    part[blockIdx.x] = s;
  }
}

// x += alpha p, r -= alpha q, z = dinv r (the first pre-smoothing sweep from zero, before
// the forward body step's term, which k_mg_fwd subtracts next to the bodies); r.r.
// Pointwise, FREE nodes only; a node is FREE exactly when its Jacobi factor is positive
// (every free node lies on an active cell), so no tag is needed.  (q is also written at
// BODY nodes, for the collapsed body rows, so the test matters.)
__global__ void __launch_bounds__(NT) k_mg0_update(FineArgs a) {
  __shared__ double sh[NT / 32];
  const int v = a.tile_var[blockIdx.x];
  const VarState& S = a.st[v];
  if (S.phase != PH_CG) return;
  const DevVariant& V = a.m.var[v];
  const int2 ij = a.tile_ij[blockIdx.x];
  const int tid = linear_tid(), col = tid % CTX, r0 = (tid / CTX) * FS;
  const int i = ij.x + col;
  const float alpha = (float)S.alpha;
  const float* pc = a.p[S.buf];
  float rn[FS];
#pragma unroll
  for (int u = 0; u < FS; ++u) {
    rn[u] = 0.0f;
    const int j = ij.y + r0 + u;
    if (i <= V.nx && j <= V.ny) {
      const long long n = V.base + (long long)j * V.P + i;
      const float pn = pc[n], xn = a.x[n], rr = a.r[n], qn = a.q[n], dn = a.dinv0[n];
      if (dn > 0.0f) {
        a.x[n] = xn + alpha * pn;
        rn[u] = rr - alpha * qn;
        a.r[n] = rn[u];
        a.z[n] = dn * rn[u];
      }
    }
  }
  Acc<float> acc;
  acc.zero();
  acc.add4(0, rn, rn);
  block_dot_acc(acc, a.part, sh);
}

// One Jacobi sweep on the fine level: zo = zi + dinv (r - A zi) at FREE nodes, zi with
// the body values of the forward body step at BODY nodes (cycle_value); zo is written at
// FREE nodes only (it stays 0 at the others).  MODE 1: res = r - A zi at FREE nodes.
// MODE 2: MODE 0 and the partial r.zo.  PROL: zi is first corrected by the prolongation
// from level 1 (the correction is not stored).
template <int MODE, bool PROL>
__global__ void __launch_bounds__(NT) k_mg0_sweep(FineArgs a, const float* zi, float* zo) {
  __shared__ float ps[FH][FW];
  __shared__ uint8_t ts[FH][FW];
  __shared__ double sh[NT / 32];
  const int v = a.tile_var[blockIdx.x];
  if (a.st[v].phase != PH_CG) return;
  const DevVariant& V = a.m.var[v];
  const int2 ij = a.tile_ij[blockIdx.x];
  const int tid = linear_tid(), col = tid % CTX, r0 = (tid / CTX) * FS;
  const int i = ij.x + col;
  float rv[FS], dv[FS];
#pragma unroll
  for (int u = 0; u < FS; ++u) {
    const int j = ij.y + r0 + u;
    const bool in = i <= V.nx && j <= V.ny;
    const long long n = V.base + (long long)j * V.P + i;
    rv[u] = in ? a.r[n] : 0.0f;
    dv[u] = in && MODE != 1 ? a.dinv0[n] : 0.0f;
  }
  load_tile66<PROL>(a, v, V, ij, zi, ps, ts);
  __syncthreads();
  float zout[FS];
#pragma unroll
  for (int u = 0; u < FS; ++u) {
    zout[u] = 0.0f;
    const int j = ij.y + r0 + u;
    if (i > V.nx || j > V.ny) continue;
    const long long n = V.base + (long long)j * V.P + i;
    const int li = 1 + col, lj = 1 + r0 + u;
    const uint8_t tg = ts[lj][li];
    if ((tg & KIND_MASK) != K_FREE) continue;   // zo, res are zero there already
    const float y = q4_row<float, FW>(ps, ts, li, lj, n, V.P, a.m.K32, a.m.Vtot, V.kr32);
    const float rr = rv[u] - y;
    if (MODE == 1) {
      zo[n] = rr;
    } else {
      zout[u] = ps[lj][li] + dv[u] * rr;
      zo[n] = zout[u];
    }
  }
  if (MODE == 2) {
    Acc<float> acc;
    acc.zero();
    acc.add4(0, rv, zout);
    block_dot_acc(acc, a.part, sh);
  }
}

// p = z + beta p at FREE nodes, the body's p at BODY nodes, 0 elsewhere (into the other
// buffer); q = A p at FREE and BODY nodes; partial p.q over FREE nodes.  z is the plane t.
__global__ void __launch_bounds__(NT) k_mg0_apply(FineArgs a) {
  __shared__ float ps[FH][FW];
  __shared__ uint8_t ts[FH][FW];
  __shared__ double sh[NT / 32];
  const int v = a.tile_var[blockIdx.x];
  const VarState& S = a.st[v];
  if (S.phase != PH_CG) return;
  const DevVariant& V = a.m.var[v];
  const int2 ij = a.tile_ij[blockIdx.x];
  const float beta = (float)S.beta;
  const float* pold = a.p[S.buf];
  float* pnew = a.p[S.buf ^ 1];
  const float* pb = a.sb + 2 * a.B;
  const int tid = linear_tid(), col = tid % CTX, r0 = (tid / CTX) * FS;
  const int i = ij.x + col;
  // t + beta p_old is zero at nodes without an unknown; BODY nodes take the body's value
  auto pval = [&](long long n, uint8_t tg) -> float {
    const float f = a.t[n] + beta * pold[n];
    return (tg & KIND_MASK) == K_BODY ? pb[V.body0 + a.m.bid[n]] : f;
  };
#pragma unroll
  for (int u = 0; u < FS; ++u) {
    const int j = ij.y + r0 + u;
    const bool in = i <= V.nx && j <= V.ny;
    const long long n = V.base + (long long)j * V.P + i;
    const uint8_t tg = in ? a.m.tag[n] : K_INACT;
    ps[1 + r0 + u][1 + col] = in ? pval(n, tg) : 0.0f;
    ts[1 + r0 + u][1 + col] = tg;
  }
  if (tid < FNH) {
    int li, lj;
    halo_pos66(tid, li, lj);
    const int hi = ij.x - 1 + li, hj = ij.y - 1 + lj;
    uint8_t ht = K_INACT;
    float hv = 0.0f;
    if (hi >= 0 && hj >= 0 && hi <= V.nx && hj <= V.ny) {
      const long long hn = V.base + (long long)hj * V.P + hi;
      ht = a.m.tag[hn];
      hv = pval(hn, ht);
    }
    ps[lj][li] = hv;
    ts[lj][li] = ht;
  }
  __syncthreads();
  float pp[FS], qq[FS];
#pragma unroll
  for (int u = 0; u < FS; ++u) {
    pp[u] = 0.0f;
    qq[u] = 0.0f;
    const int j = ij.y + r0 + u;
    if (i > V.nx || j > V.ny) continue;
    const long long n = V.base + (long long)j * V.P + i;
    const int li = 1 + col, lj = 1 + r0 + u;
    const int kind = ts[lj][li] & KIND_MASK;
    if (kind != K_FREE && kind != K_BODY) continue;
    const float y = q4_row<float, FW>(ps, ts, li, lj, n, V.P, a.m.K32, a.m.Vtot, V.kr32);
    a.q[n] = y;
    if (kind == K_FREE) {
      pnew[n] = ps[lj][li];
      pp[u] = ps[lj][li];
      qq[u] = y;
    }
  }
  Acc<float> acc;
  acc.zero();
  acc.add4(0, pp, qq);
  block_dot_acc(acc, a.part, sh);
}

// Free nodes next to body gb (one CTA per body): the FREE nodes of the body's node box
// grown by one, row-major, with a BODY neighbour of this body, and their coupling
// c = sum over those neighbours m of A(n, m), read from the node's own FP32 stencil (the
// element entries are symmetric, so this is also the sum of A(m, n)).  pass 0 counts,
// pass 1 writes.
__global__ void __launch_bounds__(NT) k_mg_adj(MeshDev m, const int* body_var, const int4* bbox, int* count,
                                               const int* ptr, long long* out_n, float* out_c, int pass) {
  __shared__ int sh[NT / 32 + 1];
  const int gb = blockIdx.x;
  const DevVariant& V = m.var[body_var[gb]];
  const int k = gb - V.body0;
  const int4 bx = bbox[gb];
  const int i0 = max(0, bx.x - 1), i1 = min(V.nx, bx.y + 1), j0 = max(0, bx.z - 1), j1 = min(V.ny, bx.w + 1);
  const int w = i1 - i0 + 1;
  const long long total = (long long)w * (j1 - j0 + 1);
  int run = 0;
  for (long long s0 = 0; s0 < total; s0 += NT) {
    const long long q = s0 + linear_tid();
    int flag = 0;
    long long n = 0;
    float c = 0.0f;
    if (q < total) {
      const int i = i0 + (int)(q % w), j = j0 + (int)(q / w);
      n = V.base + (long long)j * V.P + i;
      if ((m.tag[n] & KIND_MASK) == K_FREE) {
        float st[9];
        bool any = false;
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            const int mi = i + dx, mj = j + dy;
            if (mi < 0 || mj < 0 || mi > V.nx || mj > V.ny) continue;
            const long long mn = n + (long long)dy * V.P + dx;
            if ((m.tag[mn] & KIND_MASK) == K_BODY && m.bid[mn] == k) {
              if (!any) fine_stencil32(m, V, n, i, j, st);
              any = true;
              c += st[(dy + 1) * 3 + dx + 1];
            }
          }
        flag = any;
      }
    }
    int tot;
    const int pos = block_exscan(flag, &tot, sh);
    if (pass == 1 && flag) {
      out_n[ptr[gb] + run + pos] = n;
      out_c[ptr[gb] + run + pos] = c;
    }
    run += tot;
  }
  if (pass == 0 && linear_tid() == 0) count[gb] = run;
}

// ---------------------------------------------------------------- cycle kernels, coarse levels
// r_c = P^T res_f (res_f of level l = 0 in the padded mesh layout, or of a packed level)
// and z_c = dinv r_c, for variants whose coarsest level is below this one.
__global__ void __launch_bounds__(256) k_mg_restrict(LvArgs c, int lc, const int* Lv, const VarState* st,
                                                     const DevVariant* var, const float* res_f,
                                                     const long long* off_f, const int2* dims_f) {
  LvNode q;
  if (!lv_node(c.off, c.dims, c.blkvar, q)) return;
  if (st[q.v].phase != PH_CG || lc > Lv[q.v] - 1) return;
  float rc = 0.0f;
  if (c.act[q.k]) {
    const bool fine0 = off_f == nullptr;
    const DevVariant& V = var[q.v];
    const int2 df = fine0 ? make_int2(V.nx, V.ny) : dims_f[q.v];
    const long long of = fine0 ? 0 : off_f[q.v];
    const int fx = fine_of(q.i, df.x), fy = fine_of(q.j, df.y);
    float s = 0.0f;
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
      const int ay = fy + dy;
      const float wy = (ay < 0 || ay > df.y) ? 0.0f : pwf(ay, df.y, q.j);
#pragma unroll
      for (int dx = -1; dx <= 1; ++dx) {
        const int ax = fx + dx;
        const float w = (ax < 0 || ax > df.x) ? 0.0f : pwf(ax, df.x, q.i) * wy;
        if (w == 0.0f) continue;
        const long long na = fine0 ? V.base + (long long)ay * V.P + ax : of + (long long)ay * (df.x + 1) + ax;
        s += w * res_f[na];     // res is zero at every node without an unknown
      }
    }
    rc = s;
  }
  c.r[q.k] = rc;
  c.za[q.k] = c.dinv[q.k] * rc;
}

// Jacobi sweep on a packed level: zo = zi + dinv (r - A zi); MODE 1: res = r - A zi.
template <int MODE>
__global__ void __launch_bounds__(256) k_mg_sweep(LvArgs c, int l, const int* Lv, const VarState* st,
                                                  const float* zi, float* zo) {
  LvNode q;
  if (!lv_node(c.off, c.dims, c.blkvar, q)) return;
  if (st[q.v].phase != PH_CG || l >= Lv[q.v] - 1) return;
  // the stencil, r, dinv and z are zero at inactive nodes: no activity test needed
  float y = 0.0f;
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int bi = q.i + dx, bj = q.j + dy;
      if (bi < 0 || bj < 0 || bi > q.nx || bj > q.ny) continue;
      y += c.A[((dy + 1) * 3 + dx + 1) * c.n + q.k] * zi[q.k + (long long)dy * (q.nx + 1) + dx];
    }
  const float rr = c.r[q.k] - y;
  zo[q.k] = MODE == 1 ? rr : zi[q.k] + c.dinv[q.k] * rr;
}

// za_f += P zb_c on a packed fine level (l >= 1): the pre-sweep value plus the coarse
// correction, which the post-sweep then smooths into zb_f.
__global__ void __launch_bounds__(256) k_mg_prolong(LvArgs f, LvArgs c, int l, const int* Lv, const VarState* st) {
  LvNode q;
  if (!lv_node(f.off, f.dims, f.blkvar, q)) return;
  if (st[q.v].phase != PH_CG || l >= Lv[q.v] - 1) return;
  const uint8_t act = f.act[q.k];
  const int2 dc = c.dims[q.v];
  const long long oc = c.off[q.v];
  int Ix[2], Iy[2];
  float wx[2], wy[2];
  const int nxp = parentsf(q.i, q.nx, Ix, wx), nyp = parentsf(q.j, q.ny, Iy, wy);
  float e = 0.0f;     // coarse values are zero at inactive coarse nodes
  for (int u = 0; u < nyp; ++u)
    for (int t = 0; t < nxp; ++t) e += wx[t] * wy[u] * c.zb[oc + (long long)Iy[u] * (dc.x + 1) + Ix[t]];
  if (act) f.za[q.k] = f.za[q.k] + e;
}

// Coarsest level of every variant (its own level Lv - 1): a fixed number of Jacobi
// sweeps from zero in shared memory, result in zb.  One CTA per variant.
struct CoarseTab {
  LvArgs lv[16];
};
__global__ void __launch_bounds__(256) k_mg_coarse(CoarseTab ct, const int* Lv, const VarState* st) {
  __shared__ float sA[9][MG_MAXC];
  __shared__ float sd[MG_MAXC], sr[MG_MAXC], z0[MG_MAXC], z1[MG_MAXC];
  const int v = blockIdx.x;
  if (st[v].phase != PH_CG) return;
  const LvArgs& c = ct.lv[Lv[v] - 1];
  const long long o = c.off[v];
  const int2 d = c.dims[v];
  const int nn = (d.x + 1) * (d.y + 1);
  if (o < 0 || nn > MG_MAXC) return;
  for (int k = threadIdx.x; k < nn; k += blockDim.x) {
    for (int s = 0; s < 9; ++s) sA[s][k] = c.A[s * c.n + o + k];
    sd[k] = c.dinv[o + k];
    sr[k] = c.r[o + k];
    z0[k] = 0.0f;
  }
  __syncthreads();
  float* a = z0;
  float* b = z1;
  for (int it = 0; it < MG_COARSE_SWEEPS; ++it) {
    for (int k = threadIdx.x; k < nn; k += blockDim.x) {
      const int i = k % (d.x + 1), j = k / (d.x + 1);
      float y = 0.0f;
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int bi = i + dx, bj = j + dy;
          if (bi < 0 || bj < 0 || bi > d.x || bj > d.y) continue;
          y += sA[(dy + 1) * 3 + dx + 1][k] * a[k + dy * (d.x + 1) + dx];
        }
      b[k] = a[k] + sd[k] * (sr[k] - y);
    }
    __syncthreads();
    float* tmp = a;
    a = b;
    b = tmp;
  }
  for (int k = threadIdx.x; k < nn; k += blockDim.x) c.zb[o + k] = a[k];
}

// The forward body step's term of the first pre-smoothing sweep: z -= dinv c y_b at the
// free nodes next to each body (one CTA per variant, its bodies in order, so a node next
// to two bodies takes both terms in a fixed order).
__global__ void __launch_bounds__(NT) k_mg_fwd(FineArgs a, const int* adj_ptr, const long long* adj_n,
                                               const float* adj_c) {
  const int v = blockIdx.x;
  if (a.st[v].phase != PH_CG) return;
  const DevVariant& V = a.m.var[v];
  for (int k = 0; k < V.nb; ++k) {
    const int gb = V.body0 + k;
    const float y = a.yb[gb];
    for (int e = adj_ptr[gb] + linear_tid(); e < adj_ptr[gb + 1]; e += NT) {
      const long long n = adj_n[e];
      a.z[n] -= a.dinv0[n] * (adj_c[e] * y);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- finalisers (one CTA per variant)
struct FinArgs {
  VarState* st;
  const SolveParams* prm;
  const long long* tile0;    // [nv + 1]
  const double* part;
  MeshDev m;
  float* sb;                 // [4][B]
  const double* Abb;
  const float* q;            // fine q plane (body rows gathered from it)
  float* yb;                 // [B] forward body step r_b / A_bb
  const float* t;            // the cycle's result at FREE nodes (the backward body step reads it)
  const int* adj_ptr;        // free nodes next to each body and their couplings (k_mg_adj)
  const long long* adj_n;
  const float* adj_c;
  int B;
  int* n_done;
};

__device__ double fin_sum(const FinArgs& a, int v, double* scratch) {
  double s = 0.0;
  for (long long t = a.tile0[v] + linear_tid(); t < a.tile0[v + 1]; t += NT) s += a.part[t];
  return block_sum(s, scratch);
}

// After the update: body x, r; r.r; the inner stopping test.
__global__ void __launch_bounds__(NT) k_mg_finA(FinArgs a) {
  __shared__ double scratch[NT / 32 + 1];
  const int v = blockIdx.x;
  VarState* S = &a.st[v];
  if (S->phase != PH_CG) return;
  const double rr_free = fin_sum(a, v, scratch);
  if (linear_tid() != 0) return;
  const DevVariant& V = a.m.var[v];
  const int B = a.B;
  const float alpha = (float)S->alpha;
  double rr = rr_free;
  if (!a.prm->fixed_bodies) {
    for (int k = 0; k < V.nb; ++k) {
      const int gb = V.body0 + k;
      a.sb[gb] = a.sb[gb] + alpha * a.sb[2 * B + gb];
      const float rb = a.sb[B + gb] - alpha * a.sb[3 * B + gb];
      a.sb[B + gb] = rb;
      rr += (double)rb * (double)rb;
      a.yb[gb] = a.Abb[gb] > 0.0 ? (float)(rb / a.Abb[gb]) : 0.0f;   // forward body step
    }
  } else {
    for (int k = 0; k < V.nb; ++k) a.yb[V.body0 + k] = 0.0f;   // body values are data
  }
  if (S->inner_iters == 0) S->gamma_start = rr;
  S->gamma = rr;
  if (!isfinite(rr)) {
    S->status = PF_EBREAKDOWN;
    S->phase = PH_DONE;
    atomicAdd(a.n_done, 1);
  } else if (rr <= fmax(S->thr_rel * S->gamma_start, S->thr_abs2)) {
    S->phase = PH_RESID;
  } else if (S->iters >= a.prm->k_max) {
    S->capped = 1;
    S->phase = PH_RESID;
  }
}

// After the cycle: the backward body step z_b = (r_b - A_bf z_f) / A_bb, with A_bf z_f
// the sum over the free nodes next to the body of c times the cycle's result there; r.z;
// beta; the body's new search direction.  With the forward step y_b = r_b / A_bb and the
// cycle applied to r_f - A_fb y_b, the preconditioner is
//   [I, 0; -D^-1 A_bf, I] [B, 0; 0, D^-1] [I, -A_fb D^-1; 0, I]   (D = diag of A_bb,
// B the V-cycle): symmetric positive definite, a block Gauss-Seidel sweep body, free, body.
__global__ void __launch_bounds__(NT) k_mg_finB(FinArgs a) {
  __shared__ double scratch[NT / 32 + 1];
  __shared__ double sz[MAXB];
  const int v = blockIdx.x;
  VarState* S = &a.st[v];
  if (S->phase != PH_CG) return;
  const double rz_free = fin_sum(a, v, scratch);
  const DevVariant& V = a.m.var[v];
  const int nbu = a.prm->fixed_bodies ? 0 : V.nb;
  for (int k = 0; k < nbu; ++k) {
    const int gb = V.body0 + k;
    double s = 0.0;
    for (int e = a.adj_ptr[gb] + linear_tid(); e < a.adj_ptr[gb + 1]; e += NT)
      s += (double)a.adj_c[e] * (double)a.t[a.adj_n[e]];
    s = block_sum(s, scratch);
    if (linear_tid() == 0) sz[k] = s;
  }
  if (linear_tid() != 0) return;
  const int B = a.B;
  double rz = rz_free;
  float zb[MAXB];
  for (int k = 0; k < nbu; ++k) {
    const int gb = V.body0 + k;
    const float rb = a.sb[B + gb];
    zb[k] = a.Abb[gb] > 0.0 ? (float)((rb - sz[k]) / a.Abb[gb]) : 0.0f;
    rz += (double)rb * (double)zb[k];
  }
  const double beta = S->inner_iters == 0 ? 0.0 : rz / S->rho;
  S->beta = beta;
  S->rho = rz;
  for (int k = 0; k < nbu; ++k) {
    const int gb = V.body0 + k;
    a.sb[2 * B + gb] = zb[k] + (float)beta * a.sb[2 * B + gb];
  }
}

// After the apply: collapsed body rows of q; p.q; alpha; iteration count; buffer flip.
__global__ void __launch_bounds__(NT) k_mg_finC(FinArgs a) {
  __shared__ double scratch[NT / 32 + 1];
  __shared__ double sq[MAXB];
  const int v = blockIdx.x;
  VarState* S = &a.st[v];
  if (S->phase != PH_CG) return;
  const double pq_free = fin_sum(a, v, scratch);
  const DevVariant& V = a.m.var[v];
  const int nbu = a.prm->fixed_bodies ? 0 : V.nb;
  for (int k = 0; k < nbu; ++k) {
    double s = 0.0;
    const int gb = V.body0 + k;
    for (int e = a.m.body_ptr[gb] + linear_tid(); e < a.m.body_ptr[gb + 1]; e += NT)
      s += (double)a.q[a.m.body_nodes[e]];
    s = block_sum(s, scratch);
    if (linear_tid() == 0) sq[k] = s;
  }
  if (linear_tid() != 0) return;
  const int B = a.B;
  double pq = pq_free;
  for (int k = 0; k < nbu; ++k) {
    const int gb = V.body0 + k;
    const float qb = (float)sq[k];
    a.sb[3 * B + gb] = qb;
    pq += (double)a.sb[2 * B + gb] * (double)qb;
  }
  S->pi = pq;
  S->iters += 1;
  S->inner_iters += 1;
  S->buf ^= 1;
  if (!isfinite(pq) || !(pq > 0.0)) {
    if (S->gamma == 0.0) {
      S->alpha = 0.0;
      S->phase = PH_RESID;
    } else {
      S->status = PF_EBREAKDOWN;
      S->phase = PH_DONE;
      atomicAdd(a.n_done, 1);
    }
    return;
  }
  S->alpha = S->rho / pq;
}

LvArgs lv_args(MgLevel& L) {
  LvArgs c;
  c.off = L.d_off;
  c.dims = L.d_dims;
  c.blkvar = L.d_blkvar;
  c.n = L.n;
  c.act = L.act;
  c.A = L.A32;
  c.dinv = L.dinv;
  c.r = L.r;
  c.za = L.za;
  c.zb = L.zb;
  c.res = L.res;
  return c;
}

MeshDev mesh_view(const Batch& b) {
  MeshDev m;
  m.var = b.d_var;
  m.tag = b.tag;
  m.bid = b.bid;
  m.body_ptr = b.body_ptr;
  m.body_nodes = b.body_nodes;
  m.K64 = b.K64;
  m.K32 = b.K32;
  m.Vtot = b.Vtot;
  return m;
}

}  // namespace

// The operators of the hierarchy depend on the node coordinates: after they change, the
// next preconditioned solve forms them again (the level layout and arrays are kept).
void destroy_mg(Batch& b) { b.mg_ready = false; }

static void mg_layout(Batch& b);

// The hierarchy: per-variant level counts, packed coarse levels, Galerkin operators,
// Jacobi factors, the body diagonals and the FP32 vector planes of the fine level.
void mg_setup(Batch& b) {
  if (b.mg_ready) return;
  if (b.nv > 0 && b.Vtot > 0 && !b.mg_x) {
    const size_t V = (size_t)b.Vtot * sizeof(float);
    float** planes[] = {&b.mg_x, &b.mg_r, &b.mg_z, &b.mg_t, &b.mg_res, &b.mg_p[0], &b.mg_p[1], &b.mg_q, &b.mg_dinv0};
    for (float** pl : planes) {
      *pl = (float*)dev_alloc(b, V);
      PF_CUDA(cudaMemsetAsync(*pl, 0, V, b.stream));
    }
    b.mg_part = (double*)dev_alloc(b, std::max<long long>(1, b.Tcg) * sizeof(double));
    b.mg_Abb = (double*)dev_alloc(b, std::max(1, b.B) * sizeof(double));
    b.mg_yb = (float*)dev_alloc(b, std::max(1, b.B) * sizeof(float));
    PF_CUDA(cudaMemsetAsync(b.mg_yb, 0, std::max(1, b.B) * sizeof(float), b.stream));
    // the fine-level kernels run on the fused-CG tiles (64 x 16), variant-major
    std::vector<long long> t0(b.nv + 1, 0);
    for (int v = 0; v < b.nv; ++v)
      t0[v + 1] = t0[v] + (long long)((b.hv[v].g.nx + 1 + CTX - 1) / CTX) * ((b.hv[v].g.ny + 1 + CTY - 1) / CTY);
    b.d_tile0 = (long long*)dev_alloc(b, (b.nv + 1) * sizeof(long long));
    PF_CUDA(cudaMemcpyAsync(b.d_tile0, t0.data(), (b.nv + 1) * sizeof(long long), cudaMemcpyHostToDevice, b.stream));
  }
  if (b.mg.empty()) mg_layout(b);
  const int L = b.mg_L;
  const MeshDev m = mesh_view(b);
  cudaStream_t s = b.stream;
  k_mg_dinv0<<<(unsigned)b.T, dim3(TX, TY), 0, s>>>(m, b.tile_var, b.tile_ij, b.mg_dinv0);
  if (b.B > 0) {
    k_mg_body_diag<<<b.B, dim3(TX, TY), 0, s>>>(m, b.d_body_var, b.mg_Abb);
    if (!b.mg_adj_ptr) {   // the lists depend on the topology only: counted once per handle
      int* cnt = (int*)dev_alloc(b, b.B * sizeof(int));
      k_mg_adj<<<b.B, dim3(TX, TY), 0, s>>>(m, b.d_body_var, b.d_bbox, cnt, nullptr, nullptr, nullptr, 0);
      std::vector<int> h(b.B), ptr(b.B + 1, 0);
      PF_CUDA(cudaMemcpyAsync(h.data(), cnt, b.B * sizeof(int), cudaMemcpyDeviceToHost, s));
      PF_CUDA(cudaStreamSynchronize(s));
      for (int k = 0; k < b.B; ++k) ptr[k + 1] = ptr[k] + h[k];
      b.mg_adj_ptr = (int*)dev_alloc(b, (b.B + 1) * sizeof(int));
      PF_CUDA(cudaMemcpyAsync(b.mg_adj_ptr, ptr.data(), (b.B + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
      b.mg_adj_node = (long long*)dev_alloc(b, std::max(1, ptr[b.B]) * sizeof(long long));
      b.mg_adj_c = (float*)dev_alloc(b, std::max(1, ptr[b.B]) * sizeof(float));
      PF_CUDA(cudaStreamSynchronize(s));
    }
    // the couplings follow the coordinates (recomputed with the hierarchy)
    k_mg_adj<<<b.B, dim3(TX, TY), 0, s>>>(m, b.d_body_var, b.d_bbox, nullptr, b.mg_adj_ptr, b.mg_adj_node,
                                          b.mg_adj_c, 1);
  }
  for (int l = 1; l < L; ++l) {
    MgLevel& M = b.mg[l];
    if (M.nblk == 0) continue;
    const LvArgs c = lv_args(M);
    const bool f0 = l == 1;
    MgLevel& F = b.mg[l - 1];
    k_mg_act<<<(unsigned)M.nblk, 256, 0, s>>>(c, f0 ? nullptr : F.act, f0 ? nullptr : F.d_off,
                                               f0 ? nullptr : F.d_dims, b.d_var, b.tag, M.act);
    k_mg_rap<<<(unsigned)M.nblk, 256, 0, s>>>(c, M.A32, M.dinv, m, f0 ? nullptr : F.act, f0 ? nullptr : F.A32,
                                               f0 ? nullptr : F.d_off, f0 ? nullptr : F.d_dims, f0 ? 0 : F.n);
  }
  PF_CUDA(cudaGetLastError());
  b.launches += 1 + (b.B > 0 ? 1 : 0) + 2 * (L - 1);
  b.mg_ready = true;
}

// Level counts and the packed layout of every coarse level, allocated once per handle.
static void mg_layout(Batch& b) {
  // levels per variant: coarsen while a level has more than MG_CMAX cells in a direction
  b.mg_Lv.assign(b.nv, 1);
  std::vector<std::vector<int2>> dims(b.nv);
  int L = 1;
  for (int v = 0; v < b.nv; ++v) {
    int nx = b.hv[v].g.nx, ny = b.hv[v].g.ny;
    dims[v].push_back(make_int2(nx, ny));
    do {
      nx = (nx + 1) / 2;
      ny = (ny + 1) / 2;
      dims[v].push_back(make_int2(nx, ny));
    } while (std::max(nx, ny) > MG_CMAX);
    b.mg_Lv[v] = (int)dims[v].size();
    L = std::max(L, b.mg_Lv[v]);
  }
  if (L > 16) throw Error{PF_EINVAL, "grid too large for the multigrid hierarchy"};
  b.mg_L = L;
  if (!b.d_mg_Lv) b.d_mg_Lv = (int*)dev_alloc(b, b.nv * sizeof(int));
  PF_CUDA(cudaMemcpyAsync(b.d_mg_Lv, b.mg_Lv.data(), b.nv * sizeof(int), cudaMemcpyHostToDevice, b.stream));
  b.mg.assign(L, MgLevel());
  for (int l = 1; l < L; ++l) {
    MgLevel& M = b.mg[l];
    M.off.assign(b.nv, -1);
    M.dims.assign(b.nv, make_int2(0, 0));
    long long o = 0;
    std::vector<int> blkvar;
    for (int v = 0; v < b.nv; ++v) {
      if (l >= b.mg_Lv[v]) continue;
      const int2 d = dims[v][l];
      const long long nn = (long long)(d.x + 1) * (d.y + 1);
      const long long nb = (nn + 255) / 256;
      M.off[v] = o;
      M.dims[v] = d;
      for (long long k = 0; k < nb; ++k) blkvar.push_back(v);
      o += nb * 256;
    }
    M.n = std::max<long long>(o, 256);
    M.nblk = (long long)blkvar.size();
    if (blkvar.empty()) blkvar.push_back(-1);
    M.d_off = (long long*)dev_alloc(b, b.nv * sizeof(long long));
    M.d_dims = (int2*)dev_alloc(b, b.nv * sizeof(int2));
    M.d_blkvar = (int*)dev_alloc(b, blkvar.size() * sizeof(int));
    PF_CUDA(cudaMemcpyAsync(M.d_off, M.off.data(), b.nv * sizeof(long long), cudaMemcpyHostToDevice, b.stream));
    PF_CUDA(cudaMemcpyAsync(M.d_dims, M.dims.data(), b.nv * sizeof(int2), cudaMemcpyHostToDevice, b.stream));
    PF_CUDA(cudaMemcpyAsync(M.d_blkvar, blkvar.data(), blkvar.size() * sizeof(int), cudaMemcpyHostToDevice,
                            b.stream));
    M.act = (uint8_t*)dev_alloc(b, M.n);
    M.A32 = (float*)dev_alloc(b, 9 * M.n * sizeof(float));
    M.dinv = (float*)dev_alloc(b, M.n * sizeof(float));
    M.r = (float*)dev_alloc(b, M.n * sizeof(float));
    M.za = (float*)dev_alloc(b, M.n * sizeof(float));
    M.zb = (float*)dev_alloc(b, M.n * sizeof(float));
    M.res = (float*)dev_alloc(b, M.n * sizeof(float));
    PF_CUDA(cudaMemsetAsync(M.act, 0, M.n, b.stream));
    for (float* f : {M.r, M.za, M.zb, M.res, M.dinv}) PF_CUDA(cudaMemsetAsync(f, 0, M.n * sizeof(float), b.stream));
    PF_CUDA(cudaMemsetAsync(M.A32, 0, 9 * M.n * sizeof(float), b.stream));
  }
}

// `iters` preconditioned CG iterations for every variant in the CG phase (captured as a
// graph by the solve loop).
void launch_pcg_chunk(Batch& b, int iters, cudaStream_t s) {
  FineArgs a;
  a.m = mesh_view(b);
  a.tile_var = b.tile_cg_var;
  a.tile_ij = b.tile_cg_ij;
  a.st = b.state;
  a.dinv0 = b.mg_dinv0;
  a.x = b.mg_x;
  a.r = b.mg_r;
  a.z = b.mg_z;
  a.t = b.mg_t;
  a.res = b.mg_res;
  a.q = b.mg_q;
  a.p[0] = b.mg_p[0];
  a.p[1] = b.mg_p[1];
  a.sb = b.sb32;
  a.yb = b.mg_yb;
  a.B = std::max(1, b.B);
  a.part = b.mg_part;
  a.c_off = b.mg[1].d_off;
  a.c_dims = b.mg[1].d_dims;
  a.c_zb = b.mg[1].zb;
  FinArgs f;
  f.st = b.state;
  f.prm = b.params;
  f.tile0 = b.d_tile0;
  f.part = b.mg_part;
  f.m = a.m;
  f.sb = b.sb32;
  f.Abb = b.mg_Abb;
  f.q = b.mg_q;
  f.yb = b.mg_yb;
  f.t = b.mg_t;
  f.adj_ptr = b.mg_adj_ptr;
  f.adj_n = b.mg_adj_node;
  f.adj_c = b.mg_adj_c;
  f.B = std::max(1, b.B);
  f.n_done = b.n_done;
  CoarseTab ct;
  std::memset(&ct, 0, sizeof(ct));
  for (int l = 1; l < b.mg_L; ++l) ct.lv[l] = lv_args(b.mg[l]);
  const unsigned T = (unsigned)b.Tcg, nv = (unsigned)b.nv;
  const dim3 blk(TX, TY);
  const int L = b.mg_L;
  for (int it = 0; it < iters; ++it) {
    k_mg0_update<<<T, blk, 0, s>>>(a);
    k_mg_finA<<<nv, blk, 0, s>>>(f);
    // descent: the forward body step's term of the pre-sweep (z), the residual r - A z,
    // restriction to level 1 (which also runs the level's pre-sweep from zero)
    if (b.B > 0) k_mg_fwd<<<nv, blk, 0, s>>>(a, b.mg_adj_ptr, b.mg_adj_node, b.mg_adj_c);
    k_mg0_sweep<1, false><<<T, blk, 0, s>>>(a, b.mg_z, b.mg_res);
    for (int l = 1; l < L; ++l) {
      MgLevel& M = b.mg[l];
      if (M.nblk == 0) continue;
      const LvArgs c = lv_args(M);
      if (l == 1) {
        k_mg_restrict<<<(unsigned)M.nblk, 256, 0, s>>>(c, l, b.d_mg_Lv, b.state, b.d_var, b.mg_res, nullptr, nullptr);
      } else {
        MgLevel& F = b.mg[l - 1];
        k_mg_restrict<<<(unsigned)M.nblk, 256, 0, s>>>(c, l, b.d_mg_Lv, b.state, b.d_var, F.res, F.d_off, F.d_dims);
      }
      // the level's residual after its pre-sweep (variants whose coarsest level this is
      // skip: the coarse solve below takes their restricted residual)
      k_mg_sweep<1><<<(unsigned)M.nblk, 256, 0, s>>>(c, l, b.d_mg_Lv, b.state, M.za, M.res);
    }
    k_mg_coarse<<<nv, 256, 0, s>>>(ct, b.d_mg_Lv, b.state);
    // ascent
    for (int l = L - 2; l >= 1; --l) {
      MgLevel& M = b.mg[l];
      if (M.nblk == 0) continue;
      const LvArgs c = lv_args(M);
      k_mg_prolong<<<(unsigned)M.nblk, 256, 0, s>>>(c, lv_args(b.mg[l + 1]), l, b.d_mg_Lv, b.state);
      k_mg_sweep<0><<<(unsigned)M.nblk, 256, 0, s>>>(c, l, b.d_mg_Lv, b.state, M.za, M.zb);
    }
    // post-smoothing of level 0: one sweep on z + P e (the correction from level 1), r.t
    k_mg0_sweep<2, true><<<T, blk, 0, s>>>(a, b.mg_z, b.mg_t);
    k_mg_finB<<<nv, blk, 0, s>>>(f);
    k_mg0_apply<<<T, blk, 0, s>>>(a);
    k_mg_finC<<<nv, blk, 0, s>>>(f);
  }
  PF_CUDA(cudaGetLastError());
}

}  // namespace pfq4
