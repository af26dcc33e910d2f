// Matrix-free multi-point-constraint Conjugate Gradient (Appendix A, Algorithm) on
// GB300, for one or many mesh variants at once.
//
// Per CG iteration one fused, persistent kernel (k_cg) does, for every tile of every
// unconverged variant:
//     r_k = r_{k-1} - alpha_{k-1} q_{k-1}        (residual update)
//     x_k = x_{k-1} + alpha_{k-1} p_{k-1}        (solution update)
//     p_k = r_k + beta_{k-1} p_{k-1}             (search direction, also on the halo)
//     q_k = A p_k                                (matrix-free Q4 apply, "Compute Ap")
// plus the four dot products r.r, p.q, r.q, q.q.  The body unknowns follow the
// paper's collapse / expand: q at the nodes of body k is summed into one body row
// (collapse) and the body's single search-direction value is used at all of its
// nodes (expand).  The last CTA to finish a variant reduces the per-segment partial
// sums in a fixed order and forms alpha_k = r.r / p.q and
// beta_k = |r_{k+1}|^2 / |r_k|^2 with |r_{k+1}|^2 = r.r - 2 alpha r.q + alpha^2 q.q, so a
// single grid-wide reduction per iteration suffices.  Dirichlet and inactive nodes
// keep zero search directions (constraint enforcement after every update).
//
// The CG runs on a correction: the state of a node is one record (x, r, p, q) of the
// working precision, double-buffered by parity (a launch reads one parity with its
// halo and writes the other), so a tile is one TMA box and one 16- or 32-byte store
// per node.  k_fold adds the correction x into the FP64 solution x64 and k_resid forms
// the true FP64 residual b - A x64 (Dirichlet values sit in x64, so the lifting is part
// of the same apply) and restarts the CG from it: iterative refinement, with an FP32
// inner solver in mixed precision and an FP64 one in FP64 mode.  All kernels read
// their per-variant phase from device memory, so the host launches a captured graph
// of k_cg launches followed by [k_fold, k_resid] until every variant is done.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>

#include "batch.h"
#include "tma.cuh"

namespace pfq4 {

template <typename T>
struct CGArgs {
  MeshDev m;
  Sched sc;
  VarState* st;
  const SolveParams* prm;
  State4<T>* s[2];          // ping-pong state, parity VarState::buf holds the current one
  T* sb;                    // [4][B] body x, r, p, q of the CG
  double* bq;               // [body nodes] q at each BODY node (slot order of body_nodes)
  int B;
  int* n_done;
  const uint8_t* tile_gen;  // per fused-CG tile: stored coefficients needed
  long long Rtot;           // rows of the batch's 2-D node arrays
  int* err;                 // set to 1 if a bounded wait gave up
  int poll_limit;           // polls of one mbarrier wait before it gives up
  int test_drop;            // test hook: CTA 0 never issues the copies of its first tile
};

// The refinement kernels (k_fold, k_resid) run on a (gx, variants) grid: row v handles
// variant v, its 32x8 tiles cut into gx contiguous shares, one per CTA.  A variant that
// refines is spread over gx CTAs however many variants the batch holds (a contiguous
// schedule over the whole tile list left a refining variant of a large batch on a few
// SMs), and the rows of variants that do not refine exit after one load.
template <typename T>
struct ResidArgs {
  MeshDev m;
  int gx;                   // CTAs per variant
  double* rpart;            // [variants][gx] partial sums of r.r, fixed order
  int* counter;             // [variants] CTAs of the row done in this launch
  VarState* st;
  const SolveParams* prm;
  double* x64;              // solution, Dirichlet values in place (read only here)
  double* w64;              // body-node rows of A u
  State4<T>* s[2];          // CG state to restart, in the current parity
  double* sol;              // [B] body solution values
  T* sb;                    // [4][B] CG body values
  double* sbr;              // [B] true residual body rows
  const double* rhsb;       // [B] extra right-hand side on the body rows (adjoint), or NULL
  int B;
  int mixed;
  int* n_done;
  float* rplane;            // preconditioned CG: the restarted residual goes to this FP32 plane
};

template <typename T> __device__ __forceinline__ const T* kplane(const MeshDev& m);
template <> __device__ __forceinline__ const double* kplane<double>(const MeshDev& m) { return m.K64; }
template <> __device__ __forceinline__ const float* kplane<float>(const MeshDev& m) { return m.K32; }
template <typename T> __device__ __forceinline__ const T* krect(const DevVariant& V);
template <> __device__ __forceinline__ const double* krect<double>(const DevVariant& V) { return V.kr64; }
template <> __device__ __forceinline__ const float* krect<float>(const DevVariant& V) { return V.kr32; }

// The CG vector recurrences, shared by tile owners, halo readers and the body
// finaliser so that every copy of a value is bit-identical.
template <typename T>
__device__ __forceinline__ T next_r(T r, T q, T alpha) { return r - alpha * q; }
template <typename T>
__device__ __forceinline__ T next_p(T rn, T p, T beta) { return rn + beta * p; }
template <typename T>
__device__ __forceinline__ T next_x(T x, T p, T alpha) { return x + alpha * p; }

__device__ __forceinline__ int seg_count(const Sched& sc, int v) { return sc.var_seg1[v] - sc.var_seg0[v]; }

// Sum of a node vector over the nodes of one body (fixed order), all threads get it.
template <typename T>
__device__ double body_gather(const MeshDev& m, int gb, const T* vec, double* scratch) {
  double s = 0.0;
  const int e1 = m.body_ptr[gb + 1];
  for (int e = m.body_ptr[gb] + linear_tid(); e < e1; e += NT) s += (double)__ldcg(vec + m.body_nodes[e]);
  return block_sum(s, scratch);
}

// ---------------------------------------------------------------- fused CG step
__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Shared-memory doubles the finaliser stages per pass (fixed, so that the summation
// order does not depend on the pipeline depth).
constexpr int FIN_CAP = 8192;

// What the end of an iteration needs from global memory, loaded by the consumer warps
// at the start of each segment so that the serial finaliser issues no dependent loads.
template <typename T>
struct FinCache {
  T sb[4][MAXB];             // body x, r, p, q before this iteration
  int bptr[MAXB + 1];        // body_ptr of the variant's bodies (global slots)
  double alpha, beta, gamma_start, thr_rel, thr_abs2;
  long long iters, inner_iters, k_max;
  int seg0, seg1, buf, fixed; // seg0/seg1: the variant's segments
};

// A BODY node has no x, r or p of its own (its value is the body's unknown), so the x
// field of its state record carries the node's position in body_nodes (its slot), as
// raw bits: the fused CG step then finds the node's body and stores its row of A p by
// slot with no extra memory access.
__device__ __forceinline__ float slot_bits(int e, float) { return __int_as_float(e); }
__device__ __forceinline__ double slot_bits(int e, double) { return __longlong_as_double((long long)e); }
__device__ __forceinline__ int slot_of(float x) { return __float_as_int(x); }
__device__ __forceinline__ int slot_of(double x) { return (int)__double_as_longlong(x); }

// Local index of the body whose slot range [bptr[k], bptr[k+1]) holds slot e.
__device__ __forceinline__ int body_of_slot(const int* bptr, int nb, int e) {
  int lo = 0, hi = nb;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (bptr[mid] <= e) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Runs in the last CTA of variant v to finish an iteration (all NTHR threads of the
// CTA); gbuf is the CTA's stage memory (at least FIN_CAP doubles), which no copy is
// writing once the CTA's tiles are consumed.
template <typename T, int NTHR>
__device__ __noinline__ void finalize_cg(const CGArgs<T>& a, int v, int nb, int body0, const FinCache<T>& fc, double* scratch,
                            double* sh_qb, double* gbuf) {
  VarState* S = &a.st[v];
  const int tid = linear_tid(), warp = tid >> 5, lane = tid & 31;
  constexpr int NW = NTHR / 32;
  static_assert(NW >= 5, "finaliser needs warps 0-3 for the dots and at least one body warp");
  constexpr int GB = 8;                      // independent loads in flight per thread
  constexpr int HALF = FIN_CAP / 2;          // doubles per staging region
  double* d = scratch;                       // d[0..3]: the four dots over FREE nodes
  double* gp = gbuf;                         // staged segment partials [HALF]
  double* gq = gbuf + HALF;                  // staged body-node rows of A p [HALF]
  // Both sums are staged through shared memory in passes of fixed size (independent
  // loads, one round trip per pass) and added in a fixed order: warps 0-3 take dot k =
  // warp over the variant's segment partials in segment order; warps 4.. take the
  // collapsed body rows of A p (stored by slot during the iteration), one warp per body.
  const int nparts = (fc.seg1 - fc.seg0) * 4;
  const int e0 = fc.bptr[0], nq = fc.bptr[nb] - e0;
  for (int k = tid; k < nb; k += NTHR) sh_qb[k] = 0.0;
  double dsum = 0.0;
  for (int off = 0; off < max(nparts, nq); off += HALF) {
    const int np = min(HALF, nparts - off), nqq = min(HALF, nq - off);
    for (int b = 0; b < max(np, nqq); b += GB * NTHR) {
      double vp[GB], vq[GB];
#pragma unroll
      for (int u = 0; u < GB; ++u) {
        const int e = b + u * NTHR + tid;
        vp[u] = e < np ? __ldcg(&a.sc.partial[fc.seg0 * 4 + off + e]) : 0.0;
        vq[u] = e < nqq ? __ldcg(&a.bq[e0 + off + e]) : 0.0;
      }
#pragma unroll
      for (int u = 0; u < GB; ++u) {
        const int e = b + u * NTHR + tid;
        if (e < np) gp[e] = vp[u];
        if (e < nqq) gq[e] = vq[u];
      }
    }
    __syncthreads();
    if (warp < 4) {
      for (int j = lane; j < np / 4; j += 32) dsum += gp[j * 4 + warp];
    } else {
      for (int k = warp - 4; k < nb; k += NW - 4) {
        const int b0 = max(off, fc.bptr[k] - e0), b1 = min(off + nqq, fc.bptr[k + 1] - e0);
        double sq = 0.0;
        for (int e = b0 + lane; e < b1; e += 32) sq += gq[e - off];
        sq = warp_sum(sq);
        if (lane == 0) sh_qb[k] += sq;
      }
    }
    __syncthreads();
  }
  if (warp < 4) {
    dsum = warp_sum(dsum);
    if (lane == 0) d[warp] = dsum;
  }
  __syncthreads();
  // body unknowns, one thread per body; their dot contributions are added in body order
  double* contrib = gbuf;                    // [4][MAXB]
  const T alpha = (T)fc.alpha, beta = (T)fc.beta;
  const int nbu = fc.fixed ? 0 : nb;
  const int B = a.B;
  for (int k = tid; k < nbu; k += NTHR) {
    const int gb = body0 + k;
    const T pb = fc.sb[2][k];
    const T rn = next_r(fc.sb[1][k], fc.sb[3][k], alpha);
    const T pn = next_p(rn, pb, beta);
    const T xn = next_x(fc.sb[0][k], pb, alpha);
    const T qn = (T)sh_qb[k];
    a.sb[gb] = xn;
    a.sb[B + gb] = rn;
    a.sb[2 * B + gb] = pn;
    a.sb[3 * B + gb] = qn;
    contrib[k] = (double)rn * (double)rn;
    contrib[MAXB + k] = (double)pn * (double)qn;
    contrib[2 * MAXB + k] = (double)rn * (double)qn;
    contrib[3 * MAXB + k] = (double)qn * (double)qn;
  }
  __syncthreads();
  if (tid == 0) {
    double dd[4] = {d[0], d[1], d[2], d[3]};
    for (int k = 0; k < nbu; ++k)
      for (int j = 0; j < 4; ++j) dd[j] += contrib[j * MAXB + k];
    const double g = dd[0], pi = dd[1], rho = dd[2], mu = dd[3];
    const long long iters = fc.iters + 1, inner = fc.inner_iters + 1;
    const double gs = inner == 1 ? g : fc.gamma_start;
    S->buf = fc.buf ^ 1;
    S->iters = iters;
    S->inner_iters = inner;
    if (inner == 1) S->gamma_start = g;
    S->gamma = g; S->pi = pi; S->rho = rho; S->mu = mu;
    if (!isfinite(g) || !isfinite(pi) || !(pi > 0.0)) {
      if (g == 0.0) {
        S->phase = PH_RESID;
      } else {
        S->status = PF_EBREAKDOWN;
        S->phase = PH_DONE;
        atomicAdd(a.n_done, 1);
      }
    } else if (g <= fmax(fc.thr_rel * gs, fc.thr_abs2)) {
      S->phase = PH_RESID;
    } else if (iters >= fc.k_max) {
      S->capped = 1;
      S->phase = PH_RESID;
    } else {
      const double al = g / pi;
      const double gn = g - 2.0 * al * rho + al * al * mu;
      S->alpha = al;
      S->beta = gn > 0.0 ? gn / g : 0.0;
    }
    a.sc.counter[v] = 0;
  }
}

// Shared-memory layout of one pipeline stage of k_cg (T = float or double).  Tiles are
// CTX x CTY nodes.  The state box covers nodes i0-1 .. i0+CTX and rows j0-1 .. j0+CTY
// (records of 4 values); tags cover i0-16 .. i0+CTX+15; the six element-coefficient
// planes (FP32 only) cover cells i0-4 .. i0+CTX-1, rows j0-1 .. j0+CTY-1.
template <typename T, int NS = 2>
struct CgSmem {
  static constexpr int SBW = CTX + 2;            // state box width (nodes)
  static constexpr int KBW = CTX + 4;            // coefficient box width (cells i0-4 .. i0+CTX-1)
  static constexpr int KHALF = KBW / 2;          // cells per coefficient box (two boxes of 6*KHALF floats)
  static constexpr int TBW = CTX + 32;           // tag box width
  static constexpr int SB = 4 * SBW * (CTY + 2); // elements of the state box
  static constexpr int SHALF = SBW / 2;          // nodes per state box (two boxes of 4*SHALF values per row)
  static constexpr int sbox_bytes = ((CTY + 2) * 4 * SHALF * (int)sizeof(T) + 127) / 128 * 128;
  static constexpr int sbox_recs = sbox_bytes / (4 * (int)sizeof(T));
  static constexpr int KB = KBW * (CTY + 1);     // elements of one coefficient plane box
  static constexpr bool kTmaK = sizeof(T) == 4;
  static constexpr int align(int b) { return (b + 127) / 128 * 128; }
  static constexpr int off_s = 0;
  static constexpr int off_t = off_s + 2 * sbox_bytes;
  static constexpr int off_k = off_t + align(TBW * (CTY + 2));
  // two coefficient boxes, each starting on a 128-byte boundary (TMA destination alignment)
  static constexpr int kbox_bytes = align((CTY + 1) * 6 * KHALF * (int)sizeof(T));
  static constexpr int stage_bytes = off_k + (kTmaK ? 2 * kbox_bytes : 0);
  static constexpr int tx_tag = TBW * (CTY + 2);
  static constexpr int tx_base = SB * (int)sizeof(T) + tx_tag;
  static constexpr int tx_k = kTmaK ? 6 * KB * (int)sizeof(T) : 0;
  // edge tiles: a tile whose last grid row is at most THIN - 2 rows below its first loads
  // boxes of THIN rows only (state and tags rows j0-1 .. j0+2, coefficient cell rows
  // j0-1 .. j0+2); a tile whose grid ends within its first state box loads that box alone
  static constexpr int THIN = 4;
  __host__ __device__ static constexpr int tx_sbox(bool thin) { return (thin ? THIN : CTY + 2) * 4 * SHALF * (int)sizeof(T); }
  __host__ __device__ static constexpr int tx_tbox(bool thin) { return TBW * (thin ? THIN : CTY + 2); }
  __host__ __device__ static constexpr int tx_kbox(bool thin) { return kTmaK ? (thin ? THIN : CTY + 1) * 6 * KHALF * (int)sizeof(T) : 0; }
  static_assert(2 * tx_sbox(false) == SB * (int)sizeof(T) && 2 * tx_kbox(false) == tx_k, "box byte counts");
  // after the NS stages: two p tiles with halo, two effective-tag tiles, barriers
  static constexpr int ptile_bytes = align((CTX + 2) * (CTY + 2) * (int)sizeof(T));
  static constexpr int ttile_bytes = align((CTX + 2) * (CTY + 2));
  static constexpr int off_ptile = NS * stage_bytes;
  static constexpr int off_ttile = off_ptile + 2 * ptile_bytes;
  static constexpr int off_bar = off_ttile + 2 * ttile_bytes;
  static constexpr int total = off_bar + 2 * NS * 8;
  static_assert(off_s % 128 == 0 && off_t % 128 == 0 && off_k % 128 == 0 && kbox_bytes % 128 == 0 &&
                    sbox_bytes % 128 == 0 && SBW % 2 == 0 &&
                    stage_bytes % 128 == 0,
                "TMA destinations must start on 128-byte boundaries");
};

// Row of the operator at a node whose four cells are active rectangles with the
// closed-form constants kr: K23 = K01, K12 = K03, K13 = K02, so the row is
// 2 K01 (dE + dW) + 2 K03 (dN + dS) + K02 (sum of the diagonal differences).
template <typename T>
__device__ __forceinline__ T q4_row_rect(const T (&p)[3][3], const T* kr) {
  const T pc = p[1][1];
  const T dE = p[1][2] - pc, dW = p[1][0] - pc, dN = p[2][1] - pc, dS = p[0][1] - pc;
  const T dNE = p[2][2] - pc, dNW = p[2][0] - pc, dSE = p[0][2] - pc, dSW = p[0][0] - pc;
  return T(2) * kr[0] * (dE + dW) + T(2) * kr[2] * (dN + dS) + kr[1] * ((dNE + dSW) + (dNW + dSE));
}

// Row of the operator at one node from its 3x3 neighbourhood p[3][3] (p[1][1] = the
// node, first index = row j-1, j, j+1, second = column i-1, i, i+1) and the tags of its
// four cells: c0 = (i, j), c1 = (i-1, j), c2 = (i-1, j-1), c3 = (i, j-1).  Displaced
// cells read their six coefficients from the staged boxes (STAGED: the fused kernel's
// FP32 path) or from the global planes; undisplaced cells use the closed-form rectangle
// constants kr.  HOIST (global planes only): issue all of a node's coefficient loads
// before the first use, at the cost of 12 more live registers.
template <typename T, bool STAGED = sizeof(T) == 4, bool HOIST = false>
__device__ __forceinline__ T q4_row_nb(const T (&p)[3][3], uint8_t c0, uint8_t c1, uint8_t c2, uint8_t c3,
                                       const T* ks, int kcol, int krow, long long n, int P,
                                       const T* __restrict__ Kg, long long plane, const T* kr) {
  using L = CgSmem<T>;
  const T pc = p[1][1];
  const T dE = p[1][2] - pc, dW = p[1][0] - pc, dN = p[2][1] - pc, dS = p[0][1] - pc;
  const T dNE = p[2][2] - pc, dNW = p[2][0] - pc, dSE = p[0][2] - pc, dSW = p[0][0] - pc;
  constexpr uint8_t GEN = sizeof(T) == 4 ? CELL_GEN32 : CELL_GENERAL;   // cells that need stored K_e
  constexpr uint8_t FLAGS = CELL_ACTIVE | GEN;
  if ((c0 & FLAGS) == CELL_ACTIVE && (c1 & FLAGS) == CELL_ACTIVE && (c2 & FLAGS) == CELL_ACTIVE &&
      (c3 & FLAGS) == CELL_ACTIVE)
    return q4_row_rect<T>(p, kr);
  if constexpr (!STAGED && HOIST) {
    // global planes: every coefficient load is issued before the first is used (one
    // round trip per node instead of one per displaced cell); same arithmetic as below
    T a0 = kr[0], a1 = kr[1], a2 = kr[2];         // cell (i, j):         K01 K02 K03
    T b0 = kr[0], b1 = kr[3], b2 = kr[4];         // cell (i-1, j):       K01 K12 K13
    T e0 = kr[1], e1 = kr[3], e2 = kr[5];         // cell (i-1, j-1):     K02 K12 K23
    T f0 = kr[2], f1 = kr[4], f2 = kr[5];         // cell (i, j-1):       K03 K13 K23
    if ((c0 & FLAGS) == FLAGS) { a0 = __ldg(Kg + n); a1 = __ldg(Kg + plane + n); a2 = __ldg(Kg + 2 * plane + n); }
    if ((c1 & FLAGS) == FLAGS) {
      const long long c = n - 1;
      b0 = __ldg(Kg + c); b1 = __ldg(Kg + 3 * plane + c); b2 = __ldg(Kg + 4 * plane + c);
    }
    if ((c2 & FLAGS) == FLAGS) {
      const long long c = n - P - 1;
      e0 = __ldg(Kg + plane + c); e1 = __ldg(Kg + 3 * plane + c); e2 = __ldg(Kg + 5 * plane + c);
    }
    if ((c3 & FLAGS) == FLAGS) {
      const long long c = n - P;
      f0 = __ldg(Kg + 2 * plane + c); f1 = __ldg(Kg + 4 * plane + c); f2 = __ldg(Kg + 5 * plane + c);
    }
    T y = T(0);
    if (c0 & CELL_ACTIVE) y += a0 * dE + a1 * dNE + a2 * dN;
    if (c1 & CELL_ACTIVE) y += b0 * dW + b1 * dN + b2 * dNW;
    if (c2 & CELL_ACTIVE) y += e0 * dSW + e1 * dS + e2 * dW;
    if (c3 & CELL_ACTIVE) y += f0 * dS + f1 * dSE + f2 * dE;
    return y;
  }
  // coefficient m of the cell whose corner 0 is at box column kc, box row kr_, global index g
  auto coef = [&](int m, int kr_, int kc, long long g) -> T {
    if constexpr (STAGED) {
      // two boxes of [CTY+1][6*KHALF], cells interleaved (6 coefficients per cell)
      const int half = kc >= L::KHALF;
      return ks[half * (L::kbox_bytes / (int)sizeof(T)) + kr_ * (6 * L::KHALF) + (kc - half * L::KHALF) * 6 + m];
    } else {
      return __ldg(Kg + m * plane + g);
    }
  };
  T y = T(0);
  if (c0 & CELL_ACTIVE) {                         // node is corner 0 of cell (i, j)
    T k01 = kr[0], k02 = kr[1], k03 = kr[2];
    if (c0 & GEN) { k01 = coef(0, krow, kcol, n); k02 = coef(1, krow, kcol, n); k03 = coef(2, krow, kcol, n); }
    y += k01 * dE + k02 * dNE + k03 * dN;
  }
  if (c1 & CELL_ACTIVE) {                         // corner 1 of cell (i-1, j)
    T k01 = kr[0], k12 = kr[3], k13 = kr[4];
    if (c1 & GEN) {
      k01 = coef(0, krow, kcol - 1, n - 1); k12 = coef(3, krow, kcol - 1, n - 1); k13 = coef(4, krow, kcol - 1, n - 1);
    }
    y += k01 * dW + k12 * dN + k13 * dNW;
  }
  if (c2 & CELL_ACTIVE) {                         // corner 2 of cell (i-1, j-1)
    T k02 = kr[1], k12 = kr[3], k23 = kr[5];
    if (c2 & GEN) {
      const long long c = n - P - 1;
      k02 = coef(1, krow - 1, kcol - 1, c); k12 = coef(3, krow - 1, kcol - 1, c); k23 = coef(5, krow - 1, kcol - 1, c);
    }
    y += k02 * dSW + k12 * dS + k23 * dW;
  }
  if (c3 & CELL_ACTIVE) {                         // corner 3 of cell (i, j-1)
    T k03 = kr[2], k13 = kr[4], k23 = kr[5];
    if (c3 & GEN) {
      const long long c = n - P;
      k03 = coef(2, krow - 1, kcol, c); k13 = coef(4, krow - 1, kcol, c); k23 = coef(5, krow - 1, kcol, c);
    }
    y += k03 * dS + k13 * dSE + k23 * dE;
  }
  return y;
}

// Issue the TMA loads of tile t into stage s (one thread).  thin: the grid's last row is
// at most two rows below the tile's first, so boxes of THIN rows hold every row the tile
// reads; narrow: the grid's last column is at most 30 columns right of the tile's first,
// so the first state box (nodes i0-1 .. i0+31) and the first coefficient box (cells
// i0-4 .. i0+29) hold every node and cell the tile reads.  The consumers never read the
// staged positions outside the grid, so the parts not loaded are never used.
template <typename T>
__device__ __forceinline__ void cg_issue(const CgMaps& mp, int cur, unsigned char* stage, uint64_t* bar,
                                         int2 ij, int row0, bool gen, bool plain, bool thin, bool narrow) {
  using L = CgSmem<T, 2>;   // stage layout does not depend on the stage count
  const int x0 = ij.x - 4, y0 = row0 + ij.y - 1;
  const int nbox = narrow ? 1 : 2;
  mbar_arrive_expect_tx(bar, nbox * L::tx_sbox(thin) + (plain ? 0 : L::tx_tbox(thin)) +
                                 (gen ? nbox * L::tx_kbox(thin) : 0));
  // state records viewed as a [rows][4 P] array: two boxes of SHALF nodes (long rows)
  const CUtensorMap* sm = thin ? &mp.s_thin[cur] : &mp.s[cur];
  tma_load_2d(stage + L::off_s, sm, 4 * (ij.x - 1), y0, bar);
  if (!narrow) tma_load_2d(stage + L::off_s + L::sbox_bytes, sm, 4 * (ij.x - 1 + L::SHALF), y0, bar);
  if (!plain) tma_load_2d(stage + L::off_t, thin ? &mp.tag_thin : &mp.tag, ij.x - 16, y0, bar);   // plain tiles need no tags
  if constexpr (L::kTmaK) {
    if (gen) {
      // interleaved coefficients as a [rows][6 P] array: two boxes of KHALF cells
      const CUtensorMap* km = thin ? &mp.k_thin : &mp.k;
      tma_load_2d(stage + L::off_k, km, 6 * x0, y0, bar);
      if (!narrow) tma_load_2d(stage + L::off_k + L::kbox_bytes, km, 6 * (x0 + L::KHALF), y0, bar);
    }
  }
}

// Nodes per thread (a vertical strip) and the thread -> strip mapping of a tile.
constexpr int STRIP = CTY * CTX / NT;             // 4
static_assert(STRIP * NT == CTX * CTY, "tile must split into strips");
constexpr int NTC = NT + 32;                      // 8 consumer warps + 1 TMA producer warp
constexpr int CONSUMER_BAR = 1;                   // named barrier of the consumer warps

// State record of p-tile position (li, lj) inside the two staged state boxes.
template <typename T>
__device__ __forceinline__ State4<T> staged_state(const State4<T>* Ss, int li, int lj) {
  using L = CgSmem<T>;
  const int half = li >= L::SHALF;
  return Ss[half * L::sbox_recs + lj * L::SHALF + (li - half * L::SHALF)];
}

template <typename T, int NS>
__global__ void __launch_bounds__(NTC, sizeof(T) == 4 ? 2 : 1) k_cg(CGArgs<T> a, const __grid_constant__ CgMaps mp) {
  using L = CgSmem<T, NS>;
  static_assert(L::off_bar >= FIN_CAP * 8, "the finaliser stages FIN_CAP doubles in the stage memory");
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ T s_pb[MAXB];
  __shared__ double red[NT / 32][4];
  __shared__ double scratch[NT / 32 + 1];
  __shared__ double sh_qb[MAXB];
  __shared__ FinCache<T> fc;
  __shared__ int2 s_tij[NS];                      // tile of each stage, written by the producer
  __shared__ int s_tfl[NS];                       // its flags (bit 0: coefficient boxes, bit 1: plain)
  __shared__ int s_last, s_abort, s_issued;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::off_bar);
  uint64_t* empty = full + NS;
  const int tid = threadIdx.y * TX + threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool producer = warp == NT / 32;
  const int col = tid % CTX;                      // strip column inside the tile
  const int row_lo = (tid / CTX) * STRIP;         // first strip row inside the tile
  const int B = a.B;
  const long long plane = a.m.Vtot;
  constexpr int W = CTX + 2;
  constexpr int NH = 2 * W + 2 * CTY;             // halo ring positions
  static_assert(NH <= NT, "one halo position per consumer thread at most");
  // this thread's halo-ring position (the same for every tile): li | lj << 8, or -1
  int hpos = -1;
  {
    const int h = warp + (NT / 32) * lane;
    if (!producer && h < NH) {
      int li, lj;
      if (h < W) { li = h; lj = 0; }
      else if (h < 2 * W) { li = h - W; lj = CTY + 1; }
      else if (h < 2 * W + CTY) { li = 0; lj = 1 + (h - 2 * W); }
      else { li = CTX + 1; lj = 1 + (h - 2 * W - CTY); }
      hpos = li | (lj << 8);
    }
  }
  if (tid == 0) {
    for (int k = 0; k < NS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], NT / 32);
    }
    fence_mbar_init();
    s_abort = 0;
    s_issued = 0;
  }
  __syncthreads();
  __shared__ unsigned long long s_t0;             // timed launches: start of this CTA's tile phase
  if (a.sc.cta_ns && tid == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(s_t0));
  int q = 0;                                      // tiles consumed (consumers) / issued (producer) so far
  for (int sg = a.sc.cta_seg[blockIdx.x]; sg < a.sc.cta_seg[blockIdx.x + 1]; ++sg) {
    const int v = a.sc.seg_var[sg];
    if (a.st[v].phase != PH_CG) continue;
    const DevVariant& Vg = a.m.var[v];
    const int nx = Vg.nx, ny = Vg.ny, P = Vg.P, row0 = Vg.row0, nb = Vg.nb, body0 = Vg.body0;
    const long long base = Vg.base;
    const int cur = a.st[v].buf;
    const int t0 = a.sc.seg_t0[sg], t1 = a.sc.seg_t1[sg];
    Acc<T> acc;
    acc.zero();
    if (producer) {
      // ---- TMA producer: stage s is reused once its previous tile has been released
      if (lane == 0) {
        for (int t = t0; t < t1; ++t, ++q) {
          const int s = q % NS, use = q / NS;
          if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, a.poll_limit)) {
            atomicExch(a.err, 1);
            s_abort = 1;
            break;
          }
          if (*(volatile int*)&s_abort) break;
          if (a.test_drop && blockIdx.x == 0 && q == 0) {
            s_issued = q + 1;                     // the consumers' wait on this stage must give up
            continue;
          }
          fence_proxy_async_smem();
          const int2 tij = a.sc.tile_ij[t];
          const int fl = a.tile_gen[t];
          const bool gen = (fl & (sizeof(T) == 4 ? TILE_GEN32 : TILE_GEN64)) != 0,
                     plain = (fl & (sizeof(T) == 4 ? TILE_PLAIN32 : TILE_PLAIN64)) != 0;
          s_tij[s] = tij;                         // published to the consumers by the arrive below
          s_tfl[s] = (gen ? 1 : 0) | (plain ? 2 : 0);
          cg_issue<T>(mp, cur, smem + s * L::stage_bytes, &full[s], tij, row0, gen, plain, ny - tij.y <= 2,
                      nx <= tij.x + 30);
          s_issued = q + 1;
        }
      }
      q = __shfl_sync(0xffffffffu, q, 0);
    } else {
      // ---- consumers
      T kr[6];
#pragma unroll
      for (int m = 0; m < 6; ++m) kr[m] = krect<T>(Vg)[m];
      const T alpha = (T)a.st[v].alpha, beta = (T)a.st[v].beta;
      State4<T>* __restrict__ s_new = a.s[cur ^ 1];
      if (tid < nb) {
        const int gb = body0 + tid;
        const T xb = a.sb[gb], rb = a.sb[B + gb], pb = a.sb[2 * B + gb], qb = a.sb[3 * B + gb];
        fc.sb[0][tid] = xb;
        fc.sb[1][tid] = rb;
        fc.sb[2][tid] = pb;
        fc.sb[3][tid] = qb;
        s_pb[tid] = a.prm->fixed_bodies ? T(0) : next_p(next_r(rb, qb, alpha), pb, beta);
      }
      if (tid <= nb) fc.bptr[tid] = a.m.body_ptr[body0 + tid];
      if (tid == NT - 1) {
        const VarState& S = a.st[v];
        fc.alpha = S.alpha;
        fc.beta = S.beta;
        fc.gamma_start = S.gamma_start;
        fc.thr_rel = S.thr_rel;
        fc.thr_abs2 = S.thr_abs2;
        fc.iters = S.iters;
        fc.inner_iters = S.inner_iters;
        fc.buf = cur;
        fc.k_max = a.prm->k_max;
        fc.fixed = a.prm->fixed_bodies;
        fc.seg0 = a.sc.var_seg0[v];
        fc.seg1 = a.sc.var_seg1[v];
      }
      named_bar_sync(CONSUMER_BAR, NT);
      for (int t = t0; t < t1; ++t, ++q) {
        const int s = q % NS;
        unsigned char* st = smem + s * L::stage_bytes;
        T* pt = reinterpret_cast<T*>(smem + L::off_ptile + (q & 1) * L::ptile_bytes);
        uint8_t* tt = reinterpret_cast<uint8_t*>(smem + L::off_ttile + (q & 1) * L::ttile_bytes);
        const bool ok = mbar_wait(&full[s], (q / NS) & 1, a.poll_limit);
        const int2 ij = s_tij[s];
        const bool plain = (s_tfl[s] & 2) != 0;
        const State4<T>* Ss = reinterpret_cast<const State4<T>*>(st + L::off_s);
        const uint8_t* Tg = reinterpret_cast<const uint8_t*>(st + L::off_t);
        const T* Ks = reinterpret_cast<const T*>(st + L::off_k);
        const long long tb = base + (long long)ij.y * P + ij.x;
        // pass 1: own strip and the halo ring -> p tile, effective tags
        T rn4[STRIP], pn4[STRIP], xn4[STRIP];
        int bs4[STRIP];                           // slot of a BODY node in body_nodes
        uint8_t tg4[STRIP];
        if (ok && plain) {
          // every node of the window is FREE and every cell active with rectangle constants
#pragma unroll
          for (int u = 0; u < STRIP; ++u) {
            const int li = 1 + col, lj = 1 + row_lo + u;
            const State4<T> o = staged_state<T>(Ss, li, lj);
            const T rn = next_r(o.r, o.q, alpha);
            const T pn = next_p(rn, o.p, beta);
            pt[lj * W + li] = pn;
            rn4[u] = rn; pn4[u] = pn; xn4[u] = next_x(o.x, o.p, alpha);
            tg4[u] = K_FREE;
            bs4[u] = -1;
          }
          if (hpos >= 0) {
            const int li = hpos & 255, lj = hpos >> 8;
            const State4<T> o = staged_state<T>(Ss, li, lj);
            pt[lj * W + li] = next_p(next_r(o.r, o.q, alpha), o.p, beta);
          }
        } else if (ok) {
#pragma unroll
          for (int u = 0; u < STRIP; ++u) {
            const int li = 1 + col, lj = 1 + row_lo + u;
            const int i = ij.x + col, j = ij.y + row_lo + u;
            const bool in = (i <= nx) && (j <= ny);
            const uint8_t tg = in ? Tg[lj * L::TBW + li + 15] : K_INACT;
            const int kind = tg & KIND_MASK;
            T rn = T(0), pn = T(0), xn = T(0);
            int bs = -1;
            if (kind == K_FREE) {
              const State4<T> o = staged_state<T>(Ss, li, lj);
              rn = next_r(o.r, o.q, alpha);
              xn = next_x(o.x, o.p, alpha);
              pn = next_p(rn, o.p, beta);
            } else if (kind == K_BODY) {
              const int e = slot_of(staged_state<T>(Ss, li, lj).x);
              if (e >= fc.bptr[0] && e < fc.bptr[nb]) {
                bs = e;
                pn = s_pb[body_of_slot(fc.bptr, nb, e)];
              }
            }
            bs4[u] = bs;
            pt[lj * W + li] = pn;
            tt[lj * W + li] = tg;
            rn4[u] = rn; pn4[u] = pn; xn4[u] = xn; tg4[u] = tg;
          }
          if (hpos >= 0) {
            const int li = hpos & 255, lj = hpos >> 8;
            const int i = ij.x - 1 + li, j = ij.y - 1 + lj;
            uint8_t ht = K_INACT;
            T hp = T(0);
            if (i >= 0 && j >= 0 && i <= nx && j <= ny) {
              ht = Tg[lj * L::TBW + li + 15];
              const int hk = ht & KIND_MASK;
              if (hk == K_FREE) {
                const State4<T> o = staged_state<T>(Ss, li, lj);
                hp = next_p(next_r(o.r, o.q, alpha), o.p, beta);
              } else if (hk == K_BODY) {
                const int e = slot_of(staged_state<T>(Ss, li, lj).x);
                if (e >= fc.bptr[0] && e < fc.bptr[nb]) hp = s_pb[body_of_slot(fc.bptr, nb, e)];
              }
            }
            pt[lj * W + li] = hp;
            tt[lj * W + li] = ht;
          }
        }
        if (named_bar_or(CONSUMER_BAR, NT, !ok)) {
          if (tid == 0) {
            atomicExch(a.err, 1);
            s_abort = 1;
          }
          break;
        }
        // pass 2: operator rows of the strip from a register window of the p tile
        if (plain) {
          const int li = 1 + col;
          T win[STRIP + 2][3];
#pragma unroll
          for (int r = 0; r < STRIP + 2; ++r) {
            const int lj = row_lo + r;
            win[r][0] = pt[lj * W + li - 1];
            win[r][1] = (r >= 1 && r <= STRIP) ? pn4[r - 1] : pt[lj * W + li];   // own strip in registers
            win[r][2] = pt[lj * W + li + 1];
          }
          T yq[STRIP];
#pragma unroll
          for (int u = 0; u < STRIP; ++u) {
            const long long n = tb + (long long)(row_lo + u) * P + col;
            const T nbh[3][3] = {{win[u][0], win[u][1], win[u][2]},
                                 {win[u + 1][0], win[u + 1][1], win[u + 1][2]},
                                 {win[u + 2][0], win[u + 2][1], win[u + 2][2]}};
            const T y = q4_row_rect<T>(nbh, kr);
            State4<T> o;
            o.x = xn4[u];
            o.r = rn4[u];
            o.p = pn4[u];
            o.q = y;
            s_new[n] = o;
            yq[u] = y;
          }
          acc.add4(0, rn4, rn4);
          acc.add4(1, pn4, yq);
          acc.add4(2, rn4, yq);
          acc.add4(3, yq, yq);
        } else {
          const int li = 1 + col;
          T win[STRIP + 2][3];
          uint8_t cl[STRIP + 1], cr[STRIP + 1];     // cells (i-1, j) and (i, j) for rows j0-1 .. j0+3
#pragma unroll
          for (int r = 0; r < STRIP + 2; ++r) {
            const int lj = row_lo + r;
            win[r][0] = pt[lj * W + li - 1];
            win[r][1] = (r >= 1 && r <= STRIP) ? pn4[r - 1] : pt[lj * W + li];   // own strip in registers
            win[r][2] = pt[lj * W + li + 1];
          }
#pragma unroll
          for (int r = 0; r < STRIP + 1; ++r) {
            const int lj = row_lo + r;
            cl[r] = tt[lj * W + li - 1];
            cr[r] = tt[lj * W + li];
          }
          T yq[STRIP], rr[STRIP], pp[STRIP];
#pragma unroll
          for (int u = 0; u < STRIP; ++u) {
            const int kind = tg4[u] & KIND_MASK;
            yq[u] = T(0);
            rr[u] = T(0);
            pp[u] = T(0);
            if (kind == K_FREE || kind == K_BODY) {
              const long long n = tb + (long long)(row_lo + u) * P + col;
              const T nbh[3][3] = {{win[u][0], win[u][1], win[u][2]},
                                   {win[u + 1][0], win[u + 1][1], win[u + 1][2]},
                                   {win[u + 2][0], win[u + 2][1], win[u + 2][2]}};
              const T y = q4_row_nb<T, sizeof(T) == 4, sizeof(T) == 8>(nbh, cr[u + 1], cl[u + 1], cl[u], cr[u], Ks,
                                                                       col + 4, row_lo + u + 1, n, P, kplane<T>(a.m),
                                                                       plane, kr);
              State4<T> o;
              o.x = kind == K_BODY ? slot_bits(bs4[u], T(0)) : xn4[u];
              o.r = rn4[u];
              o.p = pn4[u];
              o.q = y;
              s_new[n] = o;          // BODY nodes: x = slot bits, r = 0, p = the body's p, q = row of A p
              if (kind == K_BODY && bs4[u] >= 0) a.bq[bs4[u]] = (double)y;   // slot was range-checked
              if (kind == K_FREE) {
                yq[u] = y;
                rr[u] = rn4[u];
                pp[u] = pn4[u];
              }
            }
          }
          acc.add4(0, rr, rr);
          acc.add4(1, pp, yq);
          acc.add4(2, rr, yq);
          acc.add4(3, yq, yq);
        }
        // release the stage to the producer (one arrival per consumer warp)
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
      }
    }
    // ---- segment end: partial sums, last-CTA reduction (all warps)
    __syncthreads();
    if (s_abort) {
      // drain loads issued but not consumed (bounded), then leave
      if (tid == 0)
        for (int k = q; k < s_issued; ++k) mbar_wait(&full[k % NS], (k / NS) & 1, a.poll_limit);
      __syncthreads();
      return;
    }
    double w4[4];
    acc.warp_reduce(w4);
    if (lane == 0 && !producer)
      for (int k = 0; k < 4; ++k) red[warp][k] = w4[k];
    __syncthreads();
    if (tid == 0) {
      for (int k = 0; k < 4; ++k) {
        double sum = 0.0;
        for (int w = 0; w < NT / 32; ++w) sum += red[w][k];
        a.sc.partial[sg * 4 + k] = sum;
      }
      if (a.sc.cta_ns && sg + 1 == a.sc.cta_seg[blockIdx.x + 1]) {
        unsigned long long t_end;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t_end));
        a.sc.cta_ns[blockIdx.x] += t_end - s_t0;   // summed over the launches of a timed round
      }
      // release this CTA's stores (ordered before by the barrier), acquire the others'
      const int done = atom_add_acq_rel_gpu(&a.sc.counter[v], 1);
      s_last = (done == seg_count(a.sc, v) - 1);
    }
    __syncthreads();
    if (s_last) finalize_cg<T, NTC>(a, v, nb, body0, fc, scratch, sh_qb, reinterpret_cast<double*>(smem));
    __syncthreads();
  }
}

// ---------------------------------------------------------------- true residual
template <typename T>
__device__ void finalize_resid(const ResidArgs<T>& a, int v, double* scratch, double* sh_rb) {
  const DevVariant& V = a.m.var[v];
  VarState* S = &a.st[v];
  double d[1];
  {
    double s = 0.0;
    for (int k = linear_tid(); k < a.gx; k += NT) s += __ldcg(&a.rpart[(long long)v * a.gx + k]);
    d[0] = block_sum(s, scratch);
  }
  for (int k = 0; k < V.nb; ++k) {
    const double s = body_gather<double>(a.m, V.body0 + k, a.w64, scratch);
    if (linear_tid() == 0) sh_rb[k] = (a.rhsb ? a.rhsb[V.body0 + k] : 0.0) - s;
  }
  __syncthreads();
  if (linear_tid() == 0) {
    const int B = a.B;
    double g = d[0];
    const bool fixed = a.prm->fixed_bodies != 0;
    for (int k = 0; k < V.nb; ++k) {
      const int gb = V.body0 + k;
      const double rb = sh_rb[k];
      a.sbr[gb] = rb;
      if (fixed) {                 // given body value: its row is an output, not an equation
        a.sb[B + gb] = T(0);
        continue;
      }
      g += rb * rb;
      a.sol[gb] = a.sol[gb] + (double)a.sb[gb];   // fold the body correction
      a.sb[gb] = T(0);
      a.sb[B + gb] = (T)rb;
      a.sb[2 * B + gb] = T(0);
      a.sb[3 * B + gb] = T(0);
    }
    S->rr64 = g;
    S->n_resid += 1;
    if (S->bnorm2 < 0.0) S->bnorm2 = g;
    const double tol2 = a.prm->tol2;
    const bool paper = a.prm->paper_abs != 0;
    bool fin = false;
    if (S->bnorm2 == 0.0 || (paper ? g <= a.prm->tol_abs : g <= tol2 * S->bnorm2)) {
      S->status = PF_OK;
      fin = true;
    } else if (S->capped || !isfinite(g)) {
      S->status = isfinite(g) ? PF_ENOT_CONVERGED : PF_EBREAKDOWN;
      fin = true;
    }
    if (fin) {
      S->phase = PH_DONE;
      atomicAdd(a.n_done, 1);
    } else {
      S->phase = PH_CG;
      S->alpha = 0.0;
      S->beta = 0.0;
      S->inner_iters = 0;
      S->thr_rel = a.mixed ? a.prm->inner_rel2 : 0.0;
      // inner stop on the recurrence residual: the paper's own test sum r^2 <= tol in FP64
      // mode under PF_TOL_PAPER_ABS; otherwise below the target, so that the true residual
      // (which the FP32 recurrence tracks less closely) usually passes at the next check
      S->thr_abs2 = paper ? (a.mixed ? 0.25 : 1.0) * a.prm->tol_abs : (a.mixed ? 0.25 : 0.5) * tol2 * S->bnorm2;
    }
    a.counter[v] = 0;
  }
}

// Tiles [t0, t1) of variant v's 32x8 tile grid taken by CTA column bx of gx.
__device__ __forceinline__ void resid_share(const DevVariant& V, int gx, int bx, long long& t0, long long& t1) {
  const long long nt = (long long)V.tiles_x * V.tiles_y;
  t0 = nt * bx / gx;
  t1 = nt * (bx + 1) / gx;
}

template <typename T>
__global__ void __launch_bounds__(NT) k_resid(ResidArgs<T> a) {
  __shared__ double ps[TY + 2][SW];
  __shared__ uint8_t ts[TY + 2][SW];
  __shared__ double s_xb[MAXB];
  __shared__ double red[NT / 32];
  __shared__ double scratch[NT / 32 + 1];
  __shared__ double sh_rb[MAXB];
  __shared__ int s_last;
  const int tid = linear_tid(), lane = tid & 31, warp = tid >> 5;
  const long long plane = a.m.Vtot;
  const int v = blockIdx.y, bx = blockIdx.x;
  if (a.st[v].phase != PH_RESID) return;          // the whole row leaves: nothing to refine
  const DevVariant& V = a.m.var[v];
  if (tid < V.nb) {
    const int gb = V.body0 + tid;
    s_xb[tid] = a.sol[gb] + (double)a.sb[gb];
  }
  const int cur = a.st[v].buf;
  State4<T>* __restrict__ s_out = a.s[cur];
  __syncthreads();
  double acc = 0.0;
  long long t0, t1;
  resid_share(V, a.gx, bx, t0, t1);
  for (long long t = t0; t < t1; ++t) {
    const int2 ij = make_int2((int)(t % V.tiles_x) * TX, (int)(t / V.tiles_x) * TY);
    const int i = ij.x + threadIdx.x, j = ij.y + threadIdx.y;
    const bool in = (i <= V.nx) && (j <= V.ny);
    const long long n = V.base + (long long)j * V.P + i;
    const uint8_t tg = in ? a.m.tag[n] : K_INACT;
    const int kind = tg & KIND_MASK;
    double u = 0.0;
    if (kind == K_FREE || kind == K_DIR) u = a.x64[n];
    else if (kind == K_BODY) u = s_xb[a.m.bid[n]];
    ps[threadIdx.y + 1][threadIdx.x + 1] = u;
    ts[threadIdx.y + 1][threadIdx.x + 1] = tg;
    if (tid < NHALO) {
      int li, lj;
      halo_pos(tid, li, lj);
      const int hi = ij.x - 1 + li, hj = ij.y - 1 + lj;
      uint8_t ht = K_INACT;
      double hu = 0.0;
      if (hi >= 0 && hj >= 0 && hi <= V.nx && hj <= V.ny) {
        const long long hn = V.base + (long long)hj * V.P + hi;
        ht = a.m.tag[hn];
        const int hk = ht & KIND_MASK;
        if (hk == K_FREE || hk == K_DIR) hu = a.x64[hn];
        else if (hk == K_BODY) hu = s_xb[a.m.bid[hn]];
      }
      ps[lj][li] = hu;
      ts[lj][li] = ht;
    }
    __syncthreads();
    if (kind == K_FREE || kind == K_BODY) {
      const double y = q4_row<double>(ps, ts, threadIdx.x + 1, threadIdx.y + 1, n, V.P, a.m.K64, plane, V.kr64);
      if (kind == K_FREE) {
        const double r = -y;
        if (a.rplane) {
          a.rplane[n] = (float)r;
        } else {
          State4<T> o;
          o.x = T(0);
          o.r = (T)r;
          o.p = T(0);
          o.q = T(0);
          s_out[n] = o;
        }
        acc = fma(r, r, acc);
      } else {
        a.w64[n] = y;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    a.rpart[(long long)v * a.gx + bx] = s;
    // release this CTA's stores (ordered before by the barrier), acquire the others'
    const int done = atom_add_acq_rel_gpu(&a.counter[v], 1);
    s_last = (done == a.gx - 1);
  }
  __syncthreads();
  if (s_last) finalize_resid<T>(a, v, scratch, sh_rb);
}

// Fold the CG correction into the FP64 solution before the true residual (pointwise,
// its own launch so no tile ever sees a half-updated neighbour).  Same (gx, variants)
// grid as k_resid: a launch with no variant to refine costs one load per CTA.
template <typename T>
__global__ void __launch_bounds__(NT) k_fold(const DevVariant* var, int gx, const uint8_t* tag, const VarState* st,
                                             double* x64, State4<T>* const* sbuf, float* xplane) {
  const int v = blockIdx.y;
  if (st[v].phase != PH_RESID) return;
  const DevVariant& V = var[v];
  State4<T>* s = sbuf[st[v].buf];
  long long t0, t1;
  resid_share(V, gx, blockIdx.x, t0, t1);
  for (long long t = t0; t < t1; ++t) {
    const int i = (int)(t % V.tiles_x) * TX + threadIdx.x, j = (int)(t / V.tiles_x) * TY + threadIdx.y;
    if (i > V.nx || j > V.ny) continue;
    const long long n = V.base + (long long)j * V.P + i;
    if ((tag[n] & KIND_MASK) != K_FREE) continue;
    if (xplane) {                       // preconditioned CG keeps its correction in a plane
      x64[n] = x64[n] + (double)xplane[n];
      xplane[n] = 0.0f;
      continue;
    }
    x64[n] = x64[n] + (double)s[n].x;
    s[n].x = T(0);
  }
}

// Seed the slot bits into the x field of every BODY node's record in both ping-pong
// buffers (the fused CG step carries them forward from then on).
template <typename T>
__global__ void k_seed_slots(const long long* body_nodes, int n_slots, State4<T>* s0, State4<T>* s1) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_slots) return;
  const long long n = body_nodes[e];
  s0[n].x = slot_bits(e, T(0));
  s1[n].x = slot_bits(e, T(0));
}

// ---------------------------------------------------------------- init / export
// Dirichlet data g = U * gcoord (gcoord: the y plane of the coordinates for psi = U y, the x
// plane for phi = U x), the warm-start or zero initial guess elsewhere.
__global__ void k_init(const DevVariant* var, const int* tile_var, const int2* tile_ij, const uint8_t* tag,
                       const double* gcoord, double U0, const double* Uv, int warm, double* x64, double* w64) {
  const long long t = blockIdx.x;
  const int v = tile_var[t];
  const double U = Uv ? Uv[v] : U0;
  const DevVariant& V = var[v];
  const int2 ij = tile_ij[t];
  const int i = ij.x + threadIdx.x, j = ij.y + threadIdx.y;
  if (i >= V.P || j > V.ny) return;
  const long long n = V.base + (long long)j * V.P + i;
  const int kind = (i <= V.nx) ? (tag[n] & KIND_MASK) : K_INACT;
  double u = 0.0;
  if (kind == K_DIR) u = __dmul_rn(U, gcoord[n]);
  else if (kind == K_FREE && warm) u = x64[n];
  x64[n] = u;
  w64[n] = 0.0;
}

__global__ void k_export_psi(const DevVariant* var, int nv, const long long* lbase, const uint8_t* tag,
                             const int* bid, const double* x64, const double* xb, double* psi) {
  // one grid over all variants' logical nodes: blockIdx.y = variant
  const int v = blockIdx.y;
  const DevVariant& V = var[v];
  const long long N = (long long)(V.nx + 1) * (V.ny + 1);
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(m % (V.nx + 1)), j = (int)(m / (V.nx + 1));
    const long long n = V.base + (long long)j * V.P + i;
    const int kind = tag[n] & KIND_MASK;
    double u = 0.0;
    if (kind == K_FREE || kind == K_DIR) u = x64[n];
    else if (kind == K_BODY) u = xb[V.body0 + bid[n]];
    psi[lbase[v] + m] = u;
  }
}

// logical <-> padded copies used by pf_apply
template <typename T>
__global__ void k_to_padded(const DevVariant* var, const long long* lbase, const double* src, T* dst) {
  const int v = blockIdx.y;
  const DevVariant& V = var[v];
  const long long N = (long long)(V.nx + 1) * (V.ny + 1);
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(m % (V.nx + 1)), j = (int)(m / (V.nx + 1));
    dst[V.base + (long long)j * V.P + i] = (T)src[lbase[v] + m];
  }
}

template <typename T>
__global__ void k_from_padded(const DevVariant* var, const long long* lbase, const T* src, double* dst) {
  const int v = blockIdx.y;
  const DevVariant& V = var[v];
  const long long N = (long long)(V.nx + 1) * (V.ny + 1);
  for (long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x; m < N; m += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(m % (V.nx + 1)), j = (int)(m / (V.nx + 1));
    dst[lbase[v] + m] = (double)src[V.base + (long long)j * V.P + i];
  }
}

// Stand-alone operator y = A p on the padded vectors (pf_apply, pf_apply_timing).  The
// tile list is cut into groups of up to AG horizontally adjacent tiles of one tile row;
// a group's p window (nodes i0-4 .. i0+AG*CTX+3, rows j0-1 .. j0+CTY) has long contiguous
// rows in HBM (800 bytes of FP32 p for AG = 3).  Persistent CTAs take groups from a
// ticket counter (tiles whose cells need stored coefficients cost several times a
// plain tile, so a static split leaves SMs idle); with no reduction, the order does not
// matter.  A producer warp stages each group's p window and, unless every tile of the
// group is plain, its tag window (i0-16 .. i0+AG*CTX+15) with TMA into a ring of NS
// stages; eight consumer warps each form the rows of one 4-node vertical strip per tile
// exactly as the fused kernel does (stored coefficients come from the global planes
// for the cells that need them) and release the stage.  Nodes without an operator row
// get 0; nodes outside the grid are not written.  A wait that gives up sets *err and
// the CTA stops.
//
// Group descriptor (int4): x = i0 | tiles << 20 | FP32 plain bits << 24 | FP64 plain
// bits << 28, y = j0, z = variant, w = the batch row of j0.  Tickets: every CTA claims
// one ticket past its last group, so a launch consumes n_groups + gridDim.x tickets
// from `ticket_base` on.
constexpr int AG = 3;                             // tiles per group
static_assert(AG <= 4, "plain bits of a group: 4 per precision");
template <typename T, int NS>
struct ApSmem {
  static constexpr int AW = AG * CTX + 8;         // p box width: x start i0-4 (4 (i0-4) or 8 (i0-4) bytes)
  static constexpr int H = CTY + 2;
  static constexpr int TBW = AG * CTX + 32;       // tag box width: x start i0-16
  static constexpr int align(int b) { return (b + 127) / 128 * 128; }
  static constexpr int p_bytes = H * AW * (int)sizeof(T);
  static constexpr int t_bytes = H * TBW;
  static constexpr int off_t = align(p_bytes);
  static constexpr int stage_bytes = off_t + align(t_bytes);
  static constexpr int off_bar = NS * stage_bytes;
  static constexpr int total = off_bar + 2 * NS * 8;
  static_assert(off_t % 128 == 0 && stage_bytes % 128 == 0, "TMA destinations must start on 128-byte boundaries");
  static_assert(AW <= 256 && TBW <= 256 && (AW * sizeof(T)) % 16 == 0 && TBW % 16 == 0,
                "TMA boxes: at most 256 elements, rows of a multiple of 16 bytes");
  static_assert(CTX % 16 == 0, "box x coordinates (i0-4) sizeof(T) and i0-16 bytes must be multiples of 16");
};
template <typename T> struct ApStages;
template <> struct ApStages<float> { static constexpr int ns = 4; };
template <> struct ApStages<double> { static constexpr int ns = 3; };

template <typename T, int NS>
__global__ void __launch_bounds__(NTC, sizeof(T) == 4 ? 3 : 1) k_apply(MeshDev m, const int4* __restrict__ groups, long long n_groups,
                                               unsigned long long* ticket, unsigned long long ticket_base,
                                               T* __restrict__ y, const __grid_constant__ CgMaps mp, int* err,
                                               int poll_limit) {
  using L = ApSmem<T, NS>;
  constexpr int AW = L::AW, TBW = L::TBW;
  constexpr int PSHIFT = sizeof(T) == 4 ? 24 : 28;
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int4 s_grp[NS];                      // the group in each stage (tiles = 0: end marker)
  __shared__ int s_abort, s_issued;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + L::off_bar);
  uint64_t* empty = full + NS;
  const int tid = threadIdx.y * TX + threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    for (int k = 0; k < NS; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], NT / 32);
    }
    fence_mbar_init();
    s_abort = 0;
    s_issued = 0;
  }
  __syncthreads();
  if (warp == NT / 32) {
    // ---- TMA producer (lane 0): the next group is claimed and its descriptor loaded
    // before waiting for the current group's stage
    if (lane == 0) {
      int q = 0;
      long long item = (long long)(atomicAdd(ticket, 1ULL) - ticket_base);
      int4 d = (item >= 0 && item < n_groups) ? groups[item] : make_int4(0, 0, 0, 0);
      bool stop = false;
      while (item >= 0 && item < n_groups) {
        const long long nitem = (long long)(atomicAdd(ticket, 1ULL) - ticket_base);
        const int4 nd = (nitem >= 0 && nitem < n_groups) ? groups[nitem] : d;
        const int s = q % NS, use = q / NS;
        if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, poll_limit)) {
          atomicExch(err, 1);
          s_abort = 1;
          stop = true;
          break;
        }
        fence_proxy_async_smem();
        const int x = d.x & 0xfffff, g = (d.x >> 20) & 15, pl = (d.x >> PSHIFT) & 15;
        const bool all_plain = pl == (1 << g) - 1;
        s_grp[s] = make_int4(x, d.y, d.z, g | (pl << 4));   // published to the consumers by the arrive below
        unsigned char* st = smem + s * L::stage_bytes;
        mbar_arrive_expect_tx(&full[s], L::p_bytes + (all_plain ? 0 : L::t_bytes));
        tma_load_2d(st, &mp.s[0], x - 4, d.w - 1, &full[s]);
        if (!all_plain) tma_load_2d(st + L::off_t, &mp.tag, x - 16, d.w - 1, &full[s]);
        s_issued = ++q;
        item = nitem;
        d = nd;
      }
      // end marker: a stage with no tiles, completed by a plain arrival
      if (!stop) {
        const int s = q % NS, use = q / NS;
        if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, poll_limit)) {
          atomicExch(err, 1);
          s_abort = 1;
        } else {
          s_grp[s] = make_int4(0, 0, 0, 0);
          mbar_arrive(&full[s]);
        }
      }
    }
  } else {
    // ---- consumers: warps run independently, each releasing a stage once it is done
    const int col = tid % CTX, row_lo = (tid / CTX) * STRIP;
    int lastv = -1, nx = 0, ny = 0, P = 0;
    long long base = 0;
    T kr[6];
    for (int q = 0;; ++q) {
      const int s = q % NS;
      if (!mbar_wait(&full[s], (q / NS) & 1, poll_limit)) {
        atomicExch(err, 1);
        s_abort = 1;
        break;
      }
      const int4 gd = s_grp[s];
      const int g = gd.w & 15;
      if (g == 0) break;                          // the producer's end marker
      const int2 ij = make_int2(gd.x, gd.y);
      const int v = gd.z;
      if (v != lastv) {
        const DevVariant& V = m.var[v];
        nx = V.nx; ny = V.ny; P = V.P; base = V.base;
#pragma unroll
        for (int c = 0; c < 6; ++c) kr[c] = krect<T>(V)[c];
        lastv = v;
      }
      const unsigned char* st = smem + s * L::stage_bytes;
      const T* ps = reinterpret_cast<const T*>(st);                    // box origin (i0-4, j0-1)
      const uint8_t* Tg = st + L::off_t;                               // box origin (i0-16, j0-1)
      // flags of cell (i0 + ci, j0 + cj), 0 for cells outside the variant
      auto cellf = [&](int ci, int cj) -> uint8_t {
        return ((unsigned)(ij.x + ci) < (unsigned)nx && (unsigned)(ij.y + cj) < (unsigned)ny)
                   ? Tg[(cj + 1) * TBW + ci + 16]
                   : (uint8_t)0;
      };
      for (int u = 0; u < g; ++u) {
        const int c = u * CTX + col;              // column inside the group
        const int i = ij.x + c;
        if (i > nx) break;
        const bool plain = (gd.w >> (4 + u)) & 1;
        T win[STRIP + 2][3];                      // p around the strip: box rows row_lo .. row_lo+5
#pragma unroll
        for (int r = 0; r < STRIP + 2; ++r)
#pragma unroll
          for (int cc = 0; cc < 3; ++cc) win[r][cc] = ps[(row_lo + r) * AW + c + 3 + cc];
        if (plain) {
          // a plain tile's window is inside the grid: no bounds checks
          T* yo = y + base + (long long)(ij.y + row_lo) * P + i;
#pragma unroll
          for (int w = 0; w < STRIP; ++w) {
            const T nbh[3][3] = {{win[w][0], win[w][1], win[w][2]},
                                 {win[w + 1][0], win[w + 1][1], win[w + 1][2]},
                                 {win[w + 2][0], win[w + 2][1], win[w + 2][2]}};
            yo[(long long)w * P] = q4_row_rect<T>(nbh, kr);
          }
          continue;
        }
#pragma unroll
        for (int w = 0; w < STRIP; ++w) {
          const int rl = row_lo + w, j = ij.y + rl;
          if (j > ny) break;
          const long long n = base + (long long)j * P + i;
          const T nbh[3][3] = {{win[w][0], win[w][1], win[w][2]},
                               {win[w + 1][0], win[w + 1][1], win[w + 1][2]},
                               {win[w + 2][0], win[w + 2][1], win[w + 2][2]}};
          T out = T(0);
          const int kind = Tg[(rl + 1) * TBW + c + 16] & KIND_MASK;
          if (kind == K_FREE || kind == K_BODY)
            out = q4_row_nb<T, false, true>(nbh, cellf(c, rl), cellf(c - 1, rl), cellf(c - 1, rl - 1),
                                            cellf(c, rl - 1), nullptr, 0, 0, n, P, kplane<T>(m), m.Vtot, kr);
          y[n] = out;
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }
  __syncthreads();
  if (s_abort && tid == 0) {
    // only the last NS issued groups can still be in flight: wait for them (bounded)
    for (int k = max(0, s_issued - NS); k < s_issued; ++k) mbar_wait(&full[k % NS], (k / NS) & 1, poll_limit);
  }
  __syncthreads();
}

// collapsed body rows: one CTA per global body, fixed-order sum
template <typename T>
__global__ void __launch_bounds__(NT) k_body_sums(MeshDev m, const T* y, double* out) {
  __shared__ double scratch[NT / 32 + 1];
  const double s = body_gather<T>(m, blockIdx.x, y, scratch);
  if (linear_tid() == 0) out[blockIdx.x] = s;
}

// ---------------------------------------------------------------- host side
static MeshDev mesh_dev(const Batch& b) {
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

// Persistent schedule over a tile list: CTA c owns a contiguous range of tiles, cut into
// segments at variant boundaries.  With per-tile costs the ranges hold equal cost
// (tiles with stored coefficients move and compute more), else equal tile counts.
void make_schedule(Batch& b) {
  int dev = 0, nsm = 0;
  PF_CUDA(cudaGetDevice(&dev));
  PF_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  // refinement kernels: every variant gets the resident grid's share of CTAs, at least 64
  int oR32 = 0, oR64 = 0;
  PF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oR32, k_resid<float>, NT, 0));
  PF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&oR64, k_resid<double>, NT, 0));
  const int resident = nsm * std::max(1, std::min(oR32, oR64));
  b.rgx = std::max(64, resident / std::max(1, b.nv));
  b.rpart = (double*)dev_alloc(b, (size_t)b.nv * b.rgx * sizeof(double));
  b.rcounter = (int*)dev_alloc(b, (size_t)b.nv * sizeof(int));
  PF_CUDA(cudaMemsetAsync(b.rcounter, 0, (size_t)b.nv * sizeof(int), b.stream));
  b.nsm = nsm;
}

// Kernel instance of the fused CG step for a (precision, stages) configuration.
template <typename T, int NS>
static const void* cg_kernel() { return (const void*)k_cg<T, NS>; }

static int cg_smem(int precision, int ns) {
  if (precision == PF_FP64)
    return ns == 4 ? CgSmem<double, 4>::total : ns == 3 ? CgSmem<double, 3>::total : CgSmem<double, 2>::total;
  return ns == 4 ? CgSmem<float, 4>::total : ns == 3 ? CgSmem<float, 3>::total : CgSmem<float, 2>::total;
}

static const void* cg_func(int precision, int ns) {
  if (precision == PF_FP64)
    return ns == 4 ? cg_kernel<double, 4>() : ns == 3 ? cg_kernel<double, 3>() : cg_kernel<double, 2>();
  return ns == 4 ? cg_kernel<float, 4>() : ns == 3 ? cg_kernel<float, 3>() : cg_kernel<float, 2>();
}

// Cut points of the fused-CG schedule (contiguous tile ranges of equal estimated cost
// over the variants still marked active; tiles of finished variants count as free) and
// the segments they make at variant boundaries, written to the configuration's device
// arrays in place (graphs captured with these pointers stay valid).  The copies are
// ordered on the stream after the work already queued.
static void cg_sched_write(Batch& b, CgConfig& c) {
  const int G = c.G, T = (int)c.tile_cost.size();
  if ((int)c.active.size() != b.nv) c.active.assign(b.nv, 1);
  auto cost = [&](int t) { return c.active[c.tile_var[t]] ? c.tile_cost[t] : 0.0; };
  double total = 0.0;
  for (int t = 0; t < T; ++t) total += cost(t);
  c.cut.assign(G + 1, 0);
  int k = 0;
  double run = 0.0;
  for (int g = 0; g <= G; ++g) {
    const double target = total * g / G;
    while (k < T && run + 0.5 * cost(k) < target) run += cost(k++);
    c.cut[g] = (g == G) ? T : k;
  }
  c.h_cta_seg.assign(G + 1, 0);
  c.h_seg_var.clear();
  c.h_seg_t0.clear();
  c.h_seg_t1.clear();
  for (int g = 0; g < G; ++g) {
    c.h_cta_seg[g] = (int)c.h_seg_var.size();
    for (int t = c.cut[g]; t < c.cut[g + 1]; ++t) {
      const int v = c.tile_var[t];
      if (t == c.cut[g] || c.tile_var[t - 1] != v) {
        c.h_seg_var.push_back(v);
        c.h_seg_t0.push_back(t);
        c.h_seg_t1.push_back(t + 1);
      } else {
        c.h_seg_t1.back() = t + 1;
      }
    }
  }
  c.h_cta_seg[G] = (int)c.h_seg_var.size();
  const int S = (int)c.h_seg_var.size();
  if (S > G + b.nv) throw Error{PF_ECUDA, "internal: fused-CG schedule has too many segments"};
  c.h_vs0.assign(b.nv, 0);
  c.h_vs1.assign(b.nv, 0);
  std::vector<char> seen(b.nv, 0);
  for (int i = 0; i < S; ++i) {
    const int v = c.h_seg_var[i];
    if (!seen[v]) { c.h_vs0[v] = i; seen[v] = 1; }
    c.h_vs1[v] = i + 1;
  }
  // pageable sources: each call returns once its data is staged, so the host vectors
  // may change afterwards
  cudaStream_t s = b.stream;
  PF_CUDA(cudaMemcpyAsync(c.d_cta_seg, c.h_cta_seg.data(), (G + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  if (S > 0) {
    PF_CUDA(cudaMemcpyAsync(c.d_seg_var, c.h_seg_var.data(), S * sizeof(int), cudaMemcpyHostToDevice, s));
    PF_CUDA(cudaMemcpyAsync(c.d_seg_t0, c.h_seg_t0.data(), S * sizeof(int), cudaMemcpyHostToDevice, s));
    PF_CUDA(cudaMemcpyAsync(c.d_seg_t1, c.h_seg_t1.data(), S * sizeof(int), cudaMemcpyHostToDevice, s));
  }
  PF_CUDA(cudaMemcpyAsync(c.d_var_seg0, c.h_vs0.data(), b.nv * sizeof(int), cudaMemcpyHostToDevice, s));
  PF_CUDA(cudaMemcpyAsync(c.d_var_seg1, c.h_vs1.data(), b.nv * sizeof(int), cudaMemcpyHostToDevice, s));
}

// Re-balance rounds of the first tuned solve on a handle and launches timed per round
// (each CTA's tile-phase time is summed over the launches of a round); PFQ4_CG_TUNE_ROUNDS
// and PFQ4_CG_TUNE_LAUNCHES override them.
constexpr int CG_TUNE_ROUNDS = 4;
constexpr int CG_TUNE_LAUNCHES = 2;
static int env_int(const char* name, int dflt, int lo, int hi) {
  const char* e = getenv(name);
  if (!e) return dflt;
  const int v = atoi(e);
  return (v >= lo && v <= hi) ? v : dflt;
}

// Persistent grid (occupancy x SMs) and tile schedule of one CG configuration.  The
// first estimate of a tile's cost is a fit of measured per-CTA times of the
// five-cylinder workload on GB300: a fixed part, a part per node with an operator row
// and, for tiles that need stored coefficients, the extra coefficient boxes.
static CgConfig& cg_config(Batch& b, int precision, int ns) {
  CgConfig& c = b.cg_cfg[precision][ns - 2];
  if (c.ready) return c;
  const void* f = cg_func(precision, ns);
  const int smem = cg_smem(precision, ns);
  PF_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int occ = 0;
  PF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, NTC, smem));
  const long long T = b.Tcg;
  std::vector<uint8_t> gen(std::max<long long>(1, T));
  std::vector<int> act(std::max<long long>(1, T));
  PF_CUDA(cudaMemcpy(gen.data(), b.tile_cg_gen, T, cudaMemcpyDeviceToHost));
  PF_CUDA(cudaMemcpy(act.data(), b.tile_cg_act, T * sizeof(int), cudaMemcpyDeviceToHost));
  const int gbit = precision == PF_FP64 ? TILE_GEN64 : TILE_GEN32;
  const double w_gen = precision == PF_FP64 ? 0.6 : 1.47;
  c.tile_var.assign(T, 0);
  c.tile_cost.assign(T, 0.0);
  long long t = 0;
  for (int v = 0; v < b.nv; ++v) {
    const long long n = (long long)((b.hv[v].g.nx + 1 + CTX - 1) / CTX) * ((b.hv[v].g.ny + 1 + CTY - 1) / CTY);
    for (long long k = 0; k < n; ++k, ++t) {
      c.tile_var[t] = v;
      c.tile_cost[t] = 1.46 + 0.00042 * act[t] + ((gen[t] & gbit) ? w_gen : 0.0);
    }
  }
  c.G = (int)std::max<long long>(1, std::min<long long>((long long)b.nsm * std::max(1, occ), T));
  const int G = c.G, Smax = G + b.nv;
  c.d_cta_seg = (int*)dev_alloc(b, (G + 1) * sizeof(int));
  c.d_seg_var = (int*)dev_alloc(b, Smax * sizeof(int));
  c.d_seg_t0 = (int*)dev_alloc(b, Smax * sizeof(int));
  c.d_seg_t1 = (int*)dev_alloc(b, Smax * sizeof(int));
  c.d_var_seg0 = (int*)dev_alloc(b, b.nv * sizeof(int));
  c.d_var_seg1 = (int*)dev_alloc(b, b.nv * sizeof(int));
  c.d_cta_ns = (unsigned long long*)dev_alloc(b, G * sizeof(unsigned long long));
  int* counter = (int*)dev_alloc(b, b.nv * sizeof(int));
  PF_CUDA(cudaMemset(counter, 0, b.nv * sizeof(int)));
  Sched sc{};
  sc.cta_seg = c.d_cta_seg;
  sc.seg_var = c.d_seg_var;
  sc.seg_t0 = c.d_seg_t0;
  sc.seg_t1 = c.d_seg_t1;
  sc.var_seg0 = c.d_var_seg0;
  sc.var_seg1 = c.d_var_seg1;
  sc.counter = counter;
  sc.partial = (double*)dev_alloc(b, (size_t)Smax * 4 * sizeof(double));
  sc.n_cta = G;
  sc.tile_ij = b.tile_cg_ij;
  sc.cta_ns = nullptr;
  c.sc = sc;
  cg_sched_write(b, c);
  c.smem = smem;
  c.tune_rounds = 0;
  c.ready = true;
  return c;
}

// Re-balance from the measured tile-phase time of every CTA: the cost of each tile in
// CTA g's range is scaled by (time of g) / (estimated cost of g), then the cut points are
// recomputed.  This moves segment boundaries, so the dot products are summed in another
// order: results agree with an untuned solve to rounding, not bit for bit.
static void cg_rebalance(Batch& b, CgConfig& c, const std::vector<unsigned long long>& ns) {
  for (int g = 0; g < c.G; ++g) {
    double est = 0.0;
    for (int t = c.cut[g]; t < c.cut[g + 1]; ++t) est += c.tile_cost[t];
    if (est <= 0.0 || ns[g] == 0) continue;
    const double f = (double)ns[g] * 1e-3 / est;     // microseconds per unit of estimate
    for (int t = c.cut[g]; t < c.cut[g + 1]; ++t) c.tile_cost[t] *= f;
  }
  cg_sched_write(b, c);
}

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    PF_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q));
    if (q != cudaDriverEntryPointSuccess || !p) throw Error{PF_ECUDA, "cuTensorMapEncodeTiled is unavailable"};
    fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 2-D map over a [rows][P] array of elem_bytes elements, boxes of box_w x box_h.
static void encode_2d(CUtensorMap* map, void* base, CUtensorMapDataType dt, int elem_bytes, long long P,
                      long long rows, int box_w, int box_h) {
  const cuuint64_t dims[2] = {(cuuint64_t)P, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)P * elem_bytes};
  const cuuint32_t box[2] = {(cuuint32_t)box_w, (cuuint32_t)box_h};
  const cuuint32_t es[2] = {1, 1};
  const CUresult r = tensor_map_encoder()(map, dt, 2, base, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error{PF_ECUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")"};
}

template <typename T>
static void make_cg_maps(Batch& b, CgMaps& mp, State4<T>* const st[2], T* K) {
  using L = CgSmem<T>;
  const CUtensorMapDataType dt = sizeof(T) == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
  const int e = (int)sizeof(T);
  for (int k = 0; k < 2; ++k) {   // state records as a [rows][4 P] array, boxes of SHALF records
    encode_2d(&mp.s[k], st[k], dt, e, 4 * b.P, b.Rtot, 4 * L::SHALF, CTY + 2);
    encode_2d(&mp.s_thin[k], st[k], dt, e, 4 * b.P, b.Rtot, 4 * L::SHALF, L::THIN);
  }
  encode_2d(&mp.tag, b.tag, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, b.P, b.Rtot, L::TBW, CTY + 2);
  encode_2d(&mp.tag_thin, b.tag, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, b.P, b.Rtot, L::TBW, L::THIN);
  if (sizeof(T) == 4) {   // interleaved
    encode_2d(&mp.k, K, dt, e, 6 * b.P, b.Rtot, 6 * L::KHALF, CTY + 1);
    encode_2d(&mp.k_thin, K, dt, e, 6 * b.P, b.Rtot, 6 * L::KHALF, L::THIN);
  } else {
    encode_2d(&mp.k, K, dt, e, b.P, 6 * b.Rtot, L::KBW, CTY + 1);
    mp.k_thin = mp.k;   // the FP64 kernel reads its coefficients from the global planes
  }
}

void ensure_solver_memory(Batch& b, int precision) {
  const size_t V = (size_t)b.Vtot;
  const int B = std::max(1, b.B);
  if (!b.x64) {
    b.x64 = (double*)dev_alloc(b, V * sizeof(double));
    b.w64 = (double*)dev_alloc(b, V * sizeof(double));
    b.sol64 = (double*)dev_alloc(b, B * sizeof(double));
    b.sb64 = (double*)dev_alloc(b, 4 * B * sizeof(double));
    b.sb32 = (float*)dev_alloc(b, 4 * B * sizeof(float));
    b.sbr64 = (double*)dev_alloc(b, B * sizeof(double));
    b.state = (VarState*)dev_alloc(b, b.nv * sizeof(VarState));
    b.params = (SolveParams*)dev_alloc(b, sizeof(SolveParams));
    b.n_done = (int*)dev_alloc(b, 2 * sizeof(int));
    b.d_err = b.n_done + 1;
    b.d_sbuf = (void**)dev_alloc(b, 4 * sizeof(void*));
    PF_CUDA(cudaMemsetAsync(b.x64, 0, V * sizeof(double), b.stream));
    PF_CUDA(cudaMemsetAsync(b.sol64, 0, B * sizeof(double), b.stream));
    PF_CUDA(cudaMemsetAsync(b.sb64, 0, 4 * B * sizeof(double), b.stream));
    PF_CUDA(cudaMemsetAsync(b.sb32, 0, 4 * B * sizeof(float), b.stream));
    b.bnorm2_unit.assign(b.nv, -1.0);
    for (int k = 0; k < Batch::N_EV; ++k)
      if (!b.ev[k]) PF_CUDA(cudaEventCreate(&b.ev[k]));
  }
  if (precision == PF_FP64 && !b.st64[0]) {
    for (int k = 0; k < 2; ++k) b.st64[k] = (State4<double>*)dev_alloc(b, V * sizeof(State4<double>));
    make_cg_maps<double>(b, b.maps[0], b.st64, b.K64);
    PF_CUDA(cudaMemcpy(b.d_sbuf, b.st64, 2 * sizeof(void*), cudaMemcpyHostToDevice));
  }
  if (precision == PF_MIXED && !b.st32[0]) {
    for (int k = 0; k < 2; ++k) b.st32[k] = (State4<float>*)dev_alloc(b, V * sizeof(State4<float>));
    make_cg_maps<float>(b, b.maps[1], b.st32, b.K32i);
    PF_CUDA(cudaMemcpy(b.d_sbuf + 2, b.st32, 2 * sizeof(void*), cudaMemcpyHostToDevice));
  }
}

static std::vector<long long> logical_bases(const Batch& b) {
  std::vector<long long> lb(b.nv + 1, 0);
  for (int v = 0; v < b.nv; ++v) lb[v + 1] = lb[v] + (long long)(b.hv[v].g.nx + 1) * (b.hv[v].g.ny + 1);
  return lb;
}

long long* lbase_cached(Batch& b) {
  if (!b.d_lbase) {
    const std::vector<long long> h = logical_bases(b);
    b.d_lbase = (long long*)dev_alloc(b, h.size() * sizeof(long long));
    PF_CUDA(cudaMemcpyAsync(b.d_lbase, h.data(), h.size() * sizeof(long long), cudaMemcpyHostToDevice, b.stream));
  }
  return b.d_lbase;
}

static double* body_sum_scratch(Batch& b) {
  if (!b.d_bsum) b.d_bsum = (double*)dev_alloc(b, std::max(1, b.B) * sizeof(double));
  return b.d_bsum;
}

// The operator kernel reads p from the first scratch buffer of its precision through
// TMA descriptors made once here, and writes the second.
static void ensure_apply_buffers(Batch& b) {
  if (!b.ap64[0]) {
    for (int k = 0; k < 2; ++k) {
      b.ap64[k] = (double*)dev_alloc(b, b.Vtot * sizeof(double));
      b.ap32[k] = (float*)dev_alloc(b, b.Vtot * sizeof(float));
    }
    b.ap_err = (int*)dev_alloc(b, sizeof(int));
    PF_CUDA(cudaMemsetAsync(b.ap_err, 0, sizeof(int), b.stream));
    b.ap_ticket = (unsigned long long*)dev_alloc(b, sizeof(unsigned long long));
    PF_CUDA(cudaMemsetAsync(b.ap_ticket, 0, sizeof(unsigned long long), b.stream));
    b.ap_ticket_base = 0;
    refresh_apply_groups(b);
    using L64 = ApSmem<double, ApStages<double>::ns>;
    using L32 = ApSmem<float, ApStages<float>::ns>;
    encode_2d(&b.ap_maps[0].s[0], b.ap64[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 8, b.P, b.Rtot, L64::AW, L64::H);
    encode_2d(&b.ap_maps[0].tag, b.tag, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, b.P, b.Rtot, L64::TBW, L64::H);
    encode_2d(&b.ap_maps[1].s[0], b.ap32[0], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, b.P, b.Rtot, L32::AW, L32::H);
    encode_2d(&b.ap_maps[1].tag, b.tag, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, b.P, b.Rtot, L32::TBW, L32::H);
  }
}

// Work items of the operator kernel: up to AG consecutive tiles of one variant and tile
// row, with each tile's plain bits (written in place once the buffers exist; the tile
// flags change when node coordinates are replaced).
void refresh_apply_groups(Batch& b) {
  if (!b.ap64[0]) return;                 // made with the operator buffers on first use
  const long long T = b.Tcg;
  std::vector<int2> ij(T);
  std::vector<int> var(T);
  std::vector<uint8_t> fl(T);
  PF_CUDA(cudaMemcpyAsync(ij.data(), b.tile_cg_ij, T * sizeof(int2), cudaMemcpyDeviceToHost, b.stream));
  PF_CUDA(cudaMemcpyAsync(var.data(), b.tile_cg_var, T * sizeof(int), cudaMemcpyDeviceToHost, b.stream));
  PF_CUDA(cudaMemcpyAsync(fl.data(), b.tile_cg_gen, T, cudaMemcpyDeviceToHost, b.stream));
  PF_CUDA(cudaStreamSynchronize(b.stream));
  // groups run along tile rows: visit the tiles row-major within each variant (the list
  // itself is column-major per variant)
  std::vector<long long> ord(T);
  for (long long t = 0; t < T; ++t) ord[t] = t;
  std::stable_sort(ord.begin(), ord.end(), [&](long long a, long long c) {
    if (var[a] != var[c]) return var[a] < var[c];
    if (ij[a].y != ij[c].y) return ij[a].y < ij[c].y;
    return ij[a].x < ij[c].x;
  });
  std::vector<int4> gr;
  for (long long q = 0; q < T;) {
    const long long t = ord[q];
    int g = 1;
    while (g < AG && q + g < T && var[ord[q + g]] == var[t] && ij[ord[q + g]].y == ij[t].y) ++g;
    int pl32 = 0, pl64 = 0;
    for (int k = 0; k < g; ++k) {
      pl32 |= ((fl[ord[q + k]] & TILE_PLAIN32) != 0) << k;
      pl64 |= ((fl[ord[q + k]] & TILE_PLAIN64) != 0) << k;
    }
    if (ij[t].x >= (1 << 20)) throw Error{PF_EINVAL, "grid too wide for the operator kernel (nx >= 2^20)"};
    const HostVariant& H = b.hv[var[t]];
    const int row0 = (int)(H.base / H.P);
    gr.push_back(make_int4(ij[t].x | (g << 20) | (pl32 << 24) | (pl64 << 28), ij[t].y, var[t], row0 + ij[t].y));
    q += g;
  }
  if (!b.ap_groups) {
    b.ap_ngroups = (long long)gr.size();
    b.ap_groups = (int4*)dev_alloc(b, std::max<size_t>(1, gr.size()) * sizeof(int4));
  }
  // pageable source: the call returns once the data is staged
  PF_CUDA(cudaMemcpyAsync(b.ap_groups, gr.data(), gr.size() * sizeof(int4), cudaMemcpyHostToDevice, b.stream));
  PF_CUDA(cudaStreamSynchronize(b.stream));
}

// y = A p with p in the first scratch buffer of T's precision (persistent grid: SMs x
// resident CTAs, at most one CTA per work item).
template <typename T>
static void launch_apply(Batch& b, const MeshDev& m, T* y) {
  constexpr int NS = ApStages<T>::ns;
  using L = ApSmem<T, NS>;
  const int k = sizeof(T) == 8 ? 0 : 1;
  if (!b.ap_G[k]) {
    const void* f = (const void*)k_apply<T, NS>;
    PF_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, L::total));
    int occ = 0;
    PF_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, f, NTC, L::total));
    b.ap_G[k] = (int)std::max<long long>(1, std::min<long long>((long long)b.nsm * std::max(1, occ), b.ap_ngroups));
  }
  k_apply<T, NS><<<b.ap_G[k], dim3(TX, NTC / TX), L::total, b.stream>>>(
      m, b.ap_groups, b.ap_ngroups, b.ap_ticket, b.ap_ticket_base, y, b.ap_maps[k], b.ap_err, MBAR_POLL_LIMIT);
  b.ap_ticket_base += (unsigned long long)b.ap_ngroups + (unsigned long long)b.ap_G[k];
}

// After the stream has been synchronised: did a bounded wait of the operator kernel give up?
static void check_apply_err(Batch& b) {
  int e = 0;
  PF_CUDA(cudaMemcpyAsync(&e, b.ap_err, sizeof(int), cudaMemcpyDeviceToHost, b.stream));
  PF_CUDA(cudaStreamSynchronize(b.stream));
  if (e) {
    // a CTA that stopped early took fewer tickets: restart the count
    PF_CUDA(cudaMemsetAsync(b.ap_err, 0, sizeof(int), b.stream));
    PF_CUDA(cudaMemsetAsync(b.ap_ticket, 0, sizeof(unsigned long long), b.stream));
    b.ap_ticket_base = 0;
    throw Error{PF_ETIMEOUT, "a bounded wait in the operator kernel gave up (TMA tile not delivered)"};
  }
}

// Mean time of `reps` back-to-back stand-alone operator applications on the handle's
// padded vectors (no layout conversion, no body sums) and their algorithmic bytes: p
// read and y written at every node, one tag byte per node and the six stored
// coefficients of every cell whose coefficients differ from the rectangle's in this
// precision.
void apply_timing(Batch& b, int precision, int reps, double* us, double* bytes) {
  if (reps < 1) throw Error{PF_EINVAL, "reps must be >= 1"};
  ensure_apply_buffers(b);
  for (int k = 0; k < 2; ++k)
    if (!b.ev[k]) PF_CUDA(cudaEventCreate(&b.ev[k]));
  const MeshDev m = mesh_dev(b);
  const size_t es = precision == PF_FP64 ? sizeof(double) : sizeof(float);
  PF_CUDA(cudaMemsetAsync(precision == PF_FP64 ? (void*)b.ap64[0] : (void*)b.ap32[0], 0, b.Vtot * es, b.stream));
  auto launch = [&]() {
    if (precision == PF_FP64) launch_apply<double>(b, m, b.ap64[1]);
    else launch_apply<float>(b, m, b.ap32[1]);
  };
  for (int k = 0; k < 3; ++k) launch();      // warm-up
  PF_CUDA(cudaEventRecord(b.ev[0], b.stream));
  for (int k = 0; k < reps; ++k) launch();
  PF_CUDA(cudaEventRecord(b.ev[1], b.stream));
  PF_CUDA(cudaGetLastError());
  PF_CUDA(cudaEventSynchronize(b.ev[1]));
  float ms = 0;
  PF_CUDA(cudaEventElapsedTime(&ms, b.ev[0], b.ev[1]));
  check_apply_err(b);
  b.launches += 3 + reps;
  double by = 0.0;
  for (const HostVariant& H : b.hv) {
    const long long ng = precision == PF_FP64 ? H.stats.n_general_cells : H.n_gen32_cells;
    by += (2.0 * es + 1.0) * (double)H.stats.n_nodes + 6.0 * es * (double)ng;
  }
  if (us) *us = 1e3 * ms / reps;
  if (bytes) *bytes = by;
}

void apply_operator(Batch& b, int precision, const double* dev_p, double* dev_y, double* body_sums) {
  ensure_apply_buffers(b);
  long long* lb = lbase_cached(b);
  const MeshDev m = mesh_dev(b);
  const dim3 g2(512, b.nv);
  double* sums = body_sum_scratch(b);
  if (precision == PF_FP64) {
    k_to_padded<double><<<g2, 256, 0, b.stream>>>(b.d_var, lb, dev_p, b.ap64[0]);
    PF_CUDA(cudaMemsetAsync(b.ap64[1], 0, b.Vtot * sizeof(double), b.stream));
    launch_apply<double>(b, m, b.ap64[1]);
    k_from_padded<double><<<g2, 256, 0, b.stream>>>(b.d_var, lb, b.ap64[1], dev_y);
    if (b.B) k_body_sums<double><<<b.B, dim3(TX, TY), 0, b.stream>>>(m, b.ap64[1], sums);
  } else {
    k_to_padded<float><<<g2, 256, 0, b.stream>>>(b.d_var, lb, dev_p, b.ap32[0]);
    PF_CUDA(cudaMemsetAsync(b.ap32[1], 0, b.Vtot * sizeof(float), b.stream));
    launch_apply<float>(b, m, b.ap32[1]);
    k_from_padded<float><<<g2, 256, 0, b.stream>>>(b.d_var, lb, b.ap32[1], dev_y);
    if (b.B) k_body_sums<float><<<b.B, dim3(TX, TY), 0, b.stream>>>(m, b.ap32[1], sums);
  }
  PF_CUDA(cudaGetLastError());
  if (body_sums && b.B) {
    PF_CUDA(cudaMemcpyAsync(body_sums, sums, b.B * sizeof(double), cudaMemcpyDeviceToHost, b.stream));
  }
  PF_CUDA(cudaStreamSynchronize(b.stream));
  check_apply_err(b);
}

template <typename T>
static void fill_cg_args(Batch& b, CGArgs<T>& a, State4<T>* const st[2], T* sb, const Sched& sc) {
  a.m = mesh_dev(b);
  a.sc = sc;
  a.tile_gen = b.tile_cg_gen;
  a.Rtot = b.Rtot;
  a.err = b.d_err;
  a.st = b.state;
  a.prm = b.params;
  a.s[0] = st[0];
  a.s[1] = st[1];
  a.sb = sb;
  a.bq = b.bq;
  a.B = std::max(1, b.B);
  a.n_done = b.n_done;
  a.poll_limit = b.test_drop ? 1024 : MBAR_POLL_LIMIT;
  a.test_drop = b.test_drop;
}

template <typename T>
static void fill_resid_args(Batch& b, ResidArgs<T>& a, State4<T>* const st[2], T* sb, int mixed) {
  a.m = mesh_dev(b);
  a.gx = b.rgx;
  a.rpart = b.rpart;
  a.counter = b.rcounter;
  a.st = b.state;
  a.prm = b.params;
  a.x64 = b.x64;
  a.w64 = b.w64;
  a.s[0] = st[0];
  a.s[1] = st[1];
  a.sol = b.sol64;
  a.sb = sb;
  a.sbr = b.sbr64;
  a.rhsb = b.rhs_active ? b.d_rhsb : nullptr;
  a.B = std::max(1, b.B);
  a.mixed = mixed;
  a.n_done = b.n_done;
  a.rplane = b.pcg_active ? b.mg_r : nullptr;
}

// the k_cg launches of one chunk (captured once as a graph); timed launches record
// every CTA's tile-phase time for the schedule re-balance
static void launch_cg_chunk(Batch& b, int precision, int chunk, cudaStream_t s, bool timed = false) {
  const dim3 blk(TX, NTC / TX);
  const int ns = b.cg_stages;
  CgConfig& c = cg_config(b, precision, ns);
  Sched sc = c.sc;
  if (timed) sc.cta_ns = c.d_cta_ns;
  if (precision == PF_FP64) {
    CGArgs<double> a;
    fill_cg_args<double>(b, a, b.st64, b.sb64, sc);
    for (int k = 0; k < chunk; ++k) {
      if (ns == 4) k_cg<double, 4><<<c.G, blk, c.smem, s>>>(a, b.maps[0]);
      else if (ns == 3) k_cg<double, 3><<<c.G, blk, c.smem, s>>>(a, b.maps[0]);
      else k_cg<double, 2><<<c.G, blk, c.smem, s>>>(a, b.maps[0]);
    }
  } else {
    CGArgs<float> a;
    fill_cg_args<float>(b, a, b.st32, b.sb32, sc);
    for (int k = 0; k < chunk; ++k) {
      if (ns == 4) k_cg<float, 4><<<c.G, blk, c.smem, s>>>(a, b.maps[1]);
      else if (ns == 3) k_cg<float, 3><<<c.G, blk, c.smem, s>>>(a, b.maps[1]);
      else k_cg<float, 2><<<c.G, blk, c.smem, s>>>(a, b.maps[1]);
    }
  }
  PF_CUDA(cudaGetLastError());
}

static void launch_resid_only(Batch& b, int precision, cudaStream_t s) {
  const dim3 blk(TX, TY);
  const dim3 rg(b.rgx, b.nv);
  if (precision == PF_FP64) {
    k_fold<double><<<rg, blk, 0, s>>>(b.d_var, b.rgx, b.tag, b.state, b.x64, (State4<double>* const*)b.d_sbuf,
                                      nullptr);
    ResidArgs<double> ra;
    fill_resid_args<double>(b, ra, b.st64, b.sb64, 0);
    k_resid<double><<<rg, blk, 0, s>>>(ra);
  } else {
    k_fold<float><<<rg, blk, 0, s>>>(b.d_var, b.rgx, b.tag, b.state, b.x64, (State4<float>* const*)(b.d_sbuf + 2),
                                     b.pcg_active ? b.mg_x : nullptr);
    ResidArgs<float> ra;
    fill_resid_args<float>(b, ra, b.st32, b.sb32, 1);
    k_resid<float><<<rg, blk, 0, s>>>(ra);
  }
  PF_CUDA(cudaGetLastError());
}

static cudaGraphExec_t get_graph(Batch& b, int precision, int chunk) {
  if (b.graph[precision] && b.graph_chunk[precision] == chunk && b.graph_stages[precision] == b.cg_stages &&
      b.graph_drop[precision] == b.test_drop)
    return b.graph[precision];
  b.graph_stages[precision] = b.cg_stages;
  b.graph_drop[precision] = b.test_drop;
  cg_config(b, precision, b.cg_stages);   // schedule set-up synchronises: do it before capturing
  if (b.graph[precision]) {
    cudaGraphExecDestroy(b.graph[precision]);
    b.graph[precision] = nullptr;
  }
  cudaStream_t cs;
  PF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g;
  PF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  launch_cg_chunk(b, precision, chunk, cs);
  PF_CUDA(cudaStreamEndCapture(cs, &g));
  cudaGraphExec_t ex;
  PF_CUDA(cudaGraphInstantiate(&ex, g, 0));
  PF_CUDA(cudaGraphDestroy(g));
  PF_CUDA(cudaStreamDestroy(cs));
  b.graph[precision] = ex;
  b.graph_chunk[precision] = chunk;
  return ex;
}

// Iterations per captured graph of the preconditioned CG (each about 40 kernels).
constexpr int PCG_CHUNK = 4;

static int pcg_launches_per_iter(const Batch& b) {
  int n = 8 + (b.B > 0 ? 1 : 0);                // fine level, finalisers, the forward body step
  for (int l = 1; l < b.mg_L; ++l)
    if (b.mg[l].nblk > 0) n += 2 + (l <= b.mg_L - 2 ? 2 : 0);
  return n;
}

static cudaGraphExec_t get_pcg_graph(Batch& b, int chunk) {
  if (b.graph_pcg && b.graph_pcg_chunk == chunk) return b.graph_pcg;
  if (b.graph_pcg) {
    cudaGraphExecDestroy(b.graph_pcg);
    b.graph_pcg = nullptr;
  }
  cudaStream_t cs;
  PF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g;
  PF_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  launch_pcg_chunk(b, chunk, cs);
  PF_CUDA(cudaStreamEndCapture(cs, &g));
  cudaGraphExec_t ex;
  PF_CUDA(cudaGraphInstantiate(&ex, g, 0));
  PF_CUDA(cudaGraphDestroy(g));
  PF_CUDA(cudaStreamDestroy(cs));
  b.graph_pcg = ex;
  b.graph_pcg_chunk = chunk;
  return ex;
}

pf_status psi_solve(Batch& b, double U, const pf_solve_opts& o, double* dev_psi, double* body_psi,
                    pf_solve_info* info) {
  if (o.k_max < 1) throw Error{PF_EINVAL, "k_max must be >= 1"};
  // a Kutta condition replaces a body's symmetric equation: only the Schur form takes it
  if (b.has_kutta) return schur_solve(b, U, o, dev_psi, body_psi, info);
  b.rhs_active = false;
  b.fixed_bodies = false;
  b.Uv_active = false;
  return solve_core(b, U, o, dev_psi, body_psi, info, true);
}

// The solve proper.  With b.rhs_active the body rows carry the extra right-hand side
// b.d_rhsb (used by the adjoint); record_bnorm stores ||b||^2 at U = 1 for later warm starts.
pf_status solve_core(Batch& b, double U, const pf_solve_opts& o, double* dev_psi, double* body_psi,
                     pf_solve_info* info, bool record_bnorm) {
  if (!b.valid) throw Error{PF_EMESH_INVALID, "mesh has det J <= 0 at a Gauss point; solve refused"};
  if (o.precision != PF_FP64 && o.precision != PF_MIXED) throw Error{PF_EINVAL, "invalid precision"};
  if (!(o.tol > 0) || o.k_max < 0 || !std::isfinite(U)) throw Error{PF_EINVAL, "invalid tol, k_max or U"};
  if (o.criterion != PF_TOL_REL_TRUE && o.criterion != PF_TOL_PAPER_ABS)
    throw Error{PF_EINVAL, "invalid stopping criterion"};
  const int prec = o.precision;
  if (o.preconditioner != PF_PRECOND_NONE && o.preconditioner != PF_PRECOND_MG)
    throw Error{PF_EINVAL, "invalid preconditioner"};
  const bool pcg = o.preconditioner == PF_PRECOND_MG;
  if (pcg && prec != PF_MIXED) throw Error{PF_EINVAL, "the multigrid-preconditioned CG runs in PF_MIXED precision"};
  if (!b.rhs_active) b.last_precond = o.preconditioner;
  ensure_solver_memory(b, prec);
  // the preconditioned path is active for this solve only (also when it throws)
  struct PcgScope {
    Batch& b;
    ~PcgScope() { b.pcg_active = false; }
  } pcg_scope{b};
  b.pcg_active = pcg;
  PF_CUDA(cudaEventRecord(b.ev[3], b.stream));   // the solve's device time starts here, set-up included
  if (pcg) {
    mg_setup(b);
    for (float* f : {b.mg_x, b.mg_p[0], b.mg_p[1], b.mg_q, b.mg_r})
      PF_CUDA(cudaMemsetAsync(f, 0, b.Vtot * sizeof(float), b.stream));
  }
  {
    const char* e = getenv("PFQ4_CG_STAGES");      // a fixed pipeline depth, else the tuned one
    const int ns = e ? atoi(e) : b.tuned_stages[prec];
    b.cg_stages = (ns >= 2 && ns <= 4) ? ns : 2;
    const char* tu = getenv("PFQ4_CG_TUNE");   // overrides the option when set
    b.cg_tune = tu ? atoi(tu) != 0 : o.tune_schedule != 0;
  }
  cudaStream_t s = b.stream;
  SolveParams sp{};
  sp.tol2 = o.tol * o.tol;
  sp.tol_abs = o.tol;
  sp.paper_abs = o.criterion == PF_TOL_PAPER_ABS ? 1 : 0;
  const double itol = o.inner_tol > 0 ? o.inner_tol : PF_DEFAULT_INNER_TOL;
  sp.inner_rel2 = itol * itol;
  sp.k_max = o.k_max;
  sp.mixed = prec == PF_MIXED;
  sp.fixed_bodies = b.fixed_bodies ? 1 : 0;
  PF_CUDA(cudaMemcpyAsync(b.params, &sp, sizeof(sp), cudaMemcpyHostToDevice, s));
  const bool warm = o.warm_start && b.solved;
  std::vector<VarState> st(b.nv);
  for (int v = 0; v < b.nv; ++v) {
    VarState& S = st[v];
    memset(&S, 0, sizeof(S));
    S.phase = PH_RESID;
    S.status = PF_OK;
    S.bnorm2 = (record_bnorm && b.bnorm2_unit[v] >= 0.0) ? b.bnorm2_unit[v] * U * U : -1.0;
  }
  PF_CUDA(cudaMemcpyAsync(b.state, st.data(), b.nv * sizeof(VarState), cudaMemcpyHostToDevice, s));
  PF_CUDA(cudaMemsetAsync(b.n_done, 0, 2 * sizeof(int), s));
  const int B = std::max(1, b.B);
  if (!warm && !b.fixed_bodies) PF_CUDA(cudaMemsetAsync(b.sol64, 0, B * sizeof(double), s));
  PF_CUDA(cudaMemsetAsync(b.sb64, 0, 4 * B * sizeof(double), s));
  PF_CUDA(cudaMemsetAsync(b.sb32, 0, 4 * B * sizeof(float), s));
  for (int k = 0; k < 2; ++k) {
    if (prec == PF_FP64) PF_CUDA(cudaMemsetAsync(b.st64[k], 0, b.Vtot * sizeof(State4<double>), s));
    else PF_CUDA(cudaMemsetAsync(b.st32[k], 0, b.Vtot * sizeof(State4<float>), s));
  }
  const int n_slots = b.h_body_ptr.empty() ? 0 : b.h_body_ptr[b.B];
  if (n_slots > 0) {
    const unsigned g = (unsigned)((n_slots + 255) / 256);
    if (prec == PF_FP64) k_seed_slots<double><<<g, 256, 0, s>>>(b.body_nodes, n_slots, b.st64[0], b.st64[1]);
    else k_seed_slots<float><<<g, 256, 0, s>>>(b.body_nodes, n_slots, b.st32[0], b.st32[1]);
  }
  k_init<<<(unsigned)b.T, dim3(TX, TY), 0, s>>>(b.d_var, b.tile_var, b.tile_ij, b.tag,
                                                b.X + (b.dirichlet_x ? 0 : b.Vtot), U,
                                                b.Uv_active ? b.d_Uv : nullptr, warm, b.x64, b.w64);
  PF_CUDA(cudaGetLastError());
  launch_resid_only(b, prec, s);
  int chunk = o.chunk > 0 ? o.chunk : 0;
  if (pcg && chunk == 0) chunk = PCG_CHUNK;
  if (chunk == 0) {
    long long nodes = 0;
    for (auto& H : b.hv) nodes += H.stats.n_nodes;
    chunk = nodes > (8LL << 20) ? 16 : (nodes > (1LL << 20) ? 64 : 256);
  }
  if (!b.h_poll) PF_CUDA(cudaMallocHost(&b.h_poll, 4 * sizeof(int)));
  int* hdone = b.h_poll;
  double cg_ms = 0, res_ms = 0;
  long long launches = 0, rlaunches = 1;
  // Optional autotuning on the first tuned solve of the handle, with this solve's own CG
  // iterations run as timed launches: (1) the pipeline depth NS in {2, 3, 4} with the
  // shortest launch (each configuration has its own grid and schedule), then (2) a
  // re-balance of that configuration's cut points so that every CTA's measured tile
  // time evens out.
  auto timed_launches = [&](int n, bool per_cta) {
    PF_CUDA(cudaEventRecord(b.ev[0], s));
    launch_cg_chunk(b, prec, n, s, per_cta);
    PF_CUDA(cudaEventRecord(b.ev[1], s));
    PF_CUDA(cudaMemcpyAsync(hdone, b.n_done, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaStreamSynchronize(s));
    float ms = 0;
    PF_CUDA(cudaEventElapsedTime(&ms, b.ev[0], b.ev[1]));
    cg_ms += ms;
    launches += n;
    if (hdone[1]) throw Error{PF_ETIMEOUT, "a bounded wait in the CG kernel gave up (TMA tile not delivered)"};
    return (double)ms / n;
  };
  const bool tune = b.cg_tune && o.k_max > 0 && !getenv("PFQ4_CG_STAGES") && !pcg;
  if (tune && !b.stages_tuned[prec]) {
    double best = 1e300;
    int best_ns = b.cg_stages;
    for (int ns = 2; ns <= 4; ++ns) {
      b.cg_stages = ns;
      CgConfig& c = cg_config(b, prec, ns);
      c.active.assign(b.nv, 1);
      cg_sched_write(b, c);
      const double per = timed_launches(CG_TUNE_LAUNCHES, false);
      if (per < best) { best = per; best_ns = ns; }
    }
    b.cg_stages = best_ns;
    b.tuned_stages[prec] = best_ns;
    b.stages_tuned[prec] = true;
  }
  cudaGraphExec_t ex = pcg ? get_pcg_graph(b, chunk) : get_graph(b, prec, chunk);
  CgConfig& cc = cg_config(b, prec, b.cg_stages);
  if (!pcg &&
      (cc.active.size() != (size_t)b.nv || std::find(cc.active.begin(), cc.active.end(), 0) != cc.active.end())) {
    cc.active.assign(b.nv, 1);                   // a solve starts with every variant running
    cg_sched_write(b, cc);
  }
  if (!pcg && b.cg_tune && o.k_max > 0 && (long long)cc.tile_cost.size() >= 2LL * cc.G) {
    const int rounds = env_int("PFQ4_CG_TUNE_ROUNDS", CG_TUNE_ROUNDS, 0, 16);
    const int per_round = env_int("PFQ4_CG_TUNE_LAUNCHES", CG_TUNE_LAUNCHES, 1, 16);
    for (; cc.tune_rounds < rounds; ++cc.tune_rounds) {
      PF_CUDA(cudaMemsetAsync(cc.d_cta_ns, 0, cc.G * sizeof(unsigned long long), s));
      timed_launches(per_round, true);
      std::vector<unsigned long long> tns(cc.G);
      PF_CUDA(cudaMemcpy(tns.data(), cc.d_cta_ns, cc.G * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
      cg_rebalance(b, cc, tns);
    }
  }
  // k_max == 0 (internal use): only the initial residual, which measures ||b||
  const long long max_chunks = o.k_max == 0 ? 0 : o.k_max / chunk + 1000;
  // Chunks are queued two ahead of the host: slot k holds events (start, after the CG
  // graph, after the refinement kernels) and the pinned poll words / variant states
  // copied after it.  The host retires a slot by waiting on its last event.
  constexpr int SLOTS = 2;
  if (!b.h_vs) PF_CUDA(cudaMallocHost(&b.h_vs, SLOTS * std::max(1, b.nv) * sizeof(VarState)));
  auto cost_of_active = [&](const std::vector<char>& act) {
    double x = 0.0;
    for (size_t t = 0; t < cc.tile_cost.size(); ++t) x += act[cc.tile_var[t]] ? cc.tile_cost[t] : 0.0;
    return x;
  };
  double active_cost = cost_of_active(cc.active);   // estimated cost the schedule is balanced over
  auto issue = [&](long long c) {
    const int k = (int)(c % SLOTS);
    PF_CUDA(cudaEventRecord(b.ev[6 + 3 * k], s));
    PF_CUDA(cudaGraphLaunch(ex, s));
    PF_CUDA(cudaEventRecord(b.ev[7 + 3 * k], s));
    launch_resid_only(b, prec, s);
    PF_CUDA(cudaMemcpyAsync(hdone + 2 * k, b.n_done, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaMemcpyAsync(b.h_vs + (size_t)k * b.nv, b.state, b.nv * sizeof(VarState), cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaEventRecord(b.ev[8 + 3 * k], s));
  };
  bool finished = false;
  auto retire = [&](long long c) {
    const int k = (int)(c % SLOTS);
    PF_CUDA(cudaEventSynchronize(b.ev[8 + 3 * k]));
    float ms1 = 0, ms2 = 0;
    PF_CUDA(cudaEventElapsedTime(&ms1, b.ev[6 + 3 * k], b.ev[7 + 3 * k]));
    PF_CUDA(cudaEventElapsedTime(&ms2, b.ev[7 + 3 * k], b.ev[8 + 3 * k]));
    cg_ms += ms1;
    res_ms += ms2;
    launches += chunk;
    rlaunches += 1;
    if (hdone[2 * k + 1]) throw Error{PF_ETIMEOUT, "a bounded wait in the CG kernel gave up (TMA tile not delivered)"};
    if (hdone[2 * k] >= b.nv) {
      finished = true;
      return;
    }
    if (pcg) return;                             // its kernels take every variant's tiles each launch
    // spread the grid over the variants still running once enough work has finished
    std::vector<char> act(b.nv);
    for (int v = 0; v < b.nv; ++v) act[v] = b.h_vs[(size_t)k * b.nv + v].phase != PH_DONE;
    const double now = cost_of_active(act);
    if (now < 0.9 * active_cost) {
      cc.active = act;
      cg_sched_write(b, cc);
      active_cost = now;
    }
  };
  long long issued = 0, retired = 0;
  while (!finished && issued < max_chunks) {
    issue(issued++);
    if (issued - retired >= SLOTS) retire(retired++);
  }
  while (retired < issued) {
    // chunks queued after the last variant finished run as no-ops; account for them
    if (finished) {
      const int k = (int)(retired % SLOTS);
      PF_CUDA(cudaEventSynchronize(b.ev[8 + 3 * k]));
      ++retired;
      continue;
    }
    retire(retired++);
  }
  PF_CUDA(cudaEventRecord(b.ev[4], s));
  // kernels launched: k_init, slot seeding, the tuning launches and every queued chunk
  // (CG graph + fold + residual), no-op chunks after the last variant finished included
  const long long tuned_launches = launches - (long long)(rlaunches - 1) * chunk;
  b.launches += 1 + (n_slots > 0 ? 1 : 0) + tuned_launches + issued * chunk * (pcg ? pcg_launches_per_iter(b) : 1) +
                (1 + issued) * 2;
  std::vector<VarState> fin(b.nv);
  PF_CUDA(cudaMemcpyAsync(fin.data(), b.state, b.nv * sizeof(VarState), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  float tot = 0;
  PF_CUDA(cudaEventElapsedTime(&tot, b.ev[3], b.ev[4]));
  b.solved = true;
  b.lastU = U;
  b.last_precision = prec;
  pf_status ret = PF_OK;
  double bytes_done = 0.0;
  for (int v = 0; v < b.nv; ++v) {
    const VarState& S = fin[v];
    const pf_mesh_stats& M = b.hv[v].stats;
    if (S.phase != PH_DONE && ret == PF_OK) ret = PF_ENOT_CONVERGED;
    if (S.status != PF_OK && ret == PF_OK) ret = S.status;
    if (record_bnorm && b.bnorm2_unit[v] < 0 && S.bnorm2 >= 0 && U != 0 && !warm) b.bnorm2_unit[v] = S.bnorm2 / (U * U);
    const double per_node_free = prec == PF_MIXED ? 32.0 : 64.0;
    const double per_body = prec == PF_MIXED ? 20.0 : 36.0;
    const double per_gen = prec == PF_MIXED ? 24.0 : 48.0;
    // coefficient bytes: the cells whose stored K_e the operator of this precision reads
    const long long n_gen = prec == PF_MIXED ? b.hv[v].n_gen32_cells : M.n_general_cells;
    const double bv = per_node_free * M.n_free + per_body * M.n_body_nodes + 1.0 * M.n_nodes + per_gen * n_gen;
    if (!pcg) bytes_done += bv * (double)S.iters;
    if (info) {
      info[v].iters = S.iters;
      info[v].refinements = std::max(0, S.n_resid - 1);
      info[v].status = S.phase == PH_DONE ? S.status : PF_ENOT_CONVERGED;
      info[v].rel_true_residual = S.bnorm2 > 0 ? std::sqrt(S.rr64 / S.bnorm2) : 0.0;
      info[v].n_dof = M.n_dof;
    }
  }
  b.timing.cg_kernel_ms = cg_ms;
  b.timing.cg_launches = launches;
  b.timing.residual_kernel_ms = res_ms;
  b.timing.residual_launches = rlaunches;
  b.timing.solve_ms = tot;
  b.timing.cg_bytes_per_launch = launches > 0 ? bytes_done / (double)launches : 0.0;
  if (dev_psi) export_psi(b, dev_psi);
  if (body_psi && b.B) {
    PF_CUDA(cudaMemcpyAsync(body_psi, b.sol64, b.B * sizeof(double), cudaMemcpyDeviceToHost, s));
    PF_CUDA(cudaStreamSynchronize(s));
  }
  return ret;
}

void export_psi(Batch& b, double* dev_psi) {
  long long* lb = lbase_cached(b);
  b.launches += 1;
  k_export_psi<<<dim3(256, b.nv), 256, 0, b.stream>>>(b.d_var, b.nv, lb, b.tag, b.bid, b.x64, b.sol64, dev_psi);
  PF_CUDA(cudaGetLastError());
}

void body_values(Batch& b, std::vector<double>& C) {
  C.assign(b.B, 0.0);
  if (!b.B || !b.sol64) return;
  PF_CUDA(cudaMemcpyAsync(C.data(), b.sol64, b.B * sizeof(double), cudaMemcpyDeviceToHost, b.stream));
  PF_CUDA(cudaStreamSynchronize(b.stream));
}

}  // namespace pfq4
