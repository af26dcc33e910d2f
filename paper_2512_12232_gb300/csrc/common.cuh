// Shared definitions of the GB300 matrix-free Q4 solver library.
//
// Data layout (HBM): every variant's nodes live in padded row-major planes,
// node (i, j) at base + j*P + i with the row pitch P = round_up(nx+1, 32) so that
// every row starts on a 128-byte boundary.  Cells are stored at the index of their
// corner 0 (i, j).  Columns nx+1 .. P-1 are padding (tag INACTIVE, values 0) and are
// never read as neighbours: tile loaders bounds-check against (nx, ny).
//
// Two tilings of every variant (variant-major lists, row-major inside a variant):
// 32 x 8 nodes (mesh build and the FP64 refinement kernels, one 256-thread CTA pass
// per tile) and 64 x 16 nodes (the fused CG step, the smoothing sweeps and the
// stand-alone operator).  Row-major order keeps the 256-byte L2 lines a tile's boxes
// touch beyond its own columns in use by the next tile (a column-major walk measured
// 3-4% slower fused CG launches).  The
// fused CG step runs a persistent grid: CTA b owns a contiguous range of the 64 x 16
// list, cut into "segments" at variant boundaries.  The refinement kernels run one
// grid row per variant, each CTA a fixed share of the variant's tiles.  Either way
// partial sums are written to fixed slots and summed in a fixed order by the last CTA
// to finish a variant, so every reduction is deterministic.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pfq4.h"

namespace pfq4 {

constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NT = TX * TY;          // threads per CTA
constexpr int SW = TX + 2;           // shared tile row width with halo
constexpr int NHALO = 2 * SW + 2 * TY;
constexpr int MAXB = 64;             // bodies per variant
constexpr int CTX = 64;              // fused-CG tile: 64 x 16 nodes, a 4-node vertical strip per thread
constexpr int CTY = 16;

// node tag byte
constexpr uint8_t KIND_MASK = 3;
constexpr uint8_t K_FREE = PF_NODE_FREE, K_DIR = PF_NODE_DIRICHLET, K_BODY = PF_NODE_BODY,
                  K_INACT = PF_NODE_INACTIVE;
constexpr uint8_t CELL_ACTIVE = 4;   // cell (i, j) whose corner 0 is this node is active
constexpr uint8_t CELL_GENERAL = 8;  // ... and has a displaced corner: stored K_e is used
constexpr uint8_t DISPLACED = 16;    // node moved by the mesh generator (d != 0)
constexpr uint8_t RING = 32;         // node on the outer boundary of the box
constexpr uint8_t CELL_GEN32 = 64;   // general cell whose FP32 coefficients differ from the FP32
                                     // rectangle constants (the FP32 operator needs stored K_e)
constexpr uint8_t WAKE = 128;        // Kutta wake node: a FREE node moved onto a trailing-edge
                                     // bisector and held fixed by the mesh smoothing

// per-tile flags of the fused-CG tile list (k_tile_general)
constexpr uint8_t TILE_GEN64 = 1;     // a cell of the tile's window needs stored FP64 K_e
constexpr uint8_t TILE_GEN32 = 2;     // ... stored FP32 K_e
constexpr uint8_t TILE_PLAIN64 = 4;   // window all FREE, no TILE_GEN64 cell
constexpr uint8_t TILE_PLAIN32 = 8;   // window all FREE, no TILE_GEN32 cell

// solver phases (per variant)
constexpr int PH_CG = 0, PH_RESID = 1, PH_DONE = 2;

struct DevVariant {
  double x0, y0, hx, hy;
  long long base;      // first padded node index of the variant (= row0 * P)
  int nx, ny, P, nb;   // grid, pitch (common to all variants of a batch), bodies
  int body0;           // first global body index
  int tiles_x, tiles_y;
  int row0;            // first row of the variant in the batch's 2-D node arrays
  double kr64[6];      // K_e of an undisplaced hx-by-hy cell: K01 K02 K03 K12 K13 K23
  float kr32[6];
};

struct VarState {
  double alpha, beta;          // scalars of the next fused CG launch
  double gamma, pi, rho, mu;   // last dots  r.r, p.Ap, r.Ap, Ap.Ap
  double gamma_start;          // r.r at the start of the current inner solve
  double bnorm2;               // ||b||^2 (at U of the solve)
  double rr64;                 // last true residual ||b - A u||^2 (FP64)
  double thr_abs2;             // inner stop: gamma <= max(thr_rel * gamma_start, thr_abs2)
  double thr_rel;
  long long iters;             // all CG iterations of the solve
  long long inner_iters;       // iterations of the current inner solve
  int phase;                   // PH_CG / PH_RESID / PH_DONE
  int status;                  // pf_status
  int n_resid;                 // true-residual evaluations
  int capped;                  // k_max reached
  int buf;                     // ping-pong parity of the r, p, q buffers holding the current iterate
  int pad_;
};

// One node's CG state: x (correction), r, p, q = A p.
template <typename T> struct State4;
template <> struct __align__(16) State4<float> { float x, r, p, q; };
template <> struct __align__(32) State4<double> { double x, r, p, q; };

struct SolveParams {
  double tol2;                 // tol^2
  double tol_abs;              // paper_abs: the bound on sum r^2
  int paper_abs;               // 1: stop on sum r^2 <= tol_abs (PF_TOL_PAPER_ABS), 0: on the relative residual
  double inner_rel2;           // inner_tol^2 (mixed) or 0
  long long k_max;
  int mixed;
  int fixed_bodies;            // body values are given data (Schur sub-solves), not unknowns
};

struct Sched {                 // persistent tile schedule
  const int* cta_seg;          // [G+1] first segment of each CTA
  const int* seg_var;          // [S]
  const int* seg_t0;           // [S] first tile (global tile list)
  const int* seg_t1;           // [S] one past last tile
  const int2* tile_ij;         // [T] (i0, j0)
  const int* var_seg0;         // [nv] first segment of the variant
  const int* var_seg1;         // [nv]
  double* partial;             // [S][4]
  int* counter;                // [nv] finished segments in the current launch
  int n_cta;
  unsigned long long* cta_ns;  // [G] tile-phase time of each CTA (timed fused-CG launches), else null
};

// Shapes of the bodies (pf_batch_build_shapes): per global body its kind (PF_SHAPE_*),
// its vertices (polygons: xy[2 off[k]] .. xy[2 off[k+1]], counter-clockwise), its
// bounding box (xmin, xmax, ymin, ymax) and the trailing-edge vertex with the Kutta
// condition (-1: none).  Circles use the pf_body table only.
struct DBox {                  // axis-aligned box [x0, x1] x [y0, y1]
  double x0, x1, y0, y1;
};

struct ShapeDev {
  const int* kind;
  const int* off;            // [B + 1]
  const double* xy;
  const DBox* box;
  const int* kutta;
};

struct MeshDev {
  const DevVariant* var;
  const uint8_t* tag;
  const int* bid;              // body index local to the variant (BODY nodes), else -1
  const int* body_ptr;         // [B+1] into body_nodes
  const long long* body_nodes; // padded node indices, per body in row-major order
  const double* K64;           // [6][Vtot]
  const float* K32;            // [6][Vtot]
  long long Vtot;
};

// x * 2^-k (0 <= k <= 4), bit for bit the correctly rounded FP64 product x * 2^-k.  For
// +-0 and for normal x whose exponent field exceeds k + 1, the product is exact and is x
// with the exponent field lowered by k: one integer subtraction instead of an FP64
// multiply, which matters where the FP64 pipe is the bound (GB300 runs FP64 at a small
// fraction of its FP32 rate).  Every other x (tiny or subnormal, Inf, NaN) takes the
// FP64 multiply.
static __device__ __noinline__ double pow2_scale_rare(double x, int k) { return __dmul_rn(x, ldexp(1.0, -k)); }
static __device__ __forceinline__ double pow2_scale(double x, int k) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned e = (unsigned)(b >> 52) & 0x7ffu;
  if (e > (unsigned)k + 1u && e < 2047u) return __longlong_as_double((long long)(b - ((unsigned long long)k << 52)));
  if ((b << 1) == 0ull) return x;
  return pow2_scale_rare(x, k);
}

// ---------------------------------------------------------------- reductions

// Compensated two-float accumulation (Knuth TwoSum + exact FMA products, the Dot2
// scheme of Ogita, Rump and Oishi): every FP32 product x*y is split exactly into
// p + e with e = fma(x, y, -p), p is added to the high word with TwoSum and the two
// error terms go to the low word.  A thread's partial sum is thus as accurate as a
// sum in twice the working precision (~2^-48 relative error per addition for
// same-sign terms), and it is converted to FP64 once per warp, so no FP64
// instruction is issued per node.
struct FF { float hi, lo; };

__device__ __forceinline__ void ff_add_prod(FF& a, float x, float y) {
  float p = x * y;
  float e = fmaf(x, y, -p);           // p + e == x*y exactly
  float s = a.hi + p;
  float bb = s - a.hi;
  float err = (a.hi - (s - bb)) + (p - bb);
  a.hi = s;
  a.lo += err + e;
}

// Add one FP32 value into the two-float accumulator (TwoSum, error kept in lo).
__device__ __forceinline__ void ff_add_value(FF& a, float p) {
  float s = a.hi + p;
  float bb = s - a.hi;
  float err = (a.hi - (s - bb)) + (p - bb);
  a.hi = s;
  a.lo += err;
}

__device__ __forceinline__ FF ff_add(FF a, FF b) {
  float s = a.hi + b.hi;
  float bb = s - a.hi;
  float err = (a.hi - (s - bb)) + (b.hi - bb);
  err += a.lo + b.lo;
  float h = s + err;
  return FF{h, err - (h - s)};
}

template <typename T> struct Acc;
template <> struct Acc<double> {
  double v[4];
  __device__ void zero() { v[0] = v[1] = v[2] = v[3] = 0.0; }
  __device__ void add(int k, double x, double y) { v[k] = fma(x, y, v[k]); }
  __device__ void add2(int k, double x1, double y1, double x2, double y2) { v[k] = fma(x2, y2, fma(x1, y1, v[k])); }
  template <int N>
  __device__ void add4(int k, const double (&x)[N], const double (&y)[N]) {
#pragma unroll
    for (int u = 0; u < N; ++u) v[k] = fma(x[u], y[u], v[k]);
  }
  // warp-reduce, lane 0 returns the sums
  __device__ void warp_reduce(double out[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      double s = v[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      out[k] = s;
    }
  }
};
template <> struct Acc<float> {
  FF v[4];
  __device__ void zero() {
#pragma unroll
    for (int k = 0; k < 4; ++k) v[k] = FF{0.f, 0.f};
  }
  __device__ void add(int k, float x, float y) { ff_add_prod(v[k], x, y); }
  // a thread's two products: each split exactly into p + e (TwoProd via fmaf) and added
  // to the two-float accumulator with TwoSum, so no product is rounded
  __device__ void add2(int k, float x1, float y1, float x2, float y2) {
    ff_add_prod(v[k], x1, y1);
    ff_add_prod(v[k], x2, y2);
  }
  // a thread's N products of one tile strip, each exact (TwoProd), summed with TwoSum
  // into the two-float accumulator: the only roundings are the accumulator's own
  // (about 2^-48 relative per addition for same-sign terms, as for a double-length sum)
  template <int N>
  __device__ void add4(int k, const float (&x)[N], const float (&y)[N]) {
#pragma unroll
    for (int u = 0; u < N; ++u) ff_add_prod(v[k], x[u], y[u]);
  }
  __device__ void warp_reduce(double out[4]) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      FF s = v[k];
      s = ff_add(s, FF{0.f, 0.f});   // renormalise
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        FF t{__shfl_xor_sync(0xffffffffu, s.hi, o), __shfl_xor_sync(0xffffffffu, s.lo, o)};
        s = ff_add(s, t);
      }
      out[k] = (double)s.hi + (double)s.lo;
    }
  }
};

__device__ __forceinline__ int linear_tid() { return threadIdx.y * TX + threadIdx.x; }

// Block-wide exclusive scan of one int per thread (256 threads, 1-D linear id).
static __device__ __forceinline__ int block_exscan(int x, int* total, int* sh /* >= NT/32 + 1 */) {
  const int tid = linear_tid(), lane = tid & 31, w = tid >> 5;
  int incl = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  __syncthreads();
  if (lane == 31) sh[w] = incl;
  __syncthreads();
  if (tid == 0) {
    int s = 0;
    for (int k = 0; k < NT / 32; ++k) { int t = sh[k]; sh[k] = s; s += t; }
    sh[NT / 32] = s;
  }
  __syncthreads();
  const int r = sh[w] + incl - x;
  *total = sh[NT / 32];
  __syncthreads();
  return r;
}

// Atomic add with acquire-release semantics at GPU scope; returns the old value.  Used
// as the arrival of a CTA at a per-variant counter: it publishes the CTA's stores
// (ordered before it by a block barrier) and, in the last CTA, makes the other CTAs'
// stores visible to the threads that synchronise with it through a block barrier.
__device__ __forceinline__ int atom_add_acq_rel_gpu(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Block-wide fixed-order sum of a double; all threads get the result.
__device__ __forceinline__ double block_sum(double x, double* scratch /* >= NT/32 */) {
  const int tid = linear_tid(), lane = tid & 31, w = tid >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  __syncthreads();
  if (lane == 0) scratch[w] = x;
  __syncthreads();
  double s = 0.0;
  for (int k = 0; k < NT / 32; ++k) s += scratch[k];
  __syncthreads();
  return s;
}

// Halo position h in [0, NHALO) -> shared-tile coordinates (li, lj).
__device__ __forceinline__ void halo_pos(int h, int& li, int& lj) {
  if (h < SW) { li = h; lj = 0; }
  else if (h < 2 * SW) { li = h - SW; lj = TY + 1; }
  else if (h < 2 * SW + TY) { li = 0; lj = 1 + (h - 2 * SW); }
  else { li = TX + 1; lj = 1 + (h - 2 * SW - TY); }
}

// Row of the matrix-free Q4 operator at the node in the centre of shared tile
// position (li, lj): y = sum over the four cells around the node of
// sum_{b != a} K_e[a,b] (p_b - p_a), which equals (K_e p_e)_a because every row of
// K_e sums to zero.  Inactive cells contribute nothing.  Cell coefficients come
// from the stored planes where they differ from `kr` (the closed-form rectangle) in this
// precision (CELL_GENERAL for FP64, CELL_GEN32 for FP32) and from `kr` otherwise.
// n: padded node index, P: pitch, K: [6][plane]; W: the shared tiles' row width (tile
// width + 2).
template <typename T, int W = SW>
__device__ __forceinline__ T q4_row(const T (*ps)[W], const uint8_t (*ts)[W], int li, int lj,
                                    long long n, int P, const T* __restrict__ K, long long plane,
                                    const T* kr) {
  // stored coefficients where they differ from the rectangle constants of this precision
  // (an FP32 row reads them only for CELL_GEN32 cells: the others round to kr exactly)
  constexpr uint8_t GEN = sizeof(T) == 4 ? CELL_GEN32 : CELL_GENERAL;
  const T pc = ps[lj][li];
  const T dE = ps[lj][li + 1] - pc, dW = ps[lj][li - 1] - pc;
  const T dN = ps[lj + 1][li] - pc, dS = ps[lj - 1][li] - pc;
  const T dNE = ps[lj + 1][li + 1] - pc, dNW = ps[lj + 1][li - 1] - pc;
  const T dSE = ps[lj - 1][li + 1] - pc, dSW = ps[lj - 1][li - 1] - pc;
  // the four cells' tags, then every stored coefficient the node needs (all loads are
  // issued before the first is used), then the sum over the cells
  const uint8_t t0 = ts[lj][li];                // cell (i, j): node is corner 0
  const uint8_t t1 = ts[lj][li - 1];            // cell (i-1, j): corner 1
  const uint8_t t2 = ts[lj - 1][li - 1];        // cell (i-1, j-1): corner 2
  const uint8_t t3 = ts[lj - 1][li];            // cell (i, j-1): corner 3
  T a0 = kr[0], a1 = kr[1], a2 = kr[2];         // K01 K02 K03 of cell (i, j)
  T b0 = kr[0], b1 = kr[3], b2 = kr[4];         // K01 K12 K13 of cell (i-1, j)
  T e0 = kr[1], e1 = kr[3], e2 = kr[5];         // K02 K12 K23 of cell (i-1, j-1)
  T f0 = kr[2], f1 = kr[4], f2 = kr[5];         // K03 K13 K23 of cell (i, j-1)
  if ((t0 & (CELL_ACTIVE | GEN)) == (CELL_ACTIVE | GEN)) {
    a0 = __ldg(K + n); a1 = __ldg(K + plane + n); a2 = __ldg(K + 2 * plane + n);
  }
  if ((t1 & (CELL_ACTIVE | GEN)) == (CELL_ACTIVE | GEN)) {
    const long long c = n - 1;
    b0 = __ldg(K + c); b1 = __ldg(K + 3 * plane + c); b2 = __ldg(K + 4 * plane + c);
  }
  if ((t2 & (CELL_ACTIVE | GEN)) == (CELL_ACTIVE | GEN)) {
    const long long c = n - P - 1;
    e0 = __ldg(K + plane + c); e1 = __ldg(K + 3 * plane + c); e2 = __ldg(K + 5 * plane + c);
  }
  if ((t3 & (CELL_ACTIVE | GEN)) == (CELL_ACTIVE | GEN)) {
    const long long c = n - P;
    f0 = __ldg(K + 2 * plane + c); f1 = __ldg(K + 4 * plane + c); f2 = __ldg(K + 5 * plane + c);
  }
  T y = T(0);
  if (t0 & CELL_ACTIVE) y += a0 * dE + a1 * dNE + a2 * dN;
  if (t1 & CELL_ACTIVE) y += b0 * dW + b1 * dN + b2 * dNW;
  if (t2 & CELL_ACTIVE) y += e0 * dSW + e1 * dS + e2 * dW;
  if (t3 & CELL_ACTIVE) y += f0 * dS + f1 * dSE + f2 * dE;
  return y;
}

}  // namespace pfq4
