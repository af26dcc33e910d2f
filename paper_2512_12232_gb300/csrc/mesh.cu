// Body-conforming mesh generation on the GPU (section "Body-Conforming Grid
// Generation"): background grid, inside test, radial projection of the nodes just
// inside each body, S Jacobi sweeps of the displacement, x = x_grid + d; then the
// Q4 element matrices (section "Weak formulation", 2x2 Gauss) and the per-body node
// and boundary-edge lists used by the constraint collapse and the post-processing.
// The mixed-cell variant (pf_batch_build_cut) keeps the nodes just inside a body in
// place and gives them one surface point per grid edge to an outside neighbour (node
// splitting), smooths with those points' displacements, redistributes the points and
// forms the cut cells' triangle / quadrilateral pieces (cut.cuh).
//
// The mesh rules are evaluated with explicitly rounded FP64 intrinsics
// (__dadd_rn, __dmul_rn, __ddiv_rn, __dsqrt_rn), never contracted into FMAs, so the
// classification and the coordinates are reproducible bit for bit by any IEEE FP64
// implementation of the same operation sequence.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "batch.h"
#include "cut.cuh"

namespace pfq4 {

namespace {

__device__ __forceinline__ double grid_x(const DevVariant& V, int i) {
  return __dadd_rn(V.x0, __dmul_rn((double)i, V.hx));
}
__device__ __forceinline__ double grid_y(const DevVariant& V, int j) {
  return __dadd_rn(V.y0, __dmul_rn((double)j, V.hy));
}

struct TileCtx {
  int v, i, j;
  long long n;
  bool in;
};

__device__ __forceinline__ TileCtx tile_ctx(const DevVariant* var, const int* tile_var, const int2* tile_ij) {
  TileCtx c;
  const long long t = blockIdx.x;
  c.v = tile_var[t];
  const int2 ij = tile_ij[t];
  const DevVariant& V = var[c.v];
  c.i = ij.x + threadIdx.x;
  c.j = ij.y + threadIdx.y;
  c.in = (c.i <= V.nx) && (c.j <= V.ny);
  c.n = V.base + (long long)c.j * V.P + c.i;
  return c;
}

// Crossing-number test of (x, y) against polygon gb: an edge (a, b) is crossed when
// (a_y > y) != (b_y > y) and x < a_x + ((y - a_y)(b_x - a_x)) / (b_y - a_y); odd = inside.
__device__ bool inside_polygon(const ShapeDev& S, int gb, double x, double y) {
  const DBox bx = S.box[gb];
  if (x < bx.x0 || x > bx.x1 || y < bx.y0 || y > bx.y1) return false;   // the count is even there
  const int v0 = S.off[gb], n = S.off[gb + 1] - v0;
  const double* p = S.xy + 2 * v0;
  bool in = false;
  for (int e = 0; e < n; ++e) {
    const int f = e + 1 == n ? 0 : e + 1;
    const double ax = p[2 * e], ay = p[2 * e + 1], bxv = p[2 * f], by = p[2 * f + 1];
    if ((ay > y) != (by > y)) {
      const double xint =
          __dadd_rn(ax, __ddiv_rn(__dmul_rn(__dsub_rn(y, ay), __dsub_rn(bxv, ax)), __dsub_rn(by, ay)));
      if (x < xint) in = !in;
    }
  }
  return in;
}

// Nearest point of polygon gb's boundary to (x, y): per edge t = ((p - a).(b - a)) / |b - a|^2
// clamped to [0, 1], q = a + t (b - a); the first edge with the smallest |p - q|^2 wins.
__device__ void nearest_on_polygon(const ShapeDev& S, int gb, double x, double y, double& qx, double& qy) {
  const int v0 = S.off[gb], n = S.off[gb + 1] - v0;
  const double* p = S.xy + 2 * v0;
  double best = 1.0 / 0.0;
  qx = 0.0;
  qy = 0.0;
  for (int e = 0; e < n; ++e) {
    const int f = e + 1 == n ? 0 : e + 1;
    const double ax = p[2 * e], ay = p[2 * e + 1];
    const double dx = __dsub_rn(p[2 * f], ax), dy = __dsub_rn(p[2 * f + 1], ay);
    const double num = __dadd_rn(__dmul_rn(__dsub_rn(x, ax), dx), __dmul_rn(__dsub_rn(y, ay), dy));
    const double den = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    double t = __ddiv_rn(num, den);
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    const double cx = __dadd_rn(ax, __dmul_rn(t, dx)), cy = __dadd_rn(ay, __dmul_rn(t, dy));
    const double ex = __dsub_rn(x, cx), ey = __dsub_rn(y, cy);
    const double d2 = __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey));
    if (d2 < best) {
      best = d2;
      qx = cx;
      qy = cy;
    }
  }
}

// 1. inside test: bid[n] = body k (local) if (x-cx)^2 + (y-cy)^2 <= r^2 (circles) or the
//    crossing-number test counts odd (polygons), else -1.
__global__ void k_classify(const DevVariant* var, const int* tile_var, const int2* tile_ij,
                           const pf_body* bodies, ShapeDev shp, const int4* bbox, int* bid, int* err) {
  TileCtx c = tile_ctx(var, tile_var, tile_ij);
  const DevVariant& V = var[c.v];
  if (!c.in) return;
  const double x = grid_x(V, c.i), y = grid_y(V, c.j);
  int ib = -1;
  for (int k = 0; k < V.nb; ++k) {
    const int gb = V.body0 + k;
    // the body's node box (padded by a node or more) holds every node the test can find inside
    const int4 bx = bbox[gb];
    if (c.i < bx.x || c.i > bx.y || c.j < bx.z || c.j > bx.w) continue;
    bool in;
    if (shp.kind && shp.kind[gb] == PF_SHAPE_POLYGON) {
      in = inside_polygon(shp, gb, x, y);
    } else {
      const pf_body B = bodies[gb];
      const double dx = __dsub_rn(x, B.cx), dy = __dsub_rn(y, B.cy);
      const double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
      in = d2 <= __dmul_rn(B.r, B.r);
    }
    if (in) {
      if (ib >= 0) atomicOr(err, 1);
      ib = k;
    }
  }
  bid[c.n] = ib;
}

// 2. node kinds, cell activity, ring flag, projection displacement d0.
__global__ void k_kinds(const DevVariant* var, const int* tile_var, const int2* tile_ij,
                        const pf_body* bodies, ShapeDev shp, const int* bid, uint8_t* tag, double2* d0,
                        int bc0, int bc1, int bc2, int bc3, int cut, int* err) {
  TileCtx c = tile_ctx(var, tile_var, tile_ij);
  const DevVariant& V = var[c.v];
  if (!c.in) return;
  const int i = c.i, j = c.j, nx = V.nx, ny = V.ny, P = V.P;
  const long long n = c.n;
  auto outside = [&](int ii, int jj) -> bool { return bid[V.base + (long long)jj * P + ii] < 0; };
  auto cell_active = [&](int ci, int cj) -> bool {
    if (ci < 0 || cj < 0 || ci >= nx || cj >= ny) return false;
    return outside(ci, cj) || outside(ci + 1, cj) || outside(ci, cj + 1) || outside(ci + 1, cj + 1);
  };
  uint8_t t = 0;
  const int ib = bid[n];
  const bool ring = (i == 0) || (i == nx) || (j == 0) || (j == ny);
  if (ring) t |= RING;
  if (cell_active(i, j)) t |= CELL_ACTIVE;
  double2 d = make_double2(0.0, 0.0);
  if (ib < 0) {
    const bool dir = (i == 0 && bc0 == PF_BC_DIRICHLET_UY) || (i == nx && bc1 == PF_BC_DIRICHLET_UY) ||
                     (j == 0 && bc2 == PF_BC_DIRICHLET_UY) || (j == ny && bc3 == PF_BC_DIRICHLET_UY);
    t |= dir ? K_DIR : K_FREE;
  } else {
    const bool touch = cell_active(i - 1, j - 1) || cell_active(i, j - 1) || cell_active(i - 1, j) ||
                       cell_active(i, j);
    if (touch && cut) {
      t |= K_BODY;                     // mixed-cell mesh: the node stays, its surface points are per edge
    } else if (touch) {
      t |= K_BODY;
      const int gb = V.body0 + ib;
      const double xg = grid_x(V, i), yg = grid_y(V, j);
      double xb, yb;
      if (shp.kind && shp.kind[gb] == PF_SHAPE_POLYGON) {
        nearest_on_polygon(shp, gb, xg, yg, xb, yb);
      } else {
        const pf_body B = bodies[gb];
        const double ex = __dsub_rn(xg, B.cx), ey = __dsub_rn(yg, B.cy);
        const double rho = __dsqrt_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)));
        if (rho == 0.0) atomicOr(err, 2);
        xb = __dadd_rn(B.cx, __ddiv_rn(__dmul_rn(B.r, ex), rho));
        yb = __dadd_rn(B.cy, __ddiv_rn(__dmul_rn(B.r, ey), rho));
      }
      d = make_double2(__dsub_rn(xb, xg), __dsub_rn(yb, yg));
    } else {
      t |= K_INACT;
    }
  }
  tag[n] = t;
  d0[n] = d;
}

// Surface point of polygon gb on the grid edge from the inside node (xg, yg) to its
// outside neighbour (xk, yk) in direction d.  On a row the crossings are those of the
// inside test, x = a_x + ((y - a_y)(b_x - a_x)) / (b_y - a_y) for an edge with
// (a_y > y) != (b_y > y), of which the inside test counts an odd number in the half-open
// range from the inside node (g < x <= k towards +x, k < x <= g towards -x); the one
// nearest the inside node is taken.  On a column the same with x and y exchanged; without
// a crossing in range the crossing nearest the range (the first edge on ties) is clipped
// onto it, and without any crossing on the line the edge's midpoint is taken.
__device__ double2 polygon_crossing(const ShapeDev& S, int gb, double xg, double yg, double xk, double yk, int d) {
  const int v0 = S.off[gb], n = S.off[gb + 1] - v0;
  const double* p = S.xy + 2 * v0;
  const bool row = d == 0 || d == 2;
  const double c = row ? yg : xg;
  const double g = row ? xg : yg, k = row ? xk : yk;
  const bool up = k > g;
  const double lo = up ? g : k, hi = up ? k : g;
  double best = 0.0, fb = 0.0, fbd = 1.0 / 0.0;
  bool found = false, anyx = false;
  for (int e = 0; e < n; ++e) {
    const int f = e + 1 == n ? 0 : e + 1;
    const double ax = p[2 * e], ay = p[2 * e + 1], bx = p[2 * f], by = p[2 * f + 1];
    double t;
    if (row) {
      if ((ay > c) == (by > c)) continue;
      t = __dadd_rn(ax, __ddiv_rn(__dmul_rn(__dsub_rn(c, ay), __dsub_rn(bx, ax)), __dsub_rn(by, ay)));
    } else {
      if ((ax > c) == (bx > c)) continue;
      t = __dadd_rn(ay, __ddiv_rn(__dmul_rn(__dsub_rn(c, ax), __dsub_rn(by, ay)), __dsub_rn(bx, ax)));
    }
    anyx = true;
    const bool in = up ? (g < t && t <= k) : (k < t && t <= g);
    if (in) {
      best = !found ? t : (up ? fmin(best, t) : fmax(best, t));
      found = true;
    } else {
      const double dist = t < lo ? __dsub_rn(lo, t) : __dsub_rn(t, hi);
      if (dist < fbd) {
        fbd = dist;
        fb = t;
      }
    }
  }
  const double sv = found ? best : (anyx ? fmin(fmax(fb, lo), hi) : __dmul_rn(__dadd_rn(g, k), 0.5));
  return row ? make_double2(sv, yg) : make_double2(xg, sv);
}

// 2a. mixed-cell mesh: the surface points of every BODY node, where the grid edge
//     towards an outside neighbour crosses the body's boundary: for a circle on a row
//     (cx +- sqrt(r^2 - (y - cy)^2), y), on a column (x, cy +- sqrt(r^2 - (x - cx)^2)), the
//     sign that of the step; for a polygon polygon_crossing; NaN for the other directions
//     and for every other node.
__global__ void k_cut_points(const DevVariant* var, const int* tile_var, const int2* tile_ij,
                             const pf_body* bodies, ShapeDev shp, const int* bid, const uint8_t* tag,
                             double2* pcut, long long Vtot) {
  TileCtx c = tile_ctx(var, tile_var, tile_ij);
  const DevVariant& V = var[c.v];
  if (!c.in) return;
  const double nan = __longlong_as_double(0x7ff8000000000000LL);
  double2 out[4];
  for (int d = 0; d < 4; ++d) out[d] = make_double2(nan, nan);
  if ((tag[c.n] & KIND_MASK) == K_BODY) {
    const int gb = V.body0 + bid[c.n];
    const pf_body B = bodies[gb];
    const bool poly = shp.kind && shp.kind[gb] == PF_SHAPE_POLYGON;
    const double xg = grid_x(V, c.i), yg = grid_y(V, c.j);
    const double rr = __dmul_rn(B.r, B.r);
    const int di[4] = {1, 0, -1, 0}, dj[4] = {0, 1, 0, -1};
    for (int d = 0; d < 4; ++d) {
      const int ni = c.i + di[d], nj = c.j + dj[d];
      if (ni < 0 || nj < 0 || ni > V.nx || nj > V.ny) continue;
      if (bid[V.base + (long long)nj * V.P + ni] >= 0) continue;
      if (poly) {
        out[d] = polygon_crossing(shp, gb, xg, yg, grid_x(V, ni), grid_y(V, nj), d);
      } else if (d == 0 || d == 2) {
        const double e = __dsub_rn(yg, B.cy);
        const double sq = __dsqrt_rn(__dsub_rn(rr, __dmul_rn(e, e)));
        out[d] = make_double2(d == 0 ? __dadd_rn(B.cx, sq) : __dsub_rn(B.cx, sq), yg);
      } else {
        const double e = __dsub_rn(xg, B.cx);
        const double sq = __dsqrt_rn(__dsub_rn(rr, __dmul_rn(e, e)));
        out[d] = make_double2(xg, d == 1 ? __dadd_rn(B.cy, sq) : __dsub_rn(B.cy, sq));
      }
    }
  }
  for (int d = 0; d < 4; ++d) pcut[d * Vtot + c.n] = out[d];
}

// 2b. Kutta condition of polygon gb (one CTA per global body; others return): the wake
//     point W = T + hx w on the trailing-edge bisector w (unit, pointing out of the body),
//     the FREE node nearest to W (smallest squared distance, then smallest row-major index)
//     searched in a window of +-KUTTA_WIN cells around W, flagged WAKE and moved onto W.
constexpr int KUTTA_WIN = 8;
__global__ void __launch_bounds__(256) k_kutta(const DevVariant* var, const int* body_var, ShapeDev shp,
                                               uint8_t* tag, double2* d0, long long* wake) {
  const int gb = blockIdx.x;
  if (!shp.kind || shp.kind[gb] != PF_SHAPE_POLYGON || shp.kutta[gb] < 0) return;
  const DevVariant& V = var[body_var[gb]];
  __shared__ double sW[2];
  __shared__ double sd[256];
  __shared__ long long sk[256];
  if (threadIdx.x == 0) {
    const int v0 = shp.off[gb], n = shp.off[gb + 1] - v0, k = shp.kutta[gb];
    const double* p = shp.xy + 2 * v0;
    const int kp = k == 0 ? n - 1 : k - 1, kn = k + 1 == n ? 0 : k + 1;
    const double tx = p[2 * k], ty = p[2 * k + 1];
    const double ax = __dsub_rn(tx, p[2 * kp]), ay = __dsub_rn(ty, p[2 * kp + 1]);
    const double bx = __dsub_rn(tx, p[2 * kn]), by = __dsub_rn(ty, p[2 * kn + 1]);
    const double la = __dsqrt_rn(__dadd_rn(__dmul_rn(ax, ax), __dmul_rn(ay, ay)));
    const double lb = __dsqrt_rn(__dadd_rn(__dmul_rn(bx, bx), __dmul_rn(by, by)));
    double wx = __dadd_rn(__ddiv_rn(ax, la), __ddiv_rn(bx, lb));
    double wy = __dadd_rn(__ddiv_rn(ay, la), __ddiv_rn(by, lb));
    const double lw = __dsqrt_rn(__dadd_rn(__dmul_rn(wx, wx), __dmul_rn(wy, wy)));
    wx = __ddiv_rn(wx, lw);
    wy = __ddiv_rn(wy, lw);
    sW[0] = __dadd_rn(tx, __dmul_rn(V.hx, wx));
    sW[1] = __dadd_rn(ty, __dmul_rn(V.hx, wy));
  }
  __syncthreads();
  const double Wx = sW[0], Wy = sW[1];
  const int ic = (int)floor((Wx - V.x0) / V.hx), jc = (int)floor((Wy - V.y0) / V.hy);
  constexpr int SIDE = 2 * KUTTA_WIN + 2;
  double best = 1.0 / 0.0;
  long long bk = -1;
  for (int q = threadIdx.x; q < SIDE * SIDE; q += blockDim.x) {
    const int i = ic - KUTTA_WIN + q % SIDE, j = jc - KUTTA_WIN + q / SIDE;
    if (i < 0 || j < 0 || i > V.nx || j > V.ny) continue;
    const long long n = V.base + (long long)j * V.P + i;
    if ((tag[n] & KIND_MASK) != K_FREE) continue;
    const double ex = __dsub_rn(grid_x(V, i), Wx), ey = __dsub_rn(grid_y(V, j), Wy);
    const double d2 = __dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey));
    const long long key = (long long)j * (V.nx + 1) + i;     // row-major order of the logical grid
    if (d2 < best || (d2 == best && key < bk)) {
      best = d2;
      bk = key;
    }
  }
  sd[threadIdx.x] = best;
  sk[threadIdx.x] = bk;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int t = 1; t < blockDim.x; ++t)
      if (sk[t] >= 0 && (sd[t] < best || (sd[t] == best && (bk < 0 || sk[t] < bk)))) {
        best = sd[t];
        bk = sk[t];
      }
    if (bk >= 0) {
      const int i = (int)(bk % (V.nx + 1)), j = (int)(bk / (V.nx + 1));
      const long long n = V.base + (long long)j * V.P + i;
      d0[n] = make_double2(__dsub_rn(Wx, grid_x(V, i)), __dsub_rn(Wy, grid_y(V, j)));
      tag[n] |= WAKE;
      wake[gb] = n;
    }
  }
}

// 3. Jacobi sweeps, JK per launch (temporal blocking): nodes outside every body and off
//    the outer ring take the average of their four neighbours, summed W, E, S, N,
//    divided by 4; other nodes keep their value.  A CTA loads the window of its 64x16
//    tile with a JK-node halo once, runs the sweeps in a double-buffered shared window
//    (after s sweeps the window is exact at distance >= s from its edge) and writes its
//    tile: every node sees the same neighbour values as with one launch per sweep, so
//    the result is bit-identical.  After sweep s (0-based) the displacement is exactly
//    zero farther than s + 1 cells from every body node, so a tile farther than the
//    reach of the launch's last sweep from every body's node box is all zeros in both
//    ping-pong buffers and is skipped.
// x / 4, correctly rounded (bit for bit the oracle's division; see pow2_scale): the
// smoothing is bound by the FP64 pipe, which then runs three additions per component
// instead of three additions and a multiply.
__device__ __forceinline__ double quarter(double x) { return pow2_scale(x, 2); }

constexpr int JK = 4;
constexpr int JRW = CTX + 2 * JK, JRH = CTY + 2 * JK;      // window 72 x 24
constexpr int JACOBI_SMEM = 2 * JRW * JRH * (int)sizeof(double2) + JRW * JRH;

// CUT: the mixed-cell mesh, where a BODY neighbour contributes the displacement of its
// surface point on the common edge (P - x_grid of the neighbour) instead of its own.
__device__ __forceinline__ double2 cut_disp(const DevVariant& V, double2 p, int i, int j) {
  return make_double2(__dsub_rn(p.x, grid_x(V, i)), __dsub_rn(p.y, grid_y(V, j)));
}

template <bool CUT>
__global__ void __launch_bounds__(NT) k_jacobi(const DevVariant* var, const int* tile_var, const int2* tile_ij,
                                               const int* bid, const uint8_t* tag, const int4* bbox, int sweep0,
                                               int nsw, const double2* __restrict__ src, double2* __restrict__ dst,
                                               const double2* __restrict__ pcut, long long Vtot) {
  extern __shared__ __align__(16) unsigned char jsm[];
  double2* w0 = reinterpret_cast<double2*>(jsm);
  double2* w1 = w0 + JRW * JRH;
  uint8_t* upd = reinterpret_cast<uint8_t*>(w1 + JRW * JRH);
  const int t = blockIdx.x;
  const DevVariant& V = var[tile_var[t]];
  const int2 ij = tile_ij[t];
  {
    // a sweep moves a nonzero displacement one node in L1 distance: after `reach` sweeps
    // every node whose L1 distance from all bodies' node boxes (which hold every source:
    // BODY nodes, a Kutta wake node) exceeds reach is still +0, here and in dst
    const int reach = sweep0 + nsw;
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
  for (int q = tid; q < JRW * JRH; q += NT) {
    const int i = ij.x - JK + q % JRW, j = ij.y - JK + q / JRW;
    double2 v = make_double2(0.0, 0.0);
    uint8_t u = 0;
    if (i >= 0 && j >= 0 && i <= V.nx && j <= V.ny) {
      const long long n = V.base + (long long)j * V.P + i;
      v = src[n];
      u = bid[n] < 0 && !(tag[n] & (RING | WAKE));
      if (CUT && (tag[n] & KIND_MASK) == K_BODY) u |= 2;
    }
    w0[q] = v;
    upd[q] = u;
  }
  __syncthreads();
  double2* a = w0;
  double2* b = w1;
  for (int sw = 0; sw < nsw; ++sw) {
    // after sweep sw only nodes at distance >= sw + 1 from the window edge are read again
    // (by later sweeps, or as the tile), so the sweep covers that rectangle alone; the
    // values outside it go stale, as the edge does, and are never used
    const int rw = JRW - 2 * (sw + 1), rh = JRH - 2 * (sw + 1);
    for (int k = tid; k < rw * rh; k += NT) {
      const int ri = sw + 1 + k % rw, rj = sw + 1 + k / rw;
      const int q = rj * JRW + ri;
      double2 out = a[q];
      // an updatable node is off the ring, so its four neighbours lie in the grid
      if (upd[q] & 1) {
        double2 w = a[q - 1], e = a[q + 1], s = a[q - JRW], nn = a[q + JRW];
        if (CUT) {
          // the neighbours' surface points towards this node: W's E point, E's W point,
          // S's N point, N's S point
          const int gi = ij.x - JK + ri, gj = ij.y - JK + rj;
          const long long gn = V.base + (long long)gj * V.P + gi;
          if (upd[q - 1] & 2) w = cut_disp(V, pcut[gn - 1], gi - 1, gj);
          if (upd[q + 1] & 2) e = cut_disp(V, pcut[2 * Vtot + gn + 1], gi + 1, gj);
          if (upd[q - JRW] & 2) s = cut_disp(V, pcut[Vtot + gn - V.P], gi, gj - 1);
          if (upd[q + JRW] & 2) nn = cut_disp(V, pcut[3 * Vtot + gn + V.P], gi, gj + 1);
        }
        // four neighbours all +0 (bit for bit) give +0 without the eight FP64 operations:
        // the front of the displacement runs diagonally through the tiles it reaches
        const unsigned long long z =
            __double_as_longlong(w.x) | __double_as_longlong(w.y) | __double_as_longlong(e.x) |
            __double_as_longlong(e.y) | __double_as_longlong(s.x) | __double_as_longlong(s.y) |
            __double_as_longlong(nn.x) | __double_as_longlong(nn.y);
        if (z == 0ull) {
          out = make_double2(0.0, 0.0);
        } else {
          const double sx = __dadd_rn(__dadd_rn(__dadd_rn(w.x, e.x), s.x), nn.x);
          const double sy = __dadd_rn(__dadd_rn(__dadd_rn(w.y, e.y), s.y), nn.y);
          out = make_double2(quarter(sx), quarter(sy));
        }
      }
      b[q] = out;
    }
    __syncthreads();
    double2* tmp = a;
    a = b;
    b = tmp;
  }
  for (int q = tid; q < CTX * CTY; q += NT) {
    const int i = ij.x + q % CTX, j = ij.y + q / CTX;
    if (i <= V.nx && j <= V.ny) dst[V.base + (long long)j * V.P + i] = a[(JK + q / CTX) * JRW + JK + q % CTX];
  }
}

// 4. final coordinates x = x_grid + d and the DISPLACED flag.
__global__ void k_finalize(const DevVariant* var, const int* tile_var, const int2* tile_ij,
                           const double2* d, uint8_t* tag, double* X, long long Vtot) {
  TileCtx c = tile_ctx(var, tile_var, tile_ij);
  const DevVariant& V = var[c.v];
  if (!c.in) return;
  const double2 dd = d[c.n];
  X[c.n] = __dadd_rn(grid_x(V, c.i), dd.x);
  X[Vtot + c.n] = __dadd_rn(grid_y(V, c.j), dd.y);
  if (dd.x != 0.0 || dd.y != 0.0) tag[c.n] |= DISPLACED;
}

__device__ void atomic_min_double(double* addr, double val) {
  unsigned long long* a = (unsigned long long*)addr;
  unsigned long long old = *a, assumed;
  while (val < __longlong_as_double((long long)old)) {
    assumed = old;
    old = atomicCAS(a, assumed, (unsigned long long)__double_as_longlong(val));
    if (old == assumed) break;
  }
}

// 4b. mixed-cell mesh, boundary-point redistribution (one pass, after the smoothing): the
//     chord (A, B) of every cut cell with 0 < L = |B - A| < s_min pushes its ends apart
//     along it, A by -f (B - A) and B by +f (B - A) with f = ((s_min - L) * 0.5) / L; a
//     point adds the pushes of the two cells beside its edge (the cell below, or left of,
//     it first) and, if pushed, is projected back onto its body: radially for a circle,
//     to the nearest boundary point for a polygon.
//     s_min = sigma * min(hx, hy).  The push of one cell on point (corner a_here, d):
__device__ inline bool cut_push(const DevVariant& V, const int* bid, const double* X, long long Vtot,
                                const double2* pin, int ci, int cj, int a_here, int d, double smin, double& mx,
                                double& my) {
  mx = 0.0;
  my = 0.0;
  CutPoly p;
  if (cut_polygon(V, bid, X, Vtot, pin, V.base + (long long)cj * V.P + ci, p) != CUT_OK || p.n == 0) return false;
  int ka, kb;
  cut_chord(p, ka, kb);
  const double ex = __dsub_rn(p.x[kb], p.x[ka]), ey = __dsub_rn(p.y[kb], p.y[ka]);
  const double L = __dsqrt_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)));
  if (!(L > 0.0 && L < smin)) return false;
  const double f = __ddiv_rn(__dmul_rn(__dsub_rn(smin, L), 0.5), L);
  const int id = (a_here << 2) | d;
  if (p.pt[ka] == id) {
    mx = -__dmul_rn(f, ex);
    my = -__dmul_rn(f, ey);
    return true;
  }
  if (p.pt[kb] == id) {
    mx = __dmul_rn(f, ex);
    my = __dmul_rn(f, ey);
    return true;
  }
  return false;
}

__global__ void k_redistribute(const DevVariant* var, const int* tile_var, const int2* tile_ij,
                               const pf_body* bodies, ShapeDev shp, const int* bid, const uint8_t* tag,
                               const double* X, long long Vtot, double sigma, const double2* pin, double2* pout) {
  TileCtx c = tile_ctx(var, tile_var, tile_ij);
  const DevVariant& V = var[c.v];
  if (!c.in) return;
  const bool body = (tag[c.n] & KIND_MASK) == K_BODY;
  const double smin = __dmul_rn(sigma, fmin(V.hx, V.hy));
  for (int d = 0; d < 4; ++d) {
    double2 q = pin[d * Vtot + c.n];
    if (body && !isnan(q.x)) {
      // the cells beside the edge: below then above (E, W), left then right (N, S)
      int ci[2], cj[2];
      if (d == 0) { ci[0] = c.i; cj[0] = c.j - 1; ci[1] = c.i; cj[1] = c.j; }
      else if (d == 2) { ci[0] = c.i - 1; cj[0] = c.j - 1; ci[1] = c.i - 1; cj[1] = c.j; }
      else if (d == 1) { ci[0] = c.i - 1; cj[0] = c.j; ci[1] = c.i; cj[1] = c.j; }
      else { ci[0] = c.i - 1; cj[0] = c.j - 1; ci[1] = c.i; cj[1] = c.j - 1; }
      bool moved = false;
      double qx = q.x, qy = q.y;
      for (int k = 0; k < 2; ++k) {
        const int di = c.i - ci[k], dj = c.j - cj[k];
        double mx, my;
        moved |= cut_push(V, bid, X, Vtot, pin, ci[k], cj[k], di + 3 * dj - 2 * di * dj, d, smin, mx, my);
        qx = __dadd_rn(qx, mx);
        qy = __dadd_rn(qy, my);
      }
      const int gb = V.body0 + bid[c.n];
      if (moved && shp.kind && shp.kind[gb] == PF_SHAPE_POLYGON) {
        double px, py;
        nearest_on_polygon(shp, gb, qx, qy, px, py);
        q = make_double2(px, py);
      } else if (moved) {
        const pf_body B = bodies[gb];
        const double ux = __dsub_rn(qx, B.cx), uy = __dsub_rn(qy, B.cy);
        const double rho = __dsqrt_rn(__dadd_rn(__dmul_rn(ux, ux), __dmul_rn(uy, uy)));
        q = make_double2(__dadd_rn(B.cx, __ddiv_rn(__dmul_rn(B.r, ux), rho)),
                         __dadd_rn(B.cy, __ddiv_rn(__dmul_rn(B.r, uy), rho)));
      }
    }
    pout[d * Vtot + c.n] = q;
  }
}

// 5. element matrices, FP64 and FP32 copies, of the active cells that need stored
//    coefficients: Q4 (2x2 Gauss) of the cells with a displaced corner, and on the
//    mixed-cell mesh (pcut != NULL) the cut-cell matrices (every reader uses the
//    closed-form constants for the other cells); CELL_GENERAL / CELL_GEN32 flags,
//    per-variant counts and min det J.  err bit 4: a cut cell with two diagonal inside
//    corners; bit 8: inside corners of two bodies.
__global__ void k_stiffness(const DevVariant* var, const int* tile_var, const int2* tile_ij,
                            uint8_t* tag, const double* X, long long Vtot, double* K64, float* K32, float* K32i,
                            long long* stats_i, double* detmin, const int* bid, const double2* pcut, int* err) {
  TileCtx c = tile_ctx(var, tile_var, tile_ij);
  const DevVariant& V = var[c.v];
  __shared__ long long cnt[6];
  __shared__ double dmin;
  const int tid = linear_tid();
  if (tid < 6) cnt[tid] = 0;
  if (tid == 0) dmin = 1e300;
  __syncthreads();
  if (c.in) {
    const long long n = c.n;
    const uint8_t t = tag[n];
    const uint8_t kind = t & KIND_MASK;
    if (kind == K_FREE) atomicAdd((unsigned long long*)&cnt[0], 1ull);
    if (kind == K_BODY) atomicAdd((unsigned long long*)&cnt[1], 1ull);
    if (kind == K_INACT) atomicAdd((unsigned long long*)&cnt[2], 1ull);
    if (t & CELL_ACTIVE) {
      atomicAdd((unsigned long long*)&cnt[3], 1ull);
      const long long idx[4] = {n, n + 1, n + 1 + V.P, n + V.P};
      CutPoly cp;
      cp.n = 0;
      int cst = CUT_OK;
      if (pcut) {
        cst = cut_polygon(V, bid, X, Vtot, pcut, n, cp);
        if (cst != CUT_OK) atomicOr(err, cst == CUT_SADDLE ? 4 : 8);
      }
      bool disp = false;
      for (int a = 0; a < 4; ++a) disp |= (tag[idx[a]] & DISPLACED) != 0;
      if (cst != CUT_OK) {
        atomic_min_double(&dmin, -1.0);              // refused cell: the mesh is invalid
      } else if (cp.n == 0 && !disp) {
        // an undisplaced hx-by-hy rectangle: every reader of stored K_e uses the
        // closed-form constants for it, and det J = (hx/2)(hy/2) at every Gauss point
        atomic_min_double(&dmin, 0.25 * V.hx * V.hy);
      } else {
        double k6[6], dm;
        if (cp.n > 0) {
          dm = cut_cell_matrix(cp, k6);
        } else {
          double x[4], y[4], K[4][4];
          for (int a = 0; a < 4; ++a) {
            x[a] = X[idx[a]];
            y[a] = X[Vtot + idx[a]];
          }
          dm = q4_element(x, y, K);
          k6[0] = K[0][1]; k6[1] = K[0][2]; k6[2] = K[0][3];
          k6[3] = K[1][2]; k6[4] = K[1][3]; k6[5] = K[2][3];
        }
        for (int m = 0; m < 6; ++m) {
          K64[m * Vtot + n] = k6[m];
          K32[m * Vtot + n] = (float)k6[m];
          K32i[6 * n + m] = (float)k6[m];
        }
        bool differs32 = false;
        for (int m = 0; m < 6; ++m) differs32 |= (float)k6[m] != V.kr32[m];
        tag[n] = t | CELL_GENERAL | (differs32 ? CELL_GEN32 : 0);
        atomicAdd((unsigned long long*)&cnt[4], 1ull);
        if (differs32) atomicAdd((unsigned long long*)&cnt[5], 1ull);
        atomic_min_double(&dmin, dm);
      }
    }
  }
  __syncthreads();
  if (tid < 6 && cnt[tid]) atomicAdd((unsigned long long*)&stats_i[c.v * 6 + tid], (unsigned long long)cnt[tid]);
  if (tid == 0 && dmin < 1e300) atomic_min_double(&detmin[c.v], dmin);
}

// 5b. per fused-CG tile: does any cell used by the tile (cells i0-1 .. i0+CTX-1,
//     j0-1 .. j0+CTY-1 of its variant) carry stored coefficients (bit 0: FP64 operator,
//     bit 1: FP32 operator); is the tile "plain" for that operator (bit 2: FP64, bit 3:
//     FP32): every node of its window i0-1 .. i0+CTX, j0-1 .. j0+CTY exists and is FREE
//     (so every cell is active) and no cell needs stored coefficients, which lets the
//     fused CG step skip the tags; and how many of its nodes carry an operator row
//     (FREE or BODY)?  The counts feed the cost estimate of the fused-CG schedule.
__global__ void k_tile_general(const DevVariant* var, const int* tile_var, const int2* tile_ij, const uint8_t* tag,
                               uint8_t* gen, int* act) {
  __shared__ int sh[NT / 32 + 1];
  const long long t = blockIdx.x;
  const DevVariant& V = var[tile_var[t]];
  const int2 ij = tile_ij[t];
  int g64 = 0, g32 = 0, na = 0, allfree = 1;
  for (int q = linear_tid(); q < (CTX + 1) * (CTY + 1); q += NT) {
    const int i = ij.x - 1 + q % (CTX + 1), j = ij.y - 1 + q / (CTX + 1);
    if (i >= 0 && j >= 0 && i < V.nx && j < V.ny) {
      const uint8_t c = tag[V.base + (long long)j * V.P + i];
      g64 |= (c & CELL_GENERAL) != 0;
      g32 |= (c & CELL_GEN32) != 0;
    }
  }
  for (int q = linear_tid(); q < CTX * CTY; q += NT) {
    const int i = ij.x + q % CTX, j = ij.y + q / CTX;
    if (i <= V.nx && j <= V.ny) {
      const int k = tag[V.base + (long long)j * V.P + i] & KIND_MASK;
      na += (k == K_FREE || k == K_BODY);
    }
  }
  for (int q = linear_tid(); q < (CTX + 2) * (CTY + 2); q += NT) {
    const int i = ij.x - 1 + q % (CTX + 2), j = ij.y - 1 + q / (CTX + 2);
    if (i < 0 || j < 0 || i > V.nx || j > V.ny) allfree = 0;
    else if ((tag[V.base + (long long)j * V.P + i] & KIND_MASK) != K_FREE) allfree = 0;
  }
  g64 = __syncthreads_or(g64);
  g32 = __syncthreads_or(g32);
  allfree = __syncthreads_and(allfree);
  int tot;
  block_exscan(na, &tot, sh);
  if (linear_tid() == 0) {
    gen[t] = (uint8_t)((g64 ? TILE_GEN64 : 0) | (g32 ? TILE_GEN32 : 0) | (allfree && !g64 ? TILE_PLAIN64 : 0) |
                       (allfree && !g32 ? TILE_PLAIN32 : 0));
    act[t] = tot;
  }
}

// 6. per-body node lists (row-major inside the body's node box).  pass 0 counts,
//    pass 1 writes.  One CTA per global body.
__global__ void k_body_nodes(const DevVariant* var, const int* body_var, const int4* bbox,
                             const uint8_t* tag, const int* bid, int* count, const int* ptr,
                             long long* out, int pass) {
  __shared__ int sh[NT / 32 + 1];
  const int gb = blockIdx.x;
  const int v = body_var[gb];
  const DevVariant& V = var[v];
  const int k = gb - V.body0;
  const int4 bx = bbox[gb];
  const int w = bx.y - bx.x + 1, h = bx.w - bx.z + 1;
  const long long total = (long long)w * h;
  int run = 0;
  for (long long s = 0; s < total; s += NT) {
    const long long q = s + linear_tid();
    int flag = 0;
    long long n = 0;
    if (q < total) {
      const int i = bx.x + (int)(q % w), j = bx.z + (int)(q / w);
      n = V.base + (long long)j * V.P + i;
      flag = ((tag[n] & KIND_MASK) == K_BODY) && bid[n] == k;
    }
    int tot;
    const int pos = block_exscan(flag, &tot, sh);
    if (pass == 1 && flag) out[ptr[gb] + run + pos] = n;
    run += tot;
  }
  if (pass == 0 && linear_tid() == 0) count[gb] = run;
}

// 7. per-body boundary edges: edges (corner a -> a+1) of active cells whose two end
//    nodes are BODY nodes of this body at distinct positions; on the mixed-cell mesh
//    (pcut != NULL) the chord of every cut cell of this body whose two surface points
//    differ, recorded with a = 0.  Cells row-major in the body's box, edges by first
//    corner.  pass 0 counts, pass 1 writes.
__global__ void k_body_edges(const DevVariant* var, const int* body_var, const int4* bbox,
                             const uint8_t* tag, const int* bid, const double* X, long long Vtot,
                             int* count, const int* ptr, long long* out, int pass, const double2* pcut) {
  __shared__ int sh[NT / 32 + 1];
  const int gb = blockIdx.x;
  const int v = body_var[gb];
  const DevVariant& V = var[v];
  const int k = gb - V.body0;
  const int4 bx = bbox[gb];
  const int ci0 = bx.x, ci1 = min(bx.y, V.nx - 1), cj0 = bx.z, cj1 = min(bx.w, V.ny - 1);
  const int w = ci1 - ci0 + 1, h = cj1 - cj0 + 1;
  const long long total = (w > 0 && h > 0) ? (long long)w * h : 0;
  int run = 0;
  for (long long s = 0; s < total; s += NT) {
    const long long q = s + linear_tid();
    int cnt = 0;
    unsigned mask = 0;
    long long n = 0;
    if (q < total) {
      const int i = ci0 + (int)(q % w), j = cj0 + (int)(q / w);
      n = V.base + (long long)j * V.P + i;
      if ((tag[n] & CELL_ACTIVE) && pcut) {
        CutPoly p;
        if (cut_polygon(V, bid, X, Vtot, pcut, n, p) == CUT_OK && p.n > 0) {
          int ka, kb;
          cut_chord(p, ka, kb);
          const int g = p.pt[ka] >> 2;                       // the inside corner behind the chord
          const long long gn = n + cut_ci(g) + (long long)cut_cj(g) * V.P;
          if (bid[gn] == k && (p.x[ka] != p.x[kb] || p.y[ka] != p.y[kb])) {
            mask = 1u;
            cnt = 1;
          }
        }
      } else if (tag[n] & CELL_ACTIVE) {
        const long long idx[4] = {n, n + 1, n + 1 + V.P, n + V.P};
        bool isb[4];
        for (int a = 0; a < 4; ++a) isb[a] = ((tag[idx[a]] & KIND_MASK) == K_BODY) && bid[idx[a]] == k;
        for (int a = 0; a < 4; ++a) {
          const int b2 = (a + 1) & 3;
          if (isb[a] && isb[b2] &&
              (X[idx[a]] != X[idx[b2]] || X[Vtot + idx[a]] != X[Vtot + idx[b2]])) {
            mask |= 1u << a;
            ++cnt;
          }
        }
      }
    }
    int tot;
    const int pos = block_exscan(cnt, &tot, sh);
    if (pass == 1 && cnt) {
      int o = ptr[gb] + run + pos;
      for (int a = 0; a < 4; ++a)
        if (mask & (1u << a)) out[o++] = (n << 2) | a;
    }
    run += tot;
  }
  if (pass == 0 && linear_tid() == 0) count[gb] = run;
}

// Surface points of variant v in logical order: out[(d * N + m) * 2 + c], m = j*(nx+1) + i.
__global__ void k_export_cut(const DevVariant* var, int v, const double2* pcut, long long Vtot, double* out) {
  const DevVariant& V = var[v];
  const long long N = (long long)(V.nx + 1) * (V.ny + 1);
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (m >= N) return;
  const int i = (int)(m % (V.nx + 1)), j = (int)(m / (V.nx + 1));
  const long long n = V.base + (long long)j * V.P + i;
  for (int d = 0; d < 4; ++d) {
    const double2 q = pcut[d * Vtot + n];
    out[(d * N + m) * 2] = q.x;
    out[(d * N + m) * 2 + 1] = q.y;
  }
}

// Caller-given node coordinates of variant v (logical order, [n][2]): X and the
// DISPLACED flag (set where the node is off its background-grid position); the cell
// flags of stored coefficients are cleared for k_stiffness to set again.
__global__ void k_set_coords(const DevVariant* var, int v, const double* xy, uint8_t* tag, double* X, long long Vtot) {
  const DevVariant& V = var[v];
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long N = (long long)(V.nx + 1) * (V.ny + 1);
  if (m >= N) return;
  const int i = (int)(m % (V.nx + 1)), j = (int)(m / (V.nx + 1));
  const long long n = V.base + (long long)j * V.P + i;
  const double x = xy[2 * m], y = xy[2 * m + 1];
  X[n] = x;
  X[Vtot + n] = y;
  uint8_t t = tag[n] & (uint8_t)~(DISPLACED | CELL_GENERAL | CELL_GEN32);
  if (x != grid_x(V, i) || y != grid_y(V, j)) t |= DISPLACED;
  tag[n] = t;
}

// export kernels: padded -> logical order
__global__ void k_export_coords(const DevVariant* var, int v, const double* X, long long Vtot,
                                double* xy) {
  const DevVariant& V = var[v];
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long N = (long long)(V.nx + 1) * (V.ny + 1);
  if (m >= N) return;
  const int i = (int)(m % (V.nx + 1)), j = (int)(m / (V.nx + 1));
  const long long n = V.base + (long long)j * V.P + i;
  xy[2 * m] = X[n];
  xy[2 * m + 1] = X[Vtot + n];
}

__global__ void k_export_tags(const DevVariant* var, int v, const uint8_t* tag, const int* bid,
                              int8_t* kind, int32_t* body) {
  const DevVariant& V = var[v];
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long N = (long long)(V.nx + 1) * (V.ny + 1);
  if (m >= N) return;
  const int i = (int)(m % (V.nx + 1)), j = (int)(m / (V.nx + 1));
  const long long n = V.base + (long long)j * V.P + i;
  if (kind) kind[m] = (int8_t)(tag[n] & KIND_MASK);
  if (body) body[m] = bid[n];
}

}  // namespace

static void rect_stiffness(double hx, double hy, double k[6]) {
  // closed form of K_e for an axis-aligned hx x hy rectangle, off-diagonals
  const double b = hy / hx, a = hx / hy;
  k[0] = (-2.0 * b + a) / 6.0;   // K01
  k[1] = (-b - a) / 6.0;         // K02
  k[2] = (b - 2.0 * a) / 6.0;    // K03
  k[3] = (b - 2.0 * a) / 6.0;    // K12
  k[4] = (-b - a) / 6.0;         // K13
  k[5] = (-2.0 * b + a) / 6.0;   // K23
}

template <typename T>
static T* upload(Batch& b, const std::vector<T>& h) {
  T* d = (T*)dev_alloc(b, std::max<size_t>(1, h.size()) * sizeof(T));
  if (!h.empty()) PF_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, b.stream));
  return d;
}

void build_batch(Batch& b, const pf_grid* grids, const int* body_offsets, const pf_body* bodies,
                 int nv, int sweeps, const int bc[4], const ShapeInput* shapes) {
  if (nv < 1 || !grids || !body_offsets || sweeps < 0 || !bc) throw Error{PF_EINVAL, "invalid arguments"};
  bool any_dir = false;
  for (int s = 0; s < 4; ++s) {
    if (bc[s] != PF_BC_DIRICHLET_UY && bc[s] != PF_BC_NATURAL) throw Error{PF_EINVAL, "invalid boundary kind"};
    any_dir |= bc[s] == PF_BC_DIRICHLET_UY;
    b.bc[s] = bc[s];
  }
  if (!any_dir) throw Error{PF_EINVAL, "at least one side must carry Dirichlet data"};
  b.nv = nv;
  b.sweeps = sweeps;
  if (body_offsets[0] != 0) throw Error{PF_EINVAL, "body_offsets[0] must be 0"};
  b.body_off.assign(body_offsets, body_offsets + nv + 1);
  b.B = body_offsets[nv];
  if (b.B > 0 && !bodies) throw Error{PF_EINVAL, "bodies is NULL"};
  b.bodies.assign(bodies, bodies + b.B);
  b.shape_kind.assign(b.B, PF_SHAPE_CIRCLE);
  b.kutta.assign(b.B, -1);
  b.poly_off.assign(b.B + 1, 0);
  b.poly_xy.clear();
  b.h_wake.assign(b.B, -1);
  if (shapes && !shapes->kind.empty()) {
    b.shape_kind = shapes->kind;
    b.kutta = shapes->kutta;
    b.poly_off = shapes->off;
    b.poly_xy = shapes->xy;
  }
  b.has_polygons = std::find(b.shape_kind.begin(), b.shape_kind.end(), (int)PF_SHAPE_POLYGON) != b.shape_kind.end();
  b.has_kutta = false;
  if (b.cut && !(b.cut_sigma >= 0.0 && b.cut_sigma <= 1.0))
    throw Error{PF_EINVAL, "the minimum spacing of the mixed-cell mesh must lie in [0, 1] (times min(hx, hy))"};
  std::vector<DBox> pbox(std::max(1, b.B), DBox{0, 0, 0, 0});
  for (int k = 0; k < b.B; ++k) {
    if (b.shape_kind[k] == PF_SHAPE_POLYGON) {
      const int v0 = b.poly_off[k], n = b.poly_off[k + 1] - v0;
      if (n < 3) throw Error{PF_EINVAL, "body " + std::to_string(k) + ": a polygon needs at least 3 vertices"};
      const double* p = b.poly_xy.data() + 2 * v0;
      double area2 = 0.0;
      DBox bx{p[0], p[0], p[1], p[1]};
      for (int e = 0; e < n; ++e) {
        const int f = (e + 1) % n;
        area2 += p[2 * e] * p[2 * f + 1] - p[2 * f] * p[2 * e + 1];
        bx.x0 = std::min(bx.x0, p[2 * e]);
        bx.x1 = std::max(bx.x1, p[2 * e]);
        bx.y0 = std::min(bx.y0, p[2 * e + 1]);
        bx.y1 = std::max(bx.y1, p[2 * e + 1]);
      }
      if (!(area2 > 0)) throw Error{PF_EINVAL, "body " + std::to_string(k) + ": polygon vertices must run counter-clockwise"};
      if (b.kutta[k] >= n) throw Error{PF_EINVAL, "body " + std::to_string(k) + ": Kutta vertex out of range"};
      b.has_kutta |= b.kutta[k] >= 0;
      pbox[k] = bx;
    } else {
      const pf_body& B = b.bodies[k];
      pbox[k] = DBox{B.cx - B.r, B.cx + B.r, B.cy - B.r, B.cy + B.r};
    }
  }

  // ---- host validation and layout
  std::vector<DevVariant> dv(nv);
  std::vector<int2> tij;
  std::vector<int> tvar;
  std::vector<int4> bbox(b.B);
  std::vector<int> body_var(b.B);
  long long base = 0;
  b.hv.resize(nv);
  int max_nx = 0;
  for (int v = 0; v < nv; ++v) max_nx = std::max(max_nx, grids[v].nx);
  // one row pitch for the whole batch, so one 2-D tensor map covers every variant
  const int Pc = ((max_nx + 1 + 31) / 32) * 32;
  b.P = Pc;
  std::vector<int2> cij;
  std::vector<int> cvar;
  for (int v = 0; v < nv; ++v) {
    const pf_grid& g = grids[v];
    const int nb = body_offsets[v + 1] - body_offsets[v];
    if (g.nx < 2 || g.ny < 2 || !(g.x1 > g.x0) || !(g.y1 > g.y0) || nb < 0 || nb > MAXB)
      throw Error{PF_EINVAL, "variant " + std::to_string(v) + ": invalid grid or body count"};
    if ((long long)(g.nx + 1) * (g.ny + 1) > (1LL << 40)) throw Error{PF_EINVAL, "grid too large"};
    HostVariant& H = b.hv[v];
    H.g = g;
    H.hx = (g.x1 - g.x0) / g.nx;
    H.hy = (g.y1 - g.y0) / g.ny;
    H.P = Pc;
    H.V = (long long)(g.ny + 1) * H.P;
    H.base = base;
    base += H.V;
    H.nb = nb;
    H.body0 = body_offsets[v];
    H.tiles_x = (g.nx + 1 + TX - 1) / TX;
    H.tiles_y = (g.ny + 1 + TY - 1) / TY;
    H.tile0 = (long long)tij.size();
    for (int ty = 0; ty < H.tiles_y; ++ty)
      for (int tx = 0; tx < H.tiles_x; ++tx) {
        tij.push_back(make_int2(tx * TX, ty * TY));
        tvar.push_back(v);
      }
    for (int ty = 0; ty < (g.ny + 1 + CTY - 1) / CTY; ++ty)
      for (int tx = 0; tx < (g.nx + 1 + CTX - 1) / CTX; ++tx) {
        cij.push_back(make_int2(tx * CTX, ty * CTY));
        cvar.push_back(v);
      }
    for (int k = 0; k < nb; ++k) {
      const int gk = H.body0 + k;
      const pf_body& B = b.bodies[gk];
      const bool poly = b.shape_kind[gk] == PF_SHAPE_POLYGON;
      if (!poly && !(B.r > 0))
        throw Error{PF_EINVAL, "variant " + std::to_string(v) + ": body radius must be positive"};
      const DBox bx = pbox[gk];
      if (bx.x0 < g.x0 + 2 * H.hx || bx.x1 > g.x1 - 2 * H.hx || bx.y0 < g.y0 + 2 * H.hy || bx.y1 > g.y1 - 2 * H.hy)
        throw Error{PF_EINVAL, "variant " + std::to_string(v) + ": body within 2h of the outer boundary"};
      for (int k2 = 0; k2 < k; ++k2) {
        const int gk2 = H.body0 + k2;
        const pf_body& C = b.bodies[gk2];
        if (poly || b.shape_kind[gk2] == PF_SHAPE_POLYGON) {
          const DBox cb = pbox[gk2];   // conservative: bounding boxes of polygons may not overlap
          if (!(bx.x1 < cb.x0 || cb.x1 < bx.x0 || bx.y1 < cb.y0 || cb.y1 < bx.y0))
            throw Error{PF_EINVAL, "variant " + std::to_string(v) + ": body bounding boxes overlap"};
          continue;
        }
        const double ddx = B.cx - C.cx, ddy = B.cy - C.cy;
        if (ddx * ddx + ddy * ddy <= (B.r + C.r) * (B.r + C.r))
          throw Error{PF_EINVAL, "variant " + std::to_string(v) + ": bodies overlap or touch"};
      }
      // node box of the body (polygons: 3 more cells, a Kutta wake node lies near the box)
      const int pad = poly ? 4 : 1;
      int4 bb;
      bb.x = std::max(0, (int)std::floor((bx.x0 - g.x0) / H.hx) - pad);
      bb.y = std::min(g.nx, (int)std::ceil((bx.x1 - g.x0) / H.hx) + pad);
      bb.z = std::max(0, (int)std::floor((bx.y0 - g.y0) / H.hy) - pad);
      bb.w = std::min(g.ny, (int)std::ceil((bx.y1 - g.y0) / H.hy) + pad);
      bbox[H.body0 + k] = bb;
      body_var[H.body0 + k] = v;
    }
    DevVariant& D = dv[v];
    memset(&D, 0, sizeof(D));
    D.x0 = g.x0; D.y0 = g.y0; D.hx = H.hx; D.hy = H.hy;
    D.base = H.base; D.nx = g.nx; D.ny = g.ny; D.P = H.P; D.nb = nb; D.body0 = H.body0;
    D.tiles_x = H.tiles_x; D.tiles_y = H.tiles_y;
    D.row0 = (int)(H.base / Pc);
    rect_stiffness(H.hx, H.hy, D.kr64);
    for (int m = 0; m < 6; ++m) D.kr32[m] = (float)D.kr64[m];
  }
  b.Vtot = base;
  b.Rtot = base / Pc;
  b.T = (long long)tij.size();
  b.Tcg = (long long)cij.size();
  const long long Vt = b.Vtot;

  // ---- device arrays
  b.d_var = upload(b, dv);
  std::vector<pf_body> hb(b.bodies);
  b.d_bodies = upload(b, hb);
  b.d_body_var = upload(b, body_var);
  b.d_bbox = upload(b, bbox);
  long long* d_wake = nullptr;
  if (b.has_polygons) {
    b.shp.kind = upload(b, b.shape_kind);
    b.shp.off = upload(b, b.poly_off);
    b.shp.xy = upload(b, b.poly_xy);
    b.shp.box = upload(b, pbox);
    b.shp.kutta = upload(b, b.kutta);
    d_wake = upload(b, b.h_wake);
  } else {
    b.shp = ShapeDev{};
  }
  b.tile_ij = upload(b, tij);
  b.tile_var = upload(b, tvar);
  b.tile_cg_ij = upload(b, cij);
  b.tile_cg_var = upload(b, cvar);
  b.tile_cg_gen = (uint8_t*)dev_alloc(b, std::max<long long>(1, b.Tcg));
  b.tile_cg_act = (int*)dev_alloc(b, std::max<long long>(1, b.Tcg) * sizeof(int));
  b.tag = (uint8_t*)dev_alloc(b, Vt);
  b.bid = (int*)dev_alloc(b, Vt * sizeof(int));
  b.X = (double*)dev_alloc(b, 2 * Vt * sizeof(double));
  b.K64 = (double*)dev_alloc(b, 6 * Vt * sizeof(double));
  b.K32 = (float*)dev_alloc(b, 6 * Vt * sizeof(float));
  b.K32i = (float*)dev_alloc(b, 6 * Vt * sizeof(float));
  if (b.cut) b.pcut = (double2*)dev_alloc(b, 4 * Vt * sizeof(double2));
  double2* dA = (double2*)dev_alloc(b, Vt * sizeof(double2));
  double2* dB = (double2*)dev_alloc(b, Vt * sizeof(double2));
  int* err = (int*)dev_alloc(b, sizeof(int));
  b.d_stats_i = (long long*)dev_alloc(b, nv * 6 * sizeof(long long));
  b.d_detmin = (double*)dev_alloc(b, nv * sizeof(double));
  cudaStream_t s = b.stream;
  PF_CUDA(cudaMemsetAsync(b.tag, K_INACT, Vt, s));
  PF_CUDA(cudaMemsetAsync(b.bid, 0xff, Vt * sizeof(int), s));
  PF_CUDA(cudaMemsetAsync(b.X, 0, 2 * Vt * sizeof(double), s));
  PF_CUDA(cudaMemsetAsync(b.K64, 0, 6 * Vt * sizeof(double), s));
  PF_CUDA(cudaMemsetAsync(b.K32, 0, 6 * Vt * sizeof(float), s));
  PF_CUDA(cudaMemsetAsync(b.K32i, 0, 6 * Vt * sizeof(float), s));
  PF_CUDA(cudaMemsetAsync(dA, 0, Vt * sizeof(double2), s));
  PF_CUDA(cudaMemsetAsync(err, 0, sizeof(int), s));
  PF_CUDA(cudaMemsetAsync(b.d_stats_i, 0, nv * 6 * sizeof(long long), s));
  {
    std::vector<double> big(nv, 1e300);
    PF_CUDA(cudaMemcpyAsync(b.d_detmin, big.data(), nv * sizeof(double), cudaMemcpyHostToDevice, s));
    PF_CUDA(cudaStreamSynchronize(s));
  }

  const dim3 blk(TX, TY);
  const unsigned grid = (unsigned)b.T;
  k_classify<<<grid, blk, 0, s>>>(b.d_var, b.tile_var, b.tile_ij, b.d_bodies, b.shp, b.d_bbox, b.bid, err);
  k_kinds<<<grid, blk, 0, s>>>(b.d_var, b.tile_var, b.tile_ij, b.d_bodies, b.shp, b.bid, b.tag, dA, bc[0], bc[1],
                               bc[2], bc[3], b.cut ? 1 : 0, err);
  if (b.cut) {
    k_cut_points<<<grid, blk, 0, s>>>(b.d_var, b.tile_var, b.tile_ij, b.d_bodies, b.shp, b.bid, b.tag, b.pcut, Vt);
    b.launches += 1;
  }
  if (b.has_kutta) {
    k_kutta<<<b.B, 256, 0, s>>>(b.d_var, b.d_body_var, b.shp, b.tag, dA, d_wake);
    PF_CUDA(cudaMemcpyAsync(b.h_wake.data(), d_wake, b.B * sizeof(long long), cudaMemcpyDeviceToHost, s));
    b.launches += 1;
  }
  PF_CUDA(cudaMemcpyAsync(dB, dA, Vt * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  if (sweeps > 0) {
    PF_CUDA(cudaFuncSetAttribute(k_jacobi<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, JACOBI_SMEM));
    PF_CUDA(cudaFuncSetAttribute(k_jacobi<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, JACOBI_SMEM));
  }
  for (int it = 0; it < sweeps; it += JK) {
    const int nsw = std::min(JK, sweeps - it);
    if (b.cut)
      k_jacobi<true><<<(unsigned)b.Tcg, NT, JACOBI_SMEM, s>>>(b.d_var, b.tile_cg_var, b.tile_cg_ij, b.bid, b.tag,
                                                              b.d_bbox, it, nsw, dA, dB, b.pcut, Vt);
    else
      k_jacobi<false><<<(unsigned)b.Tcg, NT, JACOBI_SMEM, s>>>(b.d_var, b.tile_cg_var, b.tile_cg_ij, b.bid, b.tag,
                                                               b.d_bbox, it, nsw, dA, dB, nullptr, Vt);
    std::swap(dA, dB);
  }
  k_finalize<<<grid, blk, 0, s>>>(b.d_var, b.tile_var, b.tile_ij, dA, b.tag, b.X, Vt);
  if (b.cut && b.cut_sigma > 0.0) {
    double2* pn = (double2*)dev_alloc(b, 4 * Vt * sizeof(double2));
    k_redistribute<<<grid, blk, 0, s>>>(b.d_var, b.tile_var, b.tile_ij, b.d_bodies, b.shp, b.bid, b.tag, b.X, Vt,
                                        b.cut_sigma, b.pcut, pn);
    PF_CUDA(cudaGetLastError());
    std::swap(b.pcut, pn);
    PF_CUDA(cudaStreamSynchronize(s));
    dev_free(b, pn);
    b.launches += 1;
  }
  k_stiffness<<<grid, blk, 0, s>>>(b.d_var, b.tile_var, b.tile_ij, b.tag, b.X, Vt, b.K64, b.K32, b.K32i, b.d_stats_i,
                                   b.d_detmin, b.bid, b.cut ? b.pcut : nullptr, err);
  k_tile_general<<<(unsigned)b.Tcg, blk, 0, s>>>(b.d_var, b.tile_cg_var, b.tile_cg_ij, b.tag, b.tile_cg_gen,
                                                 b.tile_cg_act);
  PF_CUDA(cudaGetLastError());

  // ---- body node and edge lists
  b.body_ptr = (int*)dev_alloc(b, (b.B + 1) * sizeof(int));
  b.edge_ptr = (int*)dev_alloc(b, (b.B + 1) * sizeof(int));
  int* cnt = (int*)dev_alloc(b, std::max(1, 2 * b.B) * sizeof(int));
  std::vector<int> hcnt(2 * b.B);
  if (b.B > 0) {
    k_body_nodes<<<b.B, blk, 0, s>>>(b.d_var, b.d_body_var, b.d_bbox, b.tag, b.bid, cnt, nullptr, nullptr, 0);
    k_body_edges<<<b.B, blk, 0, s>>>(b.d_var, b.d_body_var, b.d_bbox, b.tag, b.bid, b.X, Vt, cnt + b.B, nullptr,
                                     nullptr, 0, b.cut ? b.pcut : nullptr);
    PF_CUDA(cudaMemcpyAsync(hcnt.data(), cnt, 2 * b.B * sizeof(int), cudaMemcpyDeviceToHost, s));
  }
  int herr = 0;
  PF_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  if (herr & 1) throw Error{PF_EINVAL, "a grid node lies inside two bodies"};
  if (herr & 2) throw Error{PF_EINVAL, "a grid node lies at a body centre"};
  if (herr & 4) throw Error{PF_EINVAL, "mixed-cell mesh: a cell has two diagonal inside corners"};
  if (herr & 8) throw Error{PF_EINVAL, "mixed-cell mesh: a cell has inside corners of two bodies"};
  b.h_body_ptr.assign(b.B + 1, 0);
  b.h_edge_ptr.assign(b.B + 1, 0);
  for (int k = 0; k < b.B; ++k) {
    b.h_body_ptr[k + 1] = b.h_body_ptr[k] + hcnt[k];
    b.h_edge_ptr[k + 1] = b.h_edge_ptr[k] + hcnt[b.B + k];
  }
  PF_CUDA(cudaMemcpyAsync(b.body_ptr, b.h_body_ptr.data(), (b.B + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  PF_CUDA(cudaMemcpyAsync(b.edge_ptr, b.h_edge_ptr.data(), (b.B + 1) * sizeof(int), cudaMemcpyHostToDevice, s));
  b.body_nodes = (long long*)dev_alloc(b, std::max(1, b.h_body_ptr[b.B]) * sizeof(long long));
  b.bq = (double*)dev_alloc(b, std::max(1, b.h_body_ptr[b.B]) * sizeof(double));
  b.edge_rec = (long long*)dev_alloc(b, std::max(1, b.h_edge_ptr[b.B]) * sizeof(long long));
  if (b.B > 0) {
    k_body_nodes<<<b.B, blk, 0, s>>>(b.d_var, b.d_body_var, b.d_bbox, b.tag, b.bid, nullptr, b.body_ptr,
                                     b.body_nodes, 1);
    k_body_edges<<<b.B, blk, 0, s>>>(b.d_var, b.d_body_var, b.d_bbox, b.tag, b.bid, b.X, Vt, nullptr, b.edge_ptr,
                                     b.edge_rec, 1, b.cut ? b.pcut : nullptr);
  }
  PF_CUDA(cudaGetLastError());

  // ---- stats
  std::vector<long long> st(nv * 6);
  std::vector<double> dmin(nv);
  PF_CUDA(cudaMemcpyAsync(st.data(), b.d_stats_i, nv * 6 * sizeof(long long), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaMemcpyAsync(dmin.data(), b.d_detmin, nv * sizeof(double), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  b.valid = true;
  for (int v = 0; v < nv; ++v) {
    HostVariant& H = b.hv[v];
    pf_mesh_stats& S = H.stats;
    S.n_nodes = (long long)(H.g.nx + 1) * (H.g.ny + 1);
    S.n_free = st[v * 6 + 0];
    S.n_body_nodes = st[v * 6 + 1];
    S.n_inactive = st[v * 6 + 2];
    S.n_active_cells = st[v * 6 + 3];
    S.n_general_cells = st[v * 6 + 4];
    b.hv[v].n_gen32_cells = st[v * 6 + 5];
    S.n_bodies = H.nb;
    S.n_dof = S.n_free + H.nb;
    S.n_boundary_edges = b.h_edge_ptr[H.body0 + H.nb] - b.h_edge_ptr[H.body0];
    S.min_detJ = dmin[v];
    S.h = std::max(H.hx, H.hy);
    if (!(dmin[v] > 0.0)) b.valid = false;
  }
  dev_free(b, dA);
  dev_free(b, dB);
  dev_free(b, err);
  dev_free(b, cnt);
  b.launches += 8 + (sweeps + JK - 1) / JK + (b.B > 0 ? 4 : 0);
  make_schedule(b);
}

// Per-tile flags and operator-row counts of every fused-CG tile from the handle's tags.
void tile_flags(Batch& b) {
  k_tile_general<<<(unsigned)b.Tcg, dim3(TX, TY), 0, b.stream>>>(b.d_var, b.tile_cg_var, b.tile_cg_ij, b.tag,
                                                                b.tile_cg_gen, b.tile_cg_act);
  PF_CUDA(cudaGetLastError());
}

// Replace variant v's node coordinates (topology held fixed: node kinds, body membership
// and active cells stay as built) and recompute what depends on them: the element
// matrices of cells with a displaced corner, the cell and tile flags, the per-variant
// counts and min det J.
void set_coords(Batch& b, int v, const double* dev_xy) {
  if (b.cut) throw Error{PF_EINVAL, "pf_mesh_set_coords: a mixed-cell mesh places its surface points itself"};
  HostVariant& H = b.hv[v];
  const long long N = (long long)(H.g.nx + 1) * (H.g.ny + 1);
  cudaStream_t s = b.stream;
  const long long Vt = b.Vtot;
  k_set_coords<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(b.d_var, v, dev_xy, b.tag, b.X, Vt);
  PF_CUDA(cudaMemsetAsync(b.d_stats_i + 6 * v, 0, 6 * sizeof(long long), s));
  const double big = 1e300;
  PF_CUDA(cudaMemcpyAsync(b.d_detmin + v, &big, sizeof(double), cudaMemcpyHostToDevice, s));
  const dim3 blk(TX, TY);
  const unsigned nt = (unsigned)((long long)H.tiles_x * H.tiles_y);
  k_stiffness<<<nt, blk, 0, s>>>(b.d_var, b.tile_var + H.tile0, b.tile_ij + H.tile0, b.tag, b.X, Vt, b.K64, b.K32,
                                 b.K32i, b.d_stats_i, b.d_detmin, b.bid, nullptr, nullptr);
  // the variant's fused-CG tiles follow those of the variants before it
  long long t0 = 0;
  for (int u = 0; u < v; ++u)
    t0 += (long long)((b.hv[u].g.nx + 1 + CTX - 1) / CTX) * ((b.hv[u].g.ny + 1 + CTY - 1) / CTY);
  const unsigned ntc = (unsigned)((long long)((H.g.nx + 1 + CTX - 1) / CTX) * ((H.g.ny + 1 + CTY - 1) / CTY));
  k_tile_general<<<ntc, blk, 0, s>>>(b.d_var, b.tile_cg_var + t0, b.tile_cg_ij + t0, b.tag, b.tile_cg_gen + t0,
                                     b.tile_cg_act + t0);
  PF_CUDA(cudaGetLastError());
  long long st[6];
  double dmin = 0.0;
  PF_CUDA(cudaMemcpyAsync(st, b.d_stats_i + 6 * v, sizeof(st), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaMemcpyAsync(&dmin, b.d_detmin + v, sizeof(double), cudaMemcpyDeviceToHost, s));
  PF_CUDA(cudaStreamSynchronize(s));
  H.stats.n_general_cells = st[4];
  H.n_gen32_cells = st[5];
  H.stats.min_detJ = dmin;
  b.valid = true;
  for (const HostVariant& G : b.hv)
    if (!(G.stats.min_detJ > 0.0)) b.valid = false;
  b.launches += 3;
  refresh_apply_groups(b);   // the stand-alone operator's plain-tile bits follow the tile flags
  destroy_phi_view(b);       // its tile flags were made from the old coordinates
  destroy_mg(b);             // and the multigrid operators from the old element matrices
  b.solved = false;          // any earlier solution belongs to the old coordinates
}

void export_cut_points(Batch& b, int v, double* pts) {
  const long long N = (long long)(b.hv[v].g.nx + 1) * (b.hv[v].g.ny + 1);
  k_export_cut<<<(unsigned)((N + 255) / 256), 256, 0, b.stream>>>(b.d_var, v, b.pcut, b.Vtot, pts);
  PF_CUDA(cudaGetLastError());
  b.launches += 1;
}

void export_coords(Batch& b, int v, double* dev_xy) {
  const HostVariant& H = b.hv[v];
  const long long N = (long long)(H.g.nx + 1) * (H.g.ny + 1);
  k_export_coords<<<(unsigned)((N + 255) / 256), 256, 0, b.stream>>>(b.d_var, v, b.X, b.Vtot, dev_xy);
  PF_CUDA(cudaGetLastError());
}

void export_tags(Batch& b, int v, int8_t* kind, int32_t* body) {
  const HostVariant& H = b.hv[v];
  const long long N = (long long)(H.g.nx + 1) * (H.g.ny + 1);
  k_export_tags<<<(unsigned)((N + 255) / 256), 256, 0, b.stream>>>(b.d_var, v, b.tag, b.bid, kind, body);
  PF_CUDA(cudaGetLastError());
}

}  // namespace pfq4
