// Geometry of the mixed-cell mesh (section "Body-Conforming Grid Generation": grid points
// just inside a body move onto its surface, a point meeting the surface twice is split,
// neighbouring cells become triangles and pentagons, a pentagon is divided into a
// triangle and a quadrilateral), shared by the mesh build and the post-processing.
//
// Surface points: pcut[d * Vtot + n] is the point where the grid edge from BODY node n
// towards its neighbour in direction d (0 E, 1 N, 2 W, 3 S) crosses the body's circle,
// for an outside neighbour; NaN otherwise.  BODY nodes keep their background position in X.
#pragma once

#include "batch.h"

namespace pfq4 {

// corner a of the cell whose corner 0 is node (i, j) is node (i + cut_ci(a), j + cut_cj(a))
__device__ __forceinline__ int cut_ci(int a) { return (a == 1 || a == 2) ? 1 : 0; }
__device__ __forceinline__ int cut_cj(int a) { return a >= 2 ? 1 : 0; }

struct CutPoly {
  int n;              // vertices: 3, 4 or 5; 0 for a cell without an inside corner
  double x[5], y[5];
  int corner[5];      // the cell corner each vertex stands for
  int pt[5];          // a surface point: (inside corner << 2) | direction; -1 for a cell corner
};

enum { CUT_OK = 0, CUT_SADDLE = 1, CUT_TWO_BODIES = 2 };

// The cell polygon walked counter-clockwise from corner 0: every outside corner a, and
// after it the surface point on edge a (corner a -> a+1) when exactly one end of the edge
// is inside.  n is the cell's corner-0 node.
__device__ inline int cut_polygon(const DevVariant& V, const int* bid, const double* X, long long Vtot,
                                  const double2* pcut, long long n, CutPoly& p) {
  const long long idx[4] = {n, n + 1, n + 1 + V.P, n + V.P};
  bool in[4];
  int body = -1, st = CUT_OK;
  for (int a = 0; a < 4; ++a) {
    const int b = bid[idx[a]];
    in[a] = b >= 0;
    if (in[a]) {
      if (body >= 0 && b != body) st = CUT_TWO_BODIES;
      body = b;
    }
  }
  p.n = 0;
  if (body < 0) return CUT_OK;
  if (in[0] == in[2] && in[1] == in[3] && in[0] != in[1]) return CUT_SADDLE;
  if (st != CUT_OK) return st;
  for (int a = 0; a < 4; ++a) {
    const int b2 = (a + 1) & 3;
    if (!in[a]) {
      p.x[p.n] = X[idx[a]];
      p.y[p.n] = X[Vtot + idx[a]];
      p.corner[p.n] = a;
      p.pt[p.n] = -1;
      ++p.n;
    }
    if (in[a] != in[b2]) {
      const int g = in[a] ? a : b2, d = in[a] ? a : ((a + 2) & 3);
      const double2 q = pcut[d * Vtot + idx[g]];
      p.x[p.n] = q.x;
      p.y[p.n] = q.y;
      p.corner[p.n] = g;
      p.pt[p.n] = (g << 2) | d;
      ++p.n;
    }
  }
  return CUT_OK;
}

// Indices (into the polygon) of the chord's two surface points in the order the cell's
// boundary runs counter-clockwise.
__device__ inline void cut_chord(const CutPoly& p, int& ka, int& kb) {
  int k0 = -1, k1 = -1;
  for (int k = 0; k < p.n; ++k)
    if (p.pt[k] >= 0) {
      if (k0 < 0) k0 = k;
      else k1 = k;
    }
  if (k0 == 0 && k1 == p.n - 1) {
    ka = k1;
    kb = k0;
  } else {
    ka = k0;
    kb = k1;
  }
}

// The pieces of a cut polygon as vertex lists into it: one piece (3 or 4 vertices), or for
// a pentagon with inside corner m the triangle (P+, c_{m+1}, c_{m+2}) and the
// quadrilateral (P+, c_{m+2}, c_{m+3}, P-), P+ the point on edge m.  The walk of a
// pentagon is a rotation of (P+, c_{m+1}, c_{m+2}, c_{m+3}, P-), so both follow from the
// position of P+.  Returns the number of pieces; sizes in nv[].
__device__ inline int cut_pieces(const CutPoly& p, int piece[2][4], int nv[2]) {
  if (p.n <= 4) {
    for (int k = 0; k < p.n; ++k) piece[0][k] = k;
    nv[0] = p.n;
    return 1;
  }
  int k = 0;
  for (int q = 0; q < 5; ++q)
    if (p.pt[q] >= 0 && (p.pt[q] & 3) == (p.pt[q] >> 2)) k = q;   // P+: the point on edge m leaves m in direction m
  const int r0 = k, r1 = (k + 1) % 5, r2 = (k + 2) % 5, r3 = (k + 3) % 5, r4 = (k + 4) % 5;
  piece[0][0] = r0; piece[0][1] = r1; piece[0][2] = r2;
  nv[0] = 3;
  piece[1][0] = r0; piece[1][1] = r2; piece[1][2] = r3; piece[1][3] = r4;
  nv[1] = 4;
  return 2;
}

// Linear triangle: K_ab = (b_a b_b + c_a c_b) / (4A), b_a = y_{a+1} - y_{a+2},
// c_a = x_{a+2} - x_{a+1}; returns 2A.
__device__ inline double p1_element(const double x[3], const double y[3], double K[3][3]) {
  const double two_a = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
  const double b[3] = {y[1] - y[2], y[2] - y[0], y[0] - y[1]};
  const double c[3] = {x[2] - x[1], x[0] - x[2], x[1] - x[0]};
  const double s = 1.0 / (2.0 * two_a);
  for (int a = 0; a < 3; ++a)
    for (int e = 0; e < 3; ++e) K[a][e] = (b[a] * b[e] + c[a] * c[e]) * s;
  return two_a;
}

// Q4 element (2x2 Gauss) on corners x[4], y[4] counter-clockwise: the upper triangle of
// K_e; returns the smallest det J at the Gauss points.  The bilinear map is
// x = a0 + a1 xi + a2 eta + a3 xi eta (likewise y with b), so J = [[a1 + a3 eta, b1 + b3 eta],
// [a2 + a3 xi, b2 + b3 xi]], and with grad N_a = J^{-1} (dN_a/dxi, dN_a/deta)
//   K_ab = sum_g (A_g dxi_a dxi_b - B_g (dxi_a deta_b + deta_a dxi_b) + C_g deta_a deta_b),
//   A = (J10^2 + J11^2) / det, B = (J00 J10 + J01 J11) / det, C = (J00^2 + J01^2) / det,
// the same 2x2 Gauss sum as forming grad N at every point, in fewer FP64 operations.
__device__ inline double q4_element(const double x[4], const double y[4], double K[4][4]) {
  const double g = 0.57735026918962576451;   // 1/sqrt(3)
  const double xi_a[4] = {-1, 1, 1, -1}, eta_a[4] = {-1, -1, 1, 1};
  const double gx[4] = {-g, g, g, -g}, gy[4] = {-g, -g, g, g};
  const double a1 = 0.25 * ((x[1] - x[0]) + (x[2] - x[3])), a2 = 0.25 * ((x[3] - x[0]) + (x[2] - x[1]));
  const double a3 = 0.25 * ((x[0] - x[1]) + (x[2] - x[3]));
  const double b1 = 0.25 * ((y[1] - y[0]) + (y[2] - y[3])), b2 = 0.25 * ((y[3] - y[0]) + (y[2] - y[1]));
  const double b3 = 0.25 * ((y[0] - y[1]) + (y[2] - y[3]));
  for (int a = 0; a < 4; ++a)
    for (int e = 0; e < 4; ++e) K[a][e] = 0.0;
  double dm = 1e300;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const double j00 = a1 + a3 * gy[q], j01 = b1 + b3 * gy[q];
    const double j10 = a2 + a3 * gx[q], j11 = b2 + b3 * gx[q];
    const double det = j00 * j11 - j01 * j10;
    dm = fmin(dm, det);
    const double inv = 1.0 / det;
    const double A = (j10 * j10 + j11 * j11) * inv, B = (j00 * j10 + j01 * j11) * inv;
    const double C = (j00 * j00 + j01 * j01) * inv;
    double dxi[4], deta[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      dxi[a] = 0.25 * xi_a[a] * (1.0 + eta_a[a] * gy[q]);
      deta[a] = 0.25 * eta_a[a] * (1.0 + xi_a[a] * gx[q]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int e = a + 1; e < 4; ++e)
        K[a][e] += A * (dxi[a] * dxi[e]) - B * (dxi[a] * deta[e] + deta[a] * dxi[e]) + C * (deta[a] * deta[e]);
  }
  return dm;
}

// The cut cell's matrix on its four corners as the six off-diagonals
// (K01, K02, K03, K12, K13, K23): the pieces' element matrices scattered by the vertex ->
// corner map (couplings between two vertices of one corner belong to its diagonal, which
// every reader forms from the row sum).  Returns the smallest det J of the pieces (twice the
// area for a triangle).
__device__ inline double cut_cell_matrix(const CutPoly& p, double k6[6]) {
  double M[4][4] = {};
  int piece[2][4], nv[2];
  const int np = cut_pieces(p, piece, nv);
  double dm = 1e300;
  for (int q = 0; q < np; ++q) {
    const int* v = piece[q];
    if (nv[q] == 3) {
      const double x[3] = {p.x[v[0]], p.x[v[1]], p.x[v[2]]}, y[3] = {p.y[v[0]], p.y[v[1]], p.y[v[2]]};
      double K[3][3];
      dm = fmin(dm, p1_element(x, y, K));
      for (int a = 0; a < 3; ++a)
        for (int e = a + 1; e < 3; ++e) {
          const int ca = p.corner[v[a]], ce = p.corner[v[e]];
          if (ca != ce) M[min(ca, ce)][max(ca, ce)] += K[a][e];
        }
    } else {
      const double x[4] = {p.x[v[0]], p.x[v[1]], p.x[v[2]], p.x[v[3]]};
      const double y[4] = {p.y[v[0]], p.y[v[1]], p.y[v[2]], p.y[v[3]]};
      double K[4][4];
      dm = fmin(dm, q4_element(x, y, K));
      for (int a = 0; a < 4; ++a)
        for (int e = a + 1; e < 4; ++e) {
          const int ca = p.corner[v[a]], ce = p.corner[v[e]];
          if (ca != ce) M[min(ca, ce)][max(ca, ce)] += K[a][e];
        }
    }
  }
  k6[0] = M[0][1]; k6[1] = M[0][2]; k6[2] = M[0][3];
  k6[3] = M[1][2]; k6[4] = M[1][3]; k6[5] = M[2][3];
  return dm;
}

}  // namespace pfq4
