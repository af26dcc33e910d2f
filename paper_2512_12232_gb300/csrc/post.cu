// Surface tangential velocity on the body boundary edges (section "Velocity Field
// and Surface Tangential Velocity"): u_t ~ (psi_c - psi_b) / d_nc with psi_c the mean
// psi of the adjacent cell, psi_b the body's constant value and d_nc the distance
// from the cell's vertex centroid to the edge line.  One thread per boundary edge.
#include <algorithm>
#include <cmath>

#include "batch.h"
#include "cut.cuh"

namespace pfq4 {

namespace {

// On the mixed-cell mesh (pcut != NULL) the edge is the chord of a cut cell: psi_c is the
// mean over the cell polygon's vertices (surface points carry the body's value), the
// centroid the mean of those vertices, and theta the polar angle of the chord midpoint.
__global__ void k_surface_velocity(const DevVariant* var, int v, int gb, const pf_body* bodies,
                                   const uint8_t* tag, const int* bid, const double* X, long long Vtot,
                                   const double* x64, const double* xb, const int* edge_ptr,
                                   const long long* edge_rec, double* theta, double* ut, const double2* pcut) {
  const DevVariant& V = var[v];
  const int e0 = edge_ptr[gb], e1 = edge_ptr[gb + 1];
  const int e = e0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= e1) return;
  const long long rec = edge_rec[e];
  const long long n = rec >> 2;
  const int a = (int)(rec & 3);
  if (pcut) {
    CutPoly p;
    cut_polygon(V, bid, X, Vtot, pcut, n, p);
    const long long idx[4] = {n, n + 1, n + 1 + V.P, n + V.P};
    double ps = 0.0, sx = 0.0, sy = 0.0;
    for (int k = 0; k < p.n; ++k) {
      ps += p.pt[k] >= 0 ? xb[gb] : x64[idx[p.corner[k]]];
      sx += p.x[k];
      sy += p.y[k];
    }
    const double psic = ps / p.n, gx = sx / p.n, gy = sy / p.n;
    int ka, kb;
    cut_chord(p, ka, kb);
    const double ex = p.x[kb] - p.x[ka], ey = p.y[kb] - p.y[ka];
    const double dnc = fabs(ex * (gy - p.y[ka]) - ey * (gx - p.x[ka])) / hypot(ex, ey);
    ut[e - e0] = (psic - xb[gb]) / dnc;
    const pf_body B = bodies[gb];
    const double mx = 0.5 * (p.x[ka] + p.x[kb]), my = 0.5 * (p.y[ka] + p.y[kb]);
    double t = atan2(my - B.cy, mx - B.cx) * (180.0 / 3.14159265358979323846);
    if (t < 0.0) t += 360.0;
    theta[e - e0] = t;
    return;
  }
  const long long idx[4] = {n, n + 1, n + 1 + V.P, n + V.P};
  double psi[4], x[4], y[4];
  for (int c = 0; c < 4; ++c) {
    const int kind = tag[idx[c]] & KIND_MASK;
    psi[c] = (kind == K_BODY) ? xb[V.body0 + bid[idx[c]]] : (kind == K_INACT ? 0.0 : x64[idx[c]]);
    x[c] = X[idx[c]];
    y[c] = X[Vtot + idx[c]];
  }
  const double psic = (((psi[0] + psi[1]) + psi[2]) + psi[3]) / 4.0;
  const double gx = (((x[0] + x[1]) + x[2]) + x[3]) / 4.0;
  const double gy = (((y[0] + y[1]) + y[2]) + y[3]) / 4.0;
  const int b2 = (a + 1) & 3;
  const double ex = x[b2] - x[a], ey = y[b2] - y[a];
  const double dnc = fabs(ex * (gy - y[a]) - ey * (gx - x[a])) / hypot(ex, ey);
  const double C = xb[gb];
  ut[e - e0] = (psic - C) / dnc;
  const pf_body B = bodies[gb];
  const double mx = 0.5 * (x[a] + x[b2]), my = 0.5 * (y[a] + y[b2]);
  double t = atan2(my - B.cy, mx - B.cx) * (180.0 / 3.14159265358979323846);
  if (t < 0.0) t += 360.0;
  theta[e - e0] = t;
}

// Element velocity of the solved psi: u = dpsi/dy, v = -dpsi/dx of the bilinear
// interpolant at the cell centre (xi = eta = 0), where dN_a/dxi = xi_a / 4 and
// dN_a/deta = eta_a / 4, through the isoparametric Jacobian.  One thread per logical cell
// (i, j), i < nx, j < ny, written at j*nx + i; inactive cells get 0.  Corners of an active
// cell are never inactive; BODY corners carry their body's value.
// potential = 1: the field is the velocity potential, u = dphi/dx and v = dphi/dy.
// On the mixed-cell mesh (pcut != NULL) a cut cell takes the area-weighted mean of its
// pieces' gradients: the triangle's constant gradient, the quadrilateral's at its centre.
__global__ void k_velocity_field(const DevVariant* var, int v, const uint8_t* tag, const int* bid, const double* X,
                                 long long Vtot, const double* x64, const double* xb, int potential, double* u_out,
                                 double* v_out, const double2* pcut) {
  const DevVariant& V = var[v];
  const long long m = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (m >= (long long)V.nx * V.ny) return;
  const int i = (int)(m % V.nx), j = (int)(m / V.nx);
  const long long n = V.base + (long long)j * V.P + i;
  if (!(tag[n] & CELL_ACTIVE)) {
    u_out[m] = 0.0;
    v_out[m] = 0.0;
    return;
  }
  const long long idx[4] = {n, n + 1, n + 1 + V.P, n + V.P};   // corners counter-clockwise
  const double dxi[4] = {-0.25, 0.25, 0.25, -0.25}, deta[4] = {-0.25, -0.25, 0.25, 0.25};
  if (pcut) {
    CutPoly p;
    cut_polygon(V, bid, X, Vtot, pcut, n, p);
    if (p.n > 0) {
      double fv[5];
      for (int k = 0; k < p.n; ++k)
        fv[k] = p.pt[k] >= 0 ? xb[V.body0 + bid[idx[p.corner[k]]]] : x64[idx[p.corner[k]]];
      int piece[2][4], nv[2];
      const int np = cut_pieces(p, piece, nv);
      double gx = 0.0, gy = 0.0, ws = 0.0;
      for (int q = 0; q < np; ++q) {
        const int* pv = piece[q];
        double px, py, w;
        if (nv[q] == 3) {
          const double x[3] = {p.x[pv[0]], p.x[pv[1]], p.x[pv[2]]}, y[3] = {p.y[pv[0]], p.y[pv[1]], p.y[pv[2]]};
          const double two_a = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
          const double bb[3] = {y[1] - y[2], y[2] - y[0], y[0] - y[1]};
          const double cc[3] = {x[2] - x[1], x[0] - x[2], x[1] - x[0]};
          px = (bb[0] * fv[pv[0]] + bb[1] * fv[pv[1]] + bb[2] * fv[pv[2]]) / two_a;
          py = (cc[0] * fv[pv[0]] + cc[1] * fv[pv[1]] + cc[2] * fv[pv[2]]) / two_a;
          w = 0.5 * two_a;
        } else {
          double q00 = 0.0, q01 = 0.0, q10 = 0.0, q11 = 0.0;
          for (int c = 0; c < 4; ++c) {
            q00 += p.x[pv[c]] * dxi[c];
            q01 += p.y[pv[c]] * dxi[c];
            q10 += p.x[pv[c]] * deta[c];
            q11 += p.y[pv[c]] * deta[c];
          }
          const double det = q00 * q11 - q01 * q10;
          px = 0.0;
          py = 0.0;
          for (int c = 0; c < 4; ++c) {
            px += (q11 * dxi[c] - q01 * deta[c]) / det * fv[pv[c]];
            py += (-q10 * dxi[c] + q00 * deta[c]) / det * fv[pv[c]];
          }
          w = 4.0 * det;
        }
        gx += w * px;
        gy += w * py;
        ws += w;
      }
      gx /= ws;
      gy /= ws;
      u_out[m] = potential ? gx : gy;
      v_out[m] = potential ? gy : -gx;
      return;
    }
  }
  double f[4], j00 = 0.0, j01 = 0.0, j10 = 0.0, j11 = 0.0;
  for (int c = 0; c < 4; ++c) {
    const int kind = tag[idx[c]] & KIND_MASK;
    f[c] = kind == K_BODY ? xb[V.body0 + bid[idx[c]]] : x64[idx[c]];
    const double x = X[idx[c]], y = X[Vtot + idx[c]];
    j00 += x * dxi[c];
    j01 += y * dxi[c];
    j10 += x * deta[c];
    j11 += y * deta[c];
  }
  const double det = j00 * j11 - j01 * j10;
  double fx = 0.0, fy = 0.0;
  for (int c = 0; c < 4; ++c) {
    fx += (j11 * dxi[c] - j01 * deta[c]) / det * f[c];
    fy += (-j10 * dxi[c] + j00 * deta[c]) / det * f[c];
  }
  u_out[m] = potential ? fx : fy;
  v_out[m] = potential ? fy : -fx;
}

}  // namespace

void velocity_field(Batch& b, int v, double* dev_u, double* dev_v, int potential) {
  if (!b.solved) throw Error{PF_EINVAL, "no solution on this handle yet"};
  if (!dev_u || !dev_v) throw Error{PF_EINVAL, "NULL output"};
  const long long ncell = (long long)b.hv[v].g.nx * b.hv[v].g.ny;
  if (ncell == 0) return;
  k_velocity_field<<<(unsigned)((ncell + 255) / 256), 256, 0, b.stream>>>(b.d_var, v, b.tag, b.bid, b.X, b.Vtot,
                                                                          b.x64, b.sol64, potential, dev_u, dev_v,
                                                                          b.cut ? b.pcut : nullptr);
  PF_CUDA(cudaGetLastError());
  b.launches += 1;
  PF_CUDA(cudaStreamSynchronize(b.stream));
}

int surface_velocity(Batch& b, int v, int body, double* theta, double* ut, int cap) {
  if (!b.solved) throw Error{PF_EINVAL, "no solution on this handle yet"};
  const int gb = b.hv[v].body0 + body;
  const int ne = b.h_edge_ptr[gb + 1] - b.h_edge_ptr[gb];
  if (ne == 0) return 0;
  double* d = (double*)dev_alloc(b, 2 * (size_t)ne * sizeof(double));
  k_surface_velocity<<<(ne + 127) / 128, 128, 0, b.stream>>>(b.d_var, v, gb, b.d_bodies, b.tag, b.bid, b.X, b.Vtot,
                                                             b.x64, b.sol64, b.edge_ptr, b.edge_rec, d, d + ne,
                                                             b.cut ? b.pcut : nullptr);
  PF_CUDA(cudaGetLastError());
  b.launches += 1;
  const int m = std::min(ne, cap);
  if (m > 0 && theta) PF_CUDA(cudaMemcpyAsync(theta, d, m * sizeof(double), cudaMemcpyDeviceToHost, b.stream));
  if (m > 0 && ut) PF_CUDA(cudaMemcpyAsync(ut, d + ne, m * sizeof(double), cudaMemcpyDeviceToHost, b.stream));
  PF_CUDA(cudaStreamSynchronize(b.stream));
  dev_free(b, d);
  return ne;
}

}  // namespace pfq4
