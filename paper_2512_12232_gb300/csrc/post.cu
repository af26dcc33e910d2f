// Surface tangential velocity on the body boundary edges (section "Velocity Field
// and Surface Tangential Velocity"): u_t ~ (psi_c - psi_b) / d_nc with psi_c the mean
// psi of the adjacent cell, psi_b the body's constant value and d_nc the distance
// from the cell's vertex centroid to the edge line.  One thread per boundary edge.
#include <algorithm>
#include <cmath>

#include "batch.h"

namespace pfq4 {

namespace {

__global__ void k_surface_velocity(const DevVariant* var, int v, int gb, const pf_body* bodies,
                                   const uint8_t* tag, const int* bid, const double* X, long long Vtot,
                                   const double* x64, const double* xb, const int* edge_ptr,
                                   const long long* edge_rec, double* theta, double* ut) {
  const DevVariant& V = var[v];
  const int e0 = edge_ptr[gb], e1 = edge_ptr[gb + 1];
  const int e = e0 + blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= e1) return;
  const long long rec = edge_rec[e];
  const long long n = rec >> 2;
  const int a = (int)(rec & 3);
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
__global__ void k_velocity_field(const DevVariant* var, int v, const uint8_t* tag, const int* bid, const double* X,
                                 long long Vtot, const double* x64, const double* xb, int potential, double* u_out,
                                 double* v_out) {
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
                                                                          b.x64, b.sol64, potential, dev_u, dev_v);
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
                                                             b.x64, b.sol64, b.edge_ptr, b.edge_rec, d, d + ne);
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
