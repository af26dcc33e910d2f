// Velocity potential phi on the body-conforming mesh (section "Governing Equation": in
// irrotational incompressible flow u = grad phi with nabla^2 phi = 0, and the contour
// lines of phi and psi form the flow net; section "Velocity Field and Surface Tangential
// Velocity" for the element velocities).
//
// phi obeys the same Laplace equation on the same Q4 mesh, so its operator is the one the
// psi solve applies, with other constraints:
//   - phi = U x on the inlet and outlet sides (x = x0, x = x1), the uniform stream;
//   - no flux (the natural condition) on the other two sides and on every body surface,
//     which are impermeable walls;
//   - every node that is neither inactive nor on the inlet / outlet is an unknown, body
//     nodes included: phi varies along a body, so there is no multi-point constraint.
// The solve runs the fused CG kernels of the psi solve on a view of the handle that shares
// the coordinates, element matrices and tile lists, with its own node tags (the kinds
// above, the cell flags unchanged), its own tile flags, no bodies and the Dirichlet data
// taken from the x coordinates.
#include <algorithm>
#include <cstring>

#include "batch.h"

namespace pfq4 {

namespace {

// Node kinds of the phi problem from the psi tags: inactive stays inactive, the inlet and
// outlet columns are Dirichlet, every other node is free.  Cell flags are kept.
__global__ void k_phi_tags(const DevVariant* var, const int* tile_var, const int2* tile_ij, const uint8_t* tag_psi,
                           uint8_t* tag_phi) {
  const long long t = blockIdx.x;
  const DevVariant& V = var[tile_var[t]];
  const int2 ij = tile_ij[t];
  const int i = ij.x + threadIdx.x, j = ij.y + threadIdx.y;
  if (i > V.nx || j > V.ny) return;
  const long long n = V.base + (long long)j * V.P + i;
  const uint8_t tp = tag_psi[n];
  const uint8_t kind = tp & KIND_MASK;
  uint8_t k = K_FREE;
  if (kind == K_INACT) k = K_INACT;
  else if (i == 0 || i == V.nx) k = K_DIR;
  tag_phi[n] = (uint8_t)((tp & ~KIND_MASK) | k);
}

}  // namespace

void destroy_phi_view(Batch& b) {
  if (!b.phi) return;
  Batch* p = b.phi;
  for (int k = 0; k < 2; ++k)
    if (p->graph[k]) cudaGraphExecDestroy(p->graph[k]);
  if (p->graph_pcg) cudaGraphExecDestroy(p->graph_pcg);
  for (int k = 0; k < Batch::N_EV; ++k)
    if (p->ev[k]) cudaEventDestroy(p->ev[k]);
  if (p->h_poll) cudaFreeHost(p->h_poll);
  if (p->h_vs) cudaFreeHost(p->h_vs);
  dev_free_all(*p);
  delete p;
  b.phi = nullptr;
}

// The phi view of handle b: shares b's coordinates, element matrices, body-index array and
// tile lists (owned by b); owns its tags, variant table, tile flags and solver memory.
static Batch& phi_view(Batch& b) {
  if (b.phi) {
    b.phi->stream = b.stream;
    return *b.phi;
  }
  Batch* pp = new Batch();
  Batch& p = *pp;
  b.phi = pp;
  p.device = b.device;
  p.stream = b.stream;
  p.alloc_fn = b.alloc_fn;
  p.free_fn = b.free_fn;
  p.alloc_ctx = b.alloc_ctx;
  p.nv = b.nv;
  p.B = 0;
  p.sweeps = b.sweeps;
  for (int k = 0; k < 4; ++k) p.bc[k] = b.bc[k];
  p.Vtot = b.Vtot;
  p.hv = b.hv;
  p.body_off.assign(b.nv + 1, 0);
  p.h_body_ptr.assign(1, 0);
  p.h_edge_ptr.assign(1, 0);
  p.valid = b.valid;
  p.dirichlet_x = true;
  p.T = b.T;
  p.Tcg = b.Tcg;
  p.P = b.P;
  p.Rtot = b.Rtot;
  p.tile_ij = b.tile_ij;
  p.tile_var = b.tile_var;
  p.tile_cg_ij = b.tile_cg_ij;
  p.tile_cg_var = b.tile_cg_var;
  p.bid = b.bid;
  p.X = b.X;
  p.K64 = b.K64;
  p.K32 = b.K32;
  p.K32i = b.K32i;
  p.d_bodies = b.d_bodies;
  std::vector<DevVariant> dv(b.nv);
  PF_CUDA(cudaMemcpyAsync(dv.data(), b.d_var, b.nv * sizeof(DevVariant), cudaMemcpyDeviceToHost, b.stream));
  PF_CUDA(cudaStreamSynchronize(b.stream));
  for (int v = 0; v < b.nv; ++v) {
    dv[v].nb = 0;
    dv[v].body0 = 0;
    HostVariant& H = p.hv[v];
    H.nb = 0;
    H.body0 = 0;
    pf_mesh_stats& S = H.stats;
    const long long n_dir = 2LL * (H.g.ny + 1);   // inlet and outlet columns (never inactive)
    S.n_free = S.n_nodes - S.n_inactive - n_dir;
    S.n_body_nodes = 0;
    S.n_bodies = 0;
    S.n_boundary_edges = 0;
    S.n_dof = S.n_free;
  }
  const cudaStream_t s = b.stream;
  p.d_var = (DevVariant*)dev_alloc(p, b.nv * sizeof(DevVariant));
  PF_CUDA(cudaMemcpyAsync(p.d_var, dv.data(), b.nv * sizeof(DevVariant), cudaMemcpyHostToDevice, s));
  p.tag = (uint8_t*)dev_alloc(p, b.Vtot);
  PF_CUDA(cudaMemsetAsync(p.tag, K_INACT, b.Vtot, s));
  k_phi_tags<<<(unsigned)b.T, dim3(TX, TY), 0, s>>>(p.d_var, b.tile_var, b.tile_ij, b.tag, p.tag);
  p.tile_cg_gen = (uint8_t*)dev_alloc(p, std::max<long long>(1, b.Tcg));
  p.tile_cg_act = (int*)dev_alloc(p, std::max<long long>(1, b.Tcg) * sizeof(int));
  tile_flags(p);
  p.body_ptr = (int*)dev_alloc(p, sizeof(int));
  PF_CUDA(cudaMemsetAsync(p.body_ptr, 0, sizeof(int), s));
  p.edge_ptr = p.body_ptr;
  p.body_nodes = (long long*)dev_alloc(p, sizeof(long long));
  p.bq = (double*)dev_alloc(p, sizeof(double));
  PF_CUDA(cudaGetLastError());
  b.launches += 2;
  make_schedule(p);
  return p;
}

pf_status phi_solve(Batch& b, double U, const pf_solve_opts& o, double* dev_phi, pf_solve_info* info) {
  if (!b.valid) throw Error{PF_EMESH_INVALID, "mesh has det J <= 0 at a Gauss point; solve refused"};
  if (b.has_kutta)
    throw Error{PF_EINVAL, "pf_phi_solve: a Kutta circulation makes phi multivalued (it needs a cut)"};
  if (b.cut)
    throw Error{PF_EINVAL, "pf_phi_solve: phi differs between the split copies of a node, one unknown per node cannot hold it"};
  if (o.k_max < 1) throw Error{PF_EINVAL, "k_max must be >= 1"};
  Batch& p = phi_view(b);
  p.rhs_active = false;
  p.fixed_bodies = false;
  p.Uv_active = false;
  const long long before = p.launches;
  const pf_status st = solve_core(p, U, o, dev_phi, nullptr, info, true);
  b.launches += p.launches - before;
  return st;
}

void phi_velocity_field(Batch& b, int v, double* dev_u, double* dev_v) {
  if (!b.phi || !b.phi->solved) throw Error{PF_EINVAL, "no phi solution on this handle yet"};
  b.phi->stream = b.stream;
  velocity_field(*b.phi, v, dev_u, dev_v, 1);
}

}  // namespace pfq4
