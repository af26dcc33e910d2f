// C ABI of the library: argument checks, error capture (no exception crosses the
// boundary), device-memory ownership of the handle, and dispatch to the mesh,
// solver, post-processing and gradient code.
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "batch.h"

namespace pfq4 {

static thread_local std::string g_err;
static pf_alloc_fn g_alloc = nullptr;
static pf_free_fn g_free = nullptr;
static void* g_ctx = nullptr;

void set_last_error(const std::string& msg) { g_err = msg; }

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    cudaGetLastError();   // clear a non-sticky error so later calls start clean
    const pf_status code = (e == cudaErrorMemoryAllocation) ? PF_ENOMEM : PF_ECUDA;
    throw Error{code, std::string(what) + ": " + cudaGetErrorString(e)};
  }
}

void* dev_alloc(Batch& b, size_t bytes) {
  void* p = nullptr;
  bytes = (bytes + 255) & ~size_t(255);
  if (b.alloc_fn) {
    p = b.alloc_fn(bytes, (void*)b.stream, b.alloc_ctx);
    if (!p) throw Error{PF_ENOMEM, "allocator hook returned NULL"};
  } else {
    const cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      throw Error{PF_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e)};
    }
  }
  b.allocs.push_back({p, bytes});
  b.bytes += bytes;
  return p;
}

void dev_free(Batch& b, void* p) {
  for (size_t k = 0; k < b.allocs.size(); ++k) {
    if (b.allocs[k].first != p) continue;
    cudaStreamSynchronize(b.stream);
    if (b.free_fn) b.free_fn(p, (void*)b.stream, b.alloc_ctx);
    else cudaFree(p);
    b.bytes -= b.allocs[k].second;
    b.allocs.erase(b.allocs.begin() + k);
    return;
  }
}

void dev_free_all(Batch& b) {
  cudaStreamSynchronize(b.stream);
  for (auto& a : b.allocs) {
    if (b.free_fn) b.free_fn(a.first, (void*)b.stream, b.alloc_ctx);
    else cudaFree(a.first);
  }
  b.allocs.clear();
  b.bytes = 0;
}

static pf_status fail(const Error& e) {
  g_err = e.msg;
  return e.code;
}

template <typename F>
static pf_status guarded(F&& f) {
  try {
    g_err.clear();
    return f();
  } catch (const Error& e) {
    return fail(e);
  } catch (const std::bad_alloc&) {
    return fail(Error{PF_ENOMEM, "host allocation failed"});
  } catch (const std::exception& e) {
    return fail(Error{PF_EINVAL, e.what()});
  }
}

static void bind(Batch* b, void* stream) {
  if (!b) throw Error{PF_EINVAL, "NULL handle"};
  int dev = -1;
  PF_CUDA(cudaGetDevice(&dev));
  if (dev != b->device) throw Error{PF_EINVAL, "call made with another device current than the handle's"};
  b->stream = (cudaStream_t)stream;
}

static void check_variant(const Batch* b, int v) {
  if (v < 0 || v >= b->nv) throw Error{PF_EINVAL, "variant index out of range"};
}

}  // namespace pfq4

using namespace pfq4;

extern "C" {

pf_status pf_set_allocator(pf_alloc_fn alloc, pf_free_fn free_fn, void* ctx) {
  if ((alloc == nullptr) != (free_fn == nullptr)) {
    g_err = "alloc and free must both be set or both be NULL";
    return PF_EINVAL;
  }
  g_alloc = alloc;
  g_free = free_fn;
  g_ctx = ctx;
  return PF_OK;
}

static pf_status build_handle(const pf_grid* grids, const int* body_offsets, const pf_body* bodies,
                              int n_variants, int sweeps, const int bc[4], void* stream, pf_batch** out,
                              const ShapeInput* shapes, bool cut = false, double cut_sigma = 0.0);

pf_status pf_batch_build(const pf_grid* grids, const int* body_offsets, const pf_body* bodies, int n_variants,
                         int sweeps, const int bc[4], void* stream, pf_batch** out) {
  return build_handle(grids, body_offsets, bodies, n_variants, sweeps, bc, stream, out, nullptr);
}

// Host copies of the bodies of a pf_shape list: circles as pf_body rows (polygons keep
// their reference point there) and the polygons' kinds, vertices and Kutta vertices.
static pf_status parse_shapes(const int* body_offsets, const pf_shape* shapes, int n_variants,
                              std::vector<pf_body>& bodies, ShapeInput& si) {
  if (!body_offsets || n_variants < 1) {
    g_err = "invalid arguments";
    return PF_EINVAL;
  }
  const int B = body_offsets[n_variants];
  if (B < 0 || (B > 0 && !shapes)) {
    g_err = "shapes is NULL";
    return PF_EINVAL;
  }
  try {
    bodies.resize(std::max(1, B));
    si.off.push_back(0);
    for (int k = 0; k < B; ++k) {
      const pf_shape& sh = shapes[k];
      if (sh.kind != PF_SHAPE_CIRCLE && sh.kind != PF_SHAPE_POLYGON) {
        g_err = "invalid shape kind";
        return PF_EINVAL;
      }
      bodies[k] = pf_body{sh.cx, sh.cy, sh.kind == PF_SHAPE_CIRCLE ? sh.r : 0.0};
      si.kind.push_back(sh.kind);
      si.kutta.push_back(sh.kind == PF_SHAPE_POLYGON ? sh.kutta_vertex : -1);
      if (sh.kind == PF_SHAPE_POLYGON) {
        if (sh.n_vertices < 3 || !sh.vertex_xy) {
          g_err = "a polygon needs at least 3 vertices";
          return PF_EINVAL;
        }
        si.xy.insert(si.xy.end(), sh.vertex_xy, sh.vertex_xy + 2 * (size_t)sh.n_vertices);
      }
      si.off.push_back((int)(si.xy.size() / 2));
    }
  } catch (const std::exception& e) {
    g_err = std::string("host allocation failed: ") + e.what();
    return PF_ENOMEM;
  }
  return PF_OK;
}

pf_status pf_batch_build_shapes(const pf_grid* grids, const int* body_offsets, const pf_shape* shapes,
                                int n_variants, int sweeps, const int bc[4], void* stream, pf_batch** out) {
  if (out) *out = nullptr;
  if (!out) {
    g_err = "invalid arguments";
    return PF_EINVAL;
  }
  std::vector<pf_body> bodies;
  ShapeInput si;
  const pf_status st = parse_shapes(body_offsets, shapes, n_variants, bodies, si);
  if (st != PF_OK) return st;
  return build_handle(grids, body_offsets, bodies.data(), n_variants, sweeps, bc, stream, out, &si);
}

pf_status pf_batch_build_cut(const pf_grid* grids, const int* body_offsets, const pf_shape* shapes, int n_variants,
                             int sweeps, const int bc[4], double min_spacing, void* stream, pf_batch** out) {
  if (out) *out = nullptr;
  if (!out) {
    g_err = "invalid arguments";
    return PF_EINVAL;
  }
  std::vector<pf_body> bodies;
  ShapeInput si;
  const pf_status st = parse_shapes(body_offsets, shapes, n_variants, bodies, si);
  if (st != PF_OK) return st;
  return build_handle(grids, body_offsets, bodies.data(), n_variants, sweeps, bc, stream, out, &si, true,
                      min_spacing);
}

static pf_status build_handle(const pf_grid* grids, const int* body_offsets, const pf_body* bodies,
                              int n_variants, int sweeps, const int bc[4], void* stream, pf_batch** out,
                              const ShapeInput* shapes, bool cut, double cut_sigma) {
  if (!out) {
    g_err = "out is NULL";
    return PF_EINVAL;
  }
  *out = nullptr;
  Batch* b = new (std::nothrow) Batch();
  if (!b) {
    g_err = "host allocation failed";
    return PF_ENOMEM;
  }
  const pf_status st = guarded([&]() -> pf_status {
    PF_CUDA(cudaGetDevice(&b->device));
    b->stream = (cudaStream_t)stream;
    b->alloc_fn = g_alloc;
    b->free_fn = g_free;
    b->alloc_ctx = g_ctx;
    b->cut = cut;
    b->cut_sigma = cut_sigma;
    build_batch(*b, grids, body_offsets, bodies, n_variants, sweeps, bc, shapes);
    if (!b->valid) throw Error{PF_EMESH_INVALID, "mesh has det J <= 0 at a Gauss point of an active cell"};
    return PF_OK;
  });
  if (st == PF_OK || st == PF_EMESH_INVALID) {
    *out = (pf_batch*)b;
  } else {
    dev_free_all(*b);
    delete b;
  }
  return st;
}

pf_status pf_mesh_build(const pf_grid* grid, const pf_body* bodies, int n_bodies, int sweeps, const int bc[4],
                        void* stream, pf_batch** out) {
  const int off[2] = {0, n_bodies};
  if (n_bodies < 0) {
    g_err = "n_bodies < 0";
    return PF_EINVAL;
  }
  return pf_batch_build(grid, off, bodies, 1, sweeps, bc, stream, out);
}

void pf_batch_destroy(pf_batch* h) {
  Batch* b = (Batch*)h;
  if (!b) return;
  destroy_phi_view(*b);
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) cudaGraphExecDestroy(b->graph[k]);
  if (b->graph_pcg) cudaGraphExecDestroy(b->graph_pcg);
  for (int k = 0; k < Batch::N_EV; ++k)
    if (b->ev[k]) cudaEventDestroy(b->ev[k]);
  if (b->h_poll) cudaFreeHost(b->h_poll);
  if (b->h_vs) cudaFreeHost(b->h_vs);
  dev_free_all(*b);
  delete b;
}

pf_status pf_batch_size(const pf_batch* h, int* n_variants, long long* total_nodes, int* total_bodies) {
  return guarded([&]() -> pf_status {
    const Batch* b = (const Batch*)h;
    if (!b) throw Error{PF_EINVAL, "NULL handle"};
    long long n = 0;
    for (auto& H : b->hv) n += H.stats.n_nodes;
    if (n_variants) *n_variants = b->nv;
    if (total_nodes) *total_nodes = n;
    if (total_bodies) *total_bodies = b->B;
    return PF_OK;
  });
}

pf_status pf_mesh_stats_get(const pf_batch* h, int variant, pf_mesh_stats* out) {
  return guarded([&]() -> pf_status {
    const Batch* b = (const Batch*)h;
    if (!b || !out) throw Error{PF_EINVAL, "NULL argument"};
    check_variant(b, variant);
    *out = b->hv[variant].stats;
    return PF_OK;
  });
}

pf_status pf_mesh_coords(const pf_batch* h, int variant, double* dev_xy, void* stream) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    bind(b, stream);
    check_variant(b, variant);
    if (!dev_xy) throw Error{PF_EINVAL, "dev_xy is NULL"};
    export_coords(*b, variant, dev_xy);
    PF_CUDA(cudaStreamSynchronize(b->stream));
    return PF_OK;
  });
}

pf_status pf_mesh_set_coords(pf_batch* h, int variant, const double* dev_xy, void* stream) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    bind(b, stream);
    check_variant(b, variant);
    if (!dev_xy) throw Error{PF_EINVAL, "dev_xy is NULL"};
    set_coords(*b, variant, dev_xy);
    return b->valid ? PF_OK : PF_EMESH_INVALID;
  });
}

pf_status pf_coords_vjp(pf_batch* h, const double* dev_gX, double* gc, void* stream) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    bind(b, stream);
    if (!dev_gX || (!gc && b->B > 0)) throw Error{PF_EINVAL, "NULL argument"};
    coords_vjp(*b, dev_gX, gc);
    return PF_OK;
  });
}

pf_status pf_mesh_cut_points(const pf_batch* h, int variant, double* dev_pts, void* stream) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    bind(b, stream);
    check_variant(b, variant);
    if (!b->cut) throw Error{PF_EINVAL, "pf_mesh_cut_points: not a mixed-cell mesh"};
    if (!dev_pts) throw Error{PF_EINVAL, "dev_pts is NULL"};
    export_cut_points(*b, variant, dev_pts);
    PF_CUDA(cudaStreamSynchronize(b->stream));
    return PF_OK;
  });
}

pf_status pf_mesh_tags(const pf_batch* h, int variant, int8_t* dev_kind, int32_t* dev_body, void* stream) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    bind(b, stream);
    check_variant(b, variant);
    export_tags(*b, variant, dev_kind, dev_body);
    PF_CUDA(cudaStreamSynchronize(b->stream));
    return PF_OK;
  });
}

pf_status pf_apply(pf_batch* h, int precision, const double* dev_p, double* dev_y, double* body_sums,
                   void* stream) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    bind(b, stream);
    if (!dev_p || !dev_y) throw Error{PF_EINVAL, "NULL vector"};
    if (precision != PF_FP64 && precision != PF_MIXED) throw Error{PF_EINVAL, "invalid precision"};
    apply_operator(*b, precision, dev_p, dev_y, body_sums);
    return PF_OK;
  });
}

pf_status pf_psi_solve(pf_batch* h, double U, const pf_solve_opts* opts, double* dev_psi, double* body_psi,
                       pf_solve_info* info, void* stream) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    bind(b, stream);
    pf_solve_opts o{};
    o.tol = 1e-8;
    o.k_max = 10000000;
    o.precision = PF_MIXED;
    o.inner_tol = PF_DEFAULT_INNER_TOL;
    if (opts) o = *opts;
    return psi_solve(*b, U, o, dev_psi, body_psi, info);
  });
}

pf_status pf_psi_solve_schur(pf_batch* h, double U, const pf_solve_opts* opts, double* dev_psi, double* body_psi,
                             pf_solve_info* info, void* stream) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    bind(b, stream);
    pf_solve_opts o{};
    o.tol = 1e-8;
    o.k_max = 10000000;
    o.precision = PF_MIXED;
    o.inner_tol = PF_DEFAULT_INNER_TOL;
    if (opts) o = *opts;
    return schur_solve(*b, U, o, dev_psi, body_psi, info);
  });
}

pf_status pf_phi_solve(pf_batch* h, double U, const pf_solve_opts* opts, double* dev_phi, pf_solve_info* info,
                       void* stream) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    bind(b, stream);
    pf_solve_opts o{};
    o.tol = 1e-8;
    o.k_max = 10000000;
    o.precision = PF_MIXED;
    o.inner_tol = PF_DEFAULT_INNER_TOL;
    if (opts) o = *opts;
    return phi_solve(*b, U, o, dev_phi, info);
  });
}

pf_status pf_phi_velocity_field(pf_batch* h, int variant, double* dev_u, double* dev_v, void* stream) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    bind(b, stream);
    check_variant(b, variant);
    phi_velocity_field(*b, variant, dev_u, dev_v);
    return PF_OK;
  });
}

pf_status pf_apply_timing(pf_batch* h, int precision, int reps, double* us, double* bytes, void* stream) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    if (!b) throw Error{PF_EINVAL, "NULL handle"};
    if (precision != PF_FP64 && precision != PF_MIXED) throw Error{PF_EINVAL, "invalid precision"};
    bind(b, stream);
    apply_timing(*b, precision, reps, us, bytes);
    return PF_OK;
  });
}

pf_status pf_test_wait_timeout(pf_batch* h, int enable) {
  return guarded([&]() -> pf_status {
    if (!h) throw Error{PF_EINVAL, "NULL handle"};
    ((Batch*)h)->test_drop = enable ? 1 : 0;
    return PF_OK;
  });
}

pf_status pf_last_timing(const pf_batch* h, pf_timing* out) {
  return guarded([&]() -> pf_status {
    const Batch* b = (const Batch*)h;
    if (!b || !out) throw Error{PF_EINVAL, "NULL argument"};
    *out = b->timing;
    out->kernel_launches = b->launches;
    out->cg_stages = b->cg_stages;
    return PF_OK;
  });
}

pf_status pf_velocity_field(pf_batch* h, int variant, double* dev_u, double* dev_v, void* stream) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    bind(b, stream);
    check_variant(b, variant);
    velocity_field(*b, variant, dev_u, dev_v);
    return PF_OK;
  });
}

pf_status pf_surface_velocity(pf_batch* h, int variant, int body, double* theta_deg, double* ut, int cap,
                              int* count, void* stream) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    bind(b, stream);
    check_variant(b, variant);
    if (body < 0 || body >= b->hv[variant].nb) throw Error{PF_EINVAL, "body index out of range"};
    if (cap < 0) throw Error{PF_EINVAL, "cap < 0"};
    const int n = surface_velocity(*b, variant, body, theta_deg, ut, cap);
    if (count) *count = n;
    return PF_OK;
  });
}

pf_status pf_copfi(const pf_batch* h, int variant, int body_lo, int body_hi, double U, double* copfi, double* q) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    if (!b) throw Error{PF_EINVAL, "NULL handle"};
    check_variant(b, variant);
    const int nb = b->hv[variant].nb;
    if (body_lo < 0 || body_hi < 0 || body_lo >= nb || body_hi >= nb || body_lo == body_hi)
      throw Error{PF_EINVAL, "body index out of range"};
    if (!b->solved) throw Error{PF_EINVAL, "no solution on this handle yet"};
    std::vector<double> C;
    body_values(*b, C);
    const int g0 = b->hv[variant].body0;
    const double Q = C[g0 + body_hi] - C[g0 + body_lo];
    const double dy = b->bodies[g0 + body_hi].cy - b->bodies[g0 + body_lo].cy;
    if (q) *q = Q;
    if (copfi) *copfi = Q / (U * dy);
    return PF_OK;
  });
}

pf_status pf_mesh_info(const pf_batch* h, long long* n_nodes, long long* n_dof, int* n_boundary_edges,
                       double* min_detJ) {
  pf_mesh_stats st;
  const pf_status rc = pf_mesh_stats_get(h, 0, &st);
  if (rc != PF_OK) return rc;
  if (n_nodes) *n_nodes = st.n_nodes;
  if (n_dof) *n_dof = st.n_dof;
  if (n_boundary_edges) *n_boundary_edges = st.n_boundary_edges;
  if (min_detJ) *min_detJ = st.min_detJ;
  return PF_OK;
}

pf_status pf_batch_solve(pf_batch* h, double U, const pf_solve_opts* opts, double* body_psi, pf_solve_info* info,
                         void* stream) {
  return pf_psi_solve(h, U, opts, nullptr, body_psi, info, stream);
}

pf_status pf_batch_grad(pf_batch* h, int objective, int body_lo, int body_hi, double U, double tol, double* dev_dJdX,
                        double* dJdc, double* J, void* stream) {
  return pf_grad(h, objective, body_lo, body_hi, U, tol, dev_dJdX, dJdc, J, stream);
}

void pf_mesh_destroy(pf_batch* h) { pf_batch_destroy(h); }

pf_status pf_grad(pf_batch* h, int objective, int body_lo, int body_hi, double U, double tol, double* dev_dJdX,
                  double* dJdc, double* J, void* stream) {
  return guarded([&]() -> pf_status {
    Batch* b = (Batch*)h;
    bind(b, stream);
    if (objective != PF_OBJ_COPFI && objective != PF_OBJ_GAP_FLOW) throw Error{PF_EINVAL, "invalid objective"};
    for (int v = 0; v < b->nv; ++v) {
      const int nb = b->hv[v].nb;
      if (body_lo < 0 || body_hi < 0 || body_lo >= nb || body_hi >= nb || body_lo == body_hi)
        throw Error{PF_EINVAL, "body index out of range"};
    }
    return shape_gradient(*b, objective, body_lo, body_hi, U, tol, dev_dJdX, dJdc, J);
  });
}

size_t pf_workspace_bytes(const pf_batch* h) {
  const Batch* b = (const Batch*)h;
  return b ? b->bytes : 0;
}

const char* pf_last_error(void) { return g_err.c_str(); }

}  // extern "C"
