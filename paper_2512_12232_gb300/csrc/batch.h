// Host-side state of a pf_batch handle (one or more mesh variants) and the
// internal entry points that the C ABI in capi.cu calls.
#pragma once
#include <string>
#include <vector>

#include "common.cuh"
#include "tma.cuh"

namespace pfq4 {

struct HostVariant {
  pf_grid g;
  double hx, hy;
  int P;
  long long base, V;
  int nb, body0;
  int tiles_x, tiles_y;
  long long tile0;             // first tile of the variant in the tile list
  pf_mesh_stats stats;
  long long n_gen32_cells = 0;  // general cells whose FP32 coefficients differ from the rectangle's
};

struct Error {                 // thrown inside the library, converted to pf_status at the ABI
  pf_status code;
  std::string msg;
};

struct CgConfig {                  // persistent grid + schedule of one fused-CG kernel instance
  bool ready = false;
  int G = 0;
  int smem = 0;
  Sched sc{};
  // schedule: host copies and the device arrays it is written to in place
  std::vector<int> tile_var;         // [tiles]
  std::vector<double> tile_cost;     // [tiles] relative cost estimate (refined by timed launches)
  std::vector<int> cut;              // [G+1] first tile of each CTA
  std::vector<char> active;          // [nv] variants the cut points were balanced over
  std::vector<int> h_cta_seg, h_seg_var, h_seg_t0, h_seg_t1, h_vs0, h_vs1;   // host copies of the arrays
  int *d_cta_seg = nullptr, *d_seg_var = nullptr, *d_seg_t0 = nullptr, *d_seg_t1 = nullptr;
  int *d_var_seg0 = nullptr, *d_var_seg1 = nullptr;
  unsigned long long* d_cta_ns = nullptr;   // [G] tile-phase time per CTA of a timed launch
  int tune_rounds = 0;               // timing-driven re-balances done
};

// One coarse level (l >= 1) of the geometric multigrid preconditioner, all variants packed:
// variant v's level-l nodes (i, j) at off[v] + j (nx_l + 1) + i, each variant's block
// starting on a multiple of 256 nodes (a 256-thread block never spans two variants).
struct MgLevel {
  long long n = 0;                   // nodes including the padding of every variant's block
  long long nblk = 0;                // 256-node blocks
  std::vector<long long> off;        // [nv] first node of the variant's block (-1: no such level)
  std::vector<int2> dims;            // [nv] (nx_l, ny_l) cells
  long long* d_off = nullptr;
  int2* d_dims = nullptr;
  int* d_blkvar = nullptr;           // [nblk] variant of each block
  uint8_t* act = nullptr;            // coarse node carries an unknown
  float* A32 = nullptr;              // [9][n] Galerkin stencil (FP32: set-up and cycle)
  float* dinv = nullptr;             // omega / diagonal at active nodes, else 0
  float *r = nullptr, *za = nullptr, *zb = nullptr, *res = nullptr;
};

struct Batch;
void* dev_alloc(Batch& b, size_t bytes);
void dev_free(Batch& b, void* p);
void dev_free_all(Batch& b);

struct Batch {
  int device = 0;
  cudaStream_t stream = nullptr;     // stream of the current call
  int nv = 0, B = 0, sweeps = 0;
  int bc[4] = {0, 0, 0, 0};
  long long Vtot = 0;
  std::vector<HostVariant> hv;
  std::vector<pf_body> bodies;
  std::vector<int> body_off;         // [nv+1]
  // body shapes (pf_batch_build_shapes): circles keep the pf_body table, polygons add
  std::vector<int> shape_kind;       // [B] PF_SHAPE_*
  std::vector<int> poly_off;         // [B+1] vertex offsets
  std::vector<double> poly_xy;       // [vertices][2]
  std::vector<int> kutta;            // [B] trailing-edge vertex or -1
  bool has_polygons = false, has_kutta = false;
  bool cut = false;                  // mixed-cell mesh: surface points per edge, cut cells (circles only)
  double cut_sigma = 0.0;            // its minimum surface-point spacing, a fraction of min(hx, hy)
  double2* pcut = nullptr;           // [4][Vtot] surface points of BODY nodes by direction (E, N, W, S), NaN elsewhere
  ShapeDev shp{};                    // device copies (null when there are no polygons)
  std::vector<long long> h_wake;     // [B] padded index of each Kutta body's wake node, or -1
  std::vector<int> h_body_ptr;       // [B+1]
  std::vector<int> h_edge_ptr;       // [B+1]
  bool valid = false;                // det J > 0 everywhere

  // device mesh
  DevVariant* d_var = nullptr;
  pf_body* d_bodies = nullptr;
  int* d_body_var = nullptr;         // [B] variant of each global body
  int4* d_bbox = nullptr;            // [B] node box (i_lo, i_hi, j_lo, j_hi)
  uint8_t* tag = nullptr;
  int* bid = nullptr;                // inside-body index (local) or -1
  double* X = nullptr;               // [2][Vtot] final coordinates
  double* K64 = nullptr;             // [6][Vtot]
  float* K32 = nullptr;              // [6][Vtot]
  float* K32i = nullptr;             // [Vtot][6] the same coefficients interleaved per cell (TMA-friendly)
  int* body_ptr = nullptr;           // [B+1]
  long long* body_nodes = nullptr;
  double* bq = nullptr;              // [body nodes] q of the last fused CG iteration, per BODY node
  int* edge_ptr = nullptr;           // [B+1]
  long long* edge_rec = nullptr;     // (cell padded index << 2) | first corner
  long long* d_stats_i = nullptr;    // [nv][6] integer counts
  double* d_detmin = nullptr;        // [nv]
  long long* d_lbase = nullptr;      // [nv+1] logical node offsets of the variants
  double* d_bsum = nullptr;          // [B] scratch for collapsed body rows

  // fused-CG tiles (CTX x CTY) and their persistent schedule
  long long Tcg = 0;
  int2* tile_cg_ij = nullptr;
  int* tile_cg_var = nullptr;
  uint8_t* tile_cg_gen = nullptr;    // bit 0 / bit 1: a cell used by the tile needs stored FP64 / FP32 coefficients
  int* tile_cg_act = nullptr;        // nodes of the tile with an operator row (FREE or BODY)
  CgConfig cg_cfg[2][3];             // [precision][stages - 2]
  int cg_stages = 2;
  bool cg_tune = false;              // re-balance the fused-CG schedule from timed launches
  int tuned_stages[2] = {2, 2};     // pipeline depth picked by the autotuner, per precision
  bool stages_tuned[2] = {false, false};
  int nsm = 0;
  long long Rtot = 0;                // rows of the batch's 2-D node arrays (Vtot / P)
  int P = 0;                         // common row pitch

  // 32x8 tiles (mesh build, refinement kernels)
  long long T = 0;
  int2* tile_ij = nullptr;           // [T]
  int* tile_var = nullptr;           // [T]
  // refinement kernels (k_fold, k_resid): a (rgx, variants) grid
  int rgx = 0;                       // CTAs per variant
  double* rpart = nullptr;           // [variants][rgx] partial sums
  int* rcounter = nullptr;           // [variants] arrivals per launch

  // solver state
  VarState* state = nullptr;         // [nv]
  SolveParams* params = nullptr;
  int* n_done = nullptr;             // device counter of finished variants
  int* d_err = nullptr;              // device flag: a bounded wait gave up
  CgMaps maps[2];                    // TMA descriptors of the fused CG kernel (FP64, mixed)
  double* x64 = nullptr;             // [Vtot] solution (Dirichlet values in place)
  double* w64 = nullptr;             // [Vtot] FP64 scratch (body-node rows of the true residual)
  // CG state records (x, r, p, q) double-buffered by parity: a launch reads one parity
  // with its halo and writes the other, so no tile sees a neighbour's new values
  State4<double>* st64[2] = {nullptr, nullptr};
  State4<float>* st32[2] = {nullptr, nullptr};
  void** d_sbuf = nullptr;           // device copy of {st64[0], st64[1], st32[0], st32[1]}
  double* sol64 = nullptr;           // [B] body solution values C_k (FP64)
  double* sb64 = nullptr;            // [4][B] FP64-mode CG body values x, r, p, q
  float* sb32 = nullptr;             // [4][B] mixed-mode CG body values x, r, p, q
  double* ap64[2] = {nullptr, nullptr};   // pf_apply scratch (padded in / out)
  float* ap32[2] = {nullptr, nullptr};
  CgMaps ap_maps[2];                 // TMA descriptors of the operator kernel (FP64, FP32): s[0] = p input, tag
  int ap_G[2] = {0, 0};              // its persistent grid per precision (0: not configured yet)
  int* ap_err = nullptr;             // device flag: a bounded wait of the operator kernel gave up
  int4* ap_groups = nullptr;         // operator kernel work items: groups of adjacent tiles (descriptors)
  long long ap_ngroups = 0;
  unsigned long long* ap_ticket = nullptr;   // its work counter (tickets taken so far)
  unsigned long long ap_ticket_base = 0;     // tickets consumed by the launches queued so far
  double* sbr64 = nullptr;           // [B] FP64 true-residual body rows
  double* d_rhsb = nullptr;          // [B] body-row right-hand side of the adjoint solve
  bool rhs_active = false;
  bool fixed_bodies = false;         // Schur sub-solves: body values are data (sol64 preset)
  double* d_Uv = nullptr;            // [nv] per-variant U of the Dirichlet data
  bool Uv_active = false;
  double* psi_save = nullptr;        // [Vtot] forward solution kept during the adjoint solve
  double* sol_save = nullptr;        // [B]
  double* gradX = nullptr;           // [2][Vtot] dJ/dX (padded), then the transposed sweeps
  double* gradT = nullptr;           // [2][Vtot] ping-pong partner of gradX
  double* cellG = nullptr;           // [8][Vtot] per-cell shape derivatives
  void** d_vecs = nullptr;           // device list of the vectors k_init clears
  // multigrid-preconditioned CG (mg.cu): hierarchy made on the first such solve
  bool pcg_active = false;           // the current solve runs the preconditioned CG
  int last_precond = PF_PRECOND_NONE; // preconditioner of the last forward solve (the adjoint reuses it)
  bool mg_ready = false;
  int mg_L = 0;                      // levels of the deepest variant
  std::vector<int> mg_Lv;            // [nv] levels per variant (>= 2)
  int* d_mg_Lv = nullptr;
  long long* d_tile0 = nullptr;      // [nv + 1] first 32x8 tile of each variant
  std::vector<MgLevel> mg;           // [mg_L]; entry 0 unused (the fine level is the mesh itself)
  float *mg_x = nullptr, *mg_r = nullptr, *mg_z = nullptr, *mg_t = nullptr, *mg_res = nullptr;
  float *mg_p[2] = {nullptr, nullptr}, *mg_q = nullptr, *mg_dinv0 = nullptr;
  double* mg_part = nullptr;         // [T] per-tile partial sums of one dot product
  double* mg_Abb = nullptr;          // [B] diagonal of the collapsed body rows
  float* mg_yb = nullptr;            // [B] body values of the forward body step of the cycle
  // free nodes next to each body (CSR over global bodies, row-major in the body's box) and
  // their coupling c = sum of A(n, m) over the body's nodes m: A_fb and A_bf of the cycle
  int* mg_adj_ptr = nullptr;
  long long* mg_adj_node = nullptr;
  float* mg_adj_c = nullptr;
  cudaGraphExec_t graph_pcg = nullptr;
  int graph_pcg_chunk = 0;
  bool dirichlet_x = false;          // Dirichlet data U x (the velocity potential) instead of U y
  Batch* phi = nullptr;              // velocity-potential view of this mesh (made on first use)
  bool solved = false;
  double lastU = 0.0;
  int last_precision = -1;
  std::vector<double> bnorm2_unit;   // ||b||^2 at U = 1, per variant (filled by the first solve)

  // graphs (one per precision) and timing events
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  cudaStream_t graph_stream[2] = {nullptr, nullptr};
  int graph_chunk[2] = {0, 0};
  int graph_stages[2] = {0, 0};
  int graph_drop[2] = {0, 0};
  int test_drop = 0;                 // test hook (pf_test_wait_timeout): see the header
  static constexpr int N_EV = 12;    // 0-5: solve-level timing, 6-11: two chunk slots x 3
  cudaEvent_t ev[N_EV] = {};
  pf_timing timing{};
  double cg_bytes_per_node[2] = {0, 0};

  int* h_poll = nullptr;             // pinned [2 slots][2]: finished variants, bounded-wait flag
  VarState* h_vs = nullptr;          // pinned [2 slots][nv]: variant states after each chunk
  long long launches = 0;            // kernel launches issued by this handle

  std::vector<std::pair<void*, size_t>> allocs;
  size_t bytes = 0;
  void* alloc_ctx = nullptr;
  pf_alloc_fn alloc_fn = nullptr;
  pf_free_fn free_fn = nullptr;
};

void check_cuda(cudaError_t e, const char* what);
void set_last_error(const std::string& msg);
#define PF_CUDA(call) ::pfq4::check_cuda((call), #call)

// mesh.cu
// Host description of polygonal bodies for build_batch: per body (in the order of
// `bodies`) its kind, its vertices and its Kutta vertex; empty vectors mean circles only.
struct ShapeInput {
  std::vector<int> kind;             // [B]
  std::vector<int> off;              // [B+1]
  std::vector<double> xy;
  std::vector<int> kutta;            // [B]
};
void build_batch(Batch& b, const pf_grid* grids, const int* body_offsets, const pf_body* bodies,
                 int nv, int sweeps, const int bc[4], const ShapeInput* shapes = nullptr);
void export_coords(Batch& b, int v, double* dev_xy);
void set_coords(Batch& b, int v, const double* dev_xy);
void tile_flags(Batch& b);
void export_tags(Batch& b, int v, int8_t* kind, int32_t* body);
void export_cut_points(Batch& b, int v, double* pts);

// solver.cu
void make_schedule(Batch& b);
void velocity_field(Batch& b, int v, double* dev_u, double* dev_v, int potential = 0);
void ensure_solver_memory(Batch& b, int precision);
void apply_timing(Batch& b, int precision, int reps, double* us, double* bytes);
void apply_operator(Batch& b, int precision, const double* dev_p, double* dev_y, double* body_sums);
void refresh_apply_groups(Batch& b);
pf_status psi_solve(Batch& b, double U, const pf_solve_opts& o, double* dev_psi, double* body_psi,
                    pf_solve_info* info);
pf_status solve_core(Batch& b, double U, const pf_solve_opts& o, double* dev_psi, double* body_psi,
                     pf_solve_info* info, bool record_bnorm);
long long* lbase_cached(Batch& b);
void export_psi(Batch& b, double* dev_psi);
void body_values(Batch& b, std::vector<double>& C);

// mg.cu
void mg_setup(Batch& b);
void launch_pcg_chunk(Batch& b, int iters, cudaStream_t s);
void destroy_mg(Batch& b);

// schur.cu
pf_status schur_solve(Batch& b, double U, const pf_solve_opts& o, double* dev_psi, double* body_psi,
                      pf_solve_info* info);

// post.cu
int surface_velocity(Batch& b, int v, int body, double* theta, double* ut, int cap);

// phi.cu
pf_status phi_solve(Batch& b, double U, const pf_solve_opts& o, double* dev_phi, pf_solve_info* info);
void phi_velocity_field(Batch& b, int v, double* dev_u, double* dev_v);
void destroy_phi_view(Batch& b);

// grad.cu
pf_status shape_gradient(Batch& b, int obj, int lo, int hi, double U, double tol, double* dev_dJdX,
                         double* dJdc, double* J);
void coords_vjp(Batch& b, const double* dev_gX, double* gc);

}  // namespace pfq4
