/*
 * pfq4.h - C ABI of the GB300 matrix-free Q4 stream-function solver.
 *
 * Method: Sadasivan & Yadav, "A Computational Approach for Multi-Body Potential-Flow
 * Interaction Effects Using Matrix-Free FEM and Body-Conforming Grids".
 *   - mesh: section "Body-Conforming Grid Generation" (background Cartesian grid,
 *     near-boundary nodes moved onto the bodies, Laplacian propagation of the
 *     displacement, x_new = x_old + d);
 *   - operator: section "Weak formulation", K_e = int (grad N)^T grad N over bilinear
 *     quadrilaterals, never assembled (section "Matrix-Free Conjugate Gradient with
 *     Multiple Constraint Enforcement");
 *   - unknowns: N_dof = N_int + N_N + N_b, one multi-point-constraint value C_i per
 *     body (section "Boundary Conditions": psi = C_i on body i);
 *   - solve: Conjugate Gradient of Appendix A (Algorithm);
 *   - outputs: surface tangential velocity (section "Velocity Field and Surface
 *     Tangential Velocity"), Q and CoPFI (section "Effect of Gap Ratio").
 *
 * Conventions for every function:
 *   - The return value is a pf_status; 0 (PF_OK) means success.  Nothing throws
 *     across the ABI.  pf_last_error() returns a message for the calling thread's
 *     last failure (valid until that thread's next call).
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Calls are ordered on that stream; functions that return host values
 *     synchronise the stream before returning.
 *   - Pointers named dev_* are device pointers owned by the caller (for example
 *     torch tensors' data_ptr()); all other pointers are host memory owned by the
 *     caller.  Opaque handles (pf_batch) own their device memory, which is
 *     allocated through the allocator installed with pf_set_allocator (default:
 *     cudaMalloc) and released by pf_batch_destroy.
 *   - Nodes are numbered logically per variant: node (i, j), 0 <= i <= nx,
 *     0 <= j <= ny, has index j*(nx+1) + i.  Node-valued outputs of a batch are the
 *     variants' logical arrays concatenated in variant order.
 *   - Every call must be made with the device that built the handle current.
 */
#ifndef PFQ4_H
#define PFQ4_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int pf_status;
enum {
    PF_OK = 0,
    PF_EINVAL = 1,          /* bad argument: sizes, NULL pointers, bodies overlapping / too close to the box */
    PF_EMESH_INVALID = 2,   /* generated mesh unusable: det J <= 0 at a Gauss point of an active cell */
    PF_ENOT_CONVERGED = 3,  /* k_max reached before the tolerance; outputs hold the last iterate */
    PF_EBREAKDOWN = 4,      /* p^T A p <= 0 or not finite in CG */
    PF_ETIMEOUT = 5,        /* a bounded device-side wait gave up */
    PF_ECUDA = 6,           /* a CUDA runtime call failed (message in pf_last_error) */
    PF_ENOMEM = 7           /* device allocation failed */
};

/* Side order for boundary conditions: left (x = x0), right (x = x1), bottom (y = y0), top (y = y1). */
enum { PF_BC_DIRICHLET_UY = 0,  /* psi = U*y on the side (the uniform stream; a reference streamline) */
       PF_BC_NATURAL = 1 };     /* zero normal derivative (inlet / outlet, section "Validation") */

enum { PF_FP64 = 0,             /* FP64 vectors, operator and reductions */
       PF_MIXED = 1 };          /* FP32 operator + vectors, FP64 reductions / scalars / true residual,
                                   iterative refinement in FP64 */

enum { PF_OBJ_COPFI = 0,        /* J = (C_hi - C_lo) / (U (cy_hi - cy_lo)) */
       PF_OBJ_GAP_FLOW = 1 };   /* J = C_hi - C_lo */

/* Node kinds reported by pf_mesh_tags. */
enum { PF_NODE_FREE = 0, PF_NODE_DIRICHLET = 1, PF_NODE_BODY = 2, PF_NODE_INACTIVE = 3 };

typedef struct pf_grid { double x0, x1, y0, y1; int nx, ny; } pf_grid;   /* background grid, nx x ny cells */
typedef struct pf_body { double cx, cy, r; } pf_body;                     /* circular body Gamma_i */

typedef struct pf_mesh_stats {
    long long n_nodes;          /* (nx+1)(ny+1) */
    long long n_free;           /* N_int + N_N */
    long long n_dof;            /* n_free + n_bodies */
    long long n_body_nodes;     /* nodes carrying a body value */
    long long n_inactive;
    long long n_active_cells;
    long long n_general_cells;  /* active cells with a displaced corner (stored K_e used) */
    int n_bodies;
    int n_boundary_edges;       /* over all bodies of the variant */
    double min_detJ;            /* minimum det J over the Gauss points of active cells */
    double h;                   /* max(hx, hy) */
} pf_mesh_stats;

/* Default inner tolerance of PF_MIXED solves.  Each inner FP32 CG stops once its
   recurrence residual has dropped by this factor (or below half the outer tolerance);
   the FP64 true residual then decides.  A tight value means fewer restarts of the inner
   CG: on the five-cylinder batch 2e-7 needs 2619 iterations for the slowest variant
   where 1e-4 needs 3170, at the same 1e-8 true residual. */
#define PF_DEFAULT_INNER_TOL 2e-7

/* Stopping rules of a solve (pf_solve_opts.criterion). */
enum { PF_TOL_REL_TRUE = 0,     /* ||b - A u||_2 / ||b||_2 <= tol, the FP64 true residual of the reduced
                                   system recomputed at every refinement (the library's default) */
       PF_TOL_PAPER_ABS = 1 };  /* the stopping test of Appendix A (Algorithm): the sum of squares of
                                   the reduced residual, sum r^2 over the free rows and the collapsed
                                   body rows, below tol (absolute; tol is compared with the square,
                                   as the algorithm compares r_norm = sum r^2).  Each inner CG stops on
                                   its recurrence residual sum r^2 <= tol as the algorithm does (PF_FP64)
                                   or at a quarter of it (PF_MIXED); the FP64 true residual then
                                   confirms sum r^2 <= tol or refines again */

/* Preconditioners of a solve (pf_solve_opts.preconditioner; an extension beyond the paper,
   whose Appendix A CG is unpreconditioned and needs a number of iterations that grows with the
   grid).  PF_PRECOND_MG: each CG iteration applies one V(1,1)-cycle of geometric multigrid on
   the logical node grid of every variant to the free unknowns (Galerkin coarse operators,
   bilinear interpolation, constraints injected on coarse nodes, damped Jacobi smoothing),
   coupled to the body unknowns by a symmetric block Gauss-Seidel sweep (body, free, body;
   each body by the diagonal of its collapsed row).  The preconditioner is a fixed symmetric
   positive-definite operator, so the iterates converge to the same solution;
   convergence is decided by the same FP64 true residual and refinement.  The hierarchy is
   built on the first such solve of a handle (and again after pf_mesh_set_coords). */
enum { PF_PRECOND_NONE = 0, PF_PRECOND_MG = 1 };

typedef struct pf_solve_opts {
    double tol;            /* PF_TOL_REL_TRUE: stop when ||b - A u||_2 / ||b||_2 <= tol (true residual,
                              FP64); PF_TOL_PAPER_ABS: stop when sum r^2 <= tol */
    long long k_max;       /* cap on the total CG iterations per variant */
    int precision;         /* PF_FP64 or PF_MIXED */
    double inner_tol;      /* PF_MIXED: relative residual reduction of each inner FP32 solve
                              (<= 0: PF_DEFAULT_INNER_TOL) */
    int chunk;             /* CG iterations per captured graph launch (0 = automatic) */
    int warm_start;        /* 1: start from the previous solution held by the handle */
    int tune_schedule;     /* 1: on the first such solve of the handle, run a few CG iterations
                              as timed launches and move the persistent kernel's tile ranges so
                              that every CTA's measured time evens out (kept for later solves).
                              This changes the order in which the dot products are summed:
                              results agree with an untuned solve to rounding, not bit for bit.
                              0: schedule from the static per-tile cost estimate (deterministic). */
    int criterion;         /* PF_TOL_REL_TRUE (0) or PF_TOL_PAPER_ABS (1); any other value: PF_EINVAL */
    int preconditioner;    /* PF_PRECOND_NONE (0): the paper's CG; PF_PRECOND_MG (1): CG preconditioned by a
                              geometric multigrid V-cycle (PF_MIXED only); any other value: PF_EINVAL */
} pf_solve_opts;

typedef struct pf_solve_info {
    long long iters;             /* CG iterations (all inner solves) */
    int refinements;             /* true-residual evaluations after the first */
    int status;                  /* per-variant pf_status */
    double rel_true_residual;    /* ||b - A u|| / ||b||, FP64 */
    long long n_dof;
} pf_solve_info;

typedef struct pf_timing {
    double cg_kernel_ms;         /* summed device time of the fused CG-iteration launches (CUDA events) */
    long long cg_launches;       /* number of such launches */
    double residual_kernel_ms;   /* summed device time of the FP64 true-residual launches */
    long long residual_launches;
    double solve_ms;             /* device time of the whole solve, events on the call's stream */
    double cg_bytes_per_launch;  /* algorithmic HBM bytes of one fused CG launch, averaged over the
                                    launches of the solve (variants already converged move nothing) */
    long long kernel_launches;   /* kernels launched by this handle since it was built (mesh + solves) */
    int cg_stages;               /* pipeline depth of the fused CG kernel in the last solve (2..4) */
} pf_timing;

typedef struct pf_batch pf_batch;   /* opaque: one or more mesh variants and their solver state */

/* Optional allocator hook (e.g. PyTorch's caching allocator).  alloc(bytes, stream, ctx) returns
   a device pointer or NULL; free(ptr, stream, ctx) releases it.  Pass NULLs to restore the default.
   Affects handles built afterwards. */
typedef void* (*pf_alloc_fn)(size_t bytes, void* stream, void* ctx);
typedef void (*pf_free_fn)(void* ptr, void* stream, void* ctx);
pf_status pf_set_allocator(pf_alloc_fn alloc, pf_free_fn free_fn, void* ctx);

/* Build the body-conforming mesh of n_variants independent problems
   (section "Body-Conforming Grid Generation").
   grids[v]: background grid of variant v (nx, ny >= 2).
   body_offsets[v] .. body_offsets[v+1]-1: rows of `bodies` belonging to variant v
     (0 <= bodies per variant <= 64).  Bodies must be disjoint, have r > 0, and lie at
     least 2h inside the box, else PF_EINVAL.
   sweeps: Jacobi smoothing sweeps S >= 0 of the displacement.
   bc[4]: PF_BC_* for left, right, bottom, top (at least one side must be Dirichlet).
   On success *out receives a handle; on PF_EMESH_INVALID the handle is still returned
   (so pf_mesh_stats can report min_detJ) but solves on it are refused. */
pf_status pf_batch_build(const pf_grid* grids, const int* body_offsets, const pf_body* bodies,
                         int n_variants, int sweeps, const int bc[4], void* stream, pf_batch** out);

/* Body shapes for pf_batch_build_shapes. */
enum { PF_SHAPE_CIRCLE = 0, PF_SHAPE_POLYGON = 1 };

typedef struct pf_shape {
    int kind;                 /* PF_SHAPE_CIRCLE or PF_SHAPE_POLYGON */
    double cx, cy, r;         /* circle: centre and radius; polygon: the reference point of the polar
                                 angle in pf_surface_velocity (r unused) */
    int n_vertices;           /* polygon: number of vertices (>= 3) */
    const double* vertex_xy;  /* polygon: host array [n_vertices][2], counter-clockwise */
    int kutta_vertex;         /* polygon: vertex (trailing edge) carrying the Kutta condition, or -1 */
} pf_shape;

/* pf_batch_build with general body shapes (section "Body-Conforming Grid Generation": each
   immersed body is a closed boundary curve; section "Boundary Conditions": the Kutta
   condition at sharp trailing edges).
   - A node is inside a polygon when the crossing-number test counts an odd number of edge
     crossings (edge (a, b) crossed when (a_y > y) != (b_y > y) and
     x < a_x + ((y - a_y)(b_x - a_x)) / (b_y - a_y)); circles as in pf_batch_build.
   - A node just inside a polygon moves to the nearest point of its boundary (first edge on
     ties); all of it in explicitly rounded FP64, reproducible bit for bit.
   - Kutta condition at vertex T: with w the unit bisector of the two edges at T pointing
     out of the body and W = T + hx w, the FREE node nearest to W (then the smallest
     row-major index) is moved onto W and held there by the smoothing.  Solves hold it at the
     body's value in place of the body's zero-circulation equation, so the body streamline
     leaves T along w and the circulation follows (pf_psi_solve then runs the Schur form, the
     only form that allows that non-symmetric equation: the small body system is eliminated
     with partial pivoting, info[v].iters sums the fixed-body solves' iterations and
     info[v].rel_true_residual is the largest of their residuals; pf_phi_solve refuses such
     a handle).
   - pf_grad and pf_coords_vjp refuse any handle with a polygon (the shape derivative is
     written for circles).
   - Polygons need >= 3 vertices in counter-clockwise order; their bounding boxes must stay
     2h inside the box and may not overlap any other body's bounding box.
   Otherwise as pf_batch_build (body_offsets index `shapes`). */
pf_status pf_batch_build_shapes(const pf_grid* grids, const int* body_offsets, const pf_shape* shapes,
                                int n_variants, int sweeps, const int bc[4], void* stream, pf_batch** out);

/* pf_batch_build_shapes with the mixed-cell mesh of section "Body-Conforming Grid
   Generation": node splitting, triangle and pentagon cells, boundary-point redistribution.
   Bodies as in pf_batch_build_shapes (circles and polygons, Kutta vertices allowed).
   - Node kinds as in pf_batch_build.  A BODY node keeps its background position; for each
     outside 4-neighbour it has a surface point where their grid edge crosses the body's
     boundary, explicitly rounded FP64: for a circle on a row (cx +- sqrt(r^2 - (y - cy)^2), y),
     on a column (x, cy +- sqrt(r^2 - (x - cx)^2)); for a polygon the crossing of the inside
     test's formula on a row (x = a_x + ((y - a_y)(b_x - a_x)) / (b_y - a_y)), or its
     transpose on a column, nearest the node within the edge (g < x <= k or k < x <= g;
     without one, the nearest crossing clipped onto the edge, or the edge's midpoint).  A
     node with two or more outside neighbours is split into that many points, all carrying
     the body's single value C_k.  A Kutta wake node is placed as in pf_batch_build_shapes.
   - The S Jacobi sweeps average the four neighbours as in pf_batch_build, a BODY neighbour
     contributing the displacement of its surface point on the common edge.
   - A cut cell (an active cell with an inside corner) is the polygon of its outside corners
     and surface points, walked counter-clockwise from corner 0: a triangle (linear element),
     a quadrilateral (Q4), or a pentagon split into the triangle (P+, c_{m+1}, c_{m+2}) and the
     quadrilateral (P+, c_{m+2}, c_{m+3}, P-) around its inside corner m, P+ the point on edge m.
     Its pieces' element matrices, scattered onto the cell's corners, are stored as the cell's
     coefficients, so every operator, solve and preconditioner of the library runs unchanged.
   - min_spacing in [0, 1]: after the smoothing, the chord of every cut cell shorter than
     s_min = min_spacing * min(hx, hy) (and not of zero length) pushes its two points apart
     along it by (s_min - L)/2 each; a point adds the pushes of its two cells and is projected
     back onto its body (radially for a circle, to the nearest boundary point for a polygon).
     0 leaves the points in place.
   - PF_EINVAL also for a cell with two diagonal inside corners or with inside corners of two
     bodies, and for min_spacing outside [0, 1].  min_detJ covers every piece (twice the area
     for a triangle).
   - pf_surface_velocity lists one chord per cut cell (u_t from the mean of the polygon's
     vertex values and the distance of its vertex centroid from the chord); pf_velocity_field
     gives a cut cell the area-weighted mean of its pieces' gradients.  pf_grad,
     pf_coords_vjp, pf_mesh_set_coords and pf_phi_solve refuse the handle (PF_EINVAL).
   pf_mesh_coords reports BODY nodes at their background position; pf_mesh_cut_points gives
   the surface points. */
pf_status pf_batch_build_cut(const pf_grid* grids, const int* body_offsets, const pf_shape* shapes, int n_variants,
                             int sweeps, const int bc[4], double min_spacing, void* stream, pf_batch** out);

/* Single-variant convenience form of pf_batch_build. */
pf_status pf_mesh_build(const pf_grid* grid, const pf_body* bodies, int n_bodies, int sweeps,
                        const int bc[4], void* stream, pf_batch** out);

void pf_batch_destroy(pf_batch* b);

pf_status pf_batch_size(const pf_batch* b, int* n_variants, long long* total_nodes, int* total_bodies);
pf_status pf_mesh_stats_get(const pf_batch* b, int variant, pf_mesh_stats* out);

/* Final node coordinates of variant v: dev_xy[n][2] (x, y), logical order, FP64. */
pf_status pf_mesh_coords(const pf_batch* b, int variant, double* dev_xy, void* stream);

/* Replace the node coordinates of variant v with caller-given ones (dev_xy[n][2], logical
   order, FP64), keeping the topology as built: node kinds, body membership, active cells
   and boundary edges do not change.  The element matrices (section "Weak formulation"),
   the cell and tile flags and min det J are recomputed from the new coordinates; a later
   pf_psi_solve, pf_grad or pf_apply works on them.  This is the input side of a shape
   optimisation over node coordinates (dJ/dX from pf_grad is the gradient at these
   coordinates).  Returns PF_EMESH_INVALID (coordinates kept) if det J <= 0 at a Gauss point
   of an active cell of any variant; the handle then refuses solves until valid coordinates
   are set.  Earlier solutions on the handle are discarded. */
pf_status pf_mesh_set_coords(pf_batch* b, int variant, const double* dev_xy, void* stream);

/* Vector-Jacobian product of the mesh generator (section "Body-Conforming Grid
   Generation"): given a cotangent dev_gX[n][2] on the final node coordinates of every
   variant (device, logical order, variants concatenated), return in gc[total bodies][2]
   (host) the cotangent on the body centres through the radial projection of the body
   nodes and the S Jacobi smoothing sweeps (which are linear in the projection
   displacement): gc = (dX/dc)^T gX at fixed topology.  pf_grad's dJdc is this product of
   its dJ/dX plus the objective's own dependence on the centres. */
pf_status pf_coords_vjp(pf_batch* b, const double* dev_gX, double* gc, void* stream);

/* Node classification of variant v: dev_kind[n] = PF_NODE_*, dev_body[n] = body index
   (local to the variant) for BODY nodes, else -1.  Either pointer may be NULL. */
pf_status pf_mesh_tags(const pf_batch* b, int variant, int8_t* dev_kind, int32_t* dev_body, void* stream);

/* Surface points of variant v of a pf_batch_build_cut handle: dev_pts is a caller-owned
   device array [4][nodes][2] of doubles, direction d (0 E, 1 N, 2 W, 3 S) then node
   m = j*(nx+1) + i then (x, y); NaN where node m has no surface point in direction d.
   PF_EINVAL for another handle, a variant out of range or a NULL output. */
pf_status pf_mesh_cut_points(const pf_batch* b, int variant, double* dev_pts, void* stream);

/* Matrix-free operator of the reduced system on nodal vectors (Appendix A, "Compute Ap"):
   y_n = sum over active cells e containing n of (K_e p_e)_n for FREE and BODY nodes,
   0 for DIRICHLET and INACTIVE nodes, where p is used as given at every node (so a
   DIRICHLET value enters as lifting).  body_sums[k] (host, optional) receives the
   collapsed body rows sum_{n in body k} y_n for the variant's bodies.
   precision PF_FP64 uses the FP64 element matrices; PF_MIXED rounds p to FP32 and
   applies the FP32 element matrices (FP32 result widened to FP64).  All variants'
   logical vectors concatenated; body_sums over all bodies. */
pf_status pf_apply(pf_batch* b, int precision, const double* dev_p, double* dev_y,
                   double* body_sums, void* stream);

/* Largest total number of bodies a handle may hold for pf_apply_noalloc (the size of its
   fixed device array of collapsed body rows). */
#define PF_NOALLOC_MAX_BODIES 4096

/* Allocation-free form of pf_apply (the paper has no counterpart: this exists for the
   library's callers).  For callers that cannot allocate device memory when they apply
   the operator - code whose device memory is all owned by a framework arena or caching
   allocator, or a loop that must not call cudaMalloc / cudaFree because they
   synchronise the device and can fail under memory pressure.  Same arguments, results
   and layout as pf_apply; it allocates nothing: the input and output vectors are read
   and written in place, and the collapsed body rows go through a fixed device array of
   PF_NOALLOC_MAX_BODIES doubles (32 KB) that every GPU loading the library keeps until
   exit.  A handle with more than PF_NOALLOC_MAX_BODIES bodies in total is rejected with
   PF_EINVAL.  The handle is only read, never modified.  The first call on a device looks
   up that array's device address (once per device) and keeps it for the life of the
   process, so the library is not to be used across a cudaDeviceReset.  The call waits
   for `stream` to finish its work before returning, so it cannot be captured: on a
   capturing stream it returns PF_EINVAL before launching anything.  Every call on a device shares the array and it keeps the last call's
   contents; each call overwrites what it reads back.  Calls that overlap on the GPU
   (e.g. on two streams at once) race on it. */
pf_status pf_apply_noalloc(const pf_batch* b, int precision, const double* dev_p, double* dev_y,
                           double* body_sums, void* stream);

/* Solve for psi on every variant (sections "Boundary Conditions" to Appendix A):
   Dirichlet sides carry psi = U*y, each body one unknown constant.
   dev_psi: optional device output [total nodes] (logical order, INACTIVE nodes = 0).
   body_psi: optional host output [total bodies], the C_i.
   info: optional host output [n_variants].
   Returns PF_OK if every variant reached tol, else the first failing variant's status. */
pf_status pf_psi_solve(pf_batch* b, double U, const pf_solve_opts* opts, double* dev_psi,
                       double* body_psi, pf_solve_info* info, void* stream);

/* The same solve through the Schur complement of the body unknowns (algebraically equal
   to the multi-point-constraint system of section "Matrix-Free Conjugate Gradient with
   Multiple Constraint Enforcement"): per variant, N_b + 1 solves with the body values held
   as data (psi_0 with the Dirichlet data, phi_k with C_k = 1) run as one internal batch;
   the body rows of K phi_k form the N_b x N_b FP64 Schur matrix, S C = -(body rows of
   K psi_0) is solved by Cholesky, and psi = psi_0 + sum_k C_k phi_k.  A warm-started MPC
   solve then reports the true residual (and iterates only if tol is not yet met).
   Arguments and outputs as pf_psi_solve; info[v].iters includes the sub-solves. */
pf_status pf_psi_solve_schur(pf_batch* b, double U, const pf_solve_opts* opts, double* dev_psi,
                             double* body_psi, pf_solve_info* info, void* stream);

/* Bandwidth measurement of the stand-alone operator (section "Matrix-Free Conjugate
   Gradient ..."; the same node-centric Q4 gather as pf_apply): `reps` back-to-back
   applications (after 3 untimed ones) on the handle's internal padded vectors, with no
   layout conversion and no body sums, timed with CUDA events on `stream`.  Outputs the
   mean microseconds per application and its algorithmic bytes (p read and y written at
   every node, one tag byte per node, six coefficients of every cell whose coefficients in
   this precision differ from the closed-form rectangle's).  PF_EINVAL for a NULL handle,
   reps < 1 or an invalid precision. */
pf_status pf_apply_timing(pf_batch* b, int precision, int reps, double* us_per_apply, double* bytes_per_apply,
                          void* stream);

/* Device-event timing of the last pf_psi_solve on this handle. */
pf_status pf_last_timing(const pf_batch* b, pf_timing* out);

/* Test hook for failure detection without a GPU fault.  With enable = 1, every fused CG
   launch of later solves on this handle has CTA 0 skip the copies of its first tile and
   caps each mbarrier wait at 1024 polls, so the consumer warps' bounded wait on that
   stage gives up: the kernel records the failure in a device flag, drains the copies it
   did issue, returns, and the solve returns PF_ETIMEOUT.  No wait is unbounded, nothing
   faults and the CUDA context stays usable.  The handle's iterate is then undefined:
   destroy it.  enable = 0 restores normal launches.  PF_EINVAL for a NULL handle. */
pf_status pf_test_wait_timeout(pf_batch* b, int enable);

/* Velocity potential phi of every variant (section "Governing Equation": u = grad phi,
   nabla^2 phi = 0; the contour lines of phi and psi form the flow net).  The same Q4
   operator and fused CG kernels as pf_psi_solve, with the constraints of phi: phi = U*x on
   the inlet and outlet sides (x = x0, x = x1), no flux (the natural condition) on the
   other two sides and on every body, and every node that is neither inactive nor on the
   inlet / outlet an unknown (body nodes included: there is no multi-point constraint).
   The boundary kinds given to pf_batch_build concern psi and are not used here.
   dev_phi: optional device output [total nodes] (logical order, inactive nodes = 0).
   info: optional host output [n_variants]; opts as pf_psi_solve (NULL: mixed, 1e-8).
   Returns PF_OK if every variant reached tol, else the first failing variant's status. */
pf_status pf_phi_solve(pf_batch* b, double U, const pf_solve_opts* opts, double* dev_phi, pf_solve_info* info,
                       void* stream);

/* Element velocity of the last pf_phi_solve, u = dphi/dx and v = dphi/dy at the centre of
   every cell of variant v (same layout and rules as pf_velocity_field).  PF_EINVAL before a
   phi solve. */
pf_status pf_phi_velocity_field(pf_batch* b, int variant, double* dev_u, double* dev_v, void* stream);

/* Element velocity field of variant v after a solve (section "Velocity Field and Surface
   Tangential Velocity", u = dpsi/dy, v = -dpsi/dx; the velocity-magnitude field of the
   results): the gradient of the bilinear interpolant of the solved psi at the centre of
   every cell, through the isoparametric map.  dev_u and dev_v are caller-owned device
   arrays of nx*ny doubles, cell (i, j) at j*nx + i; inactive cells get 0.  PF_EINVAL for a
   NULL handle or output, a variant out of range, or a handle with no solve yet. */
pf_status pf_velocity_field(pf_batch* b, int variant, double* dev_u, double* dev_v, void* stream);

/* Surface tangential velocity on body `body` of variant v after a solve
   (section "Velocity Field and Surface Tangential Velocity"): for every boundary edge
   (edge of an active cell whose end nodes are distinct BODY nodes of this body),
   u_t = (psi_c - C) / d_nc with psi_c the mean nodal psi of the cell and d_nc the
   distance from the cell's vertex centroid to the edge line; theta_deg is the polar
   angle of the edge midpoint about the body centre in [0, 360).  Edges in cell order
   (row-major), then by the edge's first corner.  Host outputs of capacity `cap`;
   *count receives the number of edges (outputs truncated to cap). */
pf_status pf_surface_velocity(pf_batch* b, int variant, int body, double* theta_deg, double* ut,
                              int cap, int* count, void* stream);

/* Q = C_hi - C_lo and CoPFI = Q / (U (cy_hi - cy_lo)) after a solve (section "Effect of Gap Ratio"). */
pf_status pf_copfi(const pf_batch* b, int variant, int body_lo, int body_hi, double U,
                   double* copfi, double* q);

/* Adjoint shape gradient of J (PF_OBJ_*) for body pair (lo, hi) of every variant after a
   solve with the same U.  dev_dJdX: optional device output [total nodes][2], the gradient
   with respect to the final node coordinates (topology held fixed); dJdc: optional host
   output [total bodies][2], with respect to the body centres through the projection and the
   S smoothing sweeps; J: optional host output [n_variants].  The adjoint system is solved
   to a relative FP64 true residual of `tol` (FP32 inner CG with FP64 refinement, as
   PF_MIXED), with the preconditioner of the handle's last pf_psi_solve (PF_PRECOND_MG
   after a multigrid-preconditioned solve, else none). */
pf_status pf_grad(pf_batch* b, int objective, int body_lo, int body_hi, double U, double tol,
                  double* dev_dJdX, double* dJdc, double* J, void* stream);

/* Bytes of device memory held by the handle. */
size_t pf_workspace_bytes(const pf_batch* b);

/* Names of the calls above for callers that think of a handle as one mesh or as a batch
   (a pf_mesh_build handle is a batch of one variant):
   pf_mesh_info: counts of variant 0 (nodes, DOF, boundary edges, min det J), any output
   may be NULL; PF_EINVAL for a NULL handle.
   pf_batch_solve: pf_psi_solve without the nodal psi output.
   pf_batch_grad: pf_grad.
   pf_mesh_destroy: pf_batch_destroy. */
pf_status pf_mesh_info(const pf_batch* b, long long* n_nodes, long long* n_dof, int* n_boundary_edges,
                       double* min_detJ);
pf_status pf_batch_solve(pf_batch* b, double U, const pf_solve_opts* opts, double* body_psi, pf_solve_info* info,
                         void* stream);
pf_status pf_batch_grad(pf_batch* b, int objective, int body_lo, int body_hi, double U, double tol,
                        double* dev_dJdX, double* dJdc, double* J, void* stream);
void pf_mesh_destroy(pf_batch* b);

const char* pf_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PFQ4_H */
