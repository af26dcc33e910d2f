"""Python binding of the GB300 matrix-free Q4 stream-function solver.

Thin layer over the C ABI (include/pfq4.h): it marshals arguments, allocates the
caller-owned outputs as torch CUDA tensors and passes torch's current stream.
Every step of the computation runs in the library's CUDA kernels; there is no CPU
fallback, and loading fails loudly when the library has not been built.

    mesh = mesh_build(grid, bodies, sweeps)          # section "Body-Conforming Grid Generation"
    res = psi_solve(mesh, U=1.0, tol=1e-8)           # Appendix A, Algorithm
    theta, ut = surface_velocity(mesh, 0, body=0)    # section "Velocity Field and ..."
    copfi, q = copfi(mesh, 0, lo=3, hi=4, U=1.0)     # section "Effect of Gap Ratio"
"""
from __future__ import annotations

import atexit
import ctypes as C
import weakref
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from ._lib import PF_FP64, PF_MIXED, PF_OBJ_COPFI, PF_OBJ_GAP_FLOW, PF_TOL_PAPER_ABS, PF_TOL_REL_TRUE, check

__all__ = ["Mesh", "SolveResult", "mesh_build", "batch_build", "psi_solve", "apply", "surface_velocity",
           "copfi", "grad", "use_torch_allocator", "PF_FP64", "PF_MIXED", "PF_OBJ_COPFI", "PF_OBJ_GAP_FLOW",
           "PF_TOL_REL_TRUE", "PF_TOL_PAPER_ABS"]


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


_LIVE = weakref.WeakSet()
_HOOKS = []


def use_torch_allocator(enable: bool = True):
    """Route the library's device allocations through torch's caching allocator
    (applies to handles built afterwards).  Rebuilding meshes in a loop then reuses
    cached blocks instead of calling cudaMalloc / cudaFree every time."""
    lib = L.load()
    if not enable:
        check(lib.pf_set_allocator(L.ALLOC_FN(), L.FREE_FN(), None))
        _HOOKS.clear()
        return

    @L.ALLOC_FN
    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
        except Exception:
            return None

    @L.FREE_FN
    def _free(ptr, stream, ctx):
        try:
            torch.cuda.caching_allocator_delete(int(ptr))
        except Exception:
            pass

    _HOOKS[:] = [_alloc, _free]
    check(lib.pf_set_allocator(_alloc, _free, None))


@atexit.register
def _close_live_handles():
    # release library memory while torch's allocator is still alive
    for m in list(_LIVE):
        try:
            m.close()
        except Exception:
            pass


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


@dataclass
class SolveResult:
    psi: torch.Tensor            # (total nodes,) float64 on the GPU, logical order per variant
    body_psi: np.ndarray         # (total bodies,) C_i
    info: list                   # per-variant dicts: iters, refinements, status, rel_true_residual, n_dof
    status: int


class Mesh:
    """A pf_batch handle: one or more body-conforming mesh variants on the GPU."""

    def __init__(self, grids, body_lists, sweeps, bc=(0, 0, 0, 0), polygon_lists=None, cut_spacing=None):
        """polygon_lists (optional): per variant, polygon bodies (objects with `vertices`
        ((n, 2), counter-clockwise), `ref` (reference point of the polar angle) and `kutta`
        (trailing-edge vertex or -1)); a variant's bodies are its circles, then its polygons.
        cut_spacing (optional): build the mixed-cell mesh (pf_batch_build_cut)
        with this minimum surface-point spacing, a fraction of min(hx, hy)."""
        lib = L.load()
        nv = len(grids)
        g = (L.pf_grid * nv)()
        for v, gr in enumerate(grids):
            x0, x1, y0, y1, nx, ny = gr
            g[v] = L.pf_grid(float(x0), float(x1), float(y0), float(y1), int(nx), int(ny))
        polygon_lists = [list(pl) for pl in polygon_lists] if polygon_lists is not None else [[] for _ in grids]
        if len(polygon_lists) != nv:
            raise ValueError("one polygon list per variant")
        offs = [0]
        flat = []
        for bl, pl in zip(body_lists, polygon_lists):
            bl = np.asarray(bl, dtype=np.float64).reshape(-1, 3)
            flat.extend(("c", row) for row in bl.tolist())
            flat.extend(("p", p) for p in pl)
            offs.append(len(flat))
        off = (C.c_int * (nv + 1))(*offs)
        bcs = (C.c_int * 4)(*[int(s) for s in bc])
        h = C.c_void_p()
        self._h = None
        if any(polygon_lists) or cut_spacing is not None:
            shapes = (L.pf_shape * max(1, len(flat)))()
            self._vertex_bufs = []
            for k, (kind, b) in enumerate(flat):
                if kind == "c":
                    shapes[k] = L.pf_shape(L.PF_SHAPE_CIRCLE, *map(float, b), 0, None, -1)
                else:
                    vx = np.ascontiguousarray(np.asarray(b.vertices, dtype=np.float64).reshape(-1, 2))
                    buf = (C.c_double * vx.size)(*vx.ravel().tolist())
                    self._vertex_bufs.append(buf)
                    shapes[k] = L.pf_shape(L.PF_SHAPE_POLYGON, float(b.ref[0]), float(b.ref[1]), 0.0, len(vx),
                                           C.cast(buf, C.POINTER(C.c_double)), int(b.kutta))
            if cut_spacing is not None:
                code = lib.pf_batch_build_cut(g, off, shapes, nv, int(sweeps), bcs, float(cut_spacing), _stream(),
                                              C.byref(h))
            else:
                code = lib.pf_batch_build_shapes(g, off, shapes, nv, int(sweeps), bcs, _stream(), C.byref(h))
        else:
            bodies = (L.pf_body * max(1, len(flat)))(*[L.pf_body(*row) for _, row in flat])
            code = lib.pf_batch_build(g, off, bodies, nv, int(sweeps), bcs, _stream(), C.byref(h))
        if code == L.PF_EMESH_INVALID:
            self._h = h
            self.valid = False
        else:
            check(code)
            self._h = h
            self.valid = True
        self.n_variants = nv
        self.grids = [tuple(gr) for gr in grids]
        self.bodies = [np.asarray(bl, dtype=np.float64).reshape(-1, 3) for bl in body_lists]
        self.polygons = polygon_lists
        self.body_offsets = offs
        self.n_nodes = [(gr[4] + 1) * (gr[5] + 1) for gr in grids]
        self.node_offsets = np.concatenate([[0], np.cumsum(self.n_nodes)]).astype(np.int64)
        self.sweeps = sweeps
        self.bc = tuple(bc)
        self.cut = cut_spacing is not None
        _LIVE.add(self)

    # ------------------------------------------------------------------ handle
    @property
    def handle(self):
        if self._h is None:
            raise RuntimeError("mesh handle is closed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            L.load().pf_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------ queries
    def stats(self, v=0) -> dict:
        s = L.pf_mesh_stats()
        check(L.load().pf_mesh_stats_get(self.handle, v, C.byref(s)))
        return {k: getattr(s, k) for k, _ in L.pf_mesh_stats._fields_}

    def workspace_bytes(self) -> int:
        return int(L.load().pf_workspace_bytes(self.handle))

    def coords(self, v=0) -> torch.Tensor:
        out = torch.empty((self.n_nodes[v], 2), dtype=torch.float64, device="cuda")
        check(L.load().pf_mesh_coords(self.handle, v, _ptr(out), _stream()))
        return out

    def set_coords(self, xy, v=0):
        """Replace variant v's node coordinates ((nodes, 2) float64), topology fixed; returns
        the status (PF_OK, or PF_EMESH_INVALID if a cell folds)."""
        xy = torch.as_tensor(xy).to(device="cuda", dtype=torch.float64).contiguous()
        if tuple(xy.shape) != (self.n_nodes[v], 2):
            raise ValueError(f"coordinates must have shape ({self.n_nodes[v]}, 2)")
        return check(L.load().pf_mesh_set_coords(self.handle, v, _ptr(xy), _stream()), allow=(L.PF_EMESH_INVALID,))

    def coords_vjp(self, gX):
        """(dX/dc)^T gX: cotangent on the body centres ((bodies, 2) numpy) of a cotangent gX on
        every variant's node coordinates ((total nodes, 2) tensor)."""
        gX = torch.as_tensor(gX).to(device="cuda", dtype=torch.float64).contiguous()
        if tuple(gX.shape) != (int(self.node_offsets[-1]), 2):
            raise ValueError("cotangent must have shape (total nodes, 2)")
        nb = self.body_offsets[-1]
        gc = (C.c_double * max(1, 2 * nb))()
        check(L.load().pf_coords_vjp(self.handle, _ptr(gX), gc, _stream()))
        return np.array(gc[:2 * nb]).reshape(nb, 2)

    def cut_points(self, v=0):
        """(4, nodes, 2) surface points of a mixed-cell mesh (E, N, W, S; NaN where none)."""
        out = torch.empty((4, self.n_nodes[v], 2), dtype=torch.float64, device="cuda")
        check(L.load().pf_mesh_cut_points(self.handle, v, _ptr(out), _stream()))
        return out

    def tags(self, v=0):
        kind = torch.empty(self.n_nodes[v], dtype=torch.int8, device="cuda")
        body = torch.empty(self.n_nodes[v], dtype=torch.int32, device="cuda")
        check(L.load().pf_mesh_tags(self.handle, v, _ptr(kind), _ptr(body), _stream()))
        return kind, body

    def timing(self) -> dict:
        t = L.pf_timing()
        check(L.load().pf_last_timing(self.handle, C.byref(t)))
        return {k: getattr(t, k) for k, _ in L.pf_timing._fields_}

    def apply_timing(self, precision=PF_MIXED, reps=100):
        """(microseconds, algorithmic bytes) of one stand-alone operator application."""
        us, by = C.c_double(), C.c_double()
        check(L.load().pf_apply_timing(self.handle, int(precision), int(reps), C.byref(us), C.byref(by), _stream()))
        return us.value, by.value

    def test_wait_timeout(self, enable=True):
        """Test hook: later solves make a bounded device wait give up (PF_ETIMEOUT)."""
        check(L.load().pf_test_wait_timeout(self.handle, int(bool(enable))))


def mesh_build(grid, bodies, sweeps, bc=(0, 0, 0, 0), polygons=None) -> Mesh:
    """One variant: grid = (x0, x1, y0, y1, nx, ny), bodies = rows of (cx, cy, r), then the
    optional polygon bodies."""
    return Mesh([grid], [bodies], sweeps, bc, None if polygons is None else [polygons])


def batch_build(cases, sweeps=None, bc=None, polygons=None, cut_spacing=None) -> Mesh:
    """Many variants (objects with .grid, .bodies, .sweeps, .bc) in one handle; polygons:
    optional per-variant lists of polygon bodies; cut_spacing: the mixed-cell mesh with this
    minimum surface-point spacing (a fraction of min(hx, hy), 0 for none)."""
    sweeps = cases[0].sweeps if sweeps is None else sweeps
    bc = cases[0].bc if bc is None else bc
    return Mesh([c.grid for c in cases], [c.bodies for c in cases], sweeps, bc, polygons, cut_spacing)


def cut_mesh_build(grid, bodies, sweeps, bc=(0, 0, 0, 0), cut_spacing=0.0, polygons=None) -> Mesh:
    """One variant of the mixed-cell mesh (node splitting, triangle / pentagon cells);
    polygons: optional polygon bodies after the circles."""
    return Mesh([grid], [bodies], sweeps, bc, None if polygons is None else [polygons], cut_spacing)


def apply(mesh: Mesh, p: torch.Tensor, precision=PF_FP64):
    """y = A p on nodal vectors (FREE and BODY rows), plus the collapsed body rows."""
    p = p.to(device="cuda", dtype=torch.float64).contiguous()
    y = torch.empty_like(p)
    nb = mesh.body_offsets[-1]
    sums = (C.c_double * max(1, nb))()
    check(L.load().pf_apply(mesh.handle, int(precision), _ptr(p), _ptr(y), sums, _stream()))
    return y, np.array(sums[:nb])


def _opts(tol, k_max, precision, inner_tol, chunk, warm_start, tune_schedule, criterion, preconditioner="none"):
    crit = {"relative": PF_TOL_REL_TRUE, "paper": PF_TOL_PAPER_ABS}.get(criterion, criterion)
    pre = {"none": L.PF_PRECOND_NONE, "mg": L.PF_PRECOND_MG}.get(preconditioner, preconditioner)
    return L.pf_solve_opts(float(tol), int(k_max), int(precision), float(inner_tol), int(chunk),
                           int(bool(warm_start)), int(bool(tune_schedule)), int(crit), int(pre))


def psi_solve(mesh: Mesh, U=1.0, tol=1e-8, precision=PF_MIXED, k_max=10_000_000, inner_tol=2e-7,
              chunk=0, warm_start=False, want_psi=True, raise_on_failure=True, method="mpc",
              tune_schedule=False, criterion="relative", preconditioner="none") -> SolveResult:
    """Solve for psi.  method="mpc": CG on the multi-point-constraint system;
    method="schur": body values through the Schur complement (N_b + 1 fixed-body solves).
    criterion="relative": stop on the FP64 true residual ||b - A u|| / ||b|| <= tol;
    criterion="paper": the Appendix A test, sum r^2 <= tol (PF_TOL_PAPER_ABS).
    preconditioner="mg": CG preconditioned by a multigrid V-cycle (PF_PRECOND_MG, mixed)."""
    opts = _opts(tol, k_max, precision, inner_tol, chunk, warm_start, tune_schedule, criterion, preconditioner)
    total = int(mesh.node_offsets[-1])
    psi = torch.empty(total, dtype=torch.float64, device="cuda") if want_psi else None
    nb = mesh.body_offsets[-1]
    bpsi = (C.c_double * max(1, nb))()
    info = (L.pf_solve_info * mesh.n_variants)()
    fn = L.load().pf_psi_solve_schur if method == "schur" else L.load().pf_psi_solve
    code = fn(mesh.handle, float(U), C.byref(opts), _ptr(psi), bpsi, info, _stream())
    if raise_on_failure:
        check(code)
    infos = [{k: getattr(i, k) for k, _ in L.pf_solve_info._fields_} for i in info]
    return SolveResult(psi, np.array(bpsi[:nb]), infos, code)


def surface_velocity(mesh: Mesh, v=0, body=0):
    """(theta_deg, u_t) on the boundary edges of one body after a solve."""
    cnt = C.c_int()
    check(L.load().pf_surface_velocity(mesh.handle, v, body, None, None, 0, C.byref(cnt), _stream()))
    n = cnt.value
    th = (C.c_double * max(1, n))()
    ut = (C.c_double * max(1, n))()
    check(L.load().pf_surface_velocity(mesh.handle, v, body, th, ut, n, C.byref(cnt), _stream()))
    return np.array(th[:n]), np.array(ut[:n])


def velocity_field(mesh: Mesh, v=0):
    """(u, v) at the centre of every cell of variant v after a solve, as (ny, nx) tensors on
    the device (u = dpsi/dy, v = -dpsi/dx; 0 on inactive cells)."""
    nx, ny = mesh.grids[v][4], mesh.grids[v][5]
    u = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    w = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    check(L.load().pf_velocity_field(mesh.handle, v, _ptr(u), _ptr(w), _stream()))
    return u, w


def phi_solve(mesh: Mesh, U=1.0, tol=1e-8, precision=PF_MIXED, k_max=10_000_000, inner_tol=2e-7, chunk=0,
              raise_on_failure=True, tune_schedule=False, criterion="relative", preconditioner="none"):
    """Velocity potential: phi = U x on the inlet and outlet sides, no flux on the walls and
    bodies.  Returns (phi (total nodes,) float64 tensor, per-variant info dicts, status)."""
    opts = _opts(tol, k_max, precision, inner_tol, chunk, False, tune_schedule, criterion, preconditioner)
    phi = torch.empty(int(mesh.node_offsets[-1]), dtype=torch.float64, device="cuda")
    info = (L.pf_solve_info * mesh.n_variants)()
    code = L.load().pf_phi_solve(mesh.handle, float(U), C.byref(opts), _ptr(phi), info, _stream())
    if raise_on_failure:
        check(code)
    return phi, [{k: getattr(i, k) for k, _ in L.pf_solve_info._fields_} for i in info], code


def phi_velocity_field(mesh: Mesh, v=0):
    """(u, v) = grad phi at the centre of every cell of variant v after a phi solve, as
    (ny, nx) tensors (0 on inactive cells)."""
    nx, ny = mesh.grids[v][4], mesh.grids[v][5]
    u = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    w = torch.empty((ny, nx), dtype=torch.float64, device="cuda")
    check(L.load().pf_phi_velocity_field(mesh.handle, v, _ptr(u), _ptr(w), _stream()))
    return u, w


def copfi(mesh: Mesh, v=0, lo=3, hi=4, U=1.0):
    """(CoPFI, Q) = ((C_hi - C_lo) / (U (cy_hi - cy_lo)), C_hi - C_lo) after a solve."""
    c = C.c_double()
    q = C.c_double()
    check(L.load().pf_copfi(mesh.handle, v, lo, hi, float(U), C.byref(c), C.byref(q)))
    return c.value, q.value


def grad(mesh: Mesh, objective=PF_OBJ_COPFI, lo=3, hi=4, U=1.0, tol=1e-12, want_dX=True):
    """Adjoint shape gradient after a solve: (dJ/dX (nodes, 2) tensor, dJ/dc (bodies, 2), J per variant)."""
    total = int(mesh.node_offsets[-1])
    dX = torch.empty((total, 2), dtype=torch.float64, device="cuda") if want_dX else None
    nb = mesh.body_offsets[-1]
    dc = (C.c_double * max(1, 2 * nb))()
    J = (C.c_double * mesh.n_variants)()
    check(L.load().pf_grad(mesh.handle, int(objective), int(lo), int(hi), float(U), float(tol), _ptr(dX), dc, J,
                           _stream()))
    return dX, np.array(dc[:2 * nb]).reshape(nb, 2), np.array(J[:])


def mesh_info(mesh: Mesh) -> dict:
    """Counts of variant 0: nodes, DOF, boundary edges and the minimum det J."""
    nn, nd, ne, dj = C.c_longlong(), C.c_longlong(), C.c_int(), C.c_double()
    check(L.load().pf_mesh_info(mesh.handle, C.byref(nn), C.byref(nd), C.byref(ne), C.byref(dj)))
    return {"n_nodes": nn.value, "n_dof": nd.value, "n_boundary_edges": ne.value, "min_detJ": dj.value}


def batch_solve(mesh: Mesh, U=1.0, tol=1e-8, precision=PF_MIXED, k_max=10_000_000, inner_tol=2e-7, chunk=0,
                warm_start=False, raise_on_failure=True, tune_schedule=False, criterion="relative",
                preconditioner="none") -> SolveResult:
    """Solve every variant of the batch; body psi and per-variant info only (no nodal psi)."""
    opts = _opts(tol, k_max, precision, inner_tol, chunk, warm_start, tune_schedule, criterion, preconditioner)
    nb = mesh.body_offsets[-1]
    bpsi = (C.c_double * max(1, nb))()
    info = (L.pf_solve_info * mesh.n_variants)()
    code = L.load().pf_batch_solve(mesh.handle, float(U), C.byref(opts), bpsi, info, _stream())
    if raise_on_failure:
        check(code)
    infos = [{k: getattr(i, k) for k, _ in L.pf_solve_info._fields_} for i in info]
    return SolveResult(None, np.array(bpsi[:nb]), infos, code)


def batch_grad(mesh: Mesh, objective=PF_OBJ_COPFI, lo=3, hi=4, U=1.0, tol=1e-12, want_dX=True):
    """Adjoint shape gradient of every variant after a solve (same outputs as grad)."""
    total = int(mesh.node_offsets[-1])
    dX = torch.empty((total, 2), dtype=torch.float64, device="cuda") if want_dX else None
    nb = mesh.body_offsets[-1]
    dc = (C.c_double * max(1, 2 * nb))()
    J = (C.c_double * mesh.n_variants)()
    check(L.load().pf_batch_grad(mesh.handle, int(objective), int(lo), int(hi), float(U), float(tol), _ptr(dX), dc,
                                 J, _stream()))
    return dX, np.array(dc[:2 * nb]).reshape(nb, 2), np.array(J[:])


def mesh_destroy(mesh: Mesh) -> None:
    """Release the handle's device memory (the Mesh object is unusable afterwards)."""
    if getattr(mesh, "_h", None) is not None:
        L.load().pf_mesh_destroy(mesh._h)
        mesh._h = None
