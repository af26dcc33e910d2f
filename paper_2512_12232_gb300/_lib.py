"""ctypes declarations of the C ABI in include/pfq4.h (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

from .build import LIB

PF_OK, PF_EINVAL, PF_EMESH_INVALID, PF_ENOT_CONVERGED, PF_EBREAKDOWN, PF_ETIMEOUT, PF_ECUDA, PF_ENOMEM = range(8)
STATUS_NAMES = {0: "PF_OK", 1: "PF_EINVAL", 2: "PF_EMESH_INVALID", 3: "PF_ENOT_CONVERGED",
                4: "PF_EBREAKDOWN", 5: "PF_ETIMEOUT", 6: "PF_ECUDA", 7: "PF_ENOMEM"}
PF_FP64, PF_MIXED = 0, 1
PF_TOL_REL_TRUE, PF_TOL_PAPER_ABS = 0, 1
PF_PRECOND_NONE, PF_PRECOND_MG = 0, 1
PF_OBJ_COPFI, PF_OBJ_GAP_FLOW = 0, 1
PF_SHAPE_CIRCLE, PF_SHAPE_POLYGON = 0, 1


class pf_grid(C.Structure):
    _fields_ = [("x0", C.c_double), ("x1", C.c_double), ("y0", C.c_double), ("y1", C.c_double),
                ("nx", C.c_int), ("ny", C.c_int)]


class pf_body(C.Structure):
    _fields_ = [("cx", C.c_double), ("cy", C.c_double), ("r", C.c_double)]


class pf_shape(C.Structure):
    _fields_ = [("kind", C.c_int), ("cx", C.c_double), ("cy", C.c_double), ("r", C.c_double),
                ("n_vertices", C.c_int), ("vertex_xy", C.POINTER(C.c_double)), ("kutta_vertex", C.c_int)]


class pf_mesh_stats(C.Structure):
    _fields_ = [("n_nodes", C.c_longlong), ("n_free", C.c_longlong), ("n_dof", C.c_longlong),
                ("n_body_nodes", C.c_longlong), ("n_inactive", C.c_longlong),
                ("n_active_cells", C.c_longlong), ("n_general_cells", C.c_longlong),
                ("n_bodies", C.c_int), ("n_boundary_edges", C.c_int), ("min_detJ", C.c_double),
                ("h", C.c_double)]


class pf_solve_opts(C.Structure):
    _fields_ = [("tol", C.c_double), ("k_max", C.c_longlong), ("precision", C.c_int),
                ("inner_tol", C.c_double), ("chunk", C.c_int), ("warm_start", C.c_int),
                ("tune_schedule", C.c_int), ("criterion", C.c_int), ("preconditioner", C.c_int)]


class pf_solve_info(C.Structure):
    _fields_ = [("iters", C.c_longlong), ("refinements", C.c_int), ("status", C.c_int),
                ("rel_true_residual", C.c_double), ("n_dof", C.c_longlong)]


class pf_timing(C.Structure):
    _fields_ = [("cg_kernel_ms", C.c_double), ("cg_launches", C.c_longlong),
                ("residual_kernel_ms", C.c_double), ("residual_launches", C.c_longlong),
                ("solve_ms", C.c_double), ("cg_bytes_per_launch", C.c_double),
                ("kernel_launches", C.c_longlong), ("cg_stages", C.c_int)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)

P = C.c_void_p
_SIGS = {
    "pf_set_allocator": (C.c_int, [ALLOC_FN, FREE_FN, P]),
    "pf_batch_build": (C.c_int, [C.POINTER(pf_grid), C.POINTER(C.c_int), C.POINTER(pf_body), C.c_int, C.c_int,
                                 C.POINTER(C.c_int), P, C.POINTER(P)]),
    "pf_batch_build_shapes": (C.c_int, [C.POINTER(pf_grid), C.POINTER(C.c_int), C.POINTER(pf_shape), C.c_int,
                                        C.c_int, C.POINTER(C.c_int), P, C.POINTER(P)]),
    "pf_mesh_build": (C.c_int, [C.POINTER(pf_grid), C.POINTER(pf_body), C.c_int, C.c_int, C.POINTER(C.c_int), P,
                                C.POINTER(P)]),
    "pf_batch_destroy": (None, [P]),
    "pf_batch_size": (C.c_int, [P, C.POINTER(C.c_int), C.POINTER(C.c_longlong), C.POINTER(C.c_int)]),
    "pf_mesh_stats_get": (C.c_int, [P, C.c_int, C.POINTER(pf_mesh_stats)]),
    "pf_mesh_coords": (C.c_int, [P, C.c_int, P, P]),
    "pf_mesh_tags": (C.c_int, [P, C.c_int, P, P, P]),
    "pf_batch_build_cut": (C.c_int, [C.POINTER(pf_grid), C.POINTER(C.c_int), C.POINTER(pf_shape), C.c_int, C.c_int,
                                     C.POINTER(C.c_int), C.c_double, P, C.POINTER(P)]),
    "pf_mesh_cut_points": (C.c_int, [P, C.c_int, P, P]),
    "pf_mesh_set_coords": (C.c_int, [P, C.c_int, P, P]),
    "pf_coords_vjp": (C.c_int, [P, P, P, P]),
    "pf_apply": (C.c_int, [P, C.c_int, P, P, P, P]),
    "pf_apply_noalloc": (C.c_int, [P, C.c_int, P, P, P, P]),
    "pf_psi_solve": (C.c_int, [P, C.c_double, C.POINTER(pf_solve_opts), P, P, P, P]),
    "pf_psi_solve_schur": (C.c_int, [P, C.c_double, C.POINTER(pf_solve_opts), P, P, P, P]),
    "pf_phi_solve": (C.c_int, [P, C.c_double, C.POINTER(pf_solve_opts), P, P, P]),
    "pf_phi_velocity_field": (C.c_int, [P, C.c_int, P, P, P]),
    "pf_test_wait_timeout": (C.c_int, [P, C.c_int]),
    "pf_apply_timing": (C.c_int, [P, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), P]),
    "pf_last_timing": (C.c_int, [P, C.POINTER(pf_timing)]),
    "pf_surface_velocity": (C.c_int, [P, C.c_int, C.c_int, P, P, C.c_int, C.POINTER(C.c_int), P]),
    "pf_velocity_field": (C.c_int, [P, C.c_int, P, P, P]),
    "pf_copfi": (C.c_int, [P, C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double),
                           C.POINTER(C.c_double)]),
    "pf_grad": (C.c_int, [P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, P, P, P, P]),
    "pf_workspace_bytes": (C.c_size_t, [P]),
    "pf_mesh_info": (C.c_int, [P, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong), C.POINTER(C.c_int),
                               C.POINTER(C.c_double)]),
    "pf_batch_solve": (C.c_int, [P, C.c_double, C.POINTER(pf_solve_opts), P, P, P]),
    "pf_batch_grad": (C.c_int, [P, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, P, P, P, P]),
    "pf_mesh_destroy": (None, [P]),
    "pf_last_error": (C.c_char_p, []),
}
EXPORTED = tuple(_SIGS)

_lib = None


def load(path: str = LIB):
    """Load the CUDA library; raises if it has not been built (there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library {path} is missing: build it with __graft_entry__.build() "
                           "(python -m paper_2512_12232_gb300.build)")
    lib = C.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class PfError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code, allow=()):
    if code != PF_OK and code not in allow:
        raise PfError(code, load().pf_last_error().decode(errors="replace"))
    return code
