"""Oracle: unknown set, multi-point constraints and the reduced linear system.

Section "Matrix-Free Conjugate Gradient with Multiple Constraint Enforcement":
the unknowns are the interior and natural-boundary nodes plus one value C_k per
immersed body, N_dof = N_int + N_N + N_b.  Dirichlet nodes carry known values
(here psi = U*y on sides marked DIRICHLET_UY, the reference streamline of section
"Boundary Conditions"), every node of body k carries the single unknown C_k
(psi|Gamma_k = C_k), and nodes inside a body that touch no active cell carry
nothing.  Section "Weak formulation": the right-hand side comes only from the
Dirichlet values (natural sides have zero flux, q_bar = 0).

The reduced matrix is the sum of element matrices with the body rows and columns
collapsed onto C_k:  A_IJ = sum_e sum_{a,b: m(a)=I, m(b)=J} K_e[a,b],
b_I = - sum_e sum_{a: m(a)=I, b Dirichlet} K_e[a,b] g_b.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .element import q4_stiffness
from .mesh import BODY, DIRICHLET, FREE, Mesh, cell_coords, cell_nodes


@dataclass
class System:
    A: sp.csr_matrix          # reduced SPD matrix (N_dof x N_dof)
    b: np.ndarray             # reduced right-hand side
    dof: np.ndarray           # (N,) node -> unknown index, or -1 (Dirichlet / inactive)
    n_free: int
    n_bodies: int
    g: np.ndarray             # (N,) Dirichlet values (0 elsewhere)
    Ke: np.ndarray            # (E_active, 4, 4) element matrices of the active cells
    cells: np.ndarray         # (E_active, 4) node indices of the active cells
    detmin: np.ndarray        # (E_active,) min det J per active cell

    @property
    def n_dof(self):
        return self.n_free + self.n_bodies


def dof_map(mesh: Mesh):
    """FREE nodes numbered in node order, then one unknown per body."""
    kind = mesh.kind.ravel()
    body = mesh.body.ravel()
    dof = np.full(kind.shape, -1, dtype=np.int64)
    free = np.flatnonzero(kind == FREE)
    dof[free] = np.arange(free.size)
    nb = len(mesh.bodies)
    isb = kind == BODY
    dof[isb] = free.size + body[isb]
    return dof, int(free.size), nb


def dirichlet_values(mesh: Mesh, U):
    """g = U*y on Dirichlet nodes (uniform stream psi = U y)."""
    g = np.zeros(mesh.n_nodes)
    d = mesh.kind.ravel() == DIRICHLET
    g[d] = U * mesh.y.ravel()[d]
    return g


def element_matrices(mesh: Mesh):
    """K_e and the corner node indices of every active cell (the cut-cell matrices of
    `oracle.cutmesh` on a mixed-cell mesh)."""
    if mesh.cut_points is not None:
        from .cutmesh import element_matrices as cut_element_matrices
        return cut_element_matrices(mesh)
    xy = cell_coords(mesh)[mesh.active]
    cells = cell_nodes(mesh.nx, mesh.ny)[mesh.active]
    Ke, detmin = q4_stiffness(xy)
    return Ke, cells, detmin


def assemble(mesh: Mesh, U=1.0, check_valid=True, g=None) -> System:
    """Reduced system for psi = U y on Dirichlet sides, or for the nodal Dirichlet
    values `g` when given (used by the patch test and the closed-form cylinder)."""
    Ke, cells, detmin = element_matrices(mesh)
    if check_valid and detmin.size and detmin.min() <= 0.0:
        raise ValueError("mesh invalid: det J <= 0 at a Gauss point")
    dof, n_free, nb = dof_map(mesh)
    if g is None:
        g = dirichlet_values(mesh, U)
    else:
        g = np.where(mesh.kind.ravel() == DIRICHLET, np.asarray(g, dtype=np.float64), 0.0)
    n_dof = n_free + nb
    I = dof[cells]                     # (E,4)
    rows = np.repeat(I, 4, axis=1).ravel()
    cols = np.tile(I, (1, 4)).ravel()
    vals = Ke.reshape(-1, 16).ravel()
    keep = (rows >= 0) & (cols >= 0)
    A = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(n_dof, n_dof)).tocsr()
    A.sum_duplicates()
    # Dirichlet lifting: b_I = - sum K_e[a,b] g_b over Dirichlet corners b
    ge = g[cells]                      # (E,4), zero at non-Dirichlet corners
    contrib = -np.einsum("eab,eb->ea", Ke, ge)
    b = np.zeros(n_dof)
    m = I >= 0
    np.add.at(b, I[m], contrib[m])
    return System(A, b, dof, n_free, nb, g, Ke, cells, detmin)


def expand(system: System, u):
    """Nodal psi from the reduced solution: unknowns, body values, Dirichlet data."""
    psi = system.g.copy()
    m = system.dof >= 0
    psi[m] = u[system.dof[m]]
    return psi


def full_operator_apply(system: System, v):
    """y = sum_e K_e v_e over active cells, for a nodal vector v (no constraints)."""
    ye = np.einsum("eab,eb->ea", system.Ke, v[system.cells])
    y = np.zeros_like(v)
    np.add.at(y, system.cells.ravel(), ye.ravel())
    return y


def kutta_rows(system: System, mesh: Mesh):
    """The reduced system with the Kutta condition (section "Boundary Conditions"): for
    every polygon body k with a Kutta condition, its equation - the collapsed body row,
    i.e. zero circulation around the body - is replaced by psi(W) - C_k = 0, W the wake
    node on the trailing-edge bisector, so that the body streamline psi = C_k leaves the
    trailing edge along the bisector and the circulation follows from the solution.
    Returns (A, b) of the modified, no longer symmetric, system."""
    A = system.A.tolil(copy=True)
    b = system.b.copy()
    n_circ = system.n_bodies - len(mesh.polygons)
    for q, nw in enumerate(mesh.wake_node):
        if nw < 0:
            continue
        row = system.n_free + n_circ + q
        A.rows[row] = []
        A.data[row] = []
        A[row, system.dof[nw]] = 1.0
        A[row, row] = -1.0
        b[row] = 0.0
    return A.tocsr(), b
