"""Oracle (test infrastructure only): velocity potential phi, element velocities and the
flow net.  Plain float64 numpy/scipy, independent of the CUDA library.

Section "Governing Equation": in incompressible, irrotational flow the velocity is
u = grad phi with nabla^2 phi = 0, and the contour lines of phi and of the stream function
psi (u = (dpsi/dy, -dpsi/dx)) are two orthogonal families of curves, the flow net.
Section "Velocity Field and Surface Tangential Velocity": once psi is known,
u = dpsi/dy and v = -dpsi/dx.  Section "Weak formulation": the same Q4 element matrices
K_e as for psi, since both fields solve the Laplace equation on the same mesh.

Readings taken where the paper is silent:
  * Boundary conditions of phi.  phi = U*x on the inlet and outlet sides (x = x0 and
    x = x1) and a zero normal derivative (the natural condition, no flux) on the two other
    sides and on every body surface.  Where no body disturbs the stream this is the uniform
    flow phi = U x that matches psi = U y on the sides.  For the pins below the Dirichlet
    set can instead be the whole outer ring with given nodal values.
  * Unknowns.  Every node that is neither inactive nor Dirichlet.  Body nodes are ordinary
    unknowns: phi varies along a body surface, only psi is constant there, so there is no
    multi-point constraint.
  * Element velocity.  The gradient of the bilinear interpolant at the element centre
    (xi = eta = 0), through the isoparametric map.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .element import shape_derivatives
from .mesh import INACTIVE, Mesh, cell_coords, cell_nodes
from .system import element_matrices


@dataclass
class PhiSystem:
    A: sp.csr_matrix          # SPD matrix over the unknowns
    b: np.ndarray             # right-hand side (Dirichlet lifting only)
    dof: np.ndarray           # (N,) node -> unknown index, or -1 (Dirichlet / inactive)
    dirichlet: np.ndarray     # (N,) bool
    g: np.ndarray             # (N,) Dirichlet values (0 elsewhere)
    Ke: np.ndarray            # (E_active, 4, 4)
    cells: np.ndarray         # (E_active, 4) node indices of the active cells


def inlet_outlet_mask(mesh: Mesh) -> np.ndarray:
    """Nodes on the x = x0 and x = x1 sides that are not inactive."""
    i = np.arange(mesh.n_nodes) % (mesh.nx + 1)
    return ((i == 0) | (i == mesh.nx)) & (mesh.kind.ravel() != INACTIVE)


def ring_mask(mesh: Mesh) -> np.ndarray:
    """Nodes on the outer boundary of the grid."""
    n = np.arange(mesh.n_nodes)
    i, j = n % (mesh.nx + 1), n // (mesh.nx + 1)
    return (i == 0) | (i == mesh.nx) | (j == 0) | (j == mesh.ny)


def assemble_phi(mesh: Mesh, U=1.0, dirichlet=None, g=None) -> PhiSystem:
    """The phi system.  Default: phi = U x on the inlet and outlet sides.  With
    `dirichlet` (a node mask) and `g` (nodal values), those nodes carry g instead."""
    Ke, cells, _ = element_matrices(mesh)
    kind = mesh.kind.ravel()
    if dirichlet is None:
        dirichlet = inlet_outlet_mask(mesh)
        gv = np.where(dirichlet, U * mesh.x.ravel(), 0.0)
    else:
        dirichlet = np.asarray(dirichlet, dtype=bool) & (kind != INACTIVE)
        gv = np.where(dirichlet, np.asarray(g, dtype=np.float64), 0.0)
    unknown = (kind != INACTIVE) & ~dirichlet
    dof = np.full(kind.shape, -1, dtype=np.int64)
    dof[unknown] = np.arange(int(unknown.sum()))
    n = int(unknown.sum())
    I = dof[cells]
    rows = np.repeat(I, 4, axis=1).ravel()
    cols = np.tile(I, (1, 4)).ravel()
    vals = Ke.reshape(-1, 16).ravel()
    keep = (rows >= 0) & (cols >= 0)
    A = sp.coo_matrix((vals[keep], (rows[keep], cols[keep])), shape=(n, n)).tocsr()
    A.sum_duplicates()
    contrib = -np.einsum("eab,eb->ea", Ke, gv[cells])   # b_I = -sum_b K_e[a,b] g_b
    b = np.zeros(n)
    m = I >= 0
    np.add.at(b, I[m], contrib[m])
    return PhiSystem(A, b, dof, dirichlet, gv, Ke, cells)


def solve_phi(system: PhiSystem) -> np.ndarray:
    """Nodal phi: a direct sparse solve for the unknowns, the Dirichlet data elsewhere
    (0 at inactive nodes)."""
    phi = system.g.copy()
    if system.A.shape[0]:
        u = spla.spsolve(system.A.tocsc(), system.b)
        m = system.dof >= 0
        phi[m] = u[system.dof[m]]
    return phi


def nodal_residual(system: PhiSystem, phi: np.ndarray) -> np.ndarray:
    """(K phi)_n summed over active cells: the flux at Dirichlet nodes, ~0 at unknowns."""
    ye = np.einsum("eab,eb->ea", system.Ke, phi[system.cells])
    r = np.zeros_like(phi)
    np.add.at(r, system.cells.ravel(), ye.ravel())
    return r


def element_gradient(mesh: Mesh, field: np.ndarray):
    """(d f/dx, d f/dy) of the bilinear interpolant of the nodal field f at the centre of
    every active cell, and the centres (mean of the four corners); each (E_active,)."""
    xy = cell_coords(mesh)[mesh.active]          # (E, 4, 2)
    cells = cell_nodes(mesh.nx, mesh.ny)[mesh.active]
    x, y = xy[..., 0], xy[..., 1]
    dxi, deta = shape_derivatives(0.0, 0.0)
    j00, j01 = x @ dxi, y @ dxi                   # dx/dxi, dy/dxi
    j10, j11 = x @ deta, y @ deta                 # dx/deta, dy/deta
    det = j00 * j11 - j01 * j10
    dndx = (j11[:, None] * dxi - j01[:, None] * deta) / det[:, None]
    dndy = (-j10[:, None] * dxi + j00[:, None] * deta) / det[:, None]
    f = field[cells]
    return (dndx * f).sum(axis=1), (dndy * f).sum(axis=1), x.mean(axis=1), y.mean(axis=1)


def velocity_from_psi(mesh: Mesh, psi: np.ndarray):
    """(u, v) = (dpsi/dy, -dpsi/dx) at the element centres."""
    fx, fy, _, _ = element_gradient(mesh, psi)
    return fy, -fx


def velocity_from_phi(mesh: Mesh, phi: np.ndarray):
    """(u, v) = grad phi at the element centres."""
    fx, fy, _, _ = element_gradient(mesh, phi)
    return fx, fy
