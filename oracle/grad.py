"""Oracle: adjoint shape gradients of CoPFI and of the transverse-gap flow.

Not in the paper, whose conclusions name shape optimisation and sensitivity
analysis as the next step.  The discrete objective is J(u, c) with u the reduced
solution of A(X) u = b(X) (section "Matrix-Free Conjugate Gradient with Multiple
Constraint Enforcement"), X the smoothed node coordinates and c the body centres:

  gap flow : J = C_hi - C_lo
  CoPFI    : J = (C_hi - C_lo) / (U (cy_hi - cy_lo))        (section "Effect of Gap Ratio")

With the residual R(u, X) = P^T K(X) psi(u, X) (P collapses body rows, psi carries
the Dirichlet data g = U y) and the adjoint A lambda = dJ/du,

  dJ/dX = - sum_e Lambda_e^T (dK_e/dX) psi_e - U (K Lambda)_n  [y of Dirichlet nodes n]

where Lambda is lambda expanded to the nodes.  The element derivative dK_e/dX is
taken by the complex step (`element.stiffness_shape_derivative`).  The mesh of
section "Body-Conforming Grid Generation" is linear in the projection
displacement: X = X_grid + M^S d0 (M one Jacobi sweep), so
dJ/dd0 = (M^T)^S dJ/dX, and d0 of a body node depends on the centre through the
radial projection, dx_b/dc = I - (r/rho)(I - u u^T).  The topology (which nodes are
inside) is held fixed.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .element import stiffness_shape_derivative
from .mesh import BODY, DIRICHLET, Mesh, smoothing_mask
from .system import System, assemble, expand, full_operator_apply
from .solve import solve_direct

OBJ_COPFI, OBJ_GAP_FLOW = 0, 1


def objective(C, bodies, lo, hi, U, obj):
    q = C[hi] - C[lo]
    if obj == OBJ_GAP_FLOW:
        return q
    return q / (U * (bodies[hi][1] - bodies[lo][1]))


def jacobi_matrix(mesh: Mesh):
    """Sparse matrix of one Jacobi sweep on logical node indices."""
    nx1, ny1 = mesh.nx + 1, mesh.ny + 1
    N = nx1 * ny1
    mask = smoothing_mask(mesh.kind, mesh.body).ravel()
    rows, cols, vals = [], [], []
    idx = np.arange(N)
    fixed = idx[~mask]
    rows.append(fixed); cols.append(fixed); vals.append(np.ones(fixed.size))
    upd = idx[mask]
    for off in (-1, 1, -nx1, nx1):
        rows.append(upd); cols.append(upd + off); vals.append(np.full(upd.size, 0.25))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(N, N))


def centre_chain(mesh: Mesh, sweeps: int, gX):
    """Cotangent on the body centres of a cotangent gX (N, 2) on the final node
    coordinates, through the mesh generator X = X_grid + M^S d0(c): S transposed Jacobi
    sweeps, then the radial projection's Jacobian at every body node's background
    position.  The topology is held fixed."""
    M = jacobi_matrix(mesh)
    MT = M.T.tocsr()
    gd = np.asarray(gX, dtype=np.float64).reshape(-1, 2).copy()
    for _ in range(sweeps):
        gd = MT @ gd
    out = np.zeros((len(mesh.bodies), 2))
    kind = mesh.kind.ravel()
    body = mesh.body.ravel()
    xg = mesh.xg.ravel()
    yg = mesh.yg.ravel()
    for k, (cx, cy, r) in enumerate(mesh.bodies):
        nodes = np.flatnonzero((kind == BODY) & (body == k))
        ex = xg[nodes] - cx
        ey = yg[nodes] - cy
        rho = np.sqrt(ex * ex + ey * ey)
        ux, uy = ex / rho, ey / rho
        s = r / rho
        # Jp = I - s (I - u u^T), symmetric
        j00 = 1.0 - s * (1.0 - ux * ux)
        j01 = s * ux * uy
        j11 = 1.0 - s * (1.0 - uy * uy)
        out[k, 0] = np.sum(j00 * gd[nodes, 0] + j01 * gd[nodes, 1])
        out[k, 1] = np.sum(j01 * gd[nodes, 0] + j11 * gd[nodes, 1])
    return out


def gradient(mesh: Mesh, sweeps: int, U: float, lo: int, hi: int, obj=OBJ_COPFI, system=None):
    """Returns (J, dJ/dX (N,2), dJ/dc (n_bodies,2), psi)."""
    if system is None:
        system = assemble(mesh, U)
    u, psi = solve_direct(system)
    nf = system.n_free
    C = u[nf:]
    bodies = mesh.bodies
    J = objective(C, bodies, lo, hi, U, obj)
    dy = bodies[hi][1] - bodies[lo][1]
    w = 1.0 if obj == OBJ_GAP_FLOW else 1.0 / (U * dy)
    rhs = np.zeros(system.n_dof)
    rhs[nf + hi] += w
    rhs[nf + lo] -= w
    lam = spla.spsolve(system.A.tocsc(), rhs)
    Lam = np.zeros(mesh.n_nodes)
    m = system.dof >= 0
    Lam[m] = lam[system.dof[m]]
    # element term: - sum_e Lambda_e^T dK_e/dx_{a,c} psi_e, scattered to the corners
    xy = np.stack([mesh.x.ravel()[system.cells], mesh.y.ravel()[system.cells]], axis=-1)
    dK = stiffness_shape_derivative(xy)                       # (E,4,2,4,4)
    contrib = -np.einsum("ei,eacij,ej->eac", Lam[system.cells], dK, psi[system.cells])
    dJdX = np.zeros((mesh.n_nodes, 2))
    np.add.at(dJdX, system.cells.ravel(), contrib.reshape(-1, 2))
    # Dirichlet data term: g_n = U y_n
    KL = full_operator_apply(system, Lam)
    dmask = mesh.kind.ravel() == DIRICHLET
    dJdX[dmask, 1] -= U * KL[dmask]
    dJdc = centre_chain(mesh, sweeps, dJdX)
    if obj == OBJ_COPFI:
        dJdc[hi, 1] += -J / dy
        dJdc[lo, 1] += J / dy
    return J, dJdX, dJdc, psi
