"""Oracle: solutions of the reduced system.

* `solve_direct`   - the definition of the discrete solution: A u = b solved by a
                     sparse LU (scipy SuperLU, with a symmetric fill-reducing
                     ordering since A is symmetric) or, for small systems, a dense
                     Cholesky factorisation written out step by step.
* `cg_paper`       - the Conjugate Gradient of Appendix A (Algorithm), performed
                     element by element on nodal vectors with the body rows summed
                     into one residual per body and the body search direction
                     copied back onto every body node, with the paper's signs
                     (r = A x - b, apval = -A xp).
* `solve_schur`    - the body values through the Schur complement of the body
                     unknowns (psi = psi_0 + sum_k C_k phi_k); algebraically the same
                     solution as the multi-point-constraint system.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from .mesh import BODY, FREE
from .system import System, expand


def dense_cholesky_solve(A, b):
    """Cholesky A = L L^T by the textbook column loop, then two triangular solves."""
    A = np.array(A, dtype=np.float64)
    n = A.shape[0]
    L = np.zeros_like(A)
    for j in range(n):
        s = A[j, j] - L[j, :j] @ L[j, :j]
        if s <= 0:
            raise np.linalg.LinAlgError("matrix not positive definite")
        L[j, j] = np.sqrt(s)
        L[j + 1:, j] = (A[j + 1:, j] - L[j + 1:, :j] @ L[j, :j]) / L[j, j]
    y = sla.solve_triangular(L, b, lower=True)
    return sla.solve_triangular(L.T, y, lower=False)


def sparse_factor(A):
    """SuperLU factorisation of the symmetric matrix A with the minimum-degree ordering of
    A^T + A and diagonal pivots preferred (the reduced matrix is SPD, so no pivoting is
    needed for stability; the symmetric ordering keeps the fill of these 2-D grid
    matrices about half that of the default column ordering)."""
    return spla.splu(A.tocsc(), permc_spec="MMD_AT_PLUS_A", options=dict(SymmetricMode=True))


def solve_direct(system: System, dense=False):
    """Unique solution of the reduced SPD system; returns (u, nodal psi)."""
    if dense:
        u = dense_cholesky_solve(system.A.toarray(), system.b)
    elif system.A.shape[0] == 0:
        u = np.zeros(0)
    else:
        u = sparse_factor(system.A).solve(system.b)
    return u, expand(system, u)


def cg_paper(system: System, kind, body, tol=1e-12, k_max=100000, criterion="paper",
             eps=0.0, x0=None):
    """Appendix A Algorithm on nodal vectors.

    kind, body: flattened node kind / body index arrays of the mesh.
    criterion "paper": continue while r_norm = sum r^2 > tol (the algorithm's test);
    criterion "relative": continue while sqrt(r_norm) > tol * ||b||.
    Returns (psi, body values, iterations, r_norm)."""
    Ke, cells = system.Ke, system.cells
    free = kind == FREE
    nb = system.n_bodies
    body_nodes = [np.flatnonzero((kind == BODY) & (body == k)) for k in range(nb)]

    def element_apply(v):
        ve = np.einsum("eab,eb->ea", Ke, v[cells])
        out = np.zeros_like(v)
        np.add.at(out, cells.ravel(), ve.ravel())
        return out

    def collapse(v):
        return np.array([v[idx].sum() for idx in body_nodes])

    # initial x: unknowns (or the given guess), Dirichlet values in place
    x = system.g.copy()
    psik = np.zeros(nb)
    if x0 is not None:
        x[free] = x0[free]
        psik = np.array([x0[idx[0]] if idx.size else 0.0 for idx in body_nodes])
    for k, idx in enumerate(body_nodes):
        x[idx] = psik[k]
    # v_e = A_e x_e - b_e (b_e = 0: no Neumann flux), assembled into r and rb
    v = element_apply(x)
    r = np.where(free, v, 0.0)
    rb = collapse(v)
    xp = r.copy()
    xpb = rb.copy()
    for k, idx in enumerate(body_nodes):
        xp[idx] = xpb[k]
    r_norm = r[free] @ r[free] + rb @ rb
    bnorm = np.sqrt(r_norm) if x0 is None else np.sqrt(_rhs_norm2(system))
    k = 0

    def going(rn):
        if criterion == "paper":
            return rn > tol
        return np.sqrt(rn) > tol * bnorm

    while going(r_norm) and k < k_max:
        a_n = r_norm
        apval_full = -element_apply(xp)
        apval = np.where(free, apval_full, 0.0)
        apvalb = collapse(apval_full)
        alpha_d = apval[free] @ xp[free] + apvalb @ xpb
        if alpha_d + eps == 0.0:
            raise FloatingPointError("CG breakdown: p^T A p = 0")
        alpha = a_n / (alpha_d + eps)
        x[free] += alpha * xp[free]
        psik += alpha * xpb
        r[free] -= alpha * apval[free]
        rb -= alpha * apvalb
        r_norm = r[free] @ r[free] + rb @ rb
        beta = r_norm / (a_n + eps)
        xp[free] = r[free] + beta * xp[free]
        xpb = rb + beta * xpb
        for kk, idx in enumerate(body_nodes):
            xp[idx] = xpb[kk]
        k += 1
    for kk, idx in enumerate(body_nodes):
        x[idx] = psik[kk]
    return x, psik, k, r_norm


def _rhs_norm2(system: System):
    return float(system.b @ system.b)


def solve_schur(system: System, kind, body):
    """Body values by the Schur complement of the body unknowns.

    Partition the reduced system into free (F) and body (B) unknowns.  psi_0 solves
    the free rows with every C_k = 0; phi_k solves them with C_k = 1 and the others
    0 and no Dirichlet data.  Then S C = b_B - A_BF psi_0 with
    S = A_BB + A_BF Phi, Phi = -A_FF^{-1} A_FB, and psi = psi_0 + Phi C."""
    nf, nb = system.n_free, system.n_bodies
    A = system.A.tocsr()
    AFF = A[:nf, :nf].tocsc()
    AFB = A[:nf, nf:].toarray()
    ABF = A[nf:, :nf]
    ABB = A[nf:, nf:].toarray()
    lu = spla.splu(AFF)
    psi0 = lu.solve(system.b[:nf])
    Phi = -lu.solve(AFB) if nb else np.zeros((nf, 0))
    S = ABB + ABF @ Phi
    rhs = system.b[nf:] - ABF @ psi0
    C = np.linalg.solve(S, rhs) if nb else np.zeros(0)
    u = np.concatenate([psi0 + Phi @ C, C])
    return u, expand(system, u), S


def solve_kutta(system: System, mesh):
    """Solution of the reduced system with the Kutta rows of `system.kutta_rows` (a sparse
    LU of the non-symmetric matrix); returns (u, nodal psi)."""
    from .system import kutta_rows
    A, b = kutta_rows(system, mesh)
    u = spla.spsolve(A.tocsc(), b) if A.shape[0] else np.zeros(0)
    return u, expand(system, u)
