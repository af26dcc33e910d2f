"""Helpers of the GPU parity tests: oracle references (cached) and error norms."""
import functools

import numpy as np

from oracle import mesh as OM, post as OP, solve as OS, system as OSY


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@functools.lru_cache(maxsize=32)
def _oracle_cached(key):
    grid, bodies, sweeps, bc, U = key
    bodies = np.array(bodies, dtype=np.float64).reshape(-1, 3)
    m = OM.build_mesh(grid, bodies, sweeps, bc)
    s = OSY.assemble(m, U)
    u, psi = OS.solve_direct(s)
    return m, s, u, psi


def oracle_solution(case, U=1.0):
    key = (tuple(case.grid), tuple(map(tuple, np.asarray(case.bodies).tolist())), case.sweeps, tuple(case.bc), U)
    return _oracle_cached(key)


@functools.lru_cache(maxsize=32)
def _lam_min_cached(key):
    import scipy.sparse.linalg as spla
    m, s, u, psi = _oracle_cached(key)
    lu = OS.sparse_factor(s.A)
    op = spla.LinearOperator(s.A.shape, matvec=lu.solve, dtype=np.float64)
    mu = spla.eigsh(op, k=1, which="LM", tol=1e-4, return_eigenvectors=False)[0]
    return 1.0 / mu


def residual_error_bound(case, tol, U=1.0):
    """Bound on ||u - u*||_2 (reduced vector, u* the direct solution) of any iterate whose
    relative true residual is <= tol: ||A^{-1} r|| <= ||r|| / lambda_min(A) with
    ||r|| <= tol ||b||.  lambda_min from a Lanczos run on the oracle's factorised A."""
    key = (tuple(case.grid), tuple(map(tuple, np.asarray(case.bodies).tolist())), case.sweeps, tuple(case.bc), U)
    m, s, u, psi = _oracle_cached(key)
    return tol * float(np.linalg.norm(s.b)) / _lam_min_cached(key)


def reduced_error(case, psi_nodal, U=1.0):
    """||u - u*||_2 of a nodal psi against the oracle's direct solution (reduced vector)."""
    m, s, u, psi = oracle_solution(case, U)
    ug = np.empty(s.n_dof)
    k = s.dof >= 0
    ug[s.dof[k]] = np.asarray(psi_nodal)[k]
    return float(np.linalg.norm(ug - u))
