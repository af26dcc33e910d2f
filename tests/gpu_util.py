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
