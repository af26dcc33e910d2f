"""Pins of the oracle's adjoint shape gradient against central finite differences.

The grid is chosen so that no node lies exactly on a circle; the tests assert the
topology (node kinds) is unchanged at +-step."""
import copy

import numpy as np
import pytest

from oracle import grad as G, mesh as M, solve as SV, system as S
from paper_2512_12232_gb300 import workloads as W

STEP = 1e-6


@pytest.fixture(scope="module")
def case():
    c = W.five_cylinder_case(0.83, 150, 76, 20)
    m = M.build_mesh(c.grid, c.bodies, c.sweeps, c.bc)
    return c, m


def J_of_bodies(c, m, bodies, obj):
    mm = M.build_mesh(c.grid, bodies, c.sweeps, c.bc)
    assert np.array_equal(mm.kind, m.kind) and np.array_equal(mm.body, m.body)
    s = S.assemble(mm, 1.0)
    u, _ = SV.solve_direct(s)
    return G.objective(u[s.n_free:], bodies, 3, 4, 1.0, obj)


def J_of_coords(m, x, y, obj):
    mm = copy.copy(m)
    mm.x, mm.y = x, y
    s = S.assemble(mm, 1.0)
    u, _ = SV.solve_direct(s)
    return G.objective(u[s.n_free:], m.bodies, 3, 4, 1.0, obj)


@pytest.mark.parametrize("obj", [G.OBJ_COPFI, G.OBJ_GAP_FLOW])
def test_centre_gradient_matches_central_differences(case, obj):
    c, m = case
    J, dX, dc, _ = G.gradient(m, c.sweeps, 1.0, 3, 4, obj)
    scale = np.abs(dc).max()
    for k in range(5):
        for a in range(2):
            bp = c.bodies.copy(); bp[k, a] += STEP
            bm = c.bodies.copy(); bm[k, a] -= STEP
            fd = (J_of_bodies(c, m, bp, obj) - J_of_bodies(c, m, bm, obj)) / (2 * STEP)
            if abs(fd) >= 1e-3 * scale:
                assert abs(dc[k, a] - fd) <= 1e-5 * abs(fd), (k, a, dc[k, a], fd)
            else:
                assert abs(dc[k, a] - fd) <= 1e-7 * scale + 1e-8


@pytest.mark.parametrize("obj", [G.OBJ_COPFI, G.OBJ_GAP_FLOW])
def test_node_coordinate_gradient_along_random_directions(case, obj):
    c, m = case
    J, dX, dc, _ = G.gradient(m, c.sweeps, 1.0, 3, 4, obj)
    rng = np.random.default_rng(5)
    live = (m.kind != M.INACTIVE).ravel()
    for t in range(4):
        v = rng.standard_normal((m.n_nodes, 2)) * live[:, None]
        v /= np.linalg.norm(v)
        xp = m.x + STEP * v[:, 0].reshape(m.x.shape)
        yp = m.y + STEP * v[:, 1].reshape(m.y.shape)
        xm = m.x - STEP * v[:, 0].reshape(m.x.shape)
        ym = m.y - STEP * v[:, 1].reshape(m.y.shape)
        fd = (J_of_coords(m, xp, yp, obj) - J_of_coords(m, xm, ym, obj)) / (2 * STEP)
        ad = float(np.sum(dX * v))
        assert abs(ad - fd) <= 1e-5 * max(abs(fd), 1e-3 * np.abs(dX).max()), (ad, fd)


def test_individual_node_coordinates_near_bodies(case):
    c, m = case
    J, dX, dc, _ = G.gradient(m, c.sweeps, 1.0, 3, 4, G.OBJ_GAP_FLOW)
    near = np.flatnonzero(((m.kind == M.FREE) & (np.abs(m.x - m.xg) > 0)).ravel())
    rng = np.random.default_rng(2)
    for n in rng.choice(near, 6, replace=False):
        for a in range(2):
            arrs = [m.x.copy(), m.y.copy()]
            arrs[a].ravel()[n] += STEP
            jp = J_of_coords(m, *arrs, G.OBJ_GAP_FLOW)
            arrs[a].ravel()[n] -= 2 * STEP
            jm = J_of_coords(m, *arrs, G.OBJ_GAP_FLOW)
            fd = (jp - jm) / (2 * STEP)
            assert abs(dX[n, a] - fd) <= 1e-5 * abs(fd) + 1e-7 * np.abs(dX).max()
