"""Pins of the oracle's body-conforming mesh (section "Body-Conforming Grid Generation").

The vectorised oracle is compared bit for bit with a brute-force pure-Python loop
restatement of the same rules on tiny grids, and against geometric facts:
no bodies -> the background grid, boundary nodes on their circles, mirror
symmetry of a centred cylinder, and convergence of the sweeps to a discrete
harmonic displacement."""
import numpy as np
import pytest

from oracle import mesh as M
from paper_2512_12232_gb300 import workloads as W


def brute_force_mesh(grid, bodies, sweeps, bc):
    x0, x1, y0, y1, nx, ny = grid
    hx = (x1 - x0) / nx
    hy = (y1 - y0) / ny
    X = [[x0 + i * hx for i in range(nx + 1)] for j in range(ny + 1)]
    Y = [[y0 + j * hy for i in range(nx + 1)] for j in range(ny + 1)]
    inside = [[-1] * (nx + 1) for _ in range(ny + 1)]
    for j in range(ny + 1):
        for i in range(nx + 1):
            for k, (cx, cy, r) in enumerate(bodies):
                dx = X[j][i] - cx
                dy = Y[j][i] - cy
                if dx * dx + dy * dy <= r * r:
                    inside[j][i] = k
    act = [[any(inside[j + b][i + a] < 0 for a in (0, 1) for b in (0, 1)) for i in range(nx)]
           for j in range(ny)]
    kind = [[0] * (nx + 1) for _ in range(ny + 1)]
    for j in range(ny + 1):
        for i in range(nx + 1):
            if inside[j][i] >= 0:
                touch = any(act[jj][ii] for jj in (j - 1, j) for ii in (i - 1, i)
                            if 0 <= jj < ny and 0 <= ii < nx)
                kind[j][i] = M.BODY if touch else M.INACTIVE
            else:
                ring = ((i == 0 and bc[0] == 0) or (i == nx and bc[1] == 0)
                        or (j == 0 and bc[2] == 0) or (j == ny and bc[3] == 0))
                kind[j][i] = M.DIRICHLET if ring else M.FREE
    dX = [[0.0] * (nx + 1) for _ in range(ny + 1)]
    dY = [[0.0] * (nx + 1) for _ in range(ny + 1)]
    for j in range(ny + 1):
        for i in range(nx + 1):
            if kind[j][i] == M.BODY:
                cx, cy, r = bodies[inside[j][i]]
                ex, ey = X[j][i] - cx, Y[j][i] - cy
                rho = np.sqrt(ex * ex + ey * ey)
                dX[j][i] = (cx + (r * ex) / rho) - X[j][i]
                dY[j][i] = (cy + (r * ey) / rho) - Y[j][i]
    for _ in range(sweeps):
        nX = [row[:] for row in dX]
        nY = [row[:] for row in dY]
        for j in range(1, ny):
            for i in range(1, nx):
                if inside[j][i] < 0:
                    nX[j][i] = (((dX[j][i - 1] + dX[j][i + 1]) + dX[j - 1][i]) + dX[j + 1][i]) / 4.0
                    nY[j][i] = (((dY[j][i - 1] + dY[j][i + 1]) + dY[j - 1][i]) + dY[j + 1][i]) / 4.0
        dX, dY = nX, nY
    xf = np.array([[X[j][i] + dX[j][i] for i in range(nx + 1)] for j in range(ny + 1)])
    yf = np.array([[Y[j][i] + dY[j][i] for i in range(nx + 1)] for j in range(ny + 1)])
    return xf, yf, np.array(kind, dtype=np.int8), np.array(act)


@pytest.mark.parametrize("case", [
    ((-3.0, 3.0, -2.0, 2.0, 24, 16), [[0.1, 0.05, 0.9]], 7, (0, 0, 0, 0)),
    ((-4.0, 4.0, -2.0, 2.0, 29, 17), [[-1.6, 0.2, 0.7], [1.3, -0.4, 0.55]], 11, (1, 1, 0, 0)),
    ((0.0, 1.0, 0.0, 0.5, 40, 21), [[0.3, 0.25, 0.1], [0.55, 0.14, 0.05], [0.55, 0.36, 0.05]], 5, (1, 0, 0, 1)),
])
def test_vectorised_mesh_equals_brute_force_bitwise(case):
    grid, bodies, S, bc = case
    m = M.build_mesh(grid, np.array(bodies), S, bc)
    xf, yf, kind, act = brute_force_mesh(grid, bodies, S, bc)
    assert np.array_equal(m.kind, kind)
    assert np.array_equal(m.active, act)
    assert np.array_equal(m.x.view(np.uint64), xf.view(np.uint64))
    assert np.array_equal(m.y.view(np.uint64), yf.view(np.uint64))


def test_no_bodies_gives_background_grid_exactly():
    m = M.build_mesh((-2.0, 3.0, -1.0, 1.5, 40, 20), np.zeros((0, 3)), 30)
    assert np.array_equal(m.x, m.xg) and np.array_equal(m.y, m.yg)
    assert np.all(m.kind[1:-1, 1:-1] == M.FREE) and np.all(m.active)
    assert np.all(m.kind[0, :] == M.DIRICHLET) and np.all(m.kind[:, 0] == M.DIRICHLET)


def test_boundary_nodes_lie_on_their_circles():
    c = W.five_cylinder_case(0.25, 256, 128, 30)
    m = M.build_mesh(c.grid, c.bodies, c.sweeps, c.bc)
    for k, (cx, cy, r) in enumerate(c.bodies):
        sel = (m.kind == M.BODY) & (m.body == k)
        assert sel.sum() > 8
        rr = np.hypot(m.x[sel] - cx, m.y[sel] - cy)
        np.testing.assert_allclose(rr, r, rtol=0, atol=4e-15 * 20)


def test_centred_cylinder_mesh_is_mirror_symmetric():
    c = W.single_cylinder()
    m = M.build_mesh(c.grid, c.bodies, c.sweeps, c.bc)
    assert np.array_equal(m.kind, m.kind[:, ::-1]) and np.array_equal(m.kind, m.kind[::-1, :])
    np.testing.assert_allclose(m.x, -m.x[:, ::-1], rtol=0, atol=4e-15)
    np.testing.assert_allclose(m.y, -m.y[::-1, :], rtol=0, atol=4e-15)
    assert np.array_equal(m.y, m.y[:, ::-1])


def test_many_sweeps_converge_to_discrete_harmonic_displacement():
    grid = (-2.0, 2.0, -2.0, 2.0, 24, 24)
    m = M.build_mesh(grid, np.array([[0.13, -0.07, 0.8]]), 4000)
    d = m.x - m.xg
    mask = M.smoothing_mask(m.kind, m.body)
    lap = np.zeros_like(d)
    lap[1:-1, 1:-1] = d[1:-1, :-2] + d[1:-1, 2:] + d[:-2, 1:-1] + d[2:, 1:-1] - 4 * d[1:-1, 1:-1]
    assert np.abs(lap[mask]).max() < 1e-12
    assert np.abs(d).max() > 1e-3        # the displacement did propagate


def test_node_classification_counts_are_consistent():
    c = W.five_cylinder_case(0.1, 512, 256, 10)
    m = M.build_mesh(c.grid, c.bodies, c.sweeps, c.bc)
    inside = m.body >= 0
    assert np.all((m.kind == M.BODY) | (m.kind == M.INACTIVE) | ~inside)
    assert np.all((m.kind == M.FREE) | (m.kind == M.DIRICHLET) | inside)
    # every active cell has at least one outside corner, every other cell none
    outside = ~inside
    any_out = outside[:-1, :-1] | outside[:-1, 1:] | outside[1:, :-1] | outside[1:, 1:]
    assert np.array_equal(any_out, m.active)


@pytest.mark.parametrize("bodies,msg", [
    ([[0.0, 0.0, 1.0], [1.5, 0.0, 0.6]], "overlap"),
    ([[2.8, 0.0, 1.0]], "2h"),
    ([[0.0, 0.0, -1.0]], "radius"),
])
def test_invalid_body_tables_are_rejected(bodies, msg):
    with pytest.raises(M.MeshError, match=msg):
        M.build_mesh((-4.0, 4.0, -3.0, 3.0, 32, 24), np.array(bodies), 5)
