"""GPU parity of polygonal bodies and the Kutta condition (pf_batch_build_shapes; paper,
sections "Body-Conforming Grid Generation" and "Boundary Conditions") against the oracle
(oracle/shapes.py, oracle/mesh.py, oracle.solve.solve_kutta):

* meshes bit for bit: node kinds, body membership and FP64 coordinates, the wake node
  included (its position on the trailing-edge bisector is part of the coordinates);
* a polygon without a Kutta condition solves by the MPC form like a circle (FP64 to 1e-10,
  mixed precision to 1e-6 in relative L2);
* with a Kutta condition the Schur form with the wake rows reaches the oracle's sparse LU
  solution of the non-symmetric system, also with the multigrid preconditioner and in a
  batch that mixes circles, polygons with and without a Kutta condition and grid sizes;
* the surface velocity of a polygon and the refusals of the entry points that do not take
  such handles."""
import functools

import numpy as np
import pytest

from oracle import mesh as OM, post as OP, solve as OS, system as OSY
from paper_2512_12232_gb300 import workloads as W
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu


def _ellipse():
    ell = W.ellipse_body(0.8, 0.4, 180, cx=0.3, cy=-0.1, angle=-0.3)
    return (-4.0, 4.0, -2.0, 2.0, 96, 48), np.zeros((0, 3)), [ell], 24


def _airfoil():
    c, polys = W.airfoil_case(128, 6.0)
    return c.grid, c.bodies, polys, c.sweeps


def _mixed():
    af = W.joukowski_airfoil(0.5, 0.08, 300, alpha=np.radians(4.0), shift=(0.6, -0.3))
    quad = W.PolygonBody(np.array([[2.4, 0.4], [3.2, 0.5], [3.1, 1.3], [2.3, 1.2]]), ref=(2.75, 0.85))
    return (-4.0, 4.0, -2.0, 2.0, 128, 64), np.array([[-2.5, 0.5, 0.5]]), [af, quad], 32


CASES = {"ellipse": _ellipse, "airfoil": _airfoil, "mixed": _mixed}


@functools.lru_cache(maxsize=8)
def reference(name, U=1.0):
    grid, circles, polys, sweeps = CASES[name]()
    m = OM.build_mesh(grid, circles, sweeps, polygons=polys)
    s = OSY.assemble(m, U)
    if any(p.kutta >= 0 for p in polys):
        u, psi = OS.solve_kutta(s, m)
    else:
        u, psi = OS.solve_direct(s)
    return m, s, u, psi


@pytest.fixture(scope="module")
def api():
    from paper_2512_12232_gb300 import api
    return api


def _build(api, name):
    grid, circles, polys, sweeps = CASES[name]()
    return api.mesh_build(grid, circles, sweeps, polygons=polys)


@pytest.mark.parametrize("name", list(CASES))
def test_polygon_mesh_is_bit_exact(api, name):
    m, *_ = reference(name)
    with _build(api, name) as g:
        xy = g.coords().cpu().numpy()
        kind, body = (t.cpu().numpy() for t in g.tags())
        st = g.stats()
    assert np.array_equal(kind, m.kind.ravel())
    assert np.array_equal(body[kind == OM.BODY], m.body.ravel()[m.kind.ravel() == OM.BODY])
    assert np.array_equal(xy[:, 0], m.x.ravel()) and np.array_equal(xy[:, 1], m.y.ravel())
    assert st["n_bodies"] == m.bodies.shape[0] and st["min_detJ"] > 0
    for nw in m.wake_node:
        if nw >= 0:
            assert kind[nw] == OM.FREE


@pytest.mark.parametrize("prec,tol,bound", [("fp64", 1e-13, 1e-10), ("mixed", 1e-12, 1e-6)])
def test_polygon_without_kutta_solves_like_a_circle(api, prec, tol, bound):
    m, s, u, psi_ref = reference("ellipse")
    p = api.PF_FP64 if prec == "fp64" else api.PF_MIXED
    with _build(api, "ellipse") as g:
        res = api.psi_solve(g, U=1.0, tol=tol, precision=p)
    assert res.status == 0 and res.info[0]["rel_true_residual"] <= tol
    assert rel_l2(res.psi.cpu().numpy(), psi_ref) <= bound
    np.testing.assert_allclose(res.body_psi, u[s.n_free:], rtol=0, atol=1e-7)


@pytest.mark.parametrize("name", ["airfoil", "mixed"])
@pytest.mark.parametrize("prec,tol,bound,precond", [("fp64", 1e-13, 1e-9, "none"), ("mixed", 1e-12, 1e-6, "none"),
                                                     ("mixed", 1e-12, 1e-6, "mg")])
def test_kutta_solve_matches_oracle(api, name, prec, tol, bound, precond):
    m, s, u, psi_ref = reference(name)
    p = api.PF_FP64 if prec == "fp64" else api.PF_MIXED
    with _build(api, name) as g:
        res = api.psi_solve(g, U=1.0, tol=tol, precision=p, preconditioner=precond)
    assert res.status == 0 and res.info[0]["status"] == 0 and res.info[0]["rel_true_residual"] <= tol
    psi = res.psi.cpu().numpy()
    assert rel_l2(psi, psi_ref) <= bound, rel_l2(psi, psi_ref)
    C_ref = u[s.n_free:]
    np.testing.assert_allclose(res.body_psi, C_ref, rtol=0, atol=10 * bound * np.abs(C_ref).max())
    # the wake node carries its body's value
    n_circ = len(CASES[name]()[1])
    for q, nw in enumerate(m.wake_node):
        if nw >= 0:
            assert abs(psi[nw] - res.body_psi[n_circ + q]) <= 1e-9 * max(1.0, abs(res.body_psi[n_circ + q]))


def test_kutta_circulation_is_not_zero(api):
    """With the Kutta condition the airfoil at 6 degrees carries circulation: its body value
    differs from the zero-circulation MPC solution of the same mesh given as a polygon
    without a Kutta vertex (the same mesh apart from the wake node)."""
    grid, circles, polys, sweeps = CASES["airfoil"]()
    plain = W.PolygonBody(polys[0].vertices, ref=polys[0].ref, kutta=-1)
    with _build(api, "airfoil") as g:
        Ck = api.psi_solve(g, U=1.0, tol=1e-12).body_psi[0]
    with api.mesh_build(grid, circles, sweeps, polygons=[plain]) as g:
        C0 = api.psi_solve(g, U=1.0, tol=1e-12).body_psi[0]
    assert abs(Ck - C0) > 0.05


def test_uneven_batch_of_shapes(api):
    """Two variants of different grids, one with a circle and two polygons, one with the
    airfoil alone: each variant's solution matches its own oracle solve."""
    names = ["mixed", "airfoil"]
    specs = [CASES[n]() for n in names]
    cases = [W.Case(*sp[0][:4], sp[0][4], sp[0][5], sp[1], 32) for sp in specs]
    with api.batch_build(cases, polygons=[sp[2] for sp in specs]) as g:
        res = api.psi_solve(g, U=1.0, tol=1e-12, precision=api.PF_MIXED)
        offs = g.node_offsets
        psi = res.psi.cpu().numpy()
        xy = [g.coords(v).cpu().numpy() for v in range(2)]
    boffs = [0, 3, 4]
    for v, n in enumerate(names):
        m, s, u, psi_ref = reference(n)
        assert np.array_equal(xy[v][:, 0], m.x.ravel()) and np.array_equal(xy[v][:, 1], m.y.ravel())
        assert res.info[v]["status"] == 0
        assert rel_l2(psi[offs[v]:offs[v + 1]], psi_ref) <= 1e-6
        np.testing.assert_allclose(res.body_psi[boffs[v]:boffs[v + 1]], u[s.n_free:], rtol=0, atol=1e-6)


def test_polygon_surface_velocity(api):
    m, s, u, psi_ref = reference("ellipse")
    th_ref, ut_ref = OP.surface_velocity(m, psi_ref, u[s.n_free:], 0)
    with _build(api, "ellipse") as g:
        api.psi_solve(g, U=1.0, tol=1e-13, precision=api.PF_FP64)
        th, ut = api.surface_velocity(g, 0, 0)
    order = np.argsort(th_ref, kind="stable")
    np.testing.assert_allclose(np.sort(th), th_ref[order], rtol=0, atol=1e-12)
    np.testing.assert_allclose(np.asarray(ut)[np.argsort(th, kind="stable")], ut_ref[order], rtol=0,
                               atol=1e-8 * np.abs(ut_ref).max())


def test_shape_handles_refuse_what_they_do_not_support(api):
    with _build(api, "airfoil") as g:
        with pytest.raises(Exception, match="PF_EINVAL"):
            api.phi_solve(g, U=1.0)
        api.psi_solve(g, U=1.0, tol=1e-10)
        with pytest.raises(Exception, match="PF_EINVAL"):
            api.grad(g)
    with _build(api, "ellipse") as g:
        api.psi_solve(g, U=1.0, tol=1e-10)
        with pytest.raises(Exception, match="PF_EINVAL"):
            api.grad(g)


def test_folded_polygon_mesh_is_reported_like_the_oracle(api):
    """A small triangle with acute corners folds cells next to its vertices on this grid:
    the oracle's assembly refuses the mesh and the build reports PF_EMESH_INVALID."""
    grid = (-4.0, 4.0, -2.0, 2.0, 128, 64)
    tri = W.PolygonBody(np.array([[2.5, 0.7], [3.2, 0.8], [2.8, 1.4]]), ref=(2.83, 0.96))
    m = OM.build_mesh(grid, np.zeros((0, 3)), 32, polygons=[tri])
    with pytest.raises(ValueError, match="det J"):
        OSY.assemble(m, 1.0)
    with api.mesh_build(grid, np.zeros((0, 3)), 32, polygons=[tri]) as g:
        assert not g.valid
        xy = g.coords().cpu().numpy()
    assert np.array_equal(xy[:, 0], m.x.ravel()) and np.array_equal(xy[:, 1], m.y.ravel())
