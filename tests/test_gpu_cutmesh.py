"""GPU parity of the mixed-cell mesh (pf_batch_build_cut: node splitting, triangle and
pentagon cells, boundary-point redistribution) against `oracle.cutmesh`: the mesh bit for
bit (kinds, coordinates, surface points), the operator against the oracle's cut-cell
element sums, solves against the oracle's sparse LU, the outputs, and the refusals."""
import numpy as np
import pytest
import torch

from oracle import cutmesh as CM, mesh as OM, solve as OSV, system as OSY
from paper_2512_12232_gb300 import workloads as W
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu

SINGLE = W.Case(0.0, 8.0, 0.0, 8.0, 8, 8, np.array([[4.2, 4.3, 0.45]]), 3)        # one node split four ways
LSHAPE = W.Case(0.0, 9.0, 0.0, 9.0, 9, 9, np.array([[4.3, 4.3, 0.85]]), 2)        # triangle, quad, pentagon cells
CASES = [
    (SINGLE, 0.0),
    (LSHAPE, 0.3),
    (W.Case(-3.0, 3.0, -2.0, 2.0, 37, 23, np.array([[0.1, 0.05, 0.9]]), 9, bc=(1, 1, 0, 0)), 0.25),
    (W.five_cylinder_case(0.5, 160, 80, 30), 0.0),
    (W.five_cylinder_case(0.25, 256, 128, 40), 0.4),
    (W.five_cylinder_case(0.1, 333, 170, 60), 0.25),
]
IDS = ["single", "lshape", "one_body_natural", "five_160", "five_256_spaced", "five_333_spaced"]


@pytest.fixture(scope="module")
def api():
    from paper_2512_12232_gb300 import api
    return api


def oracle_mesh(case, sigma):
    return CM.build_cut_mesh(case.grid, case.bodies, case.sweeps, case.bc, sigma=sigma)


def bits(a):
    return np.ascontiguousarray(a, dtype=np.float64).view(np.uint64)


@pytest.mark.parametrize("case,sigma", CASES, ids=IDS)
def test_cut_mesh_is_bit_exact(api, case, sigma):
    m = oracle_mesh(case, sigma)
    with api.cut_mesh_build(case.grid, case.bodies, case.sweeps, case.bc, sigma) as g:
        xy = g.coords().cpu().numpy()
        kind, body = (t.cpu().numpy() for t in g.tags())
        pts = g.cut_points().cpu().numpy()
        st = g.stats()
    assert np.array_equal(kind, m.kind.ravel())
    assert np.array_equal(body, m.body.ravel())
    assert np.array_equal(bits(xy[:, 0]), bits(m.x.ravel()))
    assert np.array_equal(bits(xy[:, 1]), bits(m.y.ravel()))
    ref = m.cut_points.reshape(4, -1, 2)
    nan_ref, nan_gpu = np.isnan(ref), np.isnan(pts)
    assert np.array_equal(nan_ref, nan_gpu)
    assert np.array_equal(bits(pts[~nan_gpu]), bits(ref[~nan_ref]))
    s = OSY.assemble(m, 1.0)
    assert st["min_detJ"] == pytest.approx(s.detmin.min(), rel=1e-12)
    assert st["n_active_cells"] == int(m.active.sum())
    chords = 0
    for (j, i) in CM.cut_cells(m):
        (A, _, _), (B, _, _) = CM.chord(m, j, i)
        chords += int(A[0] != B[0] or A[1] != B[1])
    assert st["n_boundary_edges"] == chords


def test_batched_cut_meshes_equal_single_ones(api):
    cases = W.parametric_sweep(4, seed=5, nx_choices=(192, 256, 320))
    with api.batch_build(cases, cut_spacing=0.3) as g:
        for v, c in enumerate(cases):
            m = oracle_mesh(c, 0.3)
            xy = g.coords(v).cpu().numpy()
            pts = g.cut_points(v).cpu().numpy()
            assert np.array_equal(g.tags(v)[0].cpu().numpy(), m.kind.ravel())
            assert np.array_equal(bits(xy[:, 0]), bits(m.x.ravel()))
            assert np.array_equal(bits(xy[:, 1]), bits(m.y.ravel()))
            ref = m.cut_points.reshape(4, -1, 2)
            assert np.array_equal(np.isnan(pts), np.isnan(ref))
            assert np.array_equal(bits(pts[~np.isnan(pts)]), bits(ref[~np.isnan(ref)]))


@pytest.mark.parametrize("case,sigma", CASES[1:5], ids=IDS[1:5])
def test_cut_operator_matches_oracle(api, case, sigma):
    m = oracle_mesh(case, sigma)
    s = OSY.assemble(m, 1.0)
    p = W.random_vector(m.n_nodes, seed=17)
    p[m.kind.ravel() == OM.INACTIVE] = 0.0
    ref = OSY.full_operator_apply(s, p)
    kind = m.kind.ravel()
    rows = (kind == OM.FREE) | (kind == OM.BODY)
    ref = np.where(rows, ref, 0.0)
    body_ref = np.array([ref[(kind == OM.BODY) & (m.body.ravel() == k)].sum() for k in range(len(case.bodies))])
    with api.cut_mesh_build(case.grid, case.bodies, case.sweeps, case.bc, sigma) as g:
        y64, b64 = api.apply(g, torch.from_numpy(p), api.PF_FP64)
        y32, b32 = api.apply(g, torch.from_numpy(p), api.PF_MIXED)
    scale = np.abs(ref).max()
    assert np.abs(y64.cpu().numpy() - ref).max() <= 1e-12 * scale
    assert rel_l2(y32.cpu().numpy(), ref) <= 2e-6
    np.testing.assert_allclose(b64, body_ref, rtol=0, atol=1e-11 * scale)
    np.testing.assert_allclose(b32, body_ref, rtol=0, atol=1e-4 * scale)


@pytest.mark.parametrize("case,sigma", [CASES[2], CASES[4]], ids=[IDS[2], IDS[4]])
@pytest.mark.parametrize("mode", ["fp64", "mixed", "mg", "schur", "schur64"])
def test_cut_solve_matches_oracle(api, case, sigma, mode):
    m = oracle_mesh(case, sigma)
    s = OSY.assemble(m, 1.0)
    u, psi_ref = OSV.solve_direct(s)
    C_ref = u[s.n_free:]
    kw = {"fp64": dict(precision=api.PF_FP64, tol=1e-12),
          "mixed": dict(precision=api.PF_MIXED, tol=1e-11),
          "mg": dict(precision=api.PF_MIXED, tol=1e-11, preconditioner="mg"),
          "schur": dict(precision=api.PF_MIXED, tol=1e-11, method="schur"),
          "schur64": dict(precision=api.PF_FP64, tol=1e-12, method="schur")}[mode]
    with api.cut_mesh_build(case.grid, case.bodies, case.sweeps, case.bc, sigma) as g:
        res = api.psi_solve(g, U=1.0, **kw)
        psi = res.psi.cpu().numpy()
    assert res.status == 0
    live = m.kind.ravel() != OM.INACTIVE
    assert rel_l2(psi[live], psi_ref[live]) <= (1e-9 if mode in ("fp64", "schur64") else 1e-8)
    np.testing.assert_allclose(res.body_psi, C_ref, rtol=0, atol=1e-8 * max(1.0, np.abs(psi_ref).max()))


def test_cut_outputs_match_oracle(api):
    case, sigma = CASES[4]
    m = oracle_mesh(case, sigma)
    s = OSY.assemble(m, 1.0)
    u, psi_ref = OSV.solve_direct(s)
    C_ref = u[s.n_free:]
    with api.cut_mesh_build(case.grid, case.bodies, case.sweeps, case.bc, sigma) as g:
        api.psi_solve(g, U=1.0, precision=api.PF_FP64, tol=1e-13)
        uv = api.velocity_field(g, 0)
        sv = [api.surface_velocity(g, 0, k) for k in range(len(case.bodies))]
        cp = api.copfi(g, 0, 3, 4, 1.0)
    u_ref, v_ref = CM.velocity_field(m, psi_ref)
    act = m.active.ravel()
    u_gpu = uv[0].cpu().numpy().ravel()[act]
    v_gpu = uv[1].cpu().numpy().ravel()[act]
    sc = np.abs(u_ref).max()
    assert np.abs(u_gpu - u_ref).max() <= 1e-9 * sc
    assert np.abs(v_gpu - v_ref).max() <= 1e-9 * sc
    for k in range(len(case.bodies)):
        th_ref, ut_ref = CM.surface_velocity(m, psi_ref, C_ref, k)
        th, ut = sv[k]
        assert len(th) == len(th_ref) > 10
        np.testing.assert_allclose(th, th_ref, rtol=0, atol=1e-9)
        np.testing.assert_allclose(ut, ut_ref, rtol=0, atol=1e-8 * np.abs(ut_ref).max())
    q_ref = C_ref[4] - C_ref[3]
    assert abs(cp[1] - q_ref) <= 1e-10


def test_cut_mesh_refusals(api):
    case, sigma = CASES[3]
    with api.cut_mesh_build(case.grid, case.bodies, case.sweeps, case.bc, sigma) as g:
        api.psi_solve(g, U=1.0, precision=api.PF_FP64, tol=1e-10)
        with pytest.raises(RuntimeError, match="Q4"):
            api.grad(g, 0, 3, 4, 1.0, 1e-10)
        with pytest.raises(RuntimeError, match="split"):
            api.phi_solve(g, U=1.0)
        with pytest.raises(RuntimeError, match="surface points"):
            g.set_coords(g.coords())
    with api.mesh_build(case.grid, case.bodies, case.sweeps, case.bc) as g:
        with pytest.raises(RuntimeError, match="not a mixed-cell mesh"):
            g.cut_points()
    # a cell with inside corners of two bodies side by side, and one with two diagonal ones
    with pytest.raises(RuntimeError, match="two bodies"):
        api.cut_mesh_build((0.0, 12.0, 0.0, 12.0, 12, 12), np.array([[5.0, 5.0, 0.3], [6.0, 5.0, 0.3]]), 0)
    with pytest.raises(RuntimeError, match="two diagonal"):
        api.cut_mesh_build((0.0, 12.0, 0.0, 12.0, 12, 12), np.array([[5.0, 5.0, 0.3], [6.0, 6.0, 0.3]]), 0)
    with pytest.raises(RuntimeError, match="minimum spacing"):
        api.cut_mesh_build(case.grid, case.bodies, case.sweeps, case.bc, 1.5)


def test_full_size_cut_mesh_and_mixed_solve(api):
    """The five-cylinder layout at 1024 x 512 with S = 200: the mesh bit for bit, and a mixed
    solve to 1e-8 whose residual, recomputed with the oracle's assembled system, is below
    the tolerance."""
    case = W.five_cylinder_case(0.25, 1024, 512, 200)
    m = oracle_mesh(case, 0.25)
    with api.cut_mesh_build(case.grid, case.bodies, case.sweeps, case.bc, 0.25) as g:
        xy = g.coords().cpu().numpy()
        pts = g.cut_points().cpu().numpy()
        res = api.psi_solve(g, U=1.0, precision=api.PF_MIXED, tol=1e-8)
        psi = res.psi.cpu().numpy()
    assert np.array_equal(bits(xy[:, 0]), bits(m.x.ravel()))
    assert np.array_equal(bits(xy[:, 1]), bits(m.y.ravel()))
    ref = m.cut_points.reshape(4, -1, 2)
    assert np.array_equal(bits(pts[~np.isnan(pts)]), bits(ref[~np.isnan(ref)]))
    assert res.status == 0
    # the oracle's residual of the GPU solution (its own assembled system)
    s = OSY.assemble(m, 1.0)
    uvec = np.zeros(s.n_dof)
    free = s.dof >= 0
    uvec[s.dof[free]] = psi[free]
    uvec[s.n_free:] = res.body_psi
    r = s.b - s.A @ uvec
    assert np.linalg.norm(r) <= 2e-8 * np.linalg.norm(s.b)


# ---------------------------------------------------------------- polygon bodies
def polygon_case(kind, nx):
    if kind == "ellipse":
        body = W.ellipse_body(0.8, 0.4, 720, angle=-np.radians(10.0))
        return (-4.0, 4.0, -2.0, 2.0, nx, nx // 2), body
    if kind == "airfoil":
        body = W.joukowski_airfoil(0.5, 0.08, 400, alpha=np.radians(6.0))
        return (-3.0, 3.0, -1.5, 1.5, nx, nx // 2), body
    sq = W.PolygonBody([(2.5, 2.5), (5.5, 2.5), (5.5, 5.5), (2.5, 5.5)], ref=(4.0, 4.0))
    return (0.0, 10.0, 0.0, 10.0, 10, 10), sq


@pytest.mark.parametrize("kind,nx,sweeps,sigma", [("square", 10, 2, 0.3), ("ellipse", 192, 48, 0.25),
                                                  ("airfoil", 256, 64, 0.25), ("airfoil", 200, 30, 0.0)])
def test_polygon_cut_mesh_is_bit_exact(api, kind, nx, sweeps, sigma):
    grid, body = polygon_case(kind, nx)
    m = CM.build_cut_mesh(grid, np.zeros((0, 3)), sweeps, polygons=[body], sigma=sigma)
    with api.cut_mesh_build(grid, np.zeros((0, 3)), sweeps, (0, 0, 0, 0), sigma, polygons=[body]) as g:
        xy = g.coords().cpu().numpy()
        kind_g, body_g = (t.cpu().numpy() for t in g.tags())
        pts = g.cut_points().cpu().numpy()
        st = g.stats()
    assert np.array_equal(kind_g, m.kind.ravel()) and np.array_equal(body_g, m.body.ravel())
    assert np.array_equal(bits(xy[:, 0]), bits(m.x.ravel()))
    assert np.array_equal(bits(xy[:, 1]), bits(m.y.ravel()))
    ref = m.cut_points.reshape(4, -1, 2)
    assert np.array_equal(np.isnan(pts), np.isnan(ref))
    assert np.array_equal(bits(pts[~np.isnan(pts)]), bits(ref[~np.isnan(ref)]))
    assert st["min_detJ"] == pytest.approx(OSY.assemble(m, 1.0).detmin.min(), rel=1e-12)


def test_mixed_circle_and_polygon_cut_batch(api):
    """Circles and a polygon in one variant, a second variant with an airfoil: each variant
    as the oracle builds it."""
    c = W.five_cylinder_case(0.5, 320, 160, 30)
    ell = W.ellipse_body(0.3, 0.15, 240, cx=-6.0, cy=3.0, angle=0.3)
    grid2, af = polygon_case("airfoil", 192)
    with api.Mesh([c.grid, grid2], [c.bodies, np.zeros((0, 3))], 30, (0, 0, 0, 0), [[ell], [af]], 0.25) as g:
        for v, (grid, circ, polys) in enumerate([(c.grid, c.bodies, [ell]), (grid2, np.zeros((0, 3)), [af])]):
            m = CM.build_cut_mesh(grid, circ, 30, polygons=polys, sigma=0.25)
            xy = g.coords(v).cpu().numpy()
            pts = g.cut_points(v).cpu().numpy()
            assert np.array_equal(g.tags(v)[0].cpu().numpy(), m.kind.ravel())
            assert np.array_equal(bits(xy[:, 0]), bits(m.x.ravel()))
            assert np.array_equal(bits(xy[:, 1]), bits(m.y.ravel()))
            ref = m.cut_points.reshape(4, -1, 2)
            assert np.array_equal(bits(pts[~np.isnan(pts)]), bits(ref[~np.isnan(ref)]))


@pytest.mark.parametrize("mode", ["fp64", "mixed", "mg"])
def test_polygon_cut_solves_match_oracle(api, mode):
    """The ellipse (MPC form) and the Kutta airfoil (Schur form with the wake row) on the
    mixed-cell mesh against the oracle's direct solves."""
    kw = {"fp64": dict(precision=api.PF_FP64, tol=1e-12), "mixed": dict(precision=api.PF_MIXED, tol=1e-11),
          "mg": dict(precision=api.PF_MIXED, tol=1e-11, preconditioner="mg")}[mode]
    for kind in ("ellipse", "airfoil"):
        grid, body = polygon_case(kind, 192)
        m = CM.build_cut_mesh(grid, np.zeros((0, 3)), 48, polygons=[body], sigma=0.25)
        s = OSY.assemble(m, 1.0)
        u, psi_ref = OSV.solve_kutta(s, m) if kind == "airfoil" else OSV.solve_direct(s)
        with api.cut_mesh_build(grid, np.zeros((0, 3)), 48, (0, 0, 0, 0), 0.25, polygons=[body]) as g:
            res = api.psi_solve(g, U=1.0, **kw)
            psi = res.psi.cpu().numpy()
        assert res.status == 0
        live = m.kind.ravel() != OM.INACTIVE
        assert rel_l2(psi[live], psi_ref[live]) <= (1e-9 if mode == "fp64" else 1e-6), kind
        np.testing.assert_allclose(res.body_psi, u[s.n_free:], rtol=0, atol=1e-8)
