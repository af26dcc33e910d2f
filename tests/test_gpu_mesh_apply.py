"""GPU parity: mesh generation (bit-exact against the oracle) and the matrix-free
operator (against the oracle's assembled element sums)."""
import numpy as np
import pytest
import torch

from oracle import mesh as OM, system as OSY
from paper_2512_12232_gb300 import workloads as W
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu

CASES = [
    W.single_cylinder(),
    W.Case(-3.0, 3.0, -2.0, 2.0, 24, 16, np.array([[0.1, 0.05, 0.9]]), 7),
    W.Case(-4.0, 4.0, -2.0, 2.0, 29, 17, np.array([[-1.6, 0.2, 0.7], [1.3, -0.4, 0.55]]), 11,
           bc=(1, 1, 0, 0)),
    W.five_cylinder_case(0.25, 256, 128, 40),
    W.five_cylinder_case(0.1, 333, 170, 60),
]


@pytest.fixture(scope="module")
def api():
    from paper_2512_12232_gb300 import api
    return api


@pytest.mark.parametrize("case", CASES, ids=lambda c: c.name or f"{c.nx}x{c.ny}")
def test_mesh_is_bit_exact(api, case):
    m = OM.build_mesh(case.grid, case.bodies, case.sweeps, case.bc)
    with api.mesh_build(case.grid, case.bodies, case.sweeps, case.bc) as g:
        xy = g.coords().cpu().numpy()
        kind, body = (t.cpu().numpy() for t in g.tags())
        st = g.stats()
    assert np.array_equal(kind, m.kind.ravel())
    assert np.array_equal(body, m.body.ravel())
    assert np.array_equal(xy[:, 0].view(np.uint64), m.x.ravel().view(np.uint64))
    assert np.array_equal(xy[:, 1].view(np.uint64), m.y.ravel().view(np.uint64))
    assert st["n_free"] == int((m.kind == OM.FREE).sum())
    assert st["n_active_cells"] == int(m.active.sum())
    s = OSY.assemble(m, 1.0)
    assert st["min_detJ"] == pytest.approx(s.detmin.min(), rel=1e-12)


def test_batched_mesh_equals_single_meshes(api):
    cases = W.parametric_sweep(6, seed=3, nx_choices=(256, 288, 320))
    with api.batch_build(cases) as g:
        for v, c in enumerate(cases):
            m = OM.build_mesh(c.grid, c.bodies, c.sweeps, c.bc)
            xy = g.coords(v).cpu().numpy()
            kind, _ = g.tags(v)
            assert np.array_equal(kind.cpu().numpy(), m.kind.ravel())
            assert np.array_equal(xy[:, 0], m.x.ravel()) and np.array_equal(xy[:, 1], m.y.ravel())


@pytest.mark.parametrize("case", CASES[:4], ids=lambda c: c.name or f"{c.nx}x{c.ny}")
def test_operator_matches_oracle(api, case):
    m = OM.build_mesh(case.grid, case.bodies, case.sweeps, case.bc)
    s = OSY.assemble(m, 1.0)
    p = W.random_vector(m.n_nodes, seed=11)
    p[m.kind.ravel() == OM.INACTIVE] = 0.0
    ref = OSY.full_operator_apply(s, p)
    kind = m.kind.ravel()
    rows = (kind == OM.FREE) | (kind == OM.BODY)
    ref = np.where(rows, ref, 0.0)
    body_ref = np.array([ref[(kind == OM.BODY) & (m.body.ravel() == k)].sum() for k in range(len(case.bodies))])
    with api.mesh_build(case.grid, case.bodies, case.sweeps, case.bc) as g:
        y64, b64 = api.apply(g, torch.from_numpy(p), api.PF_FP64)
        y32, b32 = api.apply(g, torch.from_numpy(p), api.PF_MIXED)
    y64 = y64.cpu().numpy()
    y32 = y32.cpu().numpy()
    scale = np.abs(ref).max()
    assert np.abs(y64 - ref).max() <= 1e-13 * scale * 10
    assert rel_l2(y32, ref) <= 2e-6
    np.testing.assert_allclose(b64, body_ref, rtol=0, atol=1e-12 * scale * 10)
    np.testing.assert_allclose(b32, body_ref, rtol=0, atol=1e-5 * scale * 10)


def test_operator_after_many_launches(api):
    """The operator kernel hands out work from a counter that persists across launches
    and precisions: after many timed launches of both, pf_apply on a two-variant batch
    still matches the oracle, and two calls agree bit for bit (which CTA takes which
    group of tiles changes nothing in a node's arithmetic)."""
    cases = [W.five_cylinder_case(0.5, 200, 100, 20), W.five_cylinder_case(1.0, 263, 131, 20)]   # one sweep count per batch
    refs = []
    for c in cases:
        m = OM.build_mesh(c.grid, c.bodies, c.sweeps, c.bc)
        s = OSY.assemble(m, 1.0)
        p = W.random_vector(m.n_nodes, seed=5)
        p[m.kind.ravel() == OM.INACTIVE] = 0.0
        kind = m.kind.ravel()
        ref = np.where((kind == OM.FREE) | (kind == OM.BODY), OSY.full_operator_apply(s, p), 0.0)
        refs.append((p, ref))
    p_all = np.concatenate([p for p, _ in refs])
    with api.batch_build(cases) as g:
        for prec in (api.PF_MIXED, api.PF_FP64, api.PF_MIXED):
            g.apply_timing(prec, reps=7)
        out = {}
        for prec in (api.PF_FP64, api.PF_MIXED):
            y1, _ = api.apply(g, torch.from_numpy(p_all), prec)
            y2, _ = api.apply(g, torch.from_numpy(p_all), prec)
            assert torch.equal(y1, y2)
            out[prec] = y1.cpu().numpy()
    off = 0
    for p, ref in refs:
        scale = np.abs(ref).max()
        y64 = out[api.PF_FP64][off:off + p.size]
        y32 = out[api.PF_MIXED][off:off + p.size]
        assert np.abs(y64 - ref).max() <= 1e-12 * scale
        assert rel_l2(y32, ref) <= 2e-6
        off += p.size


def test_invalid_inputs_rejected(api):
    from paper_2512_12232_gb300._lib import PfError
    with pytest.raises(PfError, match="EINVAL"):
        api.mesh_build((-4.0, 4.0, -3.0, 3.0, 32, 24), [[0.0, 0.0, 1.0], [1.5, 0.0, 0.6]], 5)
    with pytest.raises(PfError, match="EINVAL"):
        api.mesh_build((-4.0, 4.0, -3.0, 3.0, 32, 24), [[2.8, 0.0, 1.0]], 5)
    with pytest.raises(PfError, match="EINVAL"):
        api.mesh_build((-4.0, 4.0, -3.0, 3.0, 1, 24), [], 5)


def test_inverted_cell_is_reported_and_solve_refused(api):
    """A coarse grid with no smoothing where one projected boundary node folds a cell
    (the oracle's minimum det J over the Gauss points is about -1.45e-3): the GPU mesh
    reports the same minimum det J and the solve refuses with PF_EMESH_INVALID."""
    from oracle import mesh as OM, element as OE
    from paper_2512_12232_gb300._lib import PfError
    grid = (-4.0, 4.0, -2.0, 2.0, 32, 16)
    body = [[-0.91, -0.45, 0.67]]
    m = OM.build_mesh(grid, np.array(body), 0, (0, 0, 0, 0))
    _, dm = OE.q4_stiffness(OM.cell_coords(m)[m.active])
    assert dm.min() < 0
    with api.mesh_build(grid, body, 0) as g:
        st = g.stats(0)
        assert st["min_detJ"] == pytest.approx(dm.min(), rel=1e-9)
        with pytest.raises(PfError, match="EMESH_INVALID"):
            api.psi_solve(g, U=1.0, tol=1e-8, precision=api.PF_MIXED)
