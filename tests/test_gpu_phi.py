"""GPU parity of the velocity-potential solve (pf_phi_solve) and its element velocities
against the oracle (oracle/potential.py): FP64 to 1e-10 and mixed precision to 1e-6 in
relative L2, single meshes and an uneven batch; the uniform stream without bodies; and
the flow net, where the velocities from phi and from psi agree as the oracle's do."""
import functools

import numpy as np
import pytest

from oracle import mesh as OM, potential as OPO
from paper_2512_12232_gb300 import workloads as W
from tests.gpu_util import oracle_solution, rel_l2

pytestmark = pytest.mark.gpu

CASES = [
    W.single_cylinder(),
    W.five_cylinder_case(0.25, 256, 128, 40),
    W.Case(-4.0, 4.0, -2.0, 2.0, 29, 17, np.array([[-1.6, 0.2, 0.7], [1.3, -0.4, 0.55]]), 11, bc=(1, 1, 0, 0)),
]
IDS = [c.name or f"{c.nx}x{c.ny}" for c in CASES]


@pytest.fixture(scope="module")
def api():
    from paper_2512_12232_gb300 import api
    return api


@functools.lru_cache(maxsize=16)
def _phi_ref(key):
    grid, bodies, sweeps, bc, U = key
    m = OM.build_mesh(grid, np.array(bodies, dtype=np.float64).reshape(-1, 3), sweeps, bc)
    s = OPO.assemble_phi(m, U)
    return m, s, OPO.solve_phi(s)


def phi_reference(case, U=1.0):
    return _phi_ref((tuple(case.grid), tuple(map(tuple, np.asarray(case.bodies).tolist())), case.sweeps,
                     tuple(case.bc), U))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=IDS)
def test_phi_matches_oracle(api, case, prec):
    U = 1.7
    m, s, phi_ref = phi_reference(case, U)
    p = api.PF_FP64 if prec == "fp64" else api.PF_MIXED
    with api.mesh_build(case.grid, case.bodies, case.sweeps, case.bc) as g:
        phi, info, code = api.phi_solve(g, U=U, tol=1e-13 if prec == "fp64" else 1e-12, precision=p)
    assert code == 0 and info[0]["status"] == 0
    assert info[0]["n_dof"] == s.A.shape[0]
    assert rel_l2(phi.cpu().numpy(), phi_ref) <= (1e-10 if prec == "fp64" else 1e-6)


def test_phi_on_an_uneven_batch(api):
    cases = [W.five_cylinder_case(0.5, 160, 80, 20), W.single_cylinder(), W.five_cylinder_case(1.0, 200, 100, 20)]
    with api.batch_build(cases, sweeps=20) as g:
        phi, info, code = api.phi_solve(g, U=1.0, tol=1e-13, precision=api.PF_FP64)
        offs = g.node_offsets
        phi = phi.cpu().numpy()
    assert code == 0
    for v, c in enumerate(cases):
        c = W.Case(c.x0, c.x1, c.y0, c.y1, c.nx, c.ny, c.bodies, 20, c.bc)
        _, _, phi_ref = phi_reference(c)
        assert rel_l2(phi[offs[v]:offs[v + 1]], phi_ref) <= 1e-10, v


def test_uniform_stream_without_bodies(api):
    """No bodies: phi = U x exactly (a linear field, reproduced by bilinear elements)."""
    c = W.Case(-3.0, 5.0, -1.0, 2.0, 40, 24, np.zeros((0, 3)), 0)
    with api.mesh_build(c.grid, c.bodies, c.sweeps, c.bc) as g:
        phi, _, _ = api.phi_solve(g, U=2.0, tol=1e-14, precision=api.PF_FP64)
        x = g.coords()[:, 0]
    np.testing.assert_allclose(phi.cpu().numpy(), 2.0 * x.cpu().numpy(), rtol=0, atol=1e-11)


def test_phi_velocity_and_flow_net(api):
    """Element velocities grad phi against the oracle's, and the flow net: the GPU's
    velocities from phi and from psi differ exactly as the oracle's two fields do
    (discretisation only)."""
    c = W.five_cylinder_case(0.25, 256, 128, 40)
    m, s, phi_ref = phi_reference(c)
    _, _, _, psi_ref = oracle_solution(c, 1.0)
    uf, vf = OPO.velocity_from_phi(m, phi_ref)
    us, vs = OPO.velocity_from_psi(m, psi_ref)
    with api.mesh_build(c.grid, c.bodies, c.sweeps, c.bc) as g:
        api.phi_solve(g, U=1.0, tol=1e-13, precision=api.PF_FP64)
        api.psi_solve(g, U=1.0, tol=1e-13, precision=api.PF_FP64)
        ugf, vgf = (t.cpu().numpy() for t in api.phi_velocity_field(g, 0))
        ugs, vgs = (t.cpu().numpy() for t in api.velocity_field(g, 0))
    scale = max(np.abs(uf).max(), np.abs(vf).max())
    np.testing.assert_allclose(ugf[m.active], uf, rtol=0, atol=1e-8 * scale)
    np.testing.assert_allclose(vgf[m.active], vf, rtol=0, atol=1e-8 * scale)
    assert np.all(ugf[~m.active] == 0.0) and np.all(vgf[~m.active] == 0.0)
    np.testing.assert_allclose(ugf[m.active] - ugs[m.active], uf - us, rtol=0, atol=2e-8 * scale)
    np.testing.assert_allclose(vgf[m.active] - vgs[m.active], vf - vs, rtol=0, atol=2e-8 * scale)
    # the two velocity fields describe the same flow: mean relative difference is small
    d = np.hypot(uf - us, vf - vs).mean() / np.hypot(us, vs).mean()
    assert d < 0.05, d


def test_phi_velocity_needs_a_phi_solve(api):
    c = W.single_cylinder()
    with api.mesh_build(c.grid, c.bodies, c.sweeps, c.bc) as g:
        api.psi_solve(g, U=1.0, tol=1e-10)
        with pytest.raises(Exception, match="PF_EINVAL"):
            api.phi_velocity_field(g, 0)


def test_phi_with_the_multigrid_preconditioner(api):
    """The phi system has no bodies and natural walls; the preconditioned CG reaches the
    oracle's phi (mixed precision, 1e-12) in far fewer iterations."""
    c = W.five_cylinder_case(0.25, 256, 128, 40)
    m, s, phi_ref = phi_reference(c)
    with api.mesh_build(c.grid, c.bodies, c.sweeps, c.bc) as g:
        phi, info, code = api.phi_solve(g, U=1.0, tol=1e-12, precision=api.PF_MIXED, preconditioner="mg")
        _, info0, _ = api.phi_solve(g, U=1.0, tol=1e-12, precision=api.PF_MIXED)
    assert code == 0 and info[0]["status"] == 0
    assert rel_l2(phi.cpu().numpy(), phi_ref) <= 1e-6
    assert 3 * info[0]["iters"] < info0[0]["iters"]
