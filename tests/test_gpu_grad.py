"""GPU parity of the adjoint shape gradients (dJ/dX and dJ/dc of CoPFI and gap flow)
against the oracle's adjoint gradient (complex-step element derivatives), against
central finite differences of GPU solves, and through torch.autograd."""
import numpy as np
import pytest
import torch

from oracle import grad as OG, mesh as OM
from paper_2512_12232_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASE = W.five_cylinder_case(0.83, 150, 76, 20)     # no node on a circle: topology stable at +-1e-6


@pytest.fixture(scope="module")
def api():
    from paper_2512_12232_gb300 import api
    return api


@pytest.mark.parametrize("obj", [0, 1], ids=["copfi", "gap_flow"])
def test_gradient_matches_oracle(api, obj):
    m = OM.build_mesh(CASE.grid, CASE.bodies, CASE.sweeps, CASE.bc)
    J_ref, dX_ref, dc_ref, _ = OG.gradient(m, CASE.sweeps, 1.0, 3, 4, obj)
    with api.mesh_build(CASE.grid, CASE.bodies, CASE.sweeps, CASE.bc) as g:
        api.psi_solve(g, U=1.0, tol=1e-13, precision=api.PF_FP64)
        dX, dc, J = api.grad(g, obj, 3, 4, 1.0, 1e-13)
        # the forward solution is restored after the adjoint
        cp, q = api.copfi(g, 0, 3, 4, 1.0)
    dX = dX.cpu().numpy()
    assert abs(J[0] - J_ref) <= 1e-10 * max(1.0, abs(J_ref))
    assert np.abs(dX - dX_ref).max() <= 1e-8 * np.abs(dX_ref).max()
    assert np.abs(dc - dc_ref).max() <= 1e-8 * np.abs(dc_ref).max()
    ref_q = J_ref if obj == 1 else J_ref * (CASE.bodies[4, 1] - CASE.bodies[3, 1])
    assert abs(q - ref_q) <= 1e-9


def test_centre_gradient_matches_finite_differences_of_gpu_solves(api):
    """Central differences of iteratively solved J: the two solves differ by ~1e-13 in J,
    so the step is 2e-5 (noise ~3e-9) rather than the oracle pin's 1e-6 (whose direct
    solves are exact); the topology is asserted unchanged at +-step."""
    ref_kind = None

    def J(bodies):
        with api.mesh_build(CASE.grid, bodies, CASE.sweeps, CASE.bc) as g:
            assert np.array_equal(g.tags()[0].cpu().numpy(), ref_kind)
            api.psi_solve(g, U=1.0, tol=1e-13, precision=api.PF_FP64)
            return api.copfi(g, 0, 3, 4, 1.0)[0]
    with api.mesh_build(CASE.grid, CASE.bodies, CASE.sweeps, CASE.bc) as g:
        ref_kind = g.tags()[0].cpu().numpy()
        api.psi_solve(g, U=1.0, tol=1e-13, precision=api.PF_FP64)
        _, dc, _ = api.grad(g, 0, 3, 4, 1.0, 1e-13, want_dX=False)
    h = 2e-5
    scale = np.abs(dc).max()
    for k in (0, 3, 4):
        for a in (0, 1):
            bp = CASE.bodies.copy(); bp[k, a] += h
            bm = CASE.bodies.copy(); bm[k, a] -= h
            fd = (J(bp) - J(bm)) / (2 * h)
            if abs(fd) >= 1e-3 * scale:
                assert abs(dc[k, a] - fd) <= 1e-5 * abs(fd), (k, a, dc[k, a], fd)
            else:   # component near zero (symmetry): finite differences only see solve noise
                assert abs(dc[k, a] - fd) <= 1e-7 * scale + 1e-8, (k, a, dc[k, a], fd)


def test_batched_gradient_equals_single(api):
    cases = W.gradient_study(3, seed=1, nx=256)
    with api.batch_build(cases) as g:
        api.psi_solve(g, U=1.0, tol=1e-12, precision=api.PF_MIXED)
        dXb, dcb, Jb = api.grad(g, 0, 3, 4, 1.0, 1e-12)
        offs = g.node_offsets
        dXb = dXb.cpu().numpy()
    for v, c in enumerate(cases):
        with api.mesh_build(c.grid, c.bodies, c.sweeps, c.bc) as g1:
            api.psi_solve(g1, U=1.0, tol=1e-12, precision=api.PF_MIXED)
            dX1, dc1, J1 = api.grad(g1, 0, 3, 4, 1.0, 1e-12)
        assert abs(Jb[v] - J1[0]) <= 1e-9
        np.testing.assert_allclose(dcb[5 * v:5 * v + 5], dc1, rtol=0, atol=1e-7 * np.abs(dc1).max())
        np.testing.assert_allclose(dXb[offs[v]:offs[v + 1]], dX1.cpu().numpy(), rtol=0,
                                   atol=1e-7 * np.abs(dX1.cpu().numpy()).max())


def test_multigrid_adjoint_gives_the_same_gradient(api):
    """pf_grad solves the adjoint with the preconditioner of the last forward solve: after a
    multigrid-preconditioned solve the adjoint is multigrid-preconditioned too (far fewer
    iterations, counted by the solve timers) and the gradient is the paper's CG's."""
    cases = W.gradient_study(3, seed=1, nx=256)
    out = {}
    for pre in ("none", "mg"):
        with api.batch_build(cases) as g:
            api.psi_solve(g, U=1.0, tol=1e-12, precision=api.PF_MIXED, preconditioner=pre)
            dX, dc, J = api.grad(g, 0, 3, 4, 1.0, 1e-12)
            out[pre] = (dX.cpu().numpy(), dc, J, g.timing()["cg_launches"])
    dX0, dc0, J0, it0 = out["none"]
    dX1, dc1, J1, it1 = out["mg"]
    assert 4 * it1 < it0, (it0, it1)
    np.testing.assert_allclose(J1, J0, rtol=0, atol=1e-9)
    np.testing.assert_allclose(dc1, dc0, rtol=0, atol=1e-7 * np.abs(dc0).max())
    np.testing.assert_allclose(dX1, dX0, rtol=0, atol=1e-7 * np.abs(dX0).max())


def test_autograd_function(api):
    from paper_2512_12232_gb300 import autograd as AG
    c = torch.tensor(CASE.bodies[:, :2], dtype=torch.float64, requires_grad=True)
    J = AG.copfi(c, CASE.bodies[:, 2], CASE.grid, CASE.sweeps)
    J.backward()
    m = OM.build_mesh(CASE.grid, CASE.bodies, CASE.sweeps, CASE.bc)
    J_ref, _, dc_ref, _ = OG.gradient(m, CASE.sweeps, 1.0, 3, 4, 0)
    assert abs(J.item() - J_ref) <= 1e-9
    np.testing.assert_allclose(c.grad.numpy(), dc_ref, rtol=0, atol=1e-7 * np.abs(dc_ref).max())


def test_batch_entry_points_agree_with_solve_and_grad(api):
    """pf_mesh_info / pf_batch_solve / pf_batch_grad / pf_mesh_destroy give what the
    calls they name give (to solve tolerance: a second solve on the same handle may
    run on a re-balanced schedule, which changes the order of the dot-product sums)."""
    cases = W.gradient_study(2, seed=3, nx=128)
    g = api.batch_build(cases)
    st = g.stats(0)
    info = api.mesh_info(g)
    assert info == {k: st[k] for k in ("n_nodes", "n_dof", "n_boundary_edges", "min_detJ")}
    r1 = api.psi_solve(g, U=1.0, tol=1e-12, precision=api.PF_MIXED)
    dX1, dc1, J1 = api.grad(g, 0, 3, 4, 1.0, 1e-12)
    r2 = api.batch_solve(g, U=1.0, tol=1e-12, precision=api.PF_MIXED)
    dX2, dc2, J2 = api.batch_grad(g, 0, 3, 4, 1.0, 1e-12)
    assert r2.psi is None
    assert all(i["status"] == 0 for i in r2.info)
    np.testing.assert_allclose(r2.body_psi, r1.body_psi, rtol=0, atol=1e-9 * np.abs(r1.body_psi).max())
    np.testing.assert_allclose(J2, J1, rtol=1e-9)
    np.testing.assert_allclose(dc2, dc1, rtol=0, atol=1e-7 * np.abs(dc1).max())
    np.testing.assert_allclose(dX2.cpu().numpy(), dX1.cpu().numpy(), rtol=0,
                               atol=1e-7 * dX1.abs().max().item())
    api.mesh_destroy(g)
    with pytest.raises(RuntimeError, match="closed"):
        g.handle


def _smooth_perturbation(m, amp):
    """A smooth displacement field that vanishes on the outer ring and on body nodes."""
    x, y = m.x, m.y
    Lx, Ly = x.max() - x.min(), y.max() - y.min()
    s = np.sin(np.pi * (x - x.min()) / Lx) * np.sin(np.pi * (y - y.min()) / Ly)
    keep = (m.kind == OM.FREE).astype(np.float64)
    return amp * s * np.cos(3.0 * y) * keep, amp * s * np.sin(2.0 * x) * keep


def test_set_coords_solves_and_differentiates_at_the_given_coordinates(api):
    """pf_mesh_set_coords: the solve and dJ/dX on caller-given node coordinates (a smooth
    perturbation of the generated mesh) match the oracle assembled on the same coordinates;
    setting the generated coordinates back reproduces the original solve bit for bit."""
    m = OM.build_mesh(CASE.grid, CASE.bodies, CASE.sweeps, CASE.bc)
    h = (CASE.x1 - CASE.x0) / CASE.nx
    px, py = _smooth_perturbation(m, 0.2 * h)
    m.x, m.y = m.x + px, m.y + py
    J_ref, dX_ref, dc_ref, psi_ref = OG.gradient(m, CASE.sweeps, 1.0, 3, 4, 0)
    xy_new = torch.from_numpy(np.stack([m.x.ravel(), m.y.ravel()], axis=1))
    with api.mesh_build(CASE.grid, CASE.bodies, CASE.sweeps, CASE.bc) as g:
        xy0 = g.coords()
        r0 = api.psi_solve(g, U=1.0, tol=1e-13, precision=api.PF_FP64).psi.cpu().numpy()
        assert g.set_coords(xy_new) == 0
        assert g.stats()["n_general_cells"] > 0
        np.testing.assert_array_equal(g.coords().cpu().numpy(), xy_new.numpy())
        r1 = api.psi_solve(g, U=1.0, tol=1e-13, precision=api.PF_FP64)
        psi1 = r1.psi.cpu().numpy()
        dX, dc, J = api.grad(g, 0, 3, 4, 1.0, 1e-13)
        assert g.set_coords(xy0) == 0
        r2 = api.psi_solve(g, U=1.0, tol=1e-13, precision=api.PF_FP64).psi.cpu().numpy()
    assert np.linalg.norm(psi1 - psi_ref) <= 1e-10 * np.linalg.norm(psi_ref)
    assert abs(J[0] - J_ref) <= 1e-10 * max(1.0, abs(J_ref))
    dX = dX.cpu().numpy()
    assert np.abs(dX - dX_ref).max() <= 1e-8 * np.abs(dX_ref).max()
    np.testing.assert_array_equal(r2, r0)


def test_set_coords_refuses_a_folded_cell(api):
    m = OM.build_mesh(CASE.grid, CASE.bodies, CASE.sweeps, CASE.bc)
    with api.mesh_build(CASE.grid, CASE.bodies, CASE.sweeps, CASE.bc) as g:
        xy = g.coords().clone()
        k = (m.ny // 2) * (m.nx + 1) + 5          # a free node far from the bodies
        xy[k, 0] += 3.0 * (CASE.x1 - CASE.x0) / CASE.nx
        assert g.set_coords(xy) == 2              # PF_EMESH_INVALID
        res = api.psi_solve(g, U=1.0, tol=1e-10, raise_on_failure=False)
        assert res.status == 2


def test_coords_vjp_matches_oracle_chain(api):
    """pf_coords_vjp against the oracle's transpose of the mesh generator (transposed
    smoothing sweeps and the projection Jacobian) on a random cotangent, on a batch."""
    cases = [CASE, W.five_cylinder_case(0.4, 128, 64, 12)]
    rng = np.random.default_rng(11)
    with api.batch_build(cases, sweeps=20) as g:
        gX = rng.standard_normal((int(g.node_offsets[-1]), 2))
        gc = g.coords_vjp(torch.from_numpy(gX))
        offs = g.node_offsets
    for v, c in enumerate(cases):
        m = OM.build_mesh(c.grid, c.bodies, 20, c.bc)
        ref = OG.centre_chain(m, 20, gX[offs[v]:offs[v + 1]])
        np.testing.assert_allclose(gc[5 * v:5 * v + 5], ref, rtol=0, atol=1e-11 * np.abs(ref).max())


def test_autograd_through_node_coordinates(api):
    """X = mesh_coords(c), J = objective_at_coords(X, c): dJ/dX equals pf_grad's (and the
    oracle's), dJ/dc equals the one-step objective(c) and the oracle's total gradient, and a
    central difference of J along a random direction in X agrees with dJ/dX."""
    from paper_2512_12232_gb300 import autograd as AG
    c = torch.tensor(CASE.bodies[:, :2], dtype=torch.float64, requires_grad=True)
    X = AG.mesh_coords(c, CASE.bodies[:, 2], CASE.grid, CASE.sweeps)
    X.retain_grad()
    J = AG.objective_at_coords(X, c, CASE.bodies[:, 2], CASE.grid, CASE.sweeps, tol=1e-13)
    J.backward()
    m = OM.build_mesh(CASE.grid, CASE.bodies, CASE.sweeps, CASE.bc)
    J_ref, dX_ref, dc_ref, _ = OG.gradient(m, CASE.sweeps, 1.0, 3, 4, 0)
    assert abs(J.item() - J_ref) <= 1e-9
    gX = X.grad.cpu().numpy()
    assert np.abs(gX - dX_ref).max() <= 1e-8 * np.abs(dX_ref).max()
    np.testing.assert_allclose(c.grad.numpy(), dc_ref, rtol=0, atol=1e-7 * np.abs(dc_ref).max())
    c2 = torch.tensor(CASE.bodies[:, :2], dtype=torch.float64, requires_grad=True)
    AG.copfi(c2, CASE.bodies[:, 2], CASE.grid, CASE.sweeps, tol=1e-13).backward()
    np.testing.assert_allclose(c.grad.numpy(), c2.grad.numpy(), rtol=0, atol=1e-9 * np.abs(dc_ref).max())
    # directional derivative along a smooth field in X-space
    px, py = _smooth_perturbation(m, 1.0)
    d = torch.from_numpy(np.stack([px.ravel(), py.ravel()], axis=1)).cuda()
    eps = 1e-6
    Js = []
    with api.mesh_build(CASE.grid, CASE.bodies, CASE.sweeps, CASE.bc) as g:
        for sgn in (1.0, -1.0):
            assert g.set_coords(X.detach() + sgn * eps * d) == 0
            api.psi_solve(g, U=1.0, tol=1e-13, precision=api.PF_FP64)
            Js.append(api.copfi(g, 0, 3, 4, 1.0)[0])
    fd = (Js[0] - Js[1]) / (2 * eps)
    an = float((X.grad * d).sum())
    assert abs(fd - an) <= 1e-5 * abs(an) + 1e-7, (fd, an)
