"""GPU checks of properties the discrete problem fixes exactly, whatever the oracle says:

* a uniform stream without bodies is reproduced exactly (psi = U y is bilinear, so the Q4
  space holds it), with Dirichlet sides and with natural inlet and outlet;
* the five-cylinder layout is mirror symmetric about y = 0 with psi = U y antisymmetric,
  so the bodies on the axis carry psi = 0 and the transverse pair carries opposite values;
* a converged psi satisfies the discrete equations: the operator applied to it (Dirichlet
  values included) vanishes on every FREE row and on every collapsed body row (the zero
  circulation of each body) up to the solve's tolerance."""
import numpy as np
import pytest
import torch

from paper_2512_12232_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2512_12232_gb300 import api
    return api


@pytest.mark.parametrize("bc", [(0, 0, 0, 0), (1, 1, 0, 0)], ids=["dirichlet", "natural_inlet_outlet"])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_uniform_stream_without_bodies_is_exact(api, bc, prec):
    c = W.Case(-3.0, 5.0, -1.5, 2.5, 96, 48, np.zeros((0, 3)), 0, bc=bc)
    U = 1.7
    p = api.PF_FP64 if prec == "fp64" else api.PF_MIXED
    with api.mesh_build(c.grid, c.bodies, c.sweeps, c.bc) as g:
        res = api.psi_solve(g, U=U, tol=1e-13 if prec == "fp64" else 1e-12, precision=p)
        y = g.coords()[:, 1].cpu().numpy()
    assert res.status == 0
    err = np.abs(res.psi.cpu().numpy() - U * y).max()
    assert err <= (1e-12 if prec == "fp64" else 1e-10) * U * np.abs(y).max(), err


@pytest.mark.parametrize("delta", [0.25, 1.0])
def test_mirror_symmetric_layout(api, delta):
    """Bodies 0-2 lie on y = 0, bodies 3 and 4 at y = -(1 + delta) and +(1 + delta)."""
    c = W.five_cylinder_case(delta, 256, 128, 40)
    b = np.asarray(c.bodies)
    assert np.all(b[:3, 1] == 0.0) and b[3, 1] == -b[4, 1]
    with api.mesh_build(c.grid, c.bodies, c.sweeps, c.bc) as g:
        res = api.psi_solve(g, U=1.0, tol=1e-13, precision=api.PF_FP64)
    C = res.body_psi
    scale = abs(C[4])
    assert scale > 0.1
    assert np.abs(C[:3]).max() <= 1e-9 * scale, C
    assert abs(C[3] + C[4]) <= 1e-9 * scale, C


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("mixed", 1e-10)])
def test_solution_satisfies_the_discrete_equations(api, prec, tol):
    """||A psi|| over the FREE and collapsed body rows against ||b||, b the lifting of the
    Dirichlet values (the operator applied to psi restricted to the Dirichlet nodes)."""
    c = W.five_cylinder_case(0.5, 320, 160, 40)
    p = api.PF_FP64 if prec == "fp64" else api.PF_MIXED
    with api.mesh_build(c.grid, c.bodies, c.sweeps, c.bc) as g:
        res = api.psi_solve(g, U=1.0, tol=tol, precision=p)
        kind = g.tags()[0].cpu().numpy()
        y, body_rows = api.apply(g, res.psi, api.PF_FP64)
        lift = torch.where(torch.from_numpy(kind == 1).cuda(), res.psi, torch.zeros_like(res.psi))
        yb, body_b = api.apply(g, lift, api.PF_FP64)
    free = kind == 0
    r = np.concatenate([y.cpu().numpy()[free], body_rows])
    b = np.concatenate([yb.cpu().numpy()[free], body_b])
    assert res.status == 0 and np.linalg.norm(b) > 0
    rel = np.linalg.norm(r) / np.linalg.norm(b)
    assert rel <= 1.05 * tol, rel
    assert rel == pytest.approx(res.info[0]["rel_true_residual"], rel=0.05, abs=1e-3 * tol)
