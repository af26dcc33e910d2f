"""GPU parity at the benchmark's own configuration: the five-cylinder batch of 5 variants
on 2048x1024 grids with 200 smoothing sweeps and delta in {0.1, 0.25, 0.5, 1, 2}, against
the oracle's direct solves of the same 5 systems.

* Mesh: every node's kind, body and FP64 coordinates bit for bit (the smoothing's
  temporal blocking, front skipping and shrinking window at S = 200).
* The benchmark's solve (mixed precision, relative true residual 1e-8, tuned schedule):
  the oracle recomputes the residual of the GPU solution with its own matrix and finds
  it within the tolerance, and the error of psi, of the body values and of CoPFI stays
  within what that residual allows: ||u - u*||_2 <= ||b - A u||_2 / lambda_min(A), with
  lambda_min(A) from a Lanczos run on the oracle's factorised A.
* Tight solves: mixed to 1e-12 (psi to 1e-6 relative L2, body values to 1e-8), the same
  with the multigrid-preconditioned CG, and FP64 to 1e-13 (psi to 1e-10).

The oracle's five solves run in a spawn pool, one process per variant."""
import multiprocessing as mp
import os

import numpy as np
import pytest

from paper_2512_12232_gb300 import workloads as W
from tests.gpu_util import rel_l2

pytestmark = pytest.mark.gpu

DELTAS = (0.1, 0.25, 0.5, 1.0, 2.0)
NX, NY, SWEEPS = 2048, 1024, 200


def _oracle_variant(case):
    """Mesh, reduced system, direct solution and lambda_min(A) of one variant (runs in a
    worker process; plain oracle code only)."""
    import scipy.sparse.linalg as spla

    from oracle import mesh as OM, solve as OS, system as OSY
    m = OM.build_mesh(case.grid, case.bodies, case.sweeps, case.bc)
    s = OSY.assemble(m, 1.0)
    lu = OS.sparse_factor(s.A)
    u = lu.solve(s.b)
    op = spla.LinearOperator(s.A.shape, matvec=lu.solve, dtype=np.float64)
    mu = spla.eigsh(op, k=1, which="LM", tol=1e-4, return_eigenvectors=False)[0]
    return {"x": m.x.ravel(), "y": m.y.ravel(), "kind": m.kind.ravel().astype(np.int8),
            "body": m.body.ravel().astype(np.int32), "psi": OSY.expand(s, u), "u": u, "n_free": s.n_free,
            "A": s.A.tocsr(), "b": s.b, "dof": s.dof, "lam_min": 1.0 / mu}


@pytest.fixture(scope="module")
def full_size():
    cases = [W.five_cylinder_case(d, NX, NY, SWEEPS) for d in DELTAS]
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    workers = max(1, min(len(cases), (os.cpu_count() or 1)))
    with mp.get_context("spawn").Pool(workers) as pool:
        ref = pool.map(_oracle_variant, cases)
    return cases, ref


@pytest.fixture(scope="module")
def api():
    from paper_2512_12232_gb300 import api
    return api


def _reduced(ref, psi):
    """Reduced vector (free unknowns, then body values) of a nodal psi."""
    u = np.empty(ref["A"].shape[0])
    m = ref["dof"] >= 0
    u[ref["dof"][m]] = psi[m]
    return u


def test_full_size_mesh_is_bit_exact(api, full_size):
    cases, ref = full_size
    with api.batch_build(cases) as g:
        for v, r in enumerate(ref):
            xy = g.coords(v).cpu().numpy()
            kind, body = (t.cpu().numpy() for t in g.tags(v))
            assert np.array_equal(kind, r["kind"]), v
            assert np.array_equal(body[kind == 2], r["body"][r["kind"] == 2]), v
            assert np.array_equal(xy[:, 0], r["x"]) and np.array_equal(xy[:, 1], r["y"]), v


def test_full_size_benchmark_solve_error_is_within_its_residual_bound(api, full_size):
    cases, ref = full_size
    tol = 1e-8
    with api.batch_build(cases) as g:
        res = api.psi_solve(g, U=1.0, tol=tol, precision=api.PF_MIXED, tune_schedule=True)
        psi = res.psi.cpu().numpy()
        offs = g.node_offsets
        cps = [api.copfi(g, v, 3, 4, 1.0)[0] for v in range(len(cases))]
    for v, (c, r) in enumerate(zip(cases, ref)):
        assert res.info[v]["status"] == 0 and res.info[v]["rel_true_residual"] <= tol
        pv = psi[offs[v]:offs[v + 1]]
        ug = _reduced(r, pv)
        bn = np.linalg.norm(r["b"])
        resid = np.linalg.norm(r["b"] - r["A"] @ ug) / bn
        assert resid <= 1.05 * tol, (v, resid)          # the GPU's own FP64 residual, recomputed
        e_bound = tol * bn / r["lam_min"]                 # ||u - u*||_2 <= ||r||_2 / lambda_min
        e = np.linalg.norm(ug - r["u"])
        assert e <= e_bound, (v, e, e_bound)
        C_ref = r["u"][r["n_free"]:]
        C = res.body_psi[5 * v:5 * v + 5]
        assert np.abs(C - C_ref).max() <= e_bound
        dy = c.bodies[4][1] - c.bodies[3][1]
        cp_ref = (C_ref[4] - C_ref[3]) / dy
        assert abs(cps[v] - cp_ref) <= 2 * e_bound / dy
        print(f"variant {v}: rel L2 psi {rel_l2(pv, r['psi']):.2e}, max |dC| {np.abs(C - C_ref).max():.2e}, "
              f"|dCoPFI| {abs(cps[v] - cp_ref):.2e}, residual {resid:.2e}, bound on |e| {e_bound:.2e}")


@pytest.mark.parametrize("prec,tol,bound", [("mixed", 1e-12, 1e-6), ("fp64", 1e-13, 1e-10), ("mixed_mg", 1e-12, 1e-6)])
def test_full_size_tight_solves_match_oracle(api, full_size, prec, tol, bound):
    cases, ref = full_size
    p = api.PF_FP64 if prec == "fp64" else api.PF_MIXED
    with api.batch_build(cases) as g:
        res = api.psi_solve(g, U=1.0, tol=tol, precision=p, preconditioner="mg" if prec == "mixed_mg" else "none")
        psi = res.psi.cpu().numpy()
        offs = g.node_offsets
    for v, r in enumerate(ref):
        assert res.info[v]["status"] == 0 and res.info[v]["rel_true_residual"] <= tol
        err = rel_l2(psi[offs[v]:offs[v + 1]], r["psi"])
        assert err <= bound, (v, err)
        np.testing.assert_allclose(res.body_psi[5 * v:5 * v + 5], r["u"][r["n_free"]:], rtol=0, atol=1e-8)
