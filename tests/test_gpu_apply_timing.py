"""The operator bandwidth measurement (pf_apply_timing) runs on a fresh handle and
reports a positive time and the algorithmic bytes implied by the mesh counts."""
import pytest

from paper_2512_12232_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_apply_timing_on_fresh_handle():
    from paper_2512_12232_gb300 import api
    c = W.five_cylinder_case(0.5, 256, 128, 20)
    with api.mesh_build(c.grid, c.bodies, c.sweeps, c.bc) as g:
        st = g.stats(0)
        for prec, es in ((api.PF_MIXED, 4), (api.PF_FP64, 8)):
            us, by = g.apply_timing(prec, reps=5)
            assert us > 0
            # p, y and tags at every node, plus the stored coefficients of the cells that
            # need them in this precision (at most every cell with a displaced corner)
            lo = (2 * es + 1) * st["n_nodes"]
            assert lo <= by <= lo + 6 * es * st["n_general_cells"]
            if prec == api.PF_FP64:
                assert by == pytest.approx(lo + 6 * es * st["n_general_cells"])
        # a solve afterwards still works on the same handle
        r = api.psi_solve(g, U=1.0, tol=1e-8, precision=api.PF_MIXED)
        assert r.status == 0
