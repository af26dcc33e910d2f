"""Failure detection without a GPU fault: a bounded device-side wait that runs out.

The test hook makes CTA 0 of the fused CG kernel skip the copies of its first tile, so
the consumer warps' mbarrier wait on that stage gives up after a capped number of polls.
The kernel records the failure, drains the copies it issued and returns; the solve must
report PF_ETIMEOUT, and the CUDA context must stay usable for a fresh handle."""
import numpy as np
import pytest

from paper_2512_12232_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_2512_12232_gb300 import api
    return api


def test_bounded_wait_gives_up_with_etimeout(api):
    from paper_2512_12232_gb300._lib import PF_ETIMEOUT
    c = W.five_cylinder_case(0.5, 256, 128, 20)
    g = api.mesh_build(c.grid, c.bodies, c.sweeps, c.bc)
    try:
        g.test_wait_timeout(True)
        res = api.psi_solve(g, U=1.0, tol=1e-8, precision=api.PF_MIXED, chunk=4, raise_on_failure=False)
        assert res.status == PF_ETIMEOUT
    finally:
        g.close()
    # the context is intact: a new handle solves normally
    with api.mesh_build(c.grid, c.bodies, c.sweeps, c.bc) as g2:
        r = api.psi_solve(g2, U=1.0, tol=1e-8, precision=api.PF_MIXED)
        assert r.status == 0 and r.info[0]["rel_true_residual"] <= 1e-8
        assert np.all(np.isfinite(r.body_psi))
