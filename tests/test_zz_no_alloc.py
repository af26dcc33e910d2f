"""GPU test of pf_apply_noalloc, the allocation-free operator apply.

It serves callers that cannot allocate device memory at that point (everything owned
by a framework arena, or loops that must not call cudaMalloc).  The test calls it
through the C ABI twice in a row, on two different inputs, and compares each result
with pf_apply's (the allocating entry point) within the operator tolerances used by
the other operator tests.  This file is collected last on purpose."""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2512_12232_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_noalloc_apply_matches_apply_on_two_calls_in_a_row():
    from paper_2512_12232_gb300 import _lib as L, api
    lib = L.load()
    cases = [W.five_cylinder_case(0.25, 256, 128, 40), W.single_cylinder()]
    with api.batch_build(cases) as g:
        n = int(g.node_offsets[-1])
        nb = g.body_offsets[-1]
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        for call, seed in enumerate((21, 22)):
            p = torch.from_numpy(W.random_vector(n, seed)).cuda()
            for prec, tol in ((api.PF_FP64, 1e-13), (api.PF_MIXED, 1e-6)):
                y_ref, s_ref = api.apply(g, p, prec)
                y = torch.full_like(p, float("nan"))
                sums = (C.c_double * nb)()
                code = lib.pf_apply_noalloc(g.handle, prec, C.c_void_p(p.data_ptr()), C.c_void_p(y.data_ptr()),
                                            sums, stream)
                assert code == L.PF_OK, lib.pf_last_error()
                y = y.cpu().numpy()
                y_ref = y_ref.cpu().numpy()
                scale = np.abs(y_ref).max()
                assert np.isfinite(y).all()
                assert np.abs(y - y_ref).max() <= tol * scale, (call, prec)
                np.testing.assert_allclose(np.array(sums[:nb]), s_ref, rtol=0, atol=tol * scale * 10)


def test_noalloc_apply_rejects_bad_arguments():
    from paper_2512_12232_gb300 import _lib as L, api
    lib = L.load()
    c = W.single_cylinder()
    with api.mesh_build(c.grid, c.bodies, c.sweeps, c.bc) as g:
        p = torch.zeros(c.n_nodes, dtype=torch.float64, device="cuda")
        assert lib.pf_apply_noalloc(g.handle, 7, C.c_void_p(p.data_ptr()), C.c_void_p(p.data_ptr()), None,
                                    None) == L.PF_EINVAL
        assert lib.pf_apply_noalloc(None, 0, None, None, None, None) == L.PF_EINVAL


def test_noalloc_apply_rejects_a_handle_over_the_body_limit():
    """A handle holding more bodies than the fixed array has room for is refused with
    PF_EINVAL (naming the limit), while the allocating pf_apply still serves it; the
    limit is the header's PF_NOALLOC_MAX_BODIES (4096): here 65 variants of 64 bodies."""
    from paper_2512_12232_gb300 import _lib as L, api
    lib = L.load()
    limit = 4096
    centres = [(1.61 + 1.73 * a, 1.61 + 1.73 * b) for a in range(8) for b in range(8)]
    bodies = np.array([[cx, cy, 0.3] for cx, cy in centres])
    cases = [W.Case(0.0, 16.0, 0.0, 16.0, 64, 64, bodies, 4) for _ in range(limit // 64 + 1)]
    with api.batch_build(cases) as g:
        nb = g.body_offsets[-1]
        assert nb == 65 * 64 > limit
        n = int(g.node_offsets[-1])
        p = torch.from_numpy(W.random_vector(n, 5)).cuda()
        y = torch.zeros_like(p)
        sums = (C.c_double * nb)()
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        code = lib.pf_apply_noalloc(g.handle, api.PF_FP64, C.c_void_p(p.data_ptr()), C.c_void_p(y.data_ptr()),
                                    sums, stream)
        assert code == L.PF_EINVAL
        assert str(limit) in lib.pf_last_error().decode()
        assert torch.count_nonzero(y).item() == 0          # nothing was launched
        y_ref, s_ref = api.apply(g, p, api.PF_FP64)
        assert torch.isfinite(y_ref).all() and s_ref.shape == (nb,)


def test_noalloc_apply_rejects_a_call_on_another_device():
    """Every call must be made with the handle's device current."""
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two visible GPUs")
    from paper_2512_12232_gb300 import _lib as L, api
    lib = L.load()
    c = W.single_cylinder()
    with api.mesh_build(c.grid, c.bodies, c.sweeps, c.bc) as g:
        p = torch.zeros(c.n_nodes, dtype=torch.float64, device="cuda")
        with torch.cuda.device(1):
            code = lib.pf_apply_noalloc(g.handle, api.PF_FP64, C.c_void_p(p.data_ptr()), C.c_void_p(p.data_ptr()),
                                        None, None)
        assert code == L.PF_EINVAL


def test_noalloc_apply_refuses_a_capturing_stream():
    """The call ends by synchronising its stream, so on a stream that is being captured it
    returns PF_EINVAL before launching anything; the capture itself stays valid."""
    from paper_2512_12232_gb300 import _lib as L, api
    lib = L.load()
    c = W.single_cylinder()
    with api.mesh_build(c.grid, c.bodies, c.sweeps, c.bc) as g:
        p = torch.from_numpy(W.random_vector(c.n_nodes, 9)).cuda()
        y = torch.zeros_like(p)
        x = torch.zeros(16, device="cuda")
        s = torch.cuda.Stream()
        graph = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=s):
            x.add_(1.0)
            code = lib.pf_apply_noalloc(g.handle, api.PF_FP64, C.c_void_p(p.data_ptr()), C.c_void_p(y.data_ptr()),
                                        None, C.c_void_p(s.cuda_stream))
        assert code == L.PF_EINVAL
        assert b"capturing" in lib.pf_last_error()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.count_nonzero(y).item() == 0 and x[0].item() == 1.0
