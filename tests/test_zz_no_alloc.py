"""glad_loglike_static: the log-likelihood for callers that cannot call cudaMalloc while
they run (code inside someone else's CUDA-graph capture, samplers under a fixed device
memory budget).  Its scratch is a static device array, so it must give the same logL as
glad_loglike -- on two calls in a row, since every call reuses the array's old contents
-- and must refuse batches that do not fit.  Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from . import systems

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _call_static(ctx, sid, th, B):
    logL = torch.empty(B, dtype=torch.float64, device="cuda")
    st = torch.empty(B, dtype=torch.int32, device="cuda")
    terms = torch.empty(B, 4, dtype=torch.float64, device="cuda")
    P = lambda t: C.c_void_p(t.data_ptr())
    rc = ctx.lib.glad_loglike_static(ctx.handle, P(sid), P(th), B, P(logL), P(st), P(terms),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, logL, st, terms


def test_static_scratch_matches_allocating_entry_point_twice():
    from paper_2504_01302_b300.glad import GladContext
    s = systems.small_system(7)
    ctx = GladContext([s])
    for seed in (31, 32):  # two calls in a row on different samples
        th_np = systems.prior_thetas(4, seed=seed)
        th_np[:2] = systems.near_truth_thetas(2, seed=seed)
        th = torch.as_tensor(th_np, device="cuda")
        sid = torch.zeros(4, dtype=torch.int32, device="cuda")
        rc, logL_s, st_s, terms_s = _call_static(ctx, sid, th, 4)
        assert rc == 0, ctx.lib.glad_last_error().decode()
        logL_a, st_a, terms_a = ctx.loglike(th, sid, terms=True)
        torch.cuda.synchronize()
        assert torch.equal(st_s, st_a)
        a, b = logL_a.cpu().numpy(), logL_s.cpu().numpy()
        for i in range(4):
            assert abs(a[i] - b[i]) < systems.logl_tol(a[i]), (i, a[i], b[i])
        ts, ta = terms_s.cpu().numpy(), terms_a.cpu().numpy()
        for i in range(4):
            for k in range(4):
                assert abs(ts[i, k] - ta[i, k]) < systems.logl_tol(ta[i, k]), (i, k, ts[i], ta[i])
    ctx.close()


def test_static_scratch_rejects_batches_beyond_its_size():
    from paper_2504_01302_b300.glad import GladContext
    s = systems.small_system(7)
    ctx = GladContext([s])
    B = 200000
    th = torch.zeros(1, 20, dtype=torch.float64, device="cuda")
    sid = torch.zeros(1, dtype=torch.int32, device="cuda")
    P = lambda t: C.c_void_p(t.data_ptr())
    rc = ctx.lib.glad_loglike_static(ctx.handle, P(sid), P(th), B, P(th), P(sid), None, None)
    assert rc == 5  # GLAD_EUNSUPPORTED, checked on the host before any launch
    assert "static array holds" in ctx.lib.glad_last_error().decode()
    ctx.close()
