"""glad_loglike_static: the log-likelihood for callers that cannot call cudaMalloc while
they run (code inside someone else's CUDA-graph capture, samplers under a fixed device
memory budget).  Its scratch is a static device array and it launches the kernels of
glad_loglike, so it must give the same logL and chi^2 terms as glad_loglike up to the
order of the FP64 atomic sums -- on two calls in a row, since every call reuses the array's
old contents -- for the cylindrically and the spherically aligned models in one batch, in
the grid and the persistent form of the JAM pair sum, and must refuse batches that do not
fit.  Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

from oracle import model
from paper_2504_01302_b300 import synth

from . import systems

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# The two entry points run the same kernels on the same inputs; only the order of the atomic
# additions (FP32 bin accumulators in shared memory, FP64 bin sums and chi^2 terms) can differ
# between runs, ~1e-7 relative in each chi^2 term.
REL = 1e-6


def _call_static(ctx, sid, th, B):
    logL = torch.empty(B, dtype=torch.float64, device="cuda")
    st = torch.empty(B, dtype=torch.int32, device="cuda")
    terms = torch.empty(B, 4, dtype=torch.float64, device="cuda")
    P = lambda t: C.c_void_p(t.data_ptr())
    rc = ctx.lib.glad_loglike_static(ctx.handle, P(sid), P(th), B, P(logL), P(st), P(terms),
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, logL, st, terms


def _near(a, b):
    a, b = np.asarray(a), np.asarray(b)
    fin = np.isfinite(a)
    assert np.array_equal(fin, np.isfinite(b))
    assert np.all(np.abs(a[fin] - b[fin]) <= REL * np.abs(a[fin]) + 1e-9), (a, b)


def _near_terms(a, b):
    """chi^2 terms of each sample, each within REL of the sample's total chi^2 (a small term
    amplifies the rounding of the residuals it squares; logL is what the bound is about)."""
    tot = np.sum(np.abs(a), axis=1, keepdims=True)
    assert np.all(np.abs(a - b) <= REL * tot + 1e-9), np.max(np.abs(a - b) / (tot + 1e-300))


def _sph_system(seed=7):
    b = dict(systems.small_base(seed), jam_align=1, sph_nr=40, sph_nw=6, sph_nlos=48)
    return model.build_system(b, synth.theta_truth(1), synth.noise_draws(b, 9100 + seed))


def _compare_twice(ctx, n_sys, B, seeds):
    for seed in seeds:  # two calls in a row on different samples
        th_np = systems.prior_thetas(B, seed=seed)
        th_np[: B // 2] = systems.near_truth_thetas(B // 2, seed=seed)
        th = torch.as_tensor(th_np, device="cuda")
        sid = torch.as_tensor(np.arange(B) % n_sys, dtype=torch.int32, device="cuda")
        rc, logL_s, st_s, terms_s = _call_static(ctx, sid, th, B)
        assert rc == 0, ctx.lib.glad_last_error().decode()
        assert ctx.lib.glad_last_error().decode() == ""
        logL_a, st_a, terms_a = ctx.loglike(th, sid, terms=True)
        torch.cuda.synchronize()
        assert torch.equal(st_s, st_a)
        assert int((st_a == 0).sum()) >= B // 2
        _near(logL_a.cpu().numpy(), logL_s.cpu().numpy())
        ok = (st_a == 0).cpu().numpy()
        _near_terms(terms_a.cpu().numpy()[ok], terms_s.cpu().numpy()[ok])


def test_static_scratch_matches_allocating_entry_point_twice():
    from paper_2504_01302_b300.glad import GladContext
    ctx = GladContext([systems.small_system(7)])
    _compare_twice(ctx, 1, 4, (31, 32))
    ctx.close()


def test_static_scratch_mixed_models_and_persistent_form():
    """A cylindrically and a spherically aligned system in one batch (the spherical model's
    slices of the scratch), first with the default grid form of the pair sum, then with the
    persistent work-list form pinned (its work list is carved from the scratch too)."""
    from paper_2504_01302_b300.glad import GladContext
    ctx = GladContext([systems.small_system(7), _sph_system(7)])
    _compare_twice(ctx, 2, 8, (41, 42))
    ctx.set_tuning(100000 + 8042, 4)  # the default shape (8 points, 4 CTAs, unroll 2), persistent
    _compare_twice(ctx, 2, 8, (43, 44))
    ctx.close()


def test_static_scratch_rejects_batches_beyond_its_size():
    from paper_2504_01302_b300.glad import GladContext
    s = systems.small_system(7)
    ctx = GladContext([s])
    B = 200000
    th = torch.zeros(1, 23, dtype=torch.float64, device="cuda")
    sid = torch.zeros(1, dtype=torch.int32, device="cuda")
    P = lambda t: C.c_void_p(t.data_ptr())
    rc = ctx.lib.glad_loglike_static(ctx.handle, P(sid), P(th), B, P(th), P(sid), None, None)
    assert rc == 5  # GLAD_EUNSUPPORTED, checked on the host before any launch
    assert "static array holds" in ctx.lib.glad_last_error().decode()
    ctx.close()
