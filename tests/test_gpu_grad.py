"""Gradient of the joint logL from the adjoint kernels against FP64 central finite
differences of the oracle (h = 1e-6 x parameter scale).

Tolerance per component (a reading of "relative 1e-3", undefined for components that
vanish): |g - g_ref| <= 1e-3 * max(|g_ref|, 1e-3 * max_i |g_ref,i|)."""
import math

import numpy as np
import pytest

from oracle import model
from paper_2504_01302_b300 import synth

from . import systems

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _ctx(sys_list):
    from paper_2504_01302_b300.glad import GladContext
    return GladContext(sys_list)


def _th(t):
    return torch.as_tensor(np.asarray(t, np.float64), device="cuda")


def assert_grad_close(g, ref, which=None):
    g = np.asarray(g, np.float64)
    ref = np.asarray(ref, np.float64)
    idx = range(len(ref)) if which is None else which
    floor = 1e-3 * np.max(np.abs(ref[list(idx)]))
    bad = []
    for i in idx:
        tol = 1e-3 * max(abs(ref[i]), floor)
        if not abs(g[i] - ref[i]) <= tol:
            bad.append((synth.THETA_NAMES[i], g[i], ref[i], abs(g[i] - ref[i]) / max(abs(ref[i]), 1e-300)))
    assert not bad, bad


@pytest.fixture(scope="module")
def small():
    s = systems.small_system(7)
    return s, _ctx([s])


def test_grad_near_truth_matches_oracle_fd(small):
    s, ctx = small
    th = systems.near_truth_thetas(2, seed=41)
    logL, grad, st = ctx.loglike_grad(_th(th))
    grad = grad.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    for b in range(len(th)):
        assert_grad_close(grad[b], model.grad_fd(th[b], s))


def test_grad_prior_draw_matches_oracle_fd(small):
    s, ctx = small
    th = systems.prior_thetas(1, seed=43)
    logL, grad, st = ctx.loglike_grad(_th(th))
    assert_grad_close(grad.cpu().numpy()[0], model.grad_fd(th[0], s))


def test_grad_logl_matches_forward_and_invalid_zero(small):
    s, ctx = small
    th = systems.near_truth_thetas(3, seed=45)
    th[2, synth.IDX["q"]] = 1.5  # invalid
    l1, st1 = ctx.loglike(_th(th))
    l2, g2, st2 = ctx.loglike_grad(_th(th))
    assert torch.equal(st1, st2)
    a, b = l1.cpu().numpy(), l2.cpu().numpy()
    assert abs(a[0] - b[0]) < 1e-6 * abs(a[0]) and abs(a[1] - b[1]) < 1e-6 * abs(a[1])
    assert np.isneginf(b[2]) and np.all(g2.cpu().numpy()[2] == 0)


def test_autograd_function(small):
    from paper_2504_01302_b300.glad import GladLogL
    s, ctx = small
    th = _th(systems.near_truth_thetas(2, seed=47)).requires_grad_(True)
    w = torch.tensor([0.3, -1.7], dtype=torch.float64, device="cuda")
    (GladLogL.apply(th, ctx) * w).sum().backward()
    _, g, _ = ctx.loglike_grad(th.detach())
    # FP64 atomics reorder between the two calls: compare with a floor at the gradient scale
    assert torch.allclose(th.grad, w[:, None] * g, rtol=1e-6, atol=1e-7 * float(g.abs().max()))


def test_grad_mixed_systems():
    sa = systems.small_system(7)
    sb = systems.small_system(8, n_px=36, ss=1, psf_k=5, sky=14, kss=4, n_mass=6, n_light=(6,),
                              n_gl=24, n_bins=9, n_sis=0, second_light=False, has_bh=False)
    ctx = _ctx([sa, sb])
    th = systems.near_truth_thetas(2, seed=49)
    sid = torch.as_tensor(np.array([1, 0], np.int32), device="cuda")
    _, g, st = ctx.loglike_grad(_th(th), sid)
    g = g.cpu().numpy()
    which = [i for i in range(synth.N_BASE) if synth.THETA_NAMES[i] not in ("upsilon", "f_bh")]
    assert_grad_close(g[0], model.grad_fd(th[0], sb), which=which)  # no BH: Upsilon, f_BH inert
    assert_grad_close(g[1], model.grad_fd(th[1], sa))


@pytest.fixture(scope="module")
def w1():
    sys_list, th, sid = systems.workload(1)
    return sys_list[0], th, _ctx(sys_list)


def test_w1_grad_full_batch_sampled(w1):
    # the benchmarked gradient launch (B = 64): every component of two of its samples, one
    # near the truth and one prior draw, against FP64 central differences of the oracle (the
    # 2 x 20 oracle evaluations of each spread over the host cores)
    s, th, ctx = w1
    th64 = systems.near_truth_thetas(64, seed=51)
    pri = systems.prior_thetas(32, seed=52)
    far = next(t for t in pri if model.check_domain(t) and model.dynamics_setup(t, s)[0] == 0)
    th64[37] = far
    _, g, st = ctx.loglike_grad(_th(th64))
    assert np.all(st.cpu().numpy() == 0)
    g = g.cpu().numpy()
    for b in (5, 37):
        assert_grad_close(g[b], systems.oracle_grad_fd_pool(th64[b], s))


def test_grad_with_image_position_term():
    s = dict(systems.small_system(7))
    s["img_sig"] = np.full(len(s["img_xy"]), 0.003)
    ctx = _ctx([s])
    th = systems.near_truth_thetas(1, seed=53)
    _, g, st = ctx.loglike_grad(_th(th))
    assert int(st.cpu().numpy()[0]) == 0
    assert_grad_close(g.cpu().numpy()[0], model.grad_fd(th[0], s))
