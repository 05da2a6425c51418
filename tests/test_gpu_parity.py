"""GPU (libglad, through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: model pixel relative 1e-4 with an absolute floor of 1e-6 * max|m|;
v_rms per bin relative 1e-4; logL absolute 0.05 near the posterior, and
0.05 + 5e-6 |logL| at arbitrary prior draws (tests/systems.logl_tol).
"""
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


def assert_image_close(g, o):
    g = np.asarray(g, np.float64)
    tol = 1e-4 * np.abs(o) + 1e-6 * np.max(np.abs(o))
    err = np.abs(g - o)
    assert np.all(err <= tol), f"max rel err {np.max(err / (np.abs(o) + 1e-30)):.3e}"


def assert_vrms_close(g, o):
    rel = np.abs(np.asarray(g, np.float64) / o - 1)
    assert np.max(rel) < 1e-4, f"max rel err {np.max(rel):.3e}"


# ------------------------------------------------------------------ workload 0

@pytest.fixture(scope="module")
def w0():
    sys_list, th, sid = systems.workload(0)
    return sys_list[0], th[0], _ctx(sys_list)


def test_w0_model_image(w0):
    s, th, ctx = w0
    o = model.evaluate(th, s)["image"]
    g = ctx.model_image(_th(th)).cpu().numpy()
    assert_image_close(g, o)


def test_w0_vrms(w0):
    s, th, ctx = w0
    o = model.evaluate(th, s)["vrms"]
    g = ctx.vrms(_th(th)).cpu().numpy()
    assert_vrms_close(g, o)


def test_w0_loglike_and_terms(w0):
    s, th, ctx = w0
    ev = model.evaluate(th, s)
    logL, st, terms = ctx.loglike(_th(th[None, :]), terms=True)
    assert int(st[0]) == 0
    assert abs(float(logL[0]) - ev["logL"]) < 0.05
    t = terms[0].cpu().numpy()
    assert abs(t[0] - ev["chi2_pix"]) < 0.05
    assert abs(t[1] - ev["chi2_dyn"]) < 0.01
    assert abs(t[2] - ev["chi2_tmd"]) < 1e-6 * max(1.0, ev["chi2_tmd"])


# ------------------------------------------------------------------ small, all features

@pytest.fixture(scope="module")
def small():
    s = systems.small_system(7)
    return s, _ctx([s])


def test_small_near_truth_absolute_005(small):
    s, ctx = small
    th = systems.near_truth_thetas(6)
    logL, st, terms = ctx.loglike(_th(th), terms=True)
    logL, terms = logL.cpu().numpy(), terms.cpu().numpy()
    for b in range(len(th)):
        ev = model.evaluate(th[b], s)
        assert ev["status"] == int(st[b]) == 0
        assert abs(logL[b] - ev["logL"]) < 0.05, (b, logL[b], ev["logL"])


def test_small_prior_batch_matches_oracle(small):
    s, ctx = small
    th = systems.prior_thetas(6)
    logL, st, terms = ctx.loglike(_th(th), terms=True)
    logL, terms = logL.cpu().numpy(), terms.cpu().numpy()
    for b in range(len(th)):
        ev = model.evaluate(th[b], s)
        assert ev["status"] == int(st[b]) == 0
        assert abs(logL[b] - ev["logL"]) < systems.logl_tol(ev["logL"]), (b, logL[b], ev["logL"])
        assert abs(terms[b, 1] - ev["chi2_dyn"]) < systems.logl_tol(ev["chi2_dyn"])
        assert abs(terms[b, 2] - ev["chi2_tmd"]) < 1e-7 * max(1.0, ev["chi2_tmd"])


def test_small_image_and_vrms_at_prior_draws(small):
    s, ctx = small
    for th in systems.prior_thetas(3, seed=21):
        ev = model.evaluate(th, s)
        assert_image_close(ctx.model_image(_th(th)).cpu().numpy(), ev["image"])
        assert_vrms_close(ctx.vrms(_th(th)).cpu().numpy(), ev["vrms"])


def test_invalid_samples_get_status_and_minus_inf(small):
    s, ctx = small
    base = systems.prior_thetas(1)[0]
    rows, want = [], []
    for name, val, st in [("q", 1.3, model.ST_DOMAIN), ("gamma", 3.2, model.ST_DOMAIN),
                          ("inc", math.radians(25), model.ST_DEPROJ), ("beta", 1.2, model.ST_DOMAIN),
                          ("H0", float("nan"), model.ST_DOMAIN)]:
        t = base.copy()
        t[synth.IDX[name]] = val
        rows.append(t)
        want.append(st)
    rows.append(base)
    want.append(0)
    logL, st = ctx.loglike(_th(np.array(rows)))
    assert list(st.cpu().numpy()) == want
    L = logL.cpu().numpy()
    assert np.all(np.isneginf(L[:-1])) and np.isfinite(L[-1])


def test_mixed_systems_in_one_batch():
    sa = systems.small_system(7)
    sb = systems.small_system(8, n_px=36, ss=1, psf_k=5, sky=14, kss=4, n_mass=6, n_light=(6,),
                              n_gl=24, n_bins=9, n_sis=0, second_light=False, has_bh=False)
    ctx = _ctx([sa, sb])
    th = systems.near_truth_thetas(8, seed=5)
    sid = np.array([0, 1, 1, 0, 1, 0, 0, 1], np.int32)
    logL, st = ctx.loglike(_th(th), torch.as_tensor(sid, device="cuda"))
    logL = logL.cpu().numpy()
    for b in range(len(th)):
        ev = model.evaluate(th[b], [sa, sb][sid[b]])
        assert abs(logL[b] - ev["logL"]) < 0.05, (b, logL[b], ev["logL"])


def test_psf_sides_in_every_convolution_form():
    # PSF sides 5 and 21 (blocked kernel, padded to 11 and 21), 31 (blocked, exact side) and
    # 35 (general kernel) in one batch: model images and logL against the oracle
    sys_list = [systems.small_system(20 + k, n_px=48 if k < 35 else 64, psf_k=k, n_bins=9)
                for k in (5, 21, 31, 35)]
    ctx = _ctx(sys_list)
    th = systems.near_truth_thetas(4, seed=9)
    sid = np.arange(4, dtype=np.int32)
    logL, st = ctx.loglike(_th(th), torch.as_tensor(sid, device="cuda"))
    logL = logL.cpu().numpy()
    for b, s in enumerate(sys_list):
        ev = model.evaluate(th[b], s)
        assert abs(logL[b] - ev["logL"]) < 0.05, (s["psf"].shape, logL[b], ev["logL"])
        assert_image_close(ctx.model_image(_th(th[b]), b).cpu().numpy(), ev["image"])


def test_degenerate_parameters_match_oracle(small):
    # the method's special cases: a round EPL (q = 1, no series terms), the SIE (gamma' = 2),
    # isotropy (beta = 0), edge-on (i = 90 deg), no black hole mass (f_BH = 0), no external
    # shear, the galaxy frame on the sky axes with the lens at the origin; one sample alone
    # (B = 1) and all together
    s, ctx = small
    I = synth.IDX
    base = systems.near_truth_thetas(1, seed=17)[0]
    cases = []
    for changes in ({"q": 1.0, "gamma": 2.0, "beta": 0.0},
                    {"inc": math.pi / 2, "f_bh": 0.0, "gamma_ext": 0.0},
                    {"phi": 0.0, "x_c": 0.0, "y_c": 0.0, "q": 1.0},
                    {"gamma": 2.0, "beta": 0.0, "inc": math.pi / 2, "f_bh": 0.0}):
        t = base.copy()
        for k, v in changes.items():
            t[I[k]] = v
        cases.append(t)
    th = np.array(cases)
    logL, st = ctx.loglike(_th(th))
    logL, st = logL.cpu().numpy(), st.cpu().numpy()
    for b, t in enumerate(th):
        ev = model.evaluate(t, s)
        assert st[b] == ev["status"] == model.ST_OK, (b, st[b], ev["status"])
        assert abs(logL[b] - ev["logL"]) < systems.logl_tol(ev["logL"]), (b, logL[b], ev["logL"])
        one, st1 = ctx.loglike(_th(t[None]))
        assert int(st1[0]) == 0 and abs(float(one[0]) - logL[b]) < 1e-6 * abs(logL[b])
        assert_image_close(ctx.model_image(_th(t)).cpu().numpy(), ev["image"])
        assert_vrms_close(ctx.vrms(_th(t)).cpu().numpy(), ev["vrms"])


def test_degenerate_parameters_gradient(small):
    # interior special cases (gamma' = 2, beta = 0, f_BH = 0 away from its bound for the FD
    # step: the oracle differences are central) against oracle central differences
    from .test_gpu_grad import assert_grad_close
    s, ctx = small
    I = synth.IDX
    t = systems.near_truth_thetas(1, seed=19)[0]
    t[I["gamma"]] = 2.0
    t[I["beta"]] = 0.0
    logL, g, st = ctx.loglike_grad(_th(t[None]))
    assert int(st[0]) == 0
    assert_grad_close(g.cpu().numpy()[0], model.grad_fd(t, s))


def test_image_position_term():
    # a system that gives image-position errors: chi^2_img joins logL (fourth term)
    s = dict(systems.small_system(7))
    s["img_sig"] = np.full(len(s["img_xy"]), 0.003)
    ctx = _ctx([s])
    th = np.vstack([systems.near_truth_thetas(3, seed=23), synth.theta_truth(1)[None]])
    logL, st, terms = ctx.loglike(_th(th), terms=True)
    logL, terms = logL.cpu().numpy(), terms.cpu().numpy()
    for b in range(len(th)):
        ev = model.evaluate(th[b], s)
        assert abs(terms[b, 3] - ev["chi2_img"]) <= 1e-9 * ev["chi2_img"] + 1e-12, (b, terms[b, 3], ev["chi2_img"])
        assert abs(logL[b] - ev["logL"]) < 0.05, (b, logL[b], ev["logL"])
    assert terms[3, 3] < 1e-12  # exact images at the truth
    # the same system without img_sig: fourth term 0, logL higher by chi^2_img / 2
    s0 = dict(s)
    del s0["img_sig"]
    l0, _, t0 = _ctx([s0]).loglike(_th(th), terms=True)
    t0 = t0.cpu().numpy()
    assert np.all(t0[:, 3] == 0.0)
    # the other three terms agree (to the run-to-run order of float atomics) and each logL
    # is -1/2 the sum of its terms
    assert np.allclose(t0[:, :3], terms[:, :3], rtol=1e-6, atol=1e-4)
    assert np.allclose(logL, -0.5 * terms.sum(axis=1), rtol=1e-12)
    assert np.allclose(l0.cpu().numpy(), -0.5 * t0.sum(axis=1), rtol=1e-12)


def test_batch_independence(small):
    # a sample's logL does not depend on which other samples share the launch
    s, ctx = small
    th = systems.prior_thetas(5, seed=3)
    full = ctx.loglike(_th(th))[0].cpu().numpy()
    for b in [0, 4]:
        one = ctx.loglike(_th(th[b:b + 1]))[0].cpu().numpy()[0]
        assert abs(one - full[b]) < 1e-9 * max(1.0, abs(full[b]))


# ------------------------------------------------------------------ workload 1, full size

@pytest.fixture(scope="module")
def w1():
    sys_list, th, sid = systems.workload(1)
    return sys_list[0], th, _ctx(sys_list)


def test_w1_full_batch_sampled_against_oracle(w1):
    s, th, ctx = w1
    logL, st, terms = ctx.loglike(_th(th), terms=True)  # B = 256, the benchmarked launch
    logL, terms = logL.cpu().numpy(), terms.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    for b in [0, 137]:
        ev = model.evaluate(th[b], s)
        assert abs(logL[b] - ev["logL"]) < systems.logl_tol(ev["logL"]), (b, logL[b], ev["logL"])
        assert abs(terms[b, 1] - ev["chi2_dyn"]) < systems.logl_tol(ev["chi2_dyn"])


def test_w1_near_truth_absolute_005(w1):
    s, _, ctx = w1
    th = systems.near_truth_thetas(2, seed=17)
    logL = ctx.loglike(_th(th))[0].cpu().numpy()
    for b in range(2):
        ev = model.evaluate(th[b], s)
        assert abs(logL[b] - ev["logL"]) < 0.05, (b, logL[b], ev["logL"])


def test_w1_image_and_vrms_one_sample(w1):
    s, th, ctx = w1
    ev = model.evaluate(th[3], s)
    assert_image_close(ctx.model_image(_th(th[3])).cpu().numpy(), ev["image"])
    assert_vrms_close(ctx.vrms(_th(th[3])).cpu().numpy(), ev["vrms"])
