"""IFU-scale system (400^2 x 3 image, 31^2 PSF, EPL + shear + 2 SIS, JAM 40 + 2 x 20 + BH
on a 128^2 x 4 sky with GL64, 400 bins) at its full size and batch (B = 4096).

The oracle evaluates this system one output at a time: the model image (1.44 M
sub-pixels), the delays, and v_rms of chosen bins through oracle.model.vrms_bins.  The
full v_rms map is out of its reach, so chi^2_dyn of the full batch is checked through the
GPU's own v_rms (a property of the reduction); the gradient is checked against central
differences of the oracle: its imaging + delay terms for parameters that only enter those,
and, on a copy of the system that keeps two bins, its restricted v_rms for the dynamics
parameters.  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

from oracle import imaging, kin, model, tdelay
from paper_2504_01302_b300 import synth

from . import systems
from .test_gpu_parity import assert_image_close, assert_vrms_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

I = synth.IDX


def _th(t):
    return torch.as_tensor(np.asarray(t, np.float64), device="cuda")


@pytest.fixture(scope="module")
def ifu():
    from paper_2504_01302_b300.glad import GladContext
    s = systems.ifu_system()
    return s, GladContext([s])


def test_ifu_image_matches_oracle(ifu):
    s, ctx = ifu
    th = systems.near_truth_thetas(1, seed=61)[0]
    g = ctx.model_image(_th(th)).cpu().numpy()
    assert_image_close(g, imaging.model_image(th, s))


def test_ifu_vrms_two_bins_match_oracle(ifu):
    s, ctx = ifu
    th = systems.near_truth_thetas(1, seed=63)[0]
    lab = np.asarray(s["bins"])
    ky, kx = lab.shape
    which = [int(lab[ky // 2, kx // 2]), int(s["n_bins"]) - 1]  # central bin, last (outer) bin
    ref, st = model.vrms_bins(th, s, which)
    assert st == model.ST_OK
    g = ctx.vrms(_th(th)).cpu().numpy()
    assert_vrms_close(g[which], ref)


def test_ifu_full_batch_sampled(ifu):
    # the full batch in one call; sampled samples against the oracle term by term
    s, ctx = ifu
    th, _ = synth.workload_thetas(4, 4096, 1)
    logL, status, terms = ctx.loglike(_th(th), terms=True)
    logL, status, terms = logL.cpu().numpy(), status.cpu().numpy(), terms.cpu().numpy()
    # status codes of the first 64 samples (domain, deprojection and density checks)
    for b in range(64):
        ref = model.ST_DOMAIN if not model.check_domain(th[b]) else model.dynamics_setup(th[b], s)[0]
        if ref == model.ST_OK:
            assert status[b] == 0 or status[b] == model.ST_NONFINITE, (b, status[b])
        else:
            assert status[b] == ref, (b, status[b], ref)
            assert np.isneginf(logL[b])
    ok = np.flatnonzero(status == 0)
    assert len(ok) > 0.5 * len(th)
    for b in (ok[0], ok[len(ok) // 2], ok[-1]):
        c_pix = imaging.chi2_pix(imaging.model_image(th[b], s), s)
        c_tmd = tdelay.chi2_tmd(tdelay.delays(th[b], s), s)
        assert abs(terms[b, 0] - c_pix) <= 2 * systems.logl_tol(0.5 * c_pix), (b, terms[b, 0], c_pix)
        assert abs(terms[b, 2] - c_tmd) <= 1e-6 * max(abs(c_tmd), 1.0), (b, terms[b, 2], c_tmd)
        v = ctx.vrms(_th(th[b])).cpu().numpy().astype(np.float64)
        # the batch and the single-sample call sum the bins in different orders (FP32 partial
        # sums): ~1e-7 relative in v, ~1e-5 of a chi^2 whose residuals are ~5 sigma
        assert abs(terms[b, 1] - kin.chi2_dyn(v, s)) <= 1e-4 * terms[b, 1]
        assert abs(logL[b] + 0.5 * terms[b].sum()) <= 1e-9 * abs(logL[b])
        # the same sample alone gives the same logL
        l1, s1 = ctx.loglike(_th(th[b:b + 1]))
        assert int(s1[0]) == 0 and abs(float(l1[0]) - logL[b]) <= 1e-6 * abs(logL[b])


def test_ifu_gradient(ifu):
    s, ctx = ifu
    # sample 0 near the truth; sample 1 a prior draw that passes the dynamics checks
    pri = systems.prior_thetas(16, seed=67)
    far = next(t for t in pri if model.check_domain(t) and model.dynamics_setup(t, s)[0] == 0)
    th = np.vstack([systems.near_truth_thetas(1, seed=65), far[None]])
    L0, g, st = ctx.loglike_grad(_th(th))
    assert np.all(st.cpu().numpy() == 0)
    g = g.cpu().numpy()
    # parameters that enter only the image and the delays: oracle central differences
    for b in (0, 1):
        for name in ("x_src", "R_e_src", "gamma_ext"):
            i = I[name]
            h = 1e-6 * synth.THETA_SCALE[i]
            f = []
            for sgn in (1, -1):
                t = th[b].copy()
                t[i] += sgn * h
                f.append(-0.5 * (imaging.chi2_pix(imaging.model_image(t, s), s) +
                                 tdelay.chi2_tmd(tdelay.delays(t, s), s)))
            ref = (f[0] - f[1]) / (2 * h)
            assert abs(g[b, i] - ref) <= 1e-3 * abs(ref) + 1e-2, (b, name, g[b, i], ref)


def test_ifu_gradient_dynamics_against_oracle(ifu):
    """The dynamics components of the IFU-scale gradient against FP64 central differences of
    the oracle.  A copy of the system keeps two bins (the central one and the outermost),
    so chi^2_dyn is a sum the oracle's restricted v_rms evaluates exactly; the gradient of
    the image and delay terms (which only theta_E of these parameters enters) comes from
    the oracle's image and delays."""
    from paper_2504_01302_b300.glad import GladContext
    s, _ = ifu
    lab = np.asarray(s["bins"])
    ky, kx = lab.shape
    s2 = systems.keep_bins(s, [int(lab[ky // 2, kx // 2]), int(s["n_bins"]) - 1])
    ctx = GladContext([s2])
    th = systems.near_truth_thetas(1, seed=65)[0]
    _, g, st = ctx.loglike_grad(_th(th[None]))
    assert int(st.cpu().numpy()[0]) == 0
    g = g.cpu().numpy()[0]
    which = [I[n] for n in ("theta_E", "inc", "beta", "upsilon", "f_bh")]
    ref = systems.oracle_dyn_grad_fd_pool(th, s2, which)
    i = I["theta_E"]
    h = 1e-6 * synth.THETA_SCALE[i]
    f = []
    for sgn in (1, -1):
        t = th.copy()
        t[i] += sgn * h
        f.append(-0.5 * (imaging.chi2_pix(imaging.model_image(t, s2), s2) +
                         tdelay.chi2_tmd(tdelay.delays(t, s2), s2)))
    ref[i] += (f[0] - f[1]) / (2 * h)
    for i in which:
        assert abs(g[i] - ref[i]) <= 1e-3 * max(abs(ref[i]), 1e-3 * np.max(np.abs(ref[which]))), \
            (synth.THETA_NAMES[i], g[i], ref[i])
