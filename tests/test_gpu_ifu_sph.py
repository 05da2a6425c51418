"""IFU-scale system (400^2 x 3 image, 31^2 PSF, EPL + shear + 2 SIS, JAM 40 + 2 x 20 + BH on a
128^2 x 4 sky with GL64, 400 bins) with the spherically aligned Jeans model (Eqs. J1/J2,
polar grid 128 x 8, 32 line-of-sight nodes), at its full size and batch (B = 4096).

As for the cylindrical model at this size (test_gpu_ifu), the oracle computes v_rms of
chosen bins through oracle.model.vrms_bins (here its polar grid in full and the line of
sight only on the sub-samples that PSF_kin carries into those bins); chi^2_dyn of the
full batch is checked through the library's own v_rms, the gradient of the dynamics
parameters through central differences of the library's logL.  Tolerances as in
test_gpu_parity."""
import numpy as np
import pytest

from oracle import kin, model
from paper_2504_01302_b300 import synth

from . import systems
from .test_gpu_parity import assert_vrms_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

I = synth.IDX


def _th(t):
    return torch.as_tensor(np.asarray(t, np.float64), device="cuda")


@pytest.fixture(scope="module")
def ifu():
    from paper_2504_01302_b300.glad import GladContext
    s = dict(systems.ifu_system(), jam_align=1, sph_nr=128, sph_nw=8, sph_nlos=32)
    return s, GladContext([s])


def test_ifu_sph_vrms_two_bins_match_oracle(ifu):
    s, ctx = ifu
    th = systems.near_truth_thetas(1, seed=61)[0]
    lab = np.asarray(s["bins"])
    ky, kx = lab.shape
    which = [int(lab[ky // 2, kx // 2]), int(s["n_bins"]) - 1]  # central bin, last (outer) bin
    ref, st = model.vrms_bins(th, s, which)
    assert st == model.ST_OK
    assert_vrms_close(ctx.vrms(_th(th)).cpu().numpy()[which], ref)


def test_ifu_sph_full_batch_sampled(ifu):
    s, ctx = ifu
    th, _ = synth.workload_thetas(6, 4096, 1)
    logL, status, terms = ctx.loglike(_th(th), terms=True)
    logL, status, terms = logL.cpu().numpy(), status.cpu().numpy(), terms.cpu().numpy()
    for b in range(64):
        ref = model.ST_DOMAIN if not model.check_domain(th[b]) else model.dynamics_setup(th[b], s)[0]
        if ref == model.ST_OK:
            assert status[b] == 0 or status[b] == model.ST_NONFINITE, (b, status[b])
        else:
            assert status[b] == ref, (b, status[b], ref)
    ok = np.flatnonzero(status == 0)
    assert len(ok) > 0.5 * len(th)
    for b in (ok[0], ok[-1]):
        v = ctx.vrms(_th(th[b])).cpu().numpy().astype(np.float64)
        assert abs(terms[b, 1] - kin.chi2_dyn(v, s)) <= 1e-4 * terms[b, 1]
        l1, s1 = ctx.loglike(_th(th[b:b + 1]))
        assert int(s1[0]) == 0 and abs(float(l1[0]) - logL[b]) <= 1e-6 * abs(logL[b])


def test_ifu_sph_gradient(ifu):
    s, ctx = ifu
    th = systems.near_truth_thetas(1, seed=65)
    _, g, st = ctx.loglike_grad(_th(th))
    assert int(st.cpu().numpy()[0]) == 0
    g = g.cpu().numpy()[0]
    # dynamics parameters (and theta_E): central differences of the library's logL, with the
    # FD error of a logL noise of 0.05 added to the bound
    for name in ("theta_E", "inc", "beta", "upsilon"):
        i = I[name]
        h = 1e-3 * synth.THETA_SCALE[i]
        tp, tm = th[0].copy(), th[0].copy()
        tp[i] += h
        tm[i] -= h
        lp, _ = ctx.loglike(_th(tp[None]))
        lm, _ = ctx.loglike(_th(tm[None]))
        fd = (float(lp[0]) - float(lm[0])) / (2 * h)
        assert abs(g[i] - fd) <= 1e-2 * abs(fd) + 0.05 / h, (name, g[i], fd)
