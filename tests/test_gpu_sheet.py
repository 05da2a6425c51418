"""The internal mass sheet of the mass class and the sampled distances (Sect. 3.3, Eqs. kappa
int and dpie_kappa; Sect. 2.3, Eq. sfd final; Table 2) through the C ABI against the oracle:
model image per pixel, v_rms per bin, logL and the chi^2 terms, status codes (lambda_int > 1
turns the EPL class's outer density negative: GLAD_SAMPLE_NEGDENS), every used gradient
component against oracle differences, the spherically aligned model with the sheet, the
exact mass-sheet transform of the model image under the ideal sheet, and the RXJ1131-scale
sheet workload's launch on sampled samples.  Tolerances as in test_gpu_parity."""
import numpy as np
import pytest

from oracle import model
from paper_2504_01302_b300 import synth

from . import systems
from .test_gpu_grad import assert_grad_close
from .test_gpu_parity import assert_image_close, assert_vrms_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

I = synth.IDX


def _th(t):
    return torch.as_tensor(np.asarray(t, np.float64), device="cuda")


def _ctx(sys_list):
    from paper_2504_01302_b300.glad import GladContext
    return GladContext(sys_list)


def sheet_truth():
    t = synth.theta_truth(1).copy()
    t[I["lam_int"]] = 0.9
    return t


def sheet_small(seed=7, **kw):
    """The small all-features system as the EPL class with the dPIE sheet in distance mode 1,
    data from the oracle at a truth with lambda_int = 0.9."""
    b = dict(systems.small_base(seed), sheet=1, distance_mode=1, **kw)
    return model.build_system(b, sheet_truth(), synth.noise_draws(b, 9300 + seed))


def near(n, seed):
    th = systems.near_truth_thetas(n, seed=seed)
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    th[:, I["lam_int"]] = 0.9 + 0.01 * rng.standard_normal(n)
    th[:, I["D_d"]] = 775.0 * (1 + 0.01 * rng.standard_normal(n))
    th[:, I["D_dt_int"]] = 1823.0 * (1 + 0.01 * rng.standard_normal(n))
    th[:, I["H0"]] = np.nan  # unused in distance mode 1
    return th


@pytest.fixture(scope="module")
def small():
    s = sheet_small(7)
    return s, _ctx([s])


def test_image_vrms_logl_near_truth(small):
    s, ctx = small
    th = near(2, 81)
    logL, st, terms = ctx.loglike(_th(th), terms=True)
    logL, terms = logL.cpu().numpy(), terms.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    for b in range(2):
        ev = model.evaluate(th[b], s)
        assert ev["status"] == 0
        assert_image_close(ctx.model_image(_th(th[b])).cpu().numpy(), ev["image"])
        assert_vrms_close(ctx.vrms(_th(th[b])).cpu().numpy(), ev["vrms"])
        assert abs(logL[b] - ev["logL"]) < 0.05, (b, logL[b], ev["logL"])
        assert abs(terms[b, 2] - ev["chi2_tmd"]) <= 1e-7 * max(1.0, ev["chi2_tmd"])


def test_prior_draws_statuses_and_negative_density(small):
    s, ctx = small
    rng = np.random.Generator(np.random.PCG64(83))
    th = synth.draw_prior_sheet(rng, 12)  # lambda_int in [0.5, 1.5] (Table 2)
    th[3, I["lam_int"]] = 1.3             # sure to be rejected (negative outer density)
    th[4, I["lam_int"]] = 0.7
    logL, st = ctx.loglike(_th(th))
    logL, st = logL.cpu().numpy(), st.cpu().numpy()
    n_neg = n_ok = 0
    for b in range(len(th)):
        ev = model.evaluate(th[b], s)
        assert st[b] == ev["status"], (b, st[b], ev["status"], th[b, I["lam_int"]])
        if ev["status"] == 0:
            n_ok += 1
            assert abs(logL[b] - ev["logL"]) < systems.logl_tol(ev["logL"]), (b, logL[b], ev["logL"])
        else:
            assert np.isneginf(logL[b])
            n_neg += ev["status"] == model.ST_NEGDENS
    assert st[3] == model.ST_NEGDENS and n_neg >= 1 and n_ok >= 2


def test_gradient_every_used_component(small):
    s, ctx = small
    th = near(1, 85)
    _, g, st = ctx.loglike_grad(_th(th))
    assert int(st.cpu().numpy()[0]) == 0
    g = g.cpu().numpy()[0]
    used = model.used_params(s)
    assert I["lam_int"] in used and I["D_dt_int"] in used and I["H0"] not in used
    assert_grad_close(g, systems.oracle_grad_fd_pool(th[0], s), which=used)
    assert g[I["H0"]] == 0.0


def test_spherically_aligned_model_with_sheet():
    s = sheet_small(7, jam_align=1, sph_nr=40, sph_nw=6, sph_nlos=48)
    ctx = _ctx([s])
    th = near(1, 87)[0]
    ev = model.evaluate(th, s)
    assert ev["status"] == 0
    assert_vrms_close(ctx.vrms(_th(th)).cpu().numpy(), ev["vrms"])
    logL = float(ctx.loglike(_th(th[None]))[0][0])
    assert abs(logL - ev["logL"]) < 0.05


def test_ideal_sheet_leaves_the_image_unchanged():
    """The mass-sheet transform (Eq. transformed MST): with the ideal sheet, lambda_int and a
    source moved and resized as beta -> lambda beta + (1 - lambda) c give the same model image
    (up to FP32 ray-shooting rounding)."""
    s = dict(systems.small_system(7), sheet=2)
    ctx = _ctx([s])
    t = systems.near_truth_thetas(1, seed=89)[0]
    t[I["lam_int"]] = 1.0
    m0 = ctx.model_image(_th(t)).cpu().numpy()
    # lambda < 1: the dynamics (which every call prepares) take the dPIE in place of the ideal
    # sheet, and above 1 it is negative and the sample rejected
    for lam in (0.8, 0.9):
        t2 = t.copy()
        t2[I["lam_int"]] = lam
        t2[I["x_src"]] = lam * t[I["x_src"]] + (1 - lam) * t[I["x_c"]]
        t2[I["y_src"]] = lam * t[I["y_src"]] + (1 - lam) * t[I["y_c"]]
        t2[I["R_e_src"]] = lam * t[I["R_e_src"]]
        m1 = ctx.model_image(_th(t2)).cpu().numpy()
        assert np.max(np.abs(m1 - m0)) <= 1e-5 * np.max(np.abs(m0)), np.max(np.abs(m1 - m0))


@pytest.fixture(scope="module")
def w7():
    sys_list, th, sid = systems.workload(7)
    return sys_list[0], th, _ctx(sys_list)


def test_w7_full_batch_sampled_against_oracle(w7):
    s, th, ctx = w7
    logL, st, terms = ctx.loglike(_th(th), terms=True)  # B = 256, the benchmarked launch
    logL, st, terms = logL.cpu().numpy(), st.cpu().numpy(), terms.cpu().numpy()
    ok = np.flatnonzero(st == 0)
    assert len(ok) > len(th) // 2
    for b in (ok[0], ok[len(ok) // 2]):
        ev = model.evaluate(th[b], s)
        assert ev["status"] == 0
        assert abs(logL[b] - ev["logL"]) < systems.logl_tol(ev["logL"]), (b, logL[b], ev["logL"])
        assert_vrms_close(ctx.vrms(_th(th[b])).cpu().numpy(), ev["vrms"])
    bad = np.flatnonzero(st != 0)[:3]
    for b in bad:
        assert model.evaluate(th[b], s)["status"] == st[b]
