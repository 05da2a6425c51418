"""The composite mass class (Sect. 3.3: kappa_int,comp = (1 - lambda_int) + lambda_int
(Upsilon_* I_light + kappa_enfw + kappa_BH), Eqs. Chameleon and kappa_enfw, App. B) with the dPIE
sheet and sampled distances, through the C ABI against the oracle: model image per pixel,
v_rms per bin, logL, chi^2 terms and status codes, every used gradient component against
oracle differences, the spherically aligned model, the mass-sheet transform of the image under
the ideal sheet, and the RXJ1131-scale composite workload's launch on sampled samples.
Tolerances as in test_gpu_parity plus the term of the two paths' own fits of the halo's CSE
decomposition (tests/systems.logl_tol_comp: up to 4e-7 of the NFW profile apart)."""
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


def comp_truth():
    t = synth.theta_truth_composite()
    t[I["lam_int"]] = 0.9
    return t


def comp_small(seed=7, sheet=1, **kw):
    """The small all-features system as the composite class with the dPIE sheet in distance
    mode 1, data from the oracle at a truth with lambda_int = 0.9."""
    b = synth.composite_light(dict(systems.small_base(seed), sheet=sheet, distance_mode=1, **kw))
    return model.build_system(b, comp_truth(), synth.noise_draws(b, 9500 + seed))


def near(n, seed):
    th = np.tile(comp_truth(), (n, 1))
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = synth.PRIOR_LO.copy()
    hi = synth.PRIOR_HI.copy()
    for i, (a, c) in synth.COMPOSITE_PRIOR.items():
        lo[i], hi[i] = a, c
    lo[I["lam_int"]], hi[I["lam_int"]] = 0.5, 1.0
    lo[I["D_d"]], hi[I["D_d"]] = 600.0, 1000.0
    span = hi - lo
    th += 0.002 * span * rng.standard_normal(th.shape)
    th[:, I["f_bh"]] = np.abs(th[:, I["f_bh"]])
    th[:, I["inc"]] = np.minimum(th[:, I["inc"]], np.pi / 2)
    th[:, I["q"]] = np.minimum(th[:, I["q"]], 1.0)
    th[:, I["H0"]] = np.nan  # unused in distance mode 1
    return th


@pytest.fixture(scope="module")
def small():
    s = comp_small(7)
    return s, _ctx([s])


def test_image_vrms_logl_near_truth(small):
    s, ctx = small
    th = near(2, 91)
    logL, st, terms = ctx.loglike(_th(th), terms=True)
    logL, terms = logL.cpu().numpy(), terms.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    for b in range(2):
        ev = model.evaluate(th[b], s)
        assert ev["status"] == 0
        assert_image_close(ctx.model_image(_th(th[b])).cpu().numpy(), ev["image"])
        assert_vrms_close(ctx.vrms(_th(th[b])).cpu().numpy(), ev["vrms"])
        assert abs(logL[b] - ev["logL"]) < 0.05, (b, logL[b], ev["logL"])
        # the two CSE fits move Fermat-potential differences by ~1e-6 of themselves
        assert abs(terms[b, 2] - ev["chi2_tmd"]) <= 1e-4 * max(1.0, ev["chi2_tmd"])


def test_prior_draws_and_statuses(small):
    s, ctx = small
    rng = np.random.Generator(np.random.PCG64(93))
    th = synth.draw_prior_composite(rng, 10, lam_hi=1.5)
    th[2, I["lam_int"]] = 1.3  # negative outer density
    th[3, I["q"]] = 1.2        # outside the domain
    logL, st = ctx.loglike(_th(th))
    logL, st = logL.cpu().numpy(), st.cpu().numpy()
    n_ok = 0
    for b in range(len(th)):
        ev = model.evaluate(th[b], s)
        assert st[b] == ev["status"], (b, st[b], ev["status"])
        if ev["status"] == 0:
            n_ok += 1
            assert abs(logL[b] - ev["logL"]) < systems.logl_tol_comp(ev["logL"]), (b, logL[b], ev["logL"])
        else:
            assert np.isneginf(logL[b])
    assert st[2] == model.ST_NEGDENS and st[3] == model.ST_DOMAIN and n_ok >= 2


def test_gradient_every_used_component(small):
    s, ctx = small
    th = near(1, 95)
    _, g, st = ctx.loglike_grad(_th(th))
    assert int(st.cpu().numpy()[0]) == 0
    g = g.cpu().numpy()[0]
    used = model.used_params(s)
    ref = systems.oracle_grad_fd_pool(th[0], s)
    # per component 1e-3 relative, with a floor of 1e-4 of the gradient's scale: the two CSE
    # fits shift the small components (source amplitude, lambda_int) by ~2e-5 of that scale
    floor = 1e-4 * np.max(np.abs(ref[used]))
    bad = [(synth.THETA_NAMES[i], g[i], ref[i]) for i in used
           if not abs(g[i] - ref[i]) <= max(1e-3 * abs(ref[i]), floor)]
    assert not bad, bad


def test_spherically_aligned_model():
    s = comp_small(7, jam_align=1, sph_nr=40, sph_nw=6, sph_nlos=48)
    ctx = _ctx([s])
    th = near(1, 97)[0]
    ev = model.evaluate(th, s)
    assert ev["status"] == 0
    assert_vrms_close(ctx.vrms(_th(th)).cpu().numpy(), ev["vrms"])
    assert abs(float(ctx.loglike(_th(th[None]))[0][0]) - ev["logL"]) < 0.05


def test_ideal_sheet_leaves_the_composite_image_unchanged():
    s = comp_small(7, sheet=2)
    ctx = _ctx([s])
    t = near(1, 99)[0]
    t[I["lam_int"]] = 1.0
    m0 = ctx.model_image(_th(t)).cpu().numpy()
    for lam in (0.8, 0.9):
        t2 = t.copy()
        t2[I["lam_int"]] = lam
        t2[I["x_src"]] = lam * t[I["x_src"]] + (1 - lam) * t[I["x_c"]]
        t2[I["y_src"]] = lam * t[I["y_src"]] + (1 - lam) * t[I["y_c"]]
        t2[I["R_e_src"]] = lam * t[I["R_e_src"]]
        m1 = ctx.model_image(_th(t2)).cpu().numpy()
        assert np.max(np.abs(m1 - m0)) <= 1e-5 * np.max(np.abs(m0)), np.max(np.abs(m1 - m0))


@pytest.fixture(scope="module")
def w8():
    sys_list, th, sid = systems.workload(8)
    return sys_list[0], th, _ctx(sys_list)


def test_w8_full_batch_sampled_against_oracle(w8):
    s, th, ctx = w8
    logL, st, terms = ctx.loglike(_th(th), terms=True)  # B = 256, the benchmarked launch
    logL, st = logL.cpu().numpy(), st.cpu().numpy()
    ok = np.flatnonzero(st == 0)
    assert len(ok) > len(th) // 2
    for b in (ok[0], ok[len(ok) // 2]):
        ev = model.evaluate(th[b], s)
        assert ev["status"] == 0
        assert abs(logL[b] - ev["logL"]) < systems.logl_tol_comp(ev["logL"]), (b, logL[b], ev["logL"])
        assert_vrms_close(ctx.vrms(_th(th[b])).cpu().numpy(), ev["vrms"])
        assert_image_close(ctx.model_image(_th(th[b])).cpu().numpy(), ev["image"])
