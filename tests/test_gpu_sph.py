"""Spherically aligned Jeans model (Eqs. J1/J2): the CUDA path against the oracle's discrete
rule (the same polar grid, characteristic and line-of-sight rules), element by element.

Tolerances as in test_gpu_parity: v_rms per bin relative 1e-4 (FP32 sums over FP64 grid
and line-of-sight rules); logL within systems.logl_tol."""
import numpy as np
import pytest

from oracle import model
from paper_2504_01302_b300 import synth

from . import systems
from .test_gpu_parity import assert_vrms_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

I = synth.IDX


def _th(t):
    return torch.as_tensor(np.asarray(t, np.float64), device="cuda")


def _ctx(sys_list):
    from paper_2504_01302_b300.glad import GladContext
    return GladContext(sys_list)


def sph_small(seed=7, **rule):
    """The small all-features system with the spherically aligned model; data from the
    oracle's spherically aligned model at the truth."""
    b = dict(systems.small_base(seed), jam_align=1, **rule)
    return model.build_system(b, synth.theta_truth(1), synth.noise_draws(b, 9100 + seed))


@pytest.fixture(scope="module")
def small():
    s = sph_small(7, sph_nr=40, sph_nw=6, sph_nlos=48)
    return s, _ctx([s])


def test_vrms_matches_oracle(small):
    s, ctx = small
    for th in systems.near_truth_thetas(2, seed=71):
        ref, st, _ = model.dynamics(th, s)
        assert st == model.ST_OK
        assert_vrms_close(ctx.vrms(_th(th)).cpu().numpy(), ref)


def test_vrms_prior_draws_match_oracle(small):
    s, ctx = small
    n = 0
    for th in systems.prior_thetas(12, seed=73):
        if not model.check_domain(th):
            continue
        ref, st, _ = model.dynamics(th, s)
        if st != model.ST_OK:
            continue
        assert_vrms_close(ctx.vrms(_th(th)).cpu().numpy(), ref)
        n += 1
    assert n >= 3


def test_loglike_batch_matches_oracle(small):
    s, ctx = small
    th = np.vstack([systems.near_truth_thetas(3, seed=75), systems.prior_thetas(5, seed=77)])
    logL, status, terms = ctx.loglike(_th(th), terms=True)
    logL, status, terms = logL.cpu().numpy(), status.cpu().numpy(), terms.cpu().numpy()
    for b in range(len(th)):
        ev = model.evaluate(th[b], s)
        assert status[b] == ev["status"], (b, status[b], ev["status"])
        if ev["status"] != model.ST_OK:
            assert np.isneginf(logL[b])
            continue
        assert abs(logL[b] - ev["logL"]) <= systems.logl_tol(ev["logL"]), (b, logL[b], ev["logL"])
        assert abs(terms[b, 1] - ev["chi2_dyn"]) <= 1e-3 * max(ev["chi2_dyn"], 1.0), (b, terms[b, 1], ev["chi2_dyn"])


@pytest.mark.parametrize("name, value", [
    ("beta", 0.0),          # isotropic: the two alignments coincide
    ("inc", np.pi / 2),     # edge-on
    ("f_bh", 0.0),          # no black hole
    ("beta", -0.29),        # tangential
])
def test_degenerate_parameters(small, name, value):
    s, ctx = small
    th = systems.near_truth_thetas(1, seed=79)[0]
    th[I[name]] = value
    ref, st, _ = model.dynamics(th, s)
    assert st == model.ST_OK
    assert_vrms_close(ctx.vrms(_th(th)).cpu().numpy(), ref)


def test_default_rule_and_isotropic_limit_against_cylindrical():
    # same system, both alignments, beta = 0: the models coincide, so the GPU v_rms differ
    # only by the spherical rule's discretisation (<= 3e-4 in Sigma v^2 on the default rule)
    cyl = systems.small_system(7)
    sph = dict(cyl, jam_align=1)
    ctx = _ctx([cyl, sph])
    th = systems.near_truth_thetas(1, seed=81)[0]
    th[I["beta"]] = 0.0
    v_c = ctx.vrms(_th(th), 0).cpu().numpy().astype(np.float64)
    v_s = ctx.vrms(_th(th), 1).cpu().numpy().astype(np.float64)
    assert np.max(np.abs(v_s / v_c - 1)) < 1e-3
    # and the default rule against the oracle
    ref, st, _ = model.dynamics(th, sph)
    assert_vrms_close(v_s, ref)


def test_mixed_alignments_in_one_batch(small):
    s, _ = small
    cyl = systems.small_system(7)
    ctx = _ctx([cyl, s])
    th = systems.near_truth_thetas(6, seed=83)
    sid = torch.as_tensor(np.array([0, 1, 1, 0, 1, 0], np.int32), device="cuda")
    logL, status = ctx.loglike(_th(th), sid)
    logL = logL.cpu().numpy()
    assert np.all(status.cpu().numpy() == 0)
    for b, i in enumerate([0, 1, 1, 0, 1, 0]):
        one = _ctx([[cyl, s][i]])
        l1, _ = one.loglike(_th(th[b:b + 1]))
        assert abs(float(l1[0]) - logL[b]) <= 1e-6 * abs(logL[b]) + 1e-6, (b, float(l1[0]), logL[b])
        one.close()


def test_gradient_matches_oracle_fd(small):
    # every component against FP64 central differences of the oracle (same rule)
    from .test_gpu_grad import assert_grad_close
    s, ctx = small
    th = systems.near_truth_thetas(2, seed=85)
    logL, grad, st = ctx.loglike_grad(_th(th))
    assert np.all(st.cpu().numpy() == 0)
    grad = grad.cpu().numpy()
    for b in range(len(th)):
        assert_grad_close(grad[b], model.grad_fd(th[b], s))


def test_gradient_prior_draw_and_logl(small):
    from .test_gpu_grad import assert_grad_close
    s, ctx = small
    pri = systems.prior_thetas(16, seed=89)
    th = next(t for t in pri if model.check_domain(t) and model.dynamics_setup(t, s)[0] == 0)
    l1, grad, st = ctx.loglike_grad(_th(th[None]))
    l0, _ = ctx.loglike(_th(th[None]))
    assert int(st[0]) == 0 and abs(float(l1[0]) - float(l0[0])) <= 1e-9 * abs(float(l0[0]))
    assert_grad_close(grad.cpu().numpy()[0], model.grad_fd(th, s))


def test_gradient_mixed_alignments(small):
    s, _ = small
    cyl = systems.small_system(7)
    ctx = _ctx([cyl, s])
    th = systems.near_truth_thetas(4, seed=91)
    ids = [1, 0, 1, 0]
    _, g, st = ctx.loglike_grad(_th(th), torch.as_tensor(np.array(ids, np.int32), device="cuda"))
    assert np.all(st.cpu().numpy() == 0)
    g = g.cpu().numpy()
    for b, i in enumerate(ids):
        one = _ctx([[cyl, s][i]])
        _, g1, _ = one.loglike_grad(_th(th[b:b + 1]))
        g1 = g1.cpu().numpy()[0]
        assert np.allclose(g[b], g1, rtol=1e-4, atol=1e-4 * np.max(np.abs(g1))), (b, g[b], g1)
        one.close()


@pytest.fixture(scope="module")
def w5():
    sys_list, th, _ = systems.workload(5)
    return sys_list[0], th, _ctx(sys_list)


def test_w5_full_batch_sampled(w5):
    # the benchmarked launch (RXJ1131 scale, B = 256); sampled samples term by term
    s, th, ctx = w5
    logL, status, terms = ctx.loglike(_th(th), terms=True)
    logL, status, terms = logL.cpu().numpy(), status.cpu().numpy(), terms.cpu().numpy()
    ok = np.flatnonzero(status == 0)
    assert len(ok) > 0.5 * len(th)
    for b in (ok[0], ok[len(ok) // 2]):
        v, st, _ = model.dynamics(th[b], s)
        assert st == model.ST_OK
        from oracle import kin
        c = kin.chi2_dyn(v, s)
        assert abs(terms[b, 1] - c) <= 1e-3 * max(c, 1.0), (b, terms[b, 1], c)
    near = systems.near_truth_thetas(2, seed=87)
    l2, s2 = ctx.loglike(_th(near))
    for b in range(2):
        ev = model.evaluate(near[b], s)
        assert int(s2[b]) == 0 and abs(float(l2[b]) - ev["logL"]) <= systems.logl_tol(ev["logL"])


@pytest.mark.parametrize("rule", [dict(sph_nr=16, sph_nw=2, sph_nlos=1),   # one node, two angles
                                  dict(sph_nr=24, sph_nw=5, sph_nlos=33)])  # odd n_los
def test_rule_edge_cases(rule):
    # the middle line-of-sight node (z' = 0) of an odd n_los, a single node, and the narrowest
    # angular grid, forward and gradient, against the oracle's same rule.  (The descriptor also
    # allows 4 radii; over 0.002" - 180" the cubic radial interpolation then overshoots to
    # negative moments, in the oracle as on the GPU, and the sample ends non-finite.)
    from .test_gpu_grad import assert_grad_close
    s = dict(sph_small(7), **rule)
    ctx = _ctx([s])
    th = systems.near_truth_thetas(1, seed=93)[0]
    ref, st, _ = model.dynamics(th, s)
    assert st == model.ST_OK
    assert_vrms_close(ctx.vrms(_th(th)).cpu().numpy(), ref)
    _, g, stg = ctx.loglike_grad(_th(th[None]))
    assert int(stg[0]) == 0
    assert_grad_close(g.cpu().numpy()[0], model.grad_fd(th, s))
    ctx.close()
