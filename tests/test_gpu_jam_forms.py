"""Forms 1-3 of the JAM pair sum (glad_set_tuning codes 1xxxxxx-3xxxxxx): two table
entries per packed operation (form 2), and the recurrence forms (1, 3), which sum the entries
whose exponent changes slowly from sky row to sky row along chains of 4 rows with two ex2 per
chain instead of one per point.  The pair sum they compute is the same (Eq. sigma_v2_jam in
the pair form of the cylindrically aligned solution): v_rms per bin against the oracle at the
parity bound (1e-4) and against the default form at 1e-5, logL within the parity bounds, in
every skipping mode, on mixed and ragged systems and at the RXJ1131-scale batch on sampled
samples."""
import numpy as np
import pytest

from oracle import model

from . import systems
from .test_gpu_parity import assert_vrms_close

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

FORMS = [1008032, 1008041, 1008042, 1016021, 1108042,
         2004042, 2004052, 2004051, 2008031, 2104042,
         3004042, 3004041, 3004051, 3008031, 3104042]
DIRECT = 8042


def _th(t):
    return torch.as_tensor(np.asarray(t, np.float64), device="cuda")


def _ctx(sys_list):
    from paper_2504_01302_b300.glad import GladContext
    return GladContext(sys_list)


@pytest.fixture(scope="module")
def small():
    s = systems.small_system(7)
    th = systems.near_truth_thetas(3, seed=71)
    rng = np.random.Generator(np.random.PCG64(72))
    from paper_2504_01302_b300 import synth
    th = np.concatenate([th, synth.draw_prior(rng, 3)])
    ev = [model.evaluate(t, s) for t in th]
    return s, th, ev, _ctx([s])


@pytest.mark.parametrize("code", FORMS)
def test_vrms_and_logl_against_oracle_and_direct(small, code):
    s, th, ev, ctx = small
    ctx.set_tuning(DIRECT, 4)
    v_dir = [ctx.vrms(_th(t)).cpu().numpy().astype(np.float64) for t in th]
    l_dir = ctx.loglike(_th(th))[0].cpu().numpy()
    ctx.set_tuning(code, 4)
    l_rec, st = ctx.loglike(_th(th))
    l_rec = l_rec.cpu().numpy()
    for b, t in enumerate(th):
        if ev[b]["status"] != 0:
            assert int(st[b]) == ev[b]["status"]
            continue
        v = ctx.vrms(_th(t)).cpu().numpy().astype(np.float64)
        assert_vrms_close(v, ev[b]["vrms"])
        assert np.max(np.abs(v / v_dir[b] - 1)) < 1e-5, (b, np.max(np.abs(v / v_dir[b] - 1)))
        assert abs(l_rec[b] - ev[b]["logL"]) < systems.logl_tol(ev[b]["logL"])
        assert abs(l_rec[b] - l_dir[b]) < 0.01 + 1e-6 * abs(l_dir[b])
    ctx.set_tuning(DIRECT, 4)


@pytest.mark.parametrize("neg", [0, 2])
@pytest.mark.parametrize("code", [1008042, 2004042, 3004042])
def test_every_skipping_mode(small, neg, code):
    s, th, ev, ctx = small
    ctx.set_tuning(code, 4)
    ctx.set_negligible(neg)
    try:
        for b in range(2):
            assert_vrms_close(ctx.vrms(_th(th[b])).cpu().numpy(), ev[b]["vrms"])
    finally:
        ctx.set_negligible(1)
        ctx.set_tuning(DIRECT, 4)


def test_mixed_ragged_systems_and_invalid_sample():
    sa = systems.small_system(7)
    sb = systems.small_system(8, n_px=36, ss=1, psf_k=5, sky=14, kss=4, n_mass=6, n_light=(6,),
                              n_gl=24, n_bins=9, n_sis=0, second_light=False, has_bh=False)
    ctx = _ctx([sa, sb])
    th_np = systems.near_truth_thetas(7, seed=73)
    th_np[3, 2] = 1.4  # q > 1: invalid
    th = _th(th_np)
    sid_np = np.array([0, 1, 1, 0, 1, 0, 1], np.int32)
    sid = torch.as_tensor(sid_np, device="cuda")
    ctx.set_tuning(DIRECT, 4)
    ref, st_ref = ctx.loglike(th, sid)
    for code in (1008042, 1108042, 1016021, 2004042, 2104042, 3004042, 3104042):
        ctx.set_tuning(code, 4)
        got, st = ctx.loglike(th, sid)
        assert torch.equal(st, st_ref)
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        ok = np.isfinite(r)
        assert np.array_equal(ok, np.isfinite(g)) and not ok[3]
        assert np.all(np.abs(g[ok] - r[ok]) < 0.01 + 1e-6 * np.abs(r[ok]))
    # one sample of the smaller, ragged system against the oracle
    b = 1
    ev = model.evaluate(th_np[b], sb)
    assert abs(float(got[b]) - ev["logL"]) < systems.logl_tol(ev["logL"])


@pytest.fixture(scope="module")
def w1():
    sys_list, th, _ = systems.workload(1)
    s = sys_list[0]
    ok = [0, 137]
    return s, th, _ctx(sys_list), {b: model.evaluate(th[b], s) for b in ok}


@pytest.mark.parametrize("code", [1008042, 2004042, 3004042])
def test_rxj1131_batch_sampled_against_oracle(w1, code):
    s, th, ctx, ev = w1
    ctx.set_tuning(code, 4)
    logL, st = ctx.loglike(_th(th))  # B = 256, the benchmarked launch
    logL, st = logL.cpu().numpy(), st.cpu().numpy()
    for b, e in ev.items():
        assert st[b] == e["status"] == 0
        assert abs(logL[b] - e["logL"]) < systems.logl_tol(e["logL"]), (b, logL[b], e["logL"])
        assert_vrms_close(ctx.vrms(_th(th[b])).cpu().numpy(), e["vrms"])
