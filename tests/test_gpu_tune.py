"""The autotuner picks a supported launch shape and does not change results."""
import numpy as np
import pytest

from . import systems

pytestmark = pytest.mark.gpu

SHAPES = [2064, 2084, 4052, 4054, 4064, 8032, 8042, 8044, 16021]
OTHER_FORMS = [1008032, 1008041, 1008042, 1016021, 2004042, 2004052, 2004051, 2008031,
               3004042, 3004041, 3004051, 3008031]

torch = pytest.importorskip("torch")


def test_autotune_keeps_results(tmp_path, monkeypatch):
    from paper_2504_01302_b300.glad import GladContext
    monkeypatch.setenv("GLAD_TUNE_CACHE", str(tmp_path / "tune.txt"))
    s = systems.small_system(7)
    ctx = GladContext([s])
    th = torch.as_tensor(systems.near_truth_thetas(5, seed=61), device="cuda")
    before = ctx.loglike(th)[0].cpu().numpy()
    g_before = ctx.loglike_grad(th)[1].cpu().numpy()
    t = ctx.autotune(th, with_grad=True)
    code = t["jam_pts"]
    assert code % 100000 + 1000000 * (code // 1000000) in SHAPES + OTHER_FORMS and t["adj_ept"] in (2, 4)
    after = ctx.loglike(th)[0].cpu().numpy()
    g_after = ctx.loglike_grad(th)[1].cpu().numpy()
    # the other forms of the pair sum round differently from the default one
    assert np.all(np.abs(after - before) < (1e-6 if code < 1000000 else 1e-5) * np.abs(before))
    assert np.allclose(g_after, g_before, rtol=1e-4, atol=1e-6 * np.max(np.abs(g_before)))
    # the cache file now holds the choice; a second context reads it back
    assert (tmp_path / "tune.txt").read_text().strip()
    ctx2 = GladContext([s])
    assert ctx2.autotune(th, with_grad=True) == t


@pytest.mark.parametrize("code", SHAPES + [100000 + c for c in (4064, 8042, 16021)])
def test_every_launch_shape_gives_the_same_logl(code):
    # mixed systems (grid form: blocks beyond a small system exit; persistent form: a
    # (sample, tile) work list), including an invalid sample that gets no work items
    from paper_2504_01302_b300.glad import GladContext
    sa = systems.small_system(7)
    sb = systems.small_system(8, n_px=36, ss=1, psf_k=5, sky=14, kss=4, n_mass=6, n_light=(6,),
                              n_gl=24, n_bins=9, n_sis=0, second_light=False, has_bh=False)
    ctx = GladContext([sa, sb])
    th_np = systems.near_truth_thetas(7, seed=63)
    th_np[3, 2] = 1.4  # q > 1: invalid
    th = torch.as_tensor(th_np, device="cuda")
    sid = torch.as_tensor(np.array([0, 1, 1, 0, 1, 0, 1], np.int32), device="cuda")
    ctx.set_tuning(8042, 4)
    ref, st_ref = ctx.loglike(th, sid)
    ctx.set_tuning(code, 2)
    got, st = ctx.loglike(th, sid)
    assert torch.equal(st, st_ref)
    r, g = ref.cpu().numpy(), got.cpu().numpy()
    ok = np.isfinite(r)
    assert np.array_equal(ok, np.isfinite(g)) and not ok[3]
    assert np.all(np.abs(g[ok] - r[ok]) < 1e-6 * np.abs(r[ok]))


def test_every_adjoint_shape_gives_the_same_gradient():
    from paper_2504_01302_b300.glad import GladContext
    ctx = GladContext([systems.small_system(7)])
    th = torch.as_tensor(systems.near_truth_thetas(3, seed=65), device="cuda")
    out = []
    for ept in (2, 4):
        ctx.set_tuning(8042, ept)
        out.append(ctx.loglike_grad(th)[1].cpu().numpy())
    scale = np.max(np.abs(out[0]), axis=1, keepdims=True)
    for g in out[1:]:
        assert np.all(np.abs(g - out[0]) <= 1e-6 * np.abs(out[0]) + 1e-7 * scale)


def test_bad_launch_shape_is_refused():
    from paper_2504_01302_b300 import _lib
    from paper_2504_01302_b300.glad import GladContext
    ctx = GladContext([systems.small_system(7)])
    with pytest.raises(_lib.GladError):
        ctx.set_tuning(8022, 4)
