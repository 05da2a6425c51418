"""The autotuner picks a supported launch shape and does not change results."""
import numpy as np
import pytest

from . import systems

pytestmark = pytest.mark.gpu

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
    assert t["jam_pts"] in (401, 801, 805, 806, 1601) and t["adj_ept"] in (2, 4)
    after = ctx.loglike(th)[0].cpu().numpy()
    g_after = ctx.loglike_grad(th)[1].cpu().numpy()
    assert np.all(np.abs(after - before) < 1e-6 * np.abs(before))
    assert np.allclose(g_after, g_before, rtol=1e-4, atol=1e-6 * np.max(np.abs(g_before)))
    # the cache file now holds the choice; a second context reads it back
    assert (tmp_path / "tune.txt").read_text().strip()
    ctx2 = GladContext([s])
    assert ctx2.autotune(th, with_grad=True) == t
