"""The oracle's restricted v_rms (bins chosen one by one, for grids whose full maps are out
of reach) against its full chain: the two must agree to rounding, since zeroing the maps
outside the PSF reach of the chosen bins changes none of their bin sums."""
import numpy as np

from oracle import model

from . import systems


def test_vrms_bins_equals_full_dynamics():
    s = systems.small_system(7)
    th = systems.near_truth_thetas(2, seed=3)
    for t in th:
        v, st, _ = model.dynamics(t, s)
        which = [0, s["n_bins"] // 2, s["n_bins"] - 1]
        vb, st2 = model.vrms_bins(t, s, which)
        assert st == st2 == model.ST_OK
        assert np.max(np.abs(vb / v[which] - 1)) < 1e-13


def test_vrms_bins_reports_invalid_samples():
    s = systems.small_system(7)
    t = systems.near_truth_thetas(1, seed=5)[0]
    t[15] = 0.3  # inclination far below what the flattest Gaussian allows
    v, st, _ = model.dynamics(t, s)
    vb, st2 = model.vrms_bins(t, s, [0])
    assert st == st2 and st != model.ST_OK and vb is None
