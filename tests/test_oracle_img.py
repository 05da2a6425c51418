"""Pins of the oracle's image-position term (Eq. chi2_img): zero at exact images, the
predicted images solve the lens equation, quadratic growth with a small displacement of
one image, and independence of H0 (a purely lensing term)."""
import numpy as np

from oracle import lens, model, tdelay
from paper_2504_01302_b300 import synth

from . import systems


def _sys():
    s = dict(systems.small_system(7))
    s["img_sig"] = np.full(len(s["img_xy"]), 0.005)
    return s


def test_zero_at_exact_images():
    s = _sys()
    assert tdelay.chi2_img(synth.theta_truth(1), s) < 1e-18


def test_predicted_images_solve_the_lens_equation():
    s = _sys()
    th = systems.near_truth_thetas(1, seed=31)[0]
    pre = tdelay.predicted_images(th, s)
    bh = tdelay.beta_hat(th, s, np.asarray(s["img_xy"]))
    ax, ay = lens.alpha_total(pre[:, 0], pre[:, 1], th, s["sis"])
    assert np.max(np.abs(pre[:, 0] - ax - bh[0])) < 1e-12
    assert np.max(np.abs(pre[:, 1] - ay - bh[1])) < 1e-12
    # each predicted image is the one near its observed counterpart
    assert np.max(np.hypot(*(pre - np.asarray(s["img_xy"])).T)) < 0.05


def test_quadratic_in_a_small_displacement():
    s = _sys()
    th = synth.theta_truth(1)
    c = []
    for d in (1e-4, 2e-4):
        t = dict(s)
        xy = np.array(s["img_xy"], np.float64, copy=True)
        xy[1, 0] += d
        t["img_xy"] = xy
        c.append(tdelay.chi2_img(th, t))
    assert abs(c[1] / c[0] - 4.0) < 1e-3, c


def test_logl_includes_the_term_and_ignores_H0():
    s = _sys()
    th = systems.near_truth_thetas(1, seed=33)[0]
    ev = model.evaluate(th, s)
    base = dict(s)
    del base["img_sig"]
    ev0 = model.evaluate(th, base)
    assert ev["chi2_img"] > 0
    assert abs((ev0["logL"] - ev["logL"]) - 0.5 * ev["chi2_img"]) < 1e-9 * abs(ev["logL"])
    t2 = th.copy()
    t2[synth.IDX["H0"]] *= 1.3
    assert abs(tdelay.chi2_img(t2, s) - ev["chi2_img"]) < 1e-12 * ev["chi2_img"]
