"""Pins of the elliptical NFW halo by cored steep ellipsoids (oracle/enfw.py), Sect. 3.3:
the 44-CSE fit against the projected NFW convergence, div alpha = 2 kappa and curl alpha = 0 of
a flattened CSE by finite differences, and the round eNFW deflection against Gauss's theorem
on the exact NFW convergence by quadrature (independent of the fit)."""
import math

import numpy as np
from scipy.integrate import quad

from oracle import enfw


def test_cse_fit():
    a, s = enfw.cse_decomposition()
    assert len(s) == 44 and np.all(a >= 0)
    u = np.geomspace(1e-4, 1e3, 777)
    fit = np.sum(a[None, :] * (u[:, None] ** 2 + s[None, :] ** 2) ** -1.5, -1)
    assert np.max(np.abs(fit / enfw.nfw_k(u) - 1)) < 1e-6


def test_cse_divergence_and_curl():
    q, s, h = 0.65, 0.3, 1e-5
    for x, y in ((0.2, 0.1), (-0.9, 0.7), (1.5, -2.0)):
        xs, ys = np.array([x]), np.array([y])
        axp, ayp = enfw.cse_alpha(xs + h, ys, s, q)
        axm, aym = enfw.cse_alpha(xs - h, ys, s, q)
        bxp, byp = enfw.cse_alpha(xs, ys + h, s, q)
        bxm, bym = enfw.cse_alpha(xs, ys - h, s, q)
        div = (axp - axm + byp - bym) / (2 * h)
        curl = (ayp - aym - bxp + bxm) / (2 * h)
        k = enfw.cse_kappa(xs, ys, s, q)
        assert abs(div[0] / (2 * k[0]) - 1) < 1e-6, (x, y, div, 2 * k)
        assert abs(curl[0]) < 1e-6 * abs(div[0])


def test_round_enfw_deflection_is_gauss():
    ks, rs = 0.3, 5.0
    for R in (0.05, 1.0, 4.0, 20.0):
        mean = 2.0 / R ** 2 * quad(lambda r: ks * enfw.nfw_k(np.array([r / rs]))[0] * r, 0.0, R,
                                   epsabs=0, epsrel=1e-12, limit=200, points=[rs] if R > rs else None)[0]
        ax, ay = enfw.enfw_alpha(np.array([0.6 * R]), np.array([0.8 * R]), ks, rs, 1.0)
        assert abs(math.hypot(ax[0], ay[0]) / (R * mean) - 1) < 1e-5, (R, math.hypot(ax[0], ay[0]), R * mean)
