"""Pins of the Chameleon profile (oracle/chameleon.py), Sect. 3.3 Eq. Chameleon:
div alpha = 2 kappa and curl alpha = 0 by finite differences for a flattened profile, the
round limit against Gauss's theorem by quadrature, and the 1-D MGE's reconstruction."""
import math

import numpy as np
from scipy.integrate import quad

from oracle import chameleon as ch

PARS = dict(I0=1.3, wc=0.05, wt=1.2)


def test_divergence_and_curl():
    q = 0.7
    h = 1e-5
    for x, y in ((0.3, 0.2), (-1.1, 0.6), (0.05, -1.9), (2.5, 2.5)):
        xs, ys = np.array([x]), np.array([y])
        axp, ayp = ch.alpha(xs + h, ys, q=q, **PARS)
        axm, aym = ch.alpha(xs - h, ys, q=q, **PARS)
        bxp, byp = ch.alpha(xs, ys + h, q=q, **PARS)
        bxm, bym = ch.alpha(xs, ys - h, q=q, **PARS)
        div = (axp - axm) / (2 * h) + (byp - bym) / (2 * h)
        curl = (ayp - aym) / (2 * h) - (bxp - bxm) / (2 * h)
        k = ch.kappa(xs, ys, q=q, **PARS)
        assert abs(div[0] / (2 * k[0]) - 1) < 1e-6, (x, y, div, 2 * k)
        assert abs(curl[0]) < 1e-6 * abs(div[0])


def test_round_limit_is_gauss():
    for R in (0.1, 0.8, 3.0):
        mean = 2.0 / R ** 2 * quad(lambda r: ch.kappa(r, 0.0, q=1.0, **PARS) * r, 0.0, R,
                                   epsabs=0, epsrel=1e-13)[0]
        ax, ay = ch.alpha(np.array([0.6 * R]), np.array([0.8 * R]), q=1.0, **PARS)
        assert abs(math.hypot(ax[0], ay[0]) / (R * mean) - 1) < 1e-10
    # and the flattened formula approaches it as q -> 1
    a1 = ch.alpha(np.array([0.7]), np.array([0.4]), q=1.0, **PARS)
    a2 = ch.alpha(np.array([0.7]), np.array([0.4]), q=1.0 - 1e-7, **PARS)
    assert abs(a2[0][0] / a1[0][0] - 1) < 1e-5 and abs(a2[1][0] / a1[1][0] - 1) < 1e-5


def test_mge_reconstruction():
    q = 0.8
    A, sig = ch.mge_of(q=q, rmin=0.005, rmax=50.0, n=30, P=10, **PARS)
    R = np.geomspace(0.01, 10.0, 100)
    rec = np.sum(A[None, :] * np.exp(-R[:, None] ** 2 / (2 * sig[None, :] ** 2)), -1)
    ref = ch.kappa(R, 0.0, q=q, **PARS)
    assert np.max(np.abs(rec / ref - 1)) < 5e-3
