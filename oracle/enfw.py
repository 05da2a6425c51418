"""Elliptical NFW halo of the composite mass class by cored steep ellipsoids (oracle, FP64;
test infrastructure).

Sect. 3.3 (kappa_int,comp, Eq. kappa_enfw): the dark matter is an NFW profile made elliptical in
its convergence, kappa(xi) = kappa_s k(xi / r_s) with xi^2 = x^2 + y^2/q^2 in the galaxy frame and
the projected NFW shape
    k(u) = 2 (1 - F(u)) / (u^2 - 1),   F(u) = arctanh(sqrt(1 - u^2))/sqrt(1 - u^2)  (u < 1),
                                          arctan(sqrt(u^2 - 1))/sqrt(u^2 - 1)    (u > 1),
k(1) = 2/3.  As in the paper, the profile is written as a sum of 44 cored steep ellipsoids
(CSE), k(u) ~ sum_i a_i / (u^2 + s_i^2)^(3/2); the paper takes the decomposition from the
literature without printing it, so here the s_i are log-spaced on [1e-5, 1e4] and the a_i >= 0
are a non-negative least-squares fit of the relative error on u in [1e-4, 1e3].

CSE deflection: 1/(xi^2 + s^2)^(3/2) = -(1/s) d/ds [1/sqrt(xi^2 + s^2)], so the deflection of a
CSE is -(1/s) d/ds of the softened isothermal ellipsoid's (oracle/chameleon.py, A = 1):
    alpha_x = 2 q x (psi + q^2 s) / (s psi ((psi + s)^2 + (1 - q^2) x^2)),
    alpha_y = 2 q^3 y (psi + s) / (s psi ((psi + q^2 s)^2 - (1 - q^2) y^2)),
    psi = sqrt(q^2 (s^2 + x^2) + y^2),
which at q = 1 is the round 2 R / (s psi (psi + s)).

Pins (tests/test_oracle_enfw.py): the fit against k(u); div alpha = 2 kappa and curl alpha = 0
of a flattened CSE by differences; the round eNFW deflection against Gauss's theorem on the
exact NFW convergence by quadrature.
"""
import functools

import numpy as np
from scipy.optimize import nnls

N_CSE = 44


def nfw_k(u):
    """Projected NFW convergence in units of kappa_s at u = xi / r_s."""
    u = np.asarray(u, np.float64)
    out = np.empty_like(u)
    lo, hi = u < 1 - 1e-6, u > 1 + 1e-6
    mid = ~(lo | hi)
    e = np.sqrt(1 - u[lo] ** 2)
    out[lo] = 2 * (1 - np.arctanh(e) / e) / (u[lo] ** 2 - 1)
    e = np.sqrt(u[hi] ** 2 - 1)
    out[hi] = 2 * (1 - np.arctan(e) / e) / (u[hi] ** 2 - 1)
    out[mid] = 2.0 / 3.0
    return out


@functools.lru_cache(maxsize=None)
def cse_decomposition(n=N_CSE, smin=1e-5, smax=1e4, umin=1e-4, umax=1e3, npts=2000):
    """(a_i, s_i) of k(u) ~ sum_i a_i (u^2 + s_i^2)^(-3/2), non-negative least squares on the
    relative error."""
    s = np.geomspace(smin, smax, n)
    u = np.geomspace(umin, umax, npts)
    G = (u[:, None] ** 2 + s[None, :] ** 2) ** -1.5
    M = G / nfw_k(u)[:, None]
    cs = np.linalg.norm(M, axis=0)
    a, _ = nnls(M / cs, np.ones_like(u), maxiter=50 * n * n)
    return a / cs, s


def cse_kappa(x, y, s, q):
    return (x * x + y * y / (q * q) + s * s) ** -1.5


def cse_alpha(x, y, s, q):
    """Deflection of 1/(x^2 + y^2/q^2 + s^2)^(3/2) in the galaxy frame."""
    e2 = 1.0 - q * q
    psi = np.sqrt(q * q * (s * s + x * x) + y * y)
    ax = 2 * q * x * (psi + q * q * s) / (s * psi * ((psi + s) ** 2 + e2 * x * x))
    ay = 2 * q ** 3 * y * (psi + s) / (s * psi * ((psi + q * q * s) ** 2 - e2 * y * y))
    return ax, ay


def enfw_kappa(x, y, kappa_s, r_s, q):
    return kappa_s * nfw_k(np.sqrt(x * x + y * y / (q * q)) / r_s)


def enfw_alpha(x, y, kappa_s, r_s, q):
    """Deflection of the CSE sum: component i has amplitude kappa_s a_i r_s^3 and core s_i r_s."""
    a, s = cse_decomposition()
    ax = np.zeros_like(np.asarray(x, np.float64))
    ay = np.zeros_like(ax)
    for ai, si in zip(a, s):
        if ai == 0.0:
            continue
        bx, by = cse_alpha(x, y, si * r_s, q)
        ax = ax + kappa_s * ai * r_s ** 3 * bx
        ay = ay + kappa_s * ai * r_s ** 3 * by
    return ax, ay
