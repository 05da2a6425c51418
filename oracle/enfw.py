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

CSE potential and Jacobian: -(1/s) d/ds of the softened isothermal ellipsoid's.  For the
dynamics the exact k(u) is expanded (Sect. 3.2) at complex u by nfw_k_complex, the CSE fit
being controlled on the real axis only.

Pins (tests/test_oracle_enfw.py): the fit against k(u); div alpha = 2 kappa and curl alpha = 0
of a flattened CSE by differences; the round eNFW deflection against Gauss's theorem on the
exact NFW convergence by quadrature; the CSE potential's gradient and the Jacobian against
differences of the deflection; nfw_k_complex against nfw_k on the real axis and against its
own Taylor branch where they meet; the eNFW MGE against the profile.
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


def cse_psi(x, y, s, q):
    """Potential of the CSE (up to a constant): -(1/s) d/ds of the softened isothermal one
    (oracle/chameleon.py, A = 1, b = 2q),
    x alpha_x + y alpha_y + (b/s) L + b (psi + s)(q^2 s/psi + 1) / ((psi + s)^2 + (1 - q^2) x^2),
    L = ln sqrt((psi + s)^2 + (1 - q^2) x^2)."""
    b = 2.0 * q
    e2 = 1.0 - q * q
    psi = np.sqrt(q * q * (s * s + x * x) + y * y)
    D = (psi + s) ** 2 + e2 * x * x
    ax, ay = cse_alpha(x, y, s, q)
    return x * ax + y * ay + b / s * 0.5 * np.log(D) + b * (psi + s) * (q * q * s / psi + 1.0) / D


def cse_jac(x, y, s, q):
    """d alpha / d (x, y) of the CSE: -(1/s) d/ds of the softened isothermal Jacobian
    (A = 1, b = 2q; a11 = b N1/D, a12 = -b x y/(psi D), a22 = b N2/(q^2 D), D = (psi + s)^2 +
    (1 - q^2) x^2, N1 = psi + s - q^2 x^2/psi, N2 = psi + q^2 s - y^2/psi) with d psi/ds =
    q^2 s / psi."""
    b = 2.0 * q
    e2 = 1.0 - q * q
    psi = np.sqrt(q * q * (s * s + x * x) + y * y)
    ps = q * q * s / psi
    D = (psi + s) ** 2 + e2 * x * x
    Ds = 2.0 * (psi + s) * (ps + 1.0)
    N1 = psi + s - q * q * x * x / psi
    N1s = ps + 1.0 + q * q * x * x * ps / (psi * psi)
    N2 = psi + q * q * s - y * y / psi
    N2s = ps + q * q + y * y * ps / (psi * psi)
    d11 = b * (N1s * D - N1 * Ds) / (D * D)
    d12 = b * x * y * (ps * D + psi * Ds) / (psi * D) ** 2
    d22 = b * (N2s * D - N2 * Ds) / (q * q * D * D)
    return -d11 / s, -d12 / s, -d12 / s, -d22 / s


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


def _cse_sum(fn, x, y, kappa_s, r_s, q):
    a, s = cse_decomposition()
    out = None
    for ai, si in zip(a, s):
        if ai == 0.0:
            continue
        v = fn(x, y, si * r_s, q)
        v = tuple(kappa_s * ai * r_s ** 3 * c for c in v) if isinstance(v, tuple) else kappa_s * ai * r_s ** 3 * v
        out = v if out is None else (tuple(o + c for o, c in zip(out, v)) if isinstance(v, tuple) else out + v)
    return out


def enfw_psi(x, y, kappa_s, r_s, q):
    return _cse_sum(cse_psi, x, y, kappa_s, r_s, q)


def enfw_jac(x, y, kappa_s, r_s, q):
    return _cse_sum(cse_jac, x, y, kappa_s, r_s, q)


def nfw_k_complex(u):
    """k(u) at complex u (Re u > 0) for the Euler inversion of the 1-D MGE: with w^2 = 1 - u^2,
    k = 2 (1 - arctanh(w)/w) / (u^2 - 1), an even function of w (so either square root), and
    k = 2 sum_n w^(2n) / (2n + 3) for |w| < 0.1 (the removable point u = 1)."""
    u = np.asarray(u, np.complex128)
    w2 = 1.0 - u * u
    w = np.sqrt(w2)
    small = np.abs(w) < 0.1
    ws = np.where(small, 0.5, w)  # keeps the direct branch free of 0/0
    direct = 2.0 * (1.0 - np.arctanh(ws) / ws) / (u * u - 1.0 + np.where(small, 1.0, 0.0))
    series = sum(2.0 * w2 ** n / (2 * n + 3) for n in range(10))
    return np.where(small, series, direct)