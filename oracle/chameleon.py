"""Chameleon profile of the composite mass class (oracle, FP64; test infrastructure).

Sect. 3.3, Eq. Chameleon: the lens light is two Chameleon profiles, each the difference of two
isothermal profiles with cores w_c < w_t,
    I(x, y) = I0/(1 + q) [1/sqrt(x^2 + y^2/q^2 + 4 w_c^2/(1+q)^2)
                          - 1/sqrt(x^2 + y^2/q^2 + 4 w_t^2/(1+q)^2)]
in the galaxy frame (major axis along x); the composite mass class uses Upsilon_* I as the
baryonic convergence (kappa_int,comp).

Each term A / sqrt(x^2 + y^2/q^2 + s^2) = q A / sqrt(q^2 (s^2 + x^2) + y^2) is a
non-singular isothermal ellipsoid, whose deflection is (the standard softened-isothermal
form, with b = 2 q A)
    alpha_x = b / sqrt(1 - q^2) arctan( sqrt(1 - q^2) x / (psi + s) ),
    alpha_y = b / sqrt(1 - q^2) arctanh( sqrt(1 - q^2) y / (psi + q^2 s) ),
    psi = sqrt(q^2 (s^2 + x^2) + y^2)
(its divergence is twice the convergence, pinned below);
at q = 1 it becomes the round alpha(R) = 2 A (sqrt(R^2 + s^2) - s)/R along the radius.  For the
dynamics the profile along the major axis, I(R) with R = sqrt(x^2 + y^2/q^2), goes through the
1-D MGE of Sect. 3.2 with axis ratio q.

Its potential is x alpha_x + y alpha_y - b s ln sqrt((psi + s)^2 + (1 - q^2) x^2) (up to a
constant), and its Jacobian follows by differentiating the deflection.

Pins (tests/test_oracle_chameleon.py): div alpha = 2 kappa and curl alpha = 0 by finite
differences (q < 1); the round limit against Gauss's theorem by quadrature; the MGE's
reconstruction of the profile; the potential's gradient and the Jacobian against
differences of the deflection.
"""
import numpy as np

from . import mge


def _cores(q, w):
    return 2.0 * w / (1.0 + q)


def kappa(x, y, I0, wc, wt, q):
    """The profile (convergence when I0 carries Upsilon_*) at galaxy-frame (x, y)."""
    m2 = x * x + y * y / (q * q)
    sc, st = _cores(q, wc), _cores(q, wt)
    return I0 / (1.0 + q) * (1.0 / np.sqrt(m2 + sc * sc) - 1.0 / np.sqrt(m2 + st * st))


def _nie_alpha(x, y, A, s, q):
    """Deflection of A / sqrt(x^2 + y^2/q^2 + s^2)."""
    b = 2.0 * q * A
    if abs(1.0 - q) < 1e-12:
        R2 = x * x + y * y
        fac = np.where(R2 > 0, 2.0 * A / (np.sqrt(R2 + s * s) + s), A / s)
        return fac * x, fac * y
    e = np.sqrt(1.0 - q * q)
    psi = np.sqrt(q * q * (s * s + x * x) + y * y)
    return (b / e * np.arctan(e * x / (psi + s)),
            b / e * np.arctanh(e * y / (psi + q * q * s)))


def _nie_psi(x, y, A, s, q):
    """Potential of A / sqrt(x^2 + y^2/q^2 + s^2) (up to a constant):
    x alpha_x + y alpha_y - b s ln sqrt((psi + s)^2 + (1 - q^2) x^2), b = 2 q A."""
    b = 2.0 * q * A
    ax, ay = _nie_alpha(x, y, A, s, q)
    psi = np.sqrt(q * q * (s * s + x * x) + y * y)
    return x * ax + y * ay - b * s * 0.5 * np.log((psi + s) ** 2 + (1.0 - q * q) * x * x)


def _nie_jac(x, y, A, s, q):
    """d alpha / d (x, y) of A / sqrt(x^2 + y^2/q^2 + s^2), by differentiating the deflection:
    a11 = b [(psi + s) - q^2 x^2/psi] / D,  a12 = a21 = -b x y / (psi D),
    a22 = b [(psi + q^2 s) - y^2/psi] / (q^2 D),  D = (psi + s)^2 + (1 - q^2) x^2."""
    b = 2.0 * q * A
    psi = np.sqrt(q * q * (s * s + x * x) + y * y)
    D = (psi + s) ** 2 + (1.0 - q * q) * x * x
    a11 = b * ((psi + s) - q * q * x * x / psi) / D
    a12 = -b * x * y / (psi * D)
    a22 = b * ((psi + q * q * s) - y * y / psi) / (q * q * D)
    return a11, a12, a12, a22


def alpha(x, y, I0, wc, wt, q):
    A = I0 / (1.0 + q)
    ax1, ay1 = _nie_alpha(x, y, A, _cores(q, wc), q)
    ax2, ay2 = _nie_alpha(x, y, A, _cores(q, wt), q)
    return ax1 - ax2, ay1 - ay2


def psi(x, y, I0, wc, wt, q):
    A = I0 / (1.0 + q)
    return _nie_psi(x, y, A, _cores(q, wc), q) - _nie_psi(x, y, A, _cores(q, wt), q)


def jac(x, y, I0, wc, wt, q):
    A = I0 / (1.0 + q)
    a = _nie_jac(x, y, A, _cores(q, wc), q)
    b = _nie_jac(x, y, A, _cores(q, wt), q)
    return tuple(u - v for u, v in zip(a, b))


def mge_of(I0, wc, wt, q, rmin, rmax, n, P):
    """(amplitudes, sigmas) of the major-axis profile; the Gaussians carry axis ratio q."""
    sc, st = _cores(q, wc), _cores(q, wt)
    F = lambda z: I0 / (1.0 + q) * (1.0 / np.sqrt(z * z + sc * sc) - 1.0 / np.sqrt(z * z + st * st))
    sig, A = mge.mge_1d(F, rmin, rmax, n, P)
    return A, sig
