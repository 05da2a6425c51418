"""Elliptical Sersic light (oracle, FP64).

The paper models light with Chameleon profiles (Eq. Chameleon); the workload
asks for elliptical Sersic source and lens light, whose standard form is
I(R) = I_e exp(-b_n [(R/R_e)^(1/n) - 1]) with R = sqrt(x'^2 + y'^2/q^2) in the
frame rotated by the position angle (same major-axis convention as App. C).
b_n is the 4th-order asymptotic series of Ciotti & Bertin (1999), used by
both paths so that it is smooth in n.

Pin: b_n against the exact root of gamma(2n, b) = Gamma(2n)/2 (scipy gammaincinv).
"""
import numpy as np


def sersic_bn(n):
    return (2.0 * n - 1.0 / 3.0 + 4.0 / (405.0 * n) + 46.0 / (25515.0 * n ** 2)
            + 131.0 / (1148175.0 * n ** 3) - 2194697.0 / (30690717750.0 * n ** 4))


def sersic_R(R, I_e, R_e, n):
    """Sersic profile at elliptical radius R (real or complex R)."""
    b = sersic_bn(n)
    return I_e * np.exp(-b * ((R / R_e) ** (1.0 / n) - 1.0))


def sersic_xy(x, y, I_e, R_e, n, q, xc, yc, phi):
    c, s = np.cos(phi), np.sin(phi)
    dx, dy = x - xc, y - yc
    xp, yp = c * dx + s * dy, -s * dx + c * dy
    R = np.sqrt(xp * xp + yp * yp / (q * q))
    return sersic_R(R, I_e, R_e, n)
