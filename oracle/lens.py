"""Lens mass model: EPL + external shear + SIS perturbers (oracle, FP64).

* Lens equation (Eq. lens_equation, Sect. 3.1.1): beta = theta - alpha(theta).
  The paper prints "theta = beta - grad psi"; the sign is garbled, the standard
  form beta = theta - alpha is used.
* EPL convergence (App. C): kappa = (3-g)/2 (b/R)^(g-1), R = sqrt(x^2 + y^2/q^2),
  b = (2/(1+q))^(1/(g-1)) theta_E, in the frame rotated by the position angle
  (counter-clockwise from +x, Table 2 footnote).  The lensing side uses the
  unsoftened profile (the softened EPL has no closed-form deflection); the MGE
  of the dynamics side uses r_soft (App. C).
* EPL deflection: the paper cites it without writing it.  It is the
  hypergeometric series of Tessore & Metcalf (2015): with t = g-1,
  b_TM = q b, R_TM = sqrt(q^2 x^2 + y^2), e^{i ph} = (q x + i y)/R_TM, f=(1-q)/(1+q):
  alpha = 2 b_TM/(1+q) (b_TM/R_TM)^(t-1) sum_n Omega_n,
  Omega_0 = e^{i ph}, Omega_n = -f (2n-(2-t))/(2n+(2-t)) e^{2 i ph} Omega_{n-1}.
  Terms are summed until f^n < 1e-16.
* EPL potential: psi = (x alpha_x + y alpha_y)/(2-t) (alpha is homogeneous).
* External shear (Sect. 3.3): psi = gamma/2 R^2 cos(2 phi - 2 phi_ext), centred
  on the lens centre.
* SIS perturber: psi = theta_Es |theta - theta_s|.

Pins: mpmath hyp2f1, the SIE closed form at g=2, the power law at q=1,
div alpha = 2 kappa and curl alpha = 0 by finite differences, mean kappa = 1
inside R = b via Gauss's theorem, psi consistent with alpha, and the shear
divergence (kappa_shear = 0).
"""
import math

import numpy as np


def frame(x, y, xc, yc, phi):
    """Sky offsets -> galaxy frame (major axis along x')."""
    c, s = math.cos(phi), math.sin(phi)
    dx, dy = x - xc, y - yc
    return c * dx + s * dy, -s * dx + c * dy


def to_sky(ax, ay, phi):
    c, s = math.cos(phi), math.sin(phi)
    return c * ax - s * ay, s * ax + c * ay


def epl_b(theta_E, g, q):
    """App. C normalisation b = (2/(1+q))^(1/(g-1)) theta_E."""
    return (2.0 / (1.0 + q)) ** (1.0 / (g - 1.0)) * theta_E


def epl_kappa_frame(xp, yp, theta_E, g, q, r_soft=0.0):
    """App. C convergence in the galaxy frame."""
    b = epl_b(theta_E, g, q)
    R2 = xp ** 2 + yp ** 2 / q ** 2
    return (3.0 - g) / 2.0 * (b / np.sqrt(R2 + r_soft ** 2)) ** (g - 1.0)


def epl_nterms(q, eps=1e-16):
    f = (1.0 - q) / (1.0 + q)
    if f <= 0.0:
        return 0
    return int(math.ceil(math.log(eps) / math.log(f)))


def epl_alpha_frame(xp, yp, theta_E, g, q, nterms=None):
    """Tessore & Metcalf (2015) deflection in the galaxy frame (complex series)."""
    t = g - 1.0
    bt = q * epl_b(theta_E, g, q)
    xp = np.asarray(xp, np.float64)
    yp = np.asarray(yp, np.float64)
    R = np.sqrt(q * q * xp * xp + yp * yp)
    # at the exact centre the direction of the deflection is undefined (|alpha| ~ R^(1-t));
    # it is taken as 0, its average over directions (the paper is silent: its lensing EPL
    # is not softened)
    at0 = R == 0.0
    R = np.where(at0, 1.0, R)
    w = (q * xp + 1j * yp) / R
    w2 = w * w
    f = (1.0 - q) / (1.0 + q)
    n_max = epl_nterms(q) if nterms is None else nterms
    om = w.copy()
    S = w.copy()
    for n in range(1, n_max + 1):
        om = -f * (2 * n - (2 - t)) / (2 * n + (2 - t)) * w2 * om
        S = S + om
    a = 2.0 * bt / (1.0 + q) * (bt / R) ** (t - 1.0) * S
    a = np.where(at0, 0.0, a)
    return a.real, a.imag


def epl_psi_frame(xp, yp, theta_E, g, q):
    ax, ay = epl_alpha_frame(xp, yp, theta_E, g, q)
    return (xp * ax + yp * ay) / (3.0 - g)


def epl_jac_frame(xp, yp, theta_E, g, q):
    """d alpha / d theta in the galaxy frame from homogeneity:
    complex shear = ((1-t) alpha - kappa z) / conj(z)."""
    t = g - 1.0
    ax, ay = epl_alpha_frame(xp, yp, theta_E, g, q)
    k = epl_kappa_frame(xp, yp, theta_E, g, q)
    z = xp + 1j * yp
    gam = ((1 - t) * (ax + 1j * ay) - k * z) / np.conj(z)
    g1, g2 = gam.real, gam.imag
    return k + g1, g2, g2, k - g1


def shear_alpha(dx, dy, gamma_ext, phi_ext):
    g1, g2 = gamma_ext * math.cos(2 * phi_ext), gamma_ext * math.sin(2 * phi_ext)
    return g1 * dx + g2 * dy, g2 * dx - g1 * dy


def shear_psi(dx, dy, gamma_ext, phi_ext):
    g1, g2 = gamma_ext * math.cos(2 * phi_ext), gamma_ext * math.sin(2 * phi_ext)
    return 0.5 * (g1 * (dx * dx - dy * dy) + 2 * g2 * dx * dy)


def sis_alpha(x, y, tE, xs, ys):
    """SIS deflection; 0 at the perturber's exact centre (as for the EPL)."""
    dx, dy = x - xs, y - ys
    r = np.sqrt(dx * dx + dy * dy)
    ri = np.where(r == 0.0, 0.0, 1.0 / np.where(r == 0.0, 1.0, r))
    return tE * dx * ri, tE * dy * ri


def sis_psi(x, y, tE, xs, ys):
    return tE * np.sqrt((x - xs) ** 2 + (y - ys) ** 2)


def sis_jac(x, y, tE, xs, ys):
    dx, dy = x - xs, y - ys
    r = np.sqrt(dx * dx + dy * dy)
    r3 = r ** 3
    return tE * dy * dy / r3, -tE * dx * dy / r3, -tE * dx * dy / r3, tE * dx * dx / r3


def alpha_total(x, y, th, sis):
    """Deflection of EPL + shear + SIS perturbers at sky positions (x, y)."""
    tE, g, q, phi, xc, yc, gext, pext = th[:8]
    xp, yp = frame(x, y, xc, yc, phi)
    axp, ayp = epl_alpha_frame(xp, yp, tE, g, q)
    ax, ay = to_sky(axp, ayp, phi)
    sx, sy = shear_alpha(x - xc, y - yc, gext, pext)
    ax = ax + sx
    ay = ay + sy
    for tEs, xs, ys in sis:
        a1, a2 = sis_alpha(x, y, tEs, xs, ys)
        ax = ax + a1
        ay = ay + a2
    return ax, ay


def psi_total(x, y, th, sis):
    tE, g, q, phi, xc, yc, gext, pext = th[:8]
    xp, yp = frame(x, y, xc, yc, phi)
    p = epl_psi_frame(xp, yp, tE, g, q) + shear_psi(x - xc, y - yc, gext, pext)
    for tEs, xs, ys in sis:
        p = p + sis_psi(x, y, tEs, xs, ys)
    return p


def jac_total(x, y, th, sis):
    """d alpha/d theta (a11, a12, a21, a22) on the sky."""
    tE, g, q, phi, xc, yc, gext, pext = th[:8]
    xp, yp = frame(x, y, xc, yc, phi)
    j11, j12, j21, j22 = epl_jac_frame(xp, yp, tE, g, q)
    c, s = math.cos(phi), math.sin(phi)
    # J_sky = Rot J Rot^T
    a11 = c * c * j11 - c * s * (j12 + j21) + s * s * j22
    a12 = c * s * (j11 - j22) + c * c * j12 - s * s * j21
    a21 = c * s * (j11 - j22) + c * c * j21 - s * s * j12
    a22 = s * s * j11 + c * s * (j12 + j21) + c * c * j22
    g1, g2 = gext * math.cos(2 * pext), gext * math.sin(2 * pext)
    a11, a12, a21, a22 = a11 + g1, a12 + g2, a21 + g2, a22 - g1
    for tEs, xs, ys in sis:
        b11, b12, b21, b22 = sis_jac(x, y, tEs, xs, ys)
        a11, a12, a21, a22 = a11 + b11, a12 + b12, a21 + b21, a22 + b22
    return a11, a12, a21, a22


def solve_images(beta, th, sis, guesses, tol=1e-13, iters=100):
    """Newton solution of beta = theta - alpha(theta) from each starting guess."""
    out = []
    for g0 in guesses:
        p = np.array(g0, np.float64)
        for _ in range(iters):
            ax, ay = alpha_total(np.array([p[0]]), np.array([p[1]]), th, sis)
            F = np.array([p[0] - ax[0] - beta[0], p[1] - ay[0] - beta[1]])
            a11, a12, a21, a22 = jac_total(np.array([p[0]]), np.array([p[1]]), th, sis)
            A = np.array([[1 - a11[0], -a12[0]], [-a21[0], 1 - a22[0]]])
            dp = np.linalg.solve(A, F)
            p = p - dp
            if np.max(np.abs(dp)) < tol:
                break
        out.append(p)
    return np.array(out)
