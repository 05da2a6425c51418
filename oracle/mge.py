"""1-D multi-Gaussian expansion by Euler inversion (oracle, FP64).

Sect. 3.2, Eq. integral_transfer ff.: a radial profile F(R) is written as a
continuous Gaussian mixture F(R) = (1/sqrt(2 pi)) int f(sigma) exp(-R^2/(2 sigma^2)) dln(sigma)
with f(sigma) = 1/(i sigma^2) sqrt(2/pi) int_C z F(z) exp(z^2/(2 sigma^2)) dz, i.e. an
inverse Laplace transform in the variable R^2.  The Euler algorithm of Abate &
Whitt (2006) approximates it by f(sigma) = sum_{m=0}^{2P} eta_m Re F(sigma chi_m) with
  chi_m = sqrt(2 P ln10 / 3 + 2 pi i m),
  eta_m = (-1)^m 2 sqrt(2 pi) 10^(P/3) xi_m,
  xi_0 = 1/2, xi_m = 1 (1 <= m <= P), xi_2P = 2^-P,
  xi_{2P-k} = xi_{2P-k+1} + 2^-P C(P, k)  (0 < k < P).
The sigma_n are log-spaced on [r_min, r_max] and
  A_n = w_n f(sigma_n) Delta(ln sigma) / sqrt(2 pi)
with trapezoid weights w_n (1/2 at the two ends).  The paper prints
exp(+R^2/(2 sigma^2)) in the reconstruction formula; the sign is garbled, the
Gaussians decay.

Pins: Euler inversion of 1/(1 + tau/(2a^2)) against its closed-form inverse
2a^2 exp(-2a^2 s); reconstruction of Sersic and power-law profiles within the
0.5 % the paper states for 21 Gaussians; the pure power law's f(sigma) is a
power law of sigma.
"""
import math

import numpy as np

from . import light


def euler_coeffs(P):
    xi = np.zeros(2 * P + 1)
    xi[0] = 0.5
    xi[1:P + 1] = 1.0
    xi[2 * P] = 2.0 ** (-P)
    for k in range(1, P):
        xi[2 * P - k] = xi[2 * P - k + 1] + 2.0 ** (-P) * math.comb(P, k)
    m = np.arange(2 * P + 1)
    eta = (-1.0) ** m * 2.0 * math.sqrt(2 * math.pi) * 10.0 ** (P / 3.0) * xi
    chi = np.sqrt(2.0 * P * math.log(10.0) / 3.0 + 2j * math.pi * m)
    return eta, chi


def f_sigma(F, sigma, P):
    """Gaussian-mixture density f(sigma) of the complex-callable profile F."""
    eta, chi = euler_coeffs(P)
    sigma = np.asarray(sigma, np.float64)
    z = sigma[..., None] * chi
    return np.sum(eta * np.real(F(z)), axis=-1)


def mge_1d(F, rmin, rmax, N, P):
    """Log-spaced sigma_n and amplitudes A_n of the 1-D MGE of F."""
    lo, hi = math.log(rmin), math.log(rmax)
    sig = np.exp(np.linspace(lo, hi, N))
    dl = (hi - lo) / (N - 1)
    w = np.ones(N)
    w[0] = w[-1] = 0.5
    A = w * f_sigma(F, sig, P) * dl / math.sqrt(2 * math.pi)
    return sig, A


def mge_eval(R, sig, A):
    R = np.asarray(R, np.float64)
    return np.sum(A * np.exp(-R[..., None] ** 2 / (2 * sig ** 2)), axis=-1)


def epl_profile(theta_E, g, q, r_soft):
    """App. C softened EPL convergence as a function of elliptical radius."""
    b = (2.0 / (1.0 + q)) ** (1.0 / (g - 1.0)) * theta_E

    def F(z):
        return (3.0 - g) / 2.0 * b ** (g - 1.0) * (z * z + r_soft * r_soft) ** (-(g - 1.0) / 2.0)
    return F


def sersic_profile(I_e, R_e, n):
    def F(z):
        return light.sersic_R(z, I_e, R_e, n)
    return F
