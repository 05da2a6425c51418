"""Deprojection and axisymmetric Jeans (JAM) line-of-sight second moment (oracle, FP64).

Deprojection (App. A, Eqs. sb_mge_2D, sb_mge_3D, smd_mge, smd_3D): a projected
Gaussian (peak I_0, dispersion sigma, axis ratio q') at inclination i deprojects to
q = sqrt(q'^2 - cos^2 i)/sin i and peak density q' I_0/(sqrt(2 pi) sigma q); this
needs cos^2 i < q'^2 for every Gaussian (App. A).  App. A swaps the indices i/j
inside the sum of Eq. sb_mge_3D; each Gaussian uses its own sigma and q.

Jeans model.  The paper's Eqs. J1/J2 are the spherically aligned equations; the
workload asks for the fixed-order Gauss-Legendre quadrature over (tracer k,
mass j) Gaussian pairs at every sky point, which is the cylindrically aligned
MGE solution (constant beta_z, v_R^2 = b v_z^2, b = 1/(1-beta)).  Its two
definitions are both written out here:

* ``sigma_v2_plain``: the definition.  Potential of each mass Gaussian
  (Emsellem et al. 1994)
    Phi_j = -sqrt(2/pi) G M_j/sigma_j int_0^1 exp[-u^2/(2 sigma_j^2) (R^2 + z^2/(1-e_j^2 u^2))]
            / sqrt(1-e_j^2 u^2) du,   M_j = (2 pi)^(3/2) rho_j sigma_j^3 q_j,
  the cylindrical Jeans equations
    nu v_z^2 = int_z^inf nu dPhi/dz' dz',
    nu v_phi^2 = b [nu v_z^2 + R d(nu v_z^2)/dR] + R nu dPhi/dR,
  the line-of-sight moment (x = x', y = y' cos i - z' sin i, z = y' sin i + z' cos i)
    nu v_los^2 = sin^2 i (nu v_R^2 sin^2 ph + nu v_phi^2 cos^2 ph) + cos^2 i nu v_z^2,
  and Sigma v_los^2(x', y') = int nu v_los^2 dz' (Eq. VLos numerator), all by
  nested numerical quadrature.

* ``table``/``sigma_v2_fast``: the same quantity after the z integrals are done
  analytically for Gaussians, leaving one integral over u in [0, 1] per pair:
    Sigma v^2 = sum_{k,j} nu_k C_j int_0^1 F(u) sqrt(pi/al) exp(-p x'^2 - (p c/al) y'^2) du
  with C_j = 4 pi G rho_j q_j sigma_j^2, a = u^2/(2 sigma_j^2), h = 1 - e_j^2 u^2,
  p = 1/(2 sigma_k^2) + a, c = 1/(2 sigma_k^2 q_k^2) + a/h, al = p sin^2 i + c cos^2 i,
  A = a/(h^(3/2) c), F = A (b sin^2 i + cos^2 i) + x'^2 sin^2 i (2a/sqrt(h) - 2 p b A).
  The u integral uses an n-point Gauss-Legendre rule in t on [0, 1] with the per-pair
  map u = u_s (exp(lam t) - 1), lam = ln(1 + 1/u_s), u_s = min(1, sigma_j / max(r_max, sigma_k)),
  r_max the largest sky-sample radius of the system: it resolves the integrand's
  scales u ~ sigma_j/r and u ~ sigma_j/sigma_k.

Pins: fast vs plain at a few sky points; the spherical isotropic limit against the
1-D Jeans integral Sigma sigma_los^2(R) = 2G int_R^inf nu M(r) sqrt(r^2-R^2)/r^2 dr;
v_rms proportional to sqrt(mass scale), independent of tracer amplitude, 4-fold
symmetric; the deprojected density integrates back along the line of sight to the
projected Gaussian.
"""
import math

import numpy as np
from scipy.integrate import quad
from scipy.special import erf

SQRT2PI = math.sqrt(2 * math.pi)


# ---------------------------------------------------------------------------
# deprojection (App. A)
# ---------------------------------------------------------------------------

def intrinsic_q(qp, inc):
    c2 = math.cos(inc) ** 2
    return np.sqrt(qp ** 2 - c2) / math.sin(inc)


def deproject(peak, sig, qp, inc):
    """Projected Gaussian peaks -> intrinsic peak densities and axis ratios."""
    q = intrinsic_q(qp, inc)
    return qp * peak / (SQRT2PI * sig * q), q


# ---------------------------------------------------------------------------
# Gauss-Legendre rule with the per-pair map
# ---------------------------------------------------------------------------

def gl01(n):
    x, w = np.polynomial.legendre.leggauss(n)
    return 0.5 * (x + 1.0), 0.5 * w


def pair_map(sig_k, sig_j, r_max):
    us = np.minimum(1.0, sig_j[None, :] / np.maximum(r_max, sig_k[:, None]))
    lam = np.log1p(1.0 / us)
    return us, lam


def nodes(sig_k, sig_j, r_max, n_gl):
    """u nodes and weights*du/dt for every (k, j, g): arrays of shape (K, J, G)."""
    t, w = gl01(n_gl)
    us, lam = pair_map(sig_k, sig_j, r_max)
    e = np.exp(lam[..., None] * t)
    u = us[..., None] * (e - 1.0)
    wu = w * us[..., None] * lam[..., None] * e
    return u, wu


# ---------------------------------------------------------------------------
# fast (single-integral) form
# ---------------------------------------------------------------------------

def table(tr, ms, inc, beta, v2u, r_max, n_gl):
    """Coefficients (T, P0, P1, ax, ay) of every (k, j, g) term.

    tr: dict(I0, sig, qp) tracer MGE (surface brightness peaks)
    ms: dict(kap0, sig, qp) mass MGE (convergence peaks)."""
    nu0, qk = deproject(tr["I0"], tr["sig"], tr["qp"], inc)
    _, qj = deproject(ms["kap0"], ms["sig"], ms["qp"], inc)
    Cj = 2.0 * SQRT2PI * v2u * ms["qp"] * ms["kap0"] * ms["sig"]    # = 4 pi G rho_j q_j sigma_j^2
    e2 = 1.0 - qj ** 2
    s2, c2 = math.sin(inc) ** 2, math.cos(inc) ** 2
    b = 1.0 / (1.0 - beta)
    u, wu = nodes(tr["sig"], ms["sig"], r_max, n_gl)
    sk = tr["sig"][:, None, None]
    qkk = qk[:, None, None]
    sj = ms["sig"][None, :, None]
    a = u * u / (2 * sj * sj)
    h = 1.0 - e2[None, :, None] * u * u
    p = 1.0 / (2 * sk * sk) + a
    c = 1.0 / (2 * sk * sk * qkk * qkk) + a / h
    al = p * s2 + c * c2
    A = a / (h ** 1.5 * c)
    P0 = A * (b * s2 + c2)
    P1 = s2 * (2 * a / np.sqrt(h) - 2 * p * b * A)
    T = nu0[:, None, None] * Cj[None, :, None] * wu * np.sqrt(math.pi / al)
    return T, P0, P1, -p, -p * c / al


def sigma_v2_fast(xp, yp, tab, chunk=2048):
    """Sigma v_los^2 at galaxy-frame sky points from the pair table."""
    T, P0, P1, ax, ay = (v.reshape(-1) for v in tab)
    xp = np.asarray(xp, np.float64).reshape(-1)
    yp = np.asarray(yp, np.float64).reshape(-1)
    out = np.empty_like(xp)
    for s in range(0, xp.size, chunk):
        X = xp[s:s + chunk, None] ** 2
        Y = yp[s:s + chunk, None] ** 2
        out[s:s + chunk] = np.sum(T * (P0 + P1 * X) * np.exp(ax * X + ay * Y), axis=1)
    return out


def surface_brightness(xp, yp, tr):
    """Projected tracer MGE (Eq. sb_mge_2D)."""
    xp = np.asarray(xp, np.float64)[..., None]
    yp = np.asarray(yp, np.float64)[..., None]
    return np.sum(tr["I0"] * np.exp(-(xp ** 2 + yp ** 2 / tr["qp"] ** 2) / (2 * tr["sig"] ** 2)), -1)


# ---------------------------------------------------------------------------
# plain definition: nested quadrature of the cylindrical Jeans equations
# ---------------------------------------------------------------------------

def _u_rule():
    edges = np.concatenate([[0.0], 10.0 ** np.linspace(-8, 0, 41)])
    x, w = np.polynomial.legendre.leggauss(24)
    lo, hi = edges[:-1, None], edges[1:, None]
    u = (0.5 * (hi - lo) * (x + 1) + lo).ravel()
    wu = (0.5 * (hi - lo) * w).ravel()
    return u, wu


_U, _WU = _u_rule()


class PlainJeans:
    """Direct evaluation of the definition, for a handful of sky points."""

    def __init__(self, tr, ms, inc, beta, v2u):
        self.nu0, self.qk = deproject(tr["I0"], tr["sig"], tr["qp"], inc)
        self.sk = tr["sig"]
        rho0, qj = deproject(ms["kap0"], ms["sig"], ms["qp"], inc)
        self.sj = ms["sig"]
        self.e2 = 1.0 - qj ** 2
        M = (2 * math.pi) ** 1.5 * rho0 * self.sj ** 3 * qj
        self.amp = math.sqrt(2 / math.pi) * v2u * M / self.sj       # sqrt(2/pi) G M_j / sigma_j
        self.inc = inc
        self.b = 1.0 / (1.0 - beta)
        self.zmax = 40.0 * float(np.max(self.sk * self.qk))

    def nu(self, R, z):
        return np.sum(self.nu0 * np.exp(-(R * R + z * z / self.qk ** 2) / (2 * self.sk ** 2)))

    def dnu_dR(self, R, z):
        return np.sum(-R / self.sk ** 2 * self.nu0 *
                      np.exp(-(R * R + z * z / self.qk ** 2) / (2 * self.sk ** 2)))

    def dphi(self, R, z):
        """(dPhi/dR, dPhi/dz, d2Phi/dRdz) from the Emsellem integral."""
        u = _U[:, None]
        h = 1.0 - self.e2 * u * u
        g = u * u / self.sj ** 2
        E = np.exp(-0.5 * g * (R * R + z * z / h)) / np.sqrt(h)
        dR = np.sum(_WU[:, None] * g * R * E * self.amp)
        dz = np.sum(_WU[:, None] * g * z / h * E * self.amp)
        dRz = np.sum(_WU[:, None] * (g * z / h) * (-g * R) * E * self.amp)
        return dR, dz, dRz

    def nuvz2(self, R, z):
        """nu v_z^2 and d(nu v_z^2)/dR at (R, |z|)."""
        z = abs(z)

        def f0(zz):
            return self.nu(R, zz) * self.dphi(R, zz)[1]

        def f1(zz):
            _, dz, dRz = self.dphi(R, zz)
            return self.dnu_dR(R, zz) * dz + self.nu(R, zz) * dRz
        v0 = quad(f0, z, z + self.zmax, epsabs=0, epsrel=1e-12, limit=400)[0]
        v1 = quad(f1, z, z + self.zmax, epsabs=0, epsrel=1e-12, limit=400)[0]
        return v0, v1

    def los_integrand(self, xp, yp, zp):
        si, ci = math.sin(self.inc), math.cos(self.inc)
        x = xp
        y = yp * ci - zp * si
        z = yp * si + zp * ci
        R = math.hypot(x, y)
        vz, dvz = self.nuvz2(R, z)
        dR = self.dphi(R, z)[0]
        vR = self.b * vz
        vphi = self.b * (vz + R * dvz) + R * self.nu(R, z) * dR
        cph2 = (x / R) ** 2
        sph2 = 1.0 - cph2
        return si * si * (vR * sph2 + vphi * cph2) + ci * ci * vz

    def sigma_v2(self, xp, yp):
        L = self.zmax
        f = lambda zp: self.los_integrand(xp, yp, zp)
        return (quad(f, -L, 0.0, epsabs=0, epsrel=1e-10, limit=400)[0]
                + quad(f, 0.0, L, epsabs=0, epsrel=1e-10, limit=400)[0])


def sigma_v2_spherical_1d(R, tr, ms, v2u):
    """Spherical isotropic limit (all q = 1, beta = 0):
    Sigma sigma_los^2(R) = 2 G int_R^inf nu(r) M(r) sqrt(r^2 - R^2)/r^2 dr."""
    nu0 = tr["I0"] / (SQRT2PI * tr["sig"])
    rho0 = ms["kap0"] / (SQRT2PI * ms["sig"])
    Mj = (2 * math.pi) ** 1.5 * rho0 * ms["sig"] ** 3

    def integrand(r):
        nu = np.sum(nu0 * np.exp(-r * r / (2 * tr["sig"] ** 2)))
        x = r / ms["sig"]
        M = np.sum(Mj * (erf(x / math.sqrt(2)) - math.sqrt(2 / math.pi) * x * np.exp(-x * x / 2)))
        return nu * M * math.sqrt(max(r * r - R * R, 0.0)) / (r * r)
    L = R + 40 * float(np.max(tr["sig"]))
    pts = [R + s for s in np.sort(np.concatenate([tr["sig"], ms["sig"]])) if R + s < L]
    return 2 * v2u * quad(integrand, R, L, points=pts[:50], epsabs=0, epsrel=1e-12, limit=500)[0]


def sigma_v2_converged(xp, yp, tr, ms, inc, beta, v2u):
    """Pair form with an adaptive u integral per sky point (measures the GL rule's
    discretisation error; not used for parity)."""
    nu0, qk = deproject(tr["I0"], tr["sig"], tr["qp"], inc)
    _, qj = deproject(ms["kap0"], ms["sig"], ms["qp"], inc)
    Cj = 2.0 * SQRT2PI * v2u * ms["qp"] * ms["kap0"] * ms["sig"]
    e2 = 1.0 - qj ** 2
    s2, c2 = math.sin(inc) ** 2, math.cos(inc) ** 2
    b = 1.0 / (1.0 - beta)
    X, Y = xp * xp, yp * yp
    tot = 0.0
    for k in range(len(nu0)):
        for j in range(len(Cj)):
            def f(u):
                a = u * u / (2 * ms["sig"][j] ** 2)
                h = 1.0 - e2[j] * u * u
                p = 1.0 / (2 * tr["sig"][k] ** 2) + a
                c = 1.0 / (2 * tr["sig"][k] ** 2 * qk[k] ** 2) + a / h
                al = p * s2 + c * c2
                A = a / (h ** 1.5 * c)
                F = A * (b * s2 + c2) + X * s2 * (2 * a / math.sqrt(h) - 2 * p * b * A)
                return F * math.sqrt(math.pi / al) * math.exp(-p * X - p * c / al * Y)
            brk = [min(1.0, ms["sig"][j] / max(math.sqrt(X + Y), 1e-12)),
                   min(1.0, ms["sig"][j] / tr["sig"][k])]
            v = quad(f, 0.0, 1.0, points=sorted(set(x for x in brk if 0 < x < 1)),
                     epsabs=0, epsrel=1e-13, limit=400)[0]
            tot += nu0[k] * Cj[j] * v
    return tot
