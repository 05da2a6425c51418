"""Spherically aligned axisymmetric Jeans model (oracle, FP64; test infrastructure).

Sect. 3.2, Eqs. J1/J2: axisymmetric tracer density nu and potential Phi, velocity
ellipsoid aligned with (r, theta, phi), constant anisotropy beta = 1 - v_theta^2/v_r^2.
Spherical coordinates r, theta (polar angle from the symmetry axis z), R = r sin(theta),
z = r cos(theta).  With P = nu v_r^2 and V = nu v_phi^2 the two equations are
    J1:  dP/dr + ((1 + beta) P - V)/r = -nu dPhi/dr,
    J2:  (1 - beta) dP/dtheta + ((1 - beta) P - V)/tan(theta) = -nu dPhi/dtheta.
The paper solves them through the published spherically aligned JAM solution and gives
no formula; the solution used here is derived from J1/J2 directly.

Eliminating V gives one first-order equation for P,
    (1 - beta) tan(theta) dP/dtheta - r dP/dr - 2 beta P = nu (r Phi_r - tan(theta) Phi_theta)
                                                         = nu r^2 Phi_z / z,
whose characteristics are r' = r e^s, sin(Theta) = sin(theta) e^{-(1 - beta) s}, i.e.
R' = R e^{beta s}.  With P -> 0 at infinity,
    P(r, theta) = int_0^inf e^{2 beta s} r'^2 nu(R', z') F_z(R', z') ds,   F_z = Phi_z / z.
J2 then gives V = (1 - beta) P + tan(theta) [(1 - beta) dP/dtheta + nu Phi_theta]; the
theta-derivative of the integral (dTheta/dtheta = tan(Theta)/tan(theta)) and
tan(theta) Phi_theta = R^2 (F_R - F_z), F_R = Phi_R / R, leave
    V - (1 - beta) P = R^2 Dt,
    Dt(r, theta) = (1 - beta) int_0^inf e^{4 beta s} r'^2 [F_z dnu + nu G](R', z') ds
                   + nu (F_R - F_z)(R, z),
    dnu = nu_R/R - nu_z/z = sum_k nu_k E_k (1/p_k^2 - 1)/s_k^2,
    G   = F_{z,R}/R - F_{z,z}/z.
Every factor is smooth (no division by R or z).  For a mass Gaussian j (Emsellem et al.
1994 potential, the same as the cylindrical model's), with h = exp(-u^2 (R^2 + z^2 w^2)
/(2 sigma_j^2)), w = (1 - e_j^2 u^2)^(-1/2), K_j = 4 pi G rho_j q_j:
    F_R = sum_j K_j int_0^1 u^2 w   h du,   F_z = sum_j K_j int_0^1 u^2 w^3 h du,
    G   = sum_j K_j / sigma_j^2 int_0^1 u^4 (w^5 - w^3) h du.

Line of sight (x = x', y = y' cos i - z' sin i, z = y' sin i + z' cos i, the cylindrical
model's geometry; n = (0, -sin i, cos i)): with the ellipsoid along (r, theta, phi),
    nu v_los^2 = P (n.r)^2 + (1 - beta) P (n.theta)^2 + V (n.phi)^2
               = P [(1 - beta) + beta mu^2] + Dt sin^2 i x^2,   mu = n.r = (z cos i - y sin i)/r,
and Sigma v_los^2(x', y') = int nu v_los^2 dz' (the numerator of Eq. VLos).

Two forms are written out:

* ``intrinsic_plain``: P and Dt at a point by adaptive quadrature along the
  characteristic and a fine fixed rule in u (for pins).
* the discrete rule (``SphRule``, ``grid_moments``, ``sigma_v2_sph``) that the CUDA path
  follows step for step:
    grid   r_a log-spaced on [r_lo, r_end] (n_r points), angular variable
           w_c = sin^2(theta_c) linear on [0, 1] (n_w points);
           r_lo = d_sub / 4, r_end = 9 max_k sigma_k of the tracer;
    P, Dt  at each grid point: s on [0, ln(r_end / r_a)] in 16 equal pieces, 4-point
           Gauss-Legendre in each (64 nodes); the u integral of mass Gaussian j by the
           n_gl-point Gauss-Legendre rule in t on [0, 1] with u = u_s (e^{lam t} - 1),
           lam = ln(1 + 1/u_s), u_s = min(1, sigma_j / r_end);
           stored as v_r^2 = P/nu and d = Dt/nu;
    LOS    n_los midpoint nodes in tau on [-tau_m, tau_m], z' = c sinh(tau),
           c = max(rho, r_lo), rho = sqrt(x'^2 + y'^2), tau_m = asinh(r_end / c);
           v_r^2 and d cubic in ln r (4-point Lagrange) and linear in w = R^2/r^2,
           clamped to the grid; nu exact at the node.
  Defaults n_r = 128, n_w = 8, n_los = 32: against the cylindrical pair form at beta = 0
  (the two models coincide there) the RXJ1131-scale sky maps agree to 2.9e-4 at sampled
  points and the binned v_rms to 3e-5 - 6e-5; the radial grid sets the error up to
  n_r ~ 160 (falling as n_r^-3.3), the angular grid beyond it (192 x 16 x 32: 6e-6 - 1.1e-5
  in v_rms); beyond 24 line-of-sight nodes it no longer depends on n_los.

Pins (tests/test_oracle_sph.py): the plain solution satisfies J1 and J2 (finite
differences); at beta = 0 it equals the cylindrical isotropic solution (nu v_z^2 and
nu v_phi^2 of jam.PlainJeans) for flattened models; with every q = 1 the projected rule
matches the textbook spherical constant-beta projection; at beta = 0 the projected rule
matches the cylindrical pair form; the discrete grid values match the plain solution.
"""
import math

import numpy as np
from scipy.integrate import quad

from . import jam

R_END_FAC = 9.0     # r_end = R_END_FAC * largest tracer sigma
R_LO_FRAC = 0.25    # r_lo = R_LO_FRAC * sky sub-sample spacing
CHAR_PIECES = 16    # pieces of the characteristic's s range
CHAR_GL = 4         # Gauss-Legendre points per piece
DEFAULT_RULE = (128, 8, 32)  # n_r, n_w, n_los


class SphModel:
    """Deprojected tracer and mass Gaussians of one sample (App. A)."""

    def __init__(self, tr, ms, inc, beta, v2u):
        self.nu0, self.pk = jam.deproject(tr["I0"], tr["sig"], tr["qp"], inc)
        self.sk = np.asarray(tr["sig"], np.float64)
        rho, qj = jam.deproject(ms["kap0"], ms["sig"], ms["qp"], inc)
        self.sj = np.asarray(ms["sig"], np.float64)
        self.e2 = 1.0 - qj ** 2
        self.Kj = 4.0 * math.pi * v2u * rho * qj
        self.inc = inc
        self.beta = beta

    # tracer ------------------------------------------------------------------
    def tracer(self, R2, z2):
        """nu and dnu = nu_R/R - nu_z/z at arrays of (R^2, z^2)."""
        R2 = np.asarray(R2, np.float64)[..., None]
        z2 = np.asarray(z2, np.float64)[..., None]
        E = self.nu0 * np.exp(-(R2 + z2 / self.pk ** 2) / (2 * self.sk ** 2))
        return E.sum(-1), (E * (1.0 / self.pk ** 2 - 1.0) / self.sk ** 2).sum(-1)

    # potential ---------------------------------------------------------------
    def potential(self, R2, z2, u, wu):
        """F_R, F_z, G at arrays of (R^2, z^2); u, wu: [J, G] nodes and weights per mass
        Gaussian (or [G] shared by all)."""
        u = np.broadcast_to(np.asarray(u, np.float64), (len(self.sj),) + np.shape(u)[-1:])
        wu = np.broadcast_to(np.asarray(wu, np.float64), u.shape)
        w2 = 1.0 / (1.0 - self.e2[:, None] * u * u)
        w = np.sqrt(w2)
        a = u * u / (2 * self.sj[:, None] ** 2)
        R2 = np.asarray(R2, np.float64)[..., None, None]
        z2 = np.asarray(z2, np.float64)[..., None, None]
        h = np.exp(-a * (R2 + z2 * w2))
        c = self.Kj[:, None] * wu * u * u
        FR = (c * w * h).sum((-2, -1))
        Fz = (c * w * w2 * h).sum((-2, -1))
        G = ((c * u * u / self.sj[:, None] ** 2) * (w * w2 * w2 - w * w2) * h).sum((-2, -1))
        return FR, Fz, G

    # LOS geometry ------------------------------------------------------------
    def los_point(self, xp, yp, zp):
        si, ci = math.sin(self.inc), math.cos(self.inc)
        x = xp
        y = yp * ci - zp * si
        z = yp * si + zp * ci
        return x, y, z


# ---------------------------------------------------------------------------
# plain form (adaptive along the characteristic, fine fixed rule in u)
# ---------------------------------------------------------------------------

def intrinsic_plain(m, r, theta, s_max=None):
    """(P, Dt) at (r, theta) by adaptive quadrature in s."""
    b = m.beta
    R, z = r * math.sin(theta), r * math.cos(theta)
    if s_max is None:
        s_max = max(math.log(60.0 * float(np.max(m.sk)) / r), 1.0)

    def node(s):
        rp, Rp = r * math.exp(s), R * math.exp(b * s)
        zp2 = max(rp * rp - Rp * Rp, 0.0)
        nu, dnu = m.tracer(Rp * Rp, zp2)
        _, Fz, G = m.potential(Rp * Rp, zp2, jam._U, jam._WU)
        return rp, float(nu), float(dnu), float(Fz), float(G)

    def fP(s):
        rp, nu, _, Fz, _ = node(s)
        return math.exp(2 * b * s) * rp * rp * nu * Fz

    def fD(s):
        rp, nu, dnu, Fz, G = node(s)
        return math.exp(4 * b * s) * rp * rp * (Fz * dnu + nu * G)

    brk = [x for x in np.log(np.concatenate([m.sk, m.sj]) / r) if 0 < x < s_max]
    brk = sorted(brk)[:60]
    P = quad(fP, 0.0, s_max, points=brk or None, epsabs=0, epsrel=1e-12, limit=800)[0]
    Di = quad(fD, 0.0, s_max, points=brk or None, epsabs=0, epsrel=1e-12, limit=800)[0]
    nu, _ = m.tracer(R * R, z * z)
    FR, Fz, _ = m.potential(R * R, z * z, jam._U, jam._WU)
    return P, (1.0 - b) * Di + float(nu) * float(FR - Fz)


def phi_derivs(m, r, theta):
    """(dPhi/dr, dPhi/dtheta) at (r, theta) from the fine u rule."""
    R, z = r * math.sin(theta), r * math.cos(theta)
    FR, Fz, _ = m.potential(R * R, z * z, jam._U, jam._WU)
    FR, Fz = float(FR), float(Fz)
    return math.sin(theta) * R * FR + math.cos(theta) * z * Fz, z * R * (FR - Fz)


# ---------------------------------------------------------------------------
# discrete rule
# ---------------------------------------------------------------------------

class SphRule:
    """Fixed geometry of the discrete rule for one system."""

    def __init__(self, sig_light, sig_mass, dsub, n_r, n_w, n_los, n_gl):
        if n_r < 4 or n_w < 2 or n_los < 1:
            raise ValueError("grid too small")
        self.r_lo = R_LO_FRAC * dsub
        self.r_end = R_END_FAC * float(np.max(sig_light))
        self.n_r, self.n_w, self.n_los = n_r, n_w, n_los
        self.lr = np.linspace(math.log(self.r_lo), math.log(self.r_end), n_r)
        self.w = np.linspace(0.0, 1.0, n_w)
        x, wt = np.polynomial.legendre.leggauss(CHAR_GL)
        self.cx, self.cw = 0.5 * (x + 1.0), 0.5 * wt
        t, wt = jam.gl01(n_gl)
        us = np.minimum(1.0, np.asarray(sig_mass, np.float64) / self.r_end)[:, None]
        lam = np.log1p(1.0 / us)
        e = np.exp(lam * t)
        self.u = us * (e - 1.0)
        self.wu = wt * us * lam * e


def grid_moments(m, rule, max_elems=4_000_000):
    """v_r^2 = P/nu and d = Dt/nu on the (n_r, n_w) grid (in blocks of radii, so that the
    temporaries over (radius, angle, node, mass Gaussian, u node) stay near max_elems)."""
    per_row = rule.n_w * CHAR_PIECES * CHAR_GL * rule.u.size
    step = max(1, max_elems // per_row)
    parts = [_grid_rows(m, rule, rule.lr[a:a + step]) for a in range(0, rule.n_r, step)]
    return np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts])


def _grid_rows(m, rule, lr):
    b = m.beta
    r = np.exp(lr)[:, None]                             # [rows, 1]
    sth = np.sqrt(rule.w)[None, :]                      # [1, n_w]
    R = r * sth
    z2 = r * r * (1.0 - rule.w)[None, :]
    smax = np.log(rule.r_end / r)                       # [n_r, 1]
    ds = smax / CHAR_PIECES
    # nodes s = (p + cx) ds, weights cw ds
    s = (np.arange(CHAR_PIECES)[:, None] + rule.cx[None, :]).reshape(-1)  # [64] in units of ds
    S = s[None, None, :] * ds[..., None]                # [n_r, 1, 64]
    W = np.tile(rule.cw, CHAR_PIECES)[None, None, :] * ds[..., None]
    rp = r[..., None] * np.exp(S)
    Rp = R[..., None] * np.exp(b * S)
    zp2 = np.maximum(rp * rp - Rp * Rp, 0.0)
    shape = np.broadcast_shapes(rp.shape, Rp.shape)
    Rp2 = np.broadcast_to(Rp * Rp, shape)
    zp2 = np.broadcast_to(zp2, shape)
    nu, dnu = m.tracer(Rp2, zp2)
    _, Fz, G = m.potential(Rp2, zp2, rule.u, rule.wu)
    P = (W * np.exp(2 * b * S) * rp * rp * nu * Fz).sum(-1)
    Di = (W * np.exp(4 * b * S) * rp * rp * (Fz * dnu + nu * G)).sum(-1)
    nu0, _ = m.tracer(R * R, z2)
    FR0, Fz0, _ = m.potential(np.broadcast_to(R * R, z2.shape), z2, rule.u, rule.wu)
    Dt = (1.0 - b) * Di + nu0 * (FR0 - Fz0)
    return P / nu0, Dt / nu0


def interp(grid, rule, lnr, w):
    """Cubic Lagrange in ln r through the 4 grid radii around the point (the stencil
    shifted inward at the ends), linear in w; both coordinates clamped to the grid."""
    fa = np.clip((lnr - rule.lr[0]) / (rule.lr[1] - rule.lr[0]), 0.0, rule.n_r - 1)
    fc = np.clip(w * (rule.n_w - 1), 0.0, rule.n_w - 1)
    i0 = np.clip(np.floor(fa).astype(np.int64) - 1, 0, rule.n_r - 4)
    c0 = np.minimum(fc.astype(np.int64), rule.n_w - 2)
    x = fa - i0
    tc = fc - c0
    L = (-(x - 1) * (x - 2) * (x - 3) / 6, x * (x - 2) * (x - 3) / 2,
         -x * (x - 1) * (x - 3) / 2, x * (x - 1) * (x - 2) / 6)
    out = 0.0
    for o in range(4):
        out = out + L[o] * ((1 - tc) * grid[i0 + o, c0] + tc * grid[i0 + o, c0 + 1])
    return out


def sigma_v2_sph(xp, yp, m, rule, grids, chunk=4096):
    """Sigma v_los^2 at galaxy-frame sky points by the discrete LOS rule."""
    vr2, dg = grids
    b = m.beta
    si = math.sin(m.inc)
    xp = np.asarray(xp, np.float64).reshape(-1)
    yp = np.asarray(yp, np.float64).reshape(-1)
    n = rule.n_los
    t = (np.arange(n) + 0.5) / n * 2.0 - 1.0            # midpoints on [-1, 1]
    out = np.empty_like(xp)
    for a in range(0, xp.size, chunk):
        X, Y = xp[a:a + chunk, None], yp[a:a + chunk, None]
        c = np.maximum(np.hypot(X, Y), rule.r_lo)
        tm = np.arcsinh(rule.r_end / c)
        tau = t[None, :] * tm
        zp = c * np.sinh(tau)
        wt = (2.0 * tm / n) * c * np.cosh(tau)
        x, y, z = m.los_point(X, Y, zp)
        R2 = x * x + y * y
        r2 = R2 + z * z
        r = np.sqrt(r2)
        w = R2 / r2
        nu, _ = m.tracer(R2, z * z)
        v = interp(vr2, rule, np.log(r), w)
        d = interp(dg, rule, np.log(r), w)
        mu = (z * math.cos(m.inc) - y * si) / r
        f = nu * (v * ((1.0 - b) + b * mu * mu) + d * si * si * x * x)
        out[a:a + chunk] = (wt * f).sum(-1)
    return out
