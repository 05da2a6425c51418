"""Lens model and unit scales of a system's mass class (oracle, FP64; test infrastructure).

Sect. 3.3 (joint modelling): the mass classes carry an internal mass sheet,
    kappa_int = (1 - lambda_int) + lambda_int kappa_gal      (Eq. kappa int),
with the constant part represented by a dPIE profile of core 45" and truncation 45.09"
(Eq. dpie_kappa) whose central convergence is 1 - lambda_int.  Here the lens model of the
class scales every deflection of the galaxy model (EPL, external shear, SIS perturbers) by
lambda_int and adds the sheet's; under an ideal (uniform) sheet this is exactly the
mass-sheet transform of Sect. 2.2 (Eq. transformed MST), with the shear scaled so that the
transform leaves the image positions and morphology unchanged.  A system chooses
    sheet = 0: no sheet (theta[20] is ignored, lambda_int = 1),
            1: the dPIE sheet of Eq. dpie_kappa (the paper's),
            2: an ideal uniform sheet kappa = 1 - lambda_int (lensing only; for the dynamics
               the dPIE stands in for it, an infinite sheet having no finite MGE).

Distances (Sect. 2.3, Eqs. critical_sfd, sfd final, D_delta_int): distance_mode 0 derives
them from H0 = theta[19] in flat LambdaCDM with D_dt,int = (1 - kappa_ext) D_dt; mode 1 samples
the lens distance D_d = theta[21] and the model time-delay distance D_dt,int = theta[22] [Mpc]
directly, as Table 2 does (H0 is then not used).  Either way
    delays:   Delta t = D_dt,int / c * Delta phi   (Eq. time delay between multiple images),
    dynamics: G Sigma_crit D_d arcsec = c^2/(4 pi) D_dt,int / ((1 + z_d) D_d) arcsec
              (Eq. sfd final: the kinematic scale depends on D_dt,int / D_d only).

The composite class (mass_class 1) replaces the EPL by the Chameleon baryons scaled by
Upsilon_*, the elliptical NFW halo and the black hole (see composite_galaxy below).

Pins: tests/test_oracle_lensmodel.py (the sheet's Jacobian by differences of its deflection,
the model's psi <-> alpha <-> Jacobian by differences, the ideal-sheet transform leaving the
images and beta_hat-mapped images unchanged and scaling delays by lambda, distance mode 1
reproducing mode 0 at the distances of the same H0).
"""
import math

import numpy as np
from scipy.special import exp1

from . import chameleon, cosmo, enfw, lens, mass_sheet, mge

IDX_LAM, IDX_DD, IDX_DDT, IDX_H0 = 20, 21, 22, 19


# ---------------------------------------------------------------------------
# composite mass class (Sect. 3.3: kappa_int,comp = (1 - lambda) + lambda (Upsilon_* I_light +
# kappa_enfw + kappa_BH)).  Parameter entries with their class meaning: theta[0] kappa_s,
# theta[1] r_s [arcsec], theta[2] q of the halo (Eq. kappa_enfw; Table 2 rho_s, r_s, q_enfw),
# theta[13] I0 and theta[14] w_t of the first Chameleon (Eq. Chameleon; its w_c and q are the
# system's ll_wc and ll_q, further Chameleons are ll2 rows (I0, w_c, w_t, q)), theta[17]
# Upsilon_*.  The baryonic convergence is Upsilon_* L_scale I_light; the black hole (mass f_BH
# Upsilon_* L_tot L_scale, L_tot the total light of the tracer MGE) is the round Gaussian of
# dispersion bh_sigma the dynamics use, in the lensing too.
# ---------------------------------------------------------------------------

def is_composite(sysd):
    return int(sysd.get("mass_class", 0)) == 1


def chameleons(th, sysd):
    """(I0, w_c, w_t, q) of each Chameleon of the lens light."""
    comps = [(float(th[13]), float(sysd["ll_wc"]), float(th[14]), float(sysd["ll_q"]))]
    comps += [tuple(float(v) for v in r) for r in np.asarray(sysd["ll2"]).reshape(-1, 4)]
    return comps


def chameleon_mges(th, sysd):
    """Per Chameleon, its 1-D MGE (Sect. 3.2) on the light range: list of (A, sigma, q)."""
    out = []
    for (I0, wc, wt, q), n in zip(chameleons(th, sysd), sysd["n_mge_light"]):
        A, sig = chameleon.mge_of(I0, wc, wt, q, sysd["light_rmin"], sysd["light_rmax"], n,
                                  sysd["mge_P"])
        out.append((A, sig, q))
    return out


def total_light(th, sysd):
    """L_tot of the tracer MGE: sum 2 pi A sigma^2 q' over its Gaussians."""
    return float(sum(np.sum(2 * math.pi * A * sig ** 2 * q) for A, sig, q in chameleon_mges(th, sysd)))


def bh_mass(th, sysd):
    if not sysd["has_bh"]:
        return 0.0
    return float(th[18] * th[17] * total_light(th, sysd) * sysd["L_scale"])


def gauss_lens(dx, dy, M, sig):
    """Round Gaussian of mass M (convergence M/(2 pi sig^2) exp(-R^2/(2 sig^2))): deflection
    M (1 - e^-t)/(pi R^2) (dx, dy), potential (M/(2 pi)) (ln t + E1(t)), t = R^2/(2 sig^2), and
    Jacobian g delta_ij + 2 g' x_i x_j, g = M (1 - e^-t)/(pi R^2)."""
    R2 = np.asarray(dx * dx + dy * dy, np.float64)
    t = R2 / (2 * sig * sig)
    # below t = 1e-4 the Taylor series of (1 - e^-t)/t (the plain form is 0/0 at the centre)
    small = t < 1e-4
    ts = np.where(small, 1.0, t)
    S0 = M / (2 * math.pi * sig * sig)
    g = np.where(small, S0 * (1 - t / 2 + t * t / 6), M * (-np.expm1(-ts)) / (math.pi * ts * 2 * sig * sig))
    gp = np.where(small, S0 * (-0.5 + t / 3) / (2 * sig * sig),
                  M / math.pi * (np.exp(-ts) / (2 * sig * sig * ts * 2 * sig * sig)
                                 - (-np.expm1(-ts)) / (ts * 2 * sig * sig) ** 2))
    psi = np.where(small, M / (2 * math.pi) * (-np.euler_gamma + t - t * t / 4),
                   M / (2 * math.pi) * (np.log(ts) + exp1(ts)))
    return (g * dx, g * dy), psi, (g + 2 * gp * dx * dx, 2 * gp * dx * dy, 2 * gp * dx * dy,
                                   g + 2 * gp * dy * dy)


def _rot_jac(j, phi):
    c, s = math.cos(phi), math.sin(phi)
    j11, j12, j21, j22 = j
    return (c * c * j11 - c * s * (j12 + j21) + s * s * j22,
            c * s * (j11 - j22) + c * c * j12 - s * s * j21,
            c * s * (j11 - j22) + c * c * j21 - s * s * j12,
            s * s * j11 + c * s * (j12 + j21) + c * c * j22)


def composite_galaxy(x, y, th, sysd):
    """Deflection, potential and Jacobian of the composite galaxy (baryons + halo + black hole,
    external shear and SIS perturbers), before the sheet."""
    ks, rs, qe, phi, xc, yc, gext, pext = (float(v) for v in th[:8])
    ups = float(th[17]) * sysd["L_scale"]
    xp, yp = lens.frame(x, y, xc, yc, phi)
    axp = np.zeros_like(np.asarray(xp, np.float64))
    ayp = np.zeros_like(axp)
    pp = np.zeros_like(axp)
    jf = [np.zeros_like(axp) for _ in range(4)]
    for I0, wc, wt, q in chameleons(th, sysd):
        a = chameleon.alpha(xp, yp, ups * I0, wc, wt, q)
        axp, ayp = axp + a[0], ayp + a[1]
        pp = pp + chameleon.psi(xp, yp, ups * I0, wc, wt, q)
        jf = [u + v for u, v in zip(jf, chameleon.jac(xp, yp, ups * I0, wc, wt, q))]
    a = enfw.enfw_alpha(xp, yp, ks, rs, qe)
    axp, ayp = axp + a[0], ayp + a[1]
    pp = pp + enfw.enfw_psi(xp, yp, ks, rs, qe)
    jf = [u + v for u, v in zip(jf, enfw.enfw_jac(xp, yp, ks, rs, qe))]
    ax, ay = lens.to_sky(axp, ayp, phi)
    j = list(_rot_jac(jf, phi))
    dx, dy = x - xc, y - yc
    M = bh_mass(th, sysd)
    if M > 0:
        (bx, by), bp, bj = gauss_lens(dx, dy, M, sysd["bh_sigma"])
        ax, ay, pp = ax + bx, ay + by, pp + bp
        j = [u + v for u, v in zip(j, bj)]
    sx, sy = lens.shear_alpha(dx, dy, gext, pext)
    ax, ay = ax + sx, ay + sy
    pp = pp + lens.shear_psi(dx, dy, gext, pext)
    g1, g2 = gext * math.cos(2 * pext), gext * math.sin(2 * pext)
    j = [j[0] + g1, j[1] + g2, j[2] + g2, j[3] - g1]
    for tEs, xs, ys in sysd["sis"]:
        a1, a2 = lens.sis_alpha(x, y, tEs, xs, ys)
        ax, ay = ax + a1, ay + a2
        pp = pp + lens.sis_psi(x, y, tEs, xs, ys)
        j = [u + v for u, v in zip(j, lens.sis_jac(x, y, tEs, xs, ys))]
    return (ax, ay), pp, tuple(j)


def enfw_mass_mge(th, sysd):
    """Halo Gaussians of the dynamics: the 1-D MGE (Euler inversion, Sect. 3.2) of the exact
    kappa_s k(R / r_s) on the mass range, axis ratio q of the halo."""
    ks, rs, qe = float(th[0]), float(th[1]), float(th[2])
    sig, A = mge.mge_1d(lambda z: ks * enfw.nfw_k_complex(z / rs), sysd["mass_rmin"],
                        sysd["mass_rmax"], sysd["n_mge_mass"], sysd["mge_P"])
    return A, sig, np.full(len(sig), qe)


def sheet_of(th, sysd):
    """The internal sheet of this system at parameters th, or None."""
    kind = int(sysd.get("sheet", 0))
    if kind == 0:
        return None
    return dict(lam=float(th[IDX_LAM]), kind="ideal" if kind == 2 else "dpie",
                rc=float(sysd.get("sheet_rc", mass_sheet.R_CORE)),
                rt=float(sysd.get("sheet_rt", mass_sheet.R_TR)))


def lam_of(th, sysd):
    return 1.0 if int(sysd.get("sheet", 0)) == 0 else float(th[IDX_LAM])


def sheet_jac(dx, dy, sheet):
    """d alpha_sheet / d theta of the dPIE sheet (radial deflection s(R^2) (dx, dy)):
    a_ij = s delta_ij + 2 s'(R^2) x_i x_j with
    s = a0 f [1/(r_c + Q_c) - 1/(r_t + Q_t)], Q = sqrt(R^2 + r^2),
    s' = a0 f [-1/(2 Q_c (r_c + Q_c)^2) + 1/(2 Q_t (r_t + Q_t)^2)]."""
    lam, rc, rt = sheet["lam"], sheet["rc"], sheet["rt"]
    if sheet["kind"] == "ideal":
        z = np.zeros_like(np.asarray(dx, np.float64))
        return z + (1 - lam), z, z, z + (1 - lam)
    a0 = mass_sheet.dpie_a0(lam, rc, rt)
    f = rt * rt / (rt * rt - rc * rc)
    R2 = dx * dx + dy * dy
    Qc, Qt = np.sqrt(R2 + rc * rc), np.sqrt(R2 + rt * rt)
    s = a0 * f * (1.0 / (rc + Qc) - 1.0 / (rt + Qt))
    sp = a0 * f * (-1.0 / (2 * Qc * (rc + Qc) ** 2) + 1.0 / (2 * Qt * (rt + Qt) ** 2))
    return s + 2 * sp * dx * dx, 2 * sp * dx * dy, 2 * sp * dx * dy, s + 2 * sp * dy * dy


def alpha(x, y, th, sysd):
    """Deflection of the class: lambda x (galaxy + shear + perturbers) + sheet."""
    if is_composite(sysd):
        ax, ay = composite_galaxy(x, y, th, sysd)[0]
    else:
        ax, ay = lens.alpha_total(x, y, th, sysd["sis"])
    sh = sheet_of(th, sysd)
    if sh is None:
        return ax, ay
    sx, sy = mass_sheet.sheet_alpha(x - th[4], y - th[5], sh)
    return sh["lam"] * ax + sx, sh["lam"] * ay + sy


def psi(x, y, th, sysd):
    p = composite_galaxy(x, y, th, sysd)[1] if is_composite(sysd) else lens.psi_total(x, y, th, sysd["sis"])
    sh = sheet_of(th, sysd)
    if sh is None:
        return p
    return sh["lam"] * p + mass_sheet.sheet_psi(x - th[4], y - th[5], sh)


def jac(x, y, th, sysd):
    a = composite_galaxy(x, y, th, sysd)[2] if is_composite(sysd) else lens.jac_total(x, y, th, sysd["sis"])
    sh = sheet_of(th, sysd)
    if sh is None:
        return a
    b = sheet_jac(x - th[4], y - th[5], sh)
    return tuple(sh["lam"] * u + v for u, v in zip(a, b))


def distances_int(th, sysd):
    """(D_d, D_dt,int) in Mpc for this system's distance mode."""
    if int(sysd.get("distance_mode", 0)) == 1:
        return float(th[IDX_DD]), float(th[IDX_DDT])
    D_d, _, _, D_dt = cosmo.distances(sysd["z_d"], sysd["z_s"], float(th[IDX_H0]), sysd["omega_m"])
    return D_d, (1.0 - sysd["kappa_ext"]) * D_dt


def delay_unit(th, sysd):
    """Days of delay per arcsec^2 of Fermat-potential difference."""
    if int(sysd.get("distance_mode", 0)) == 1:
        return float(th[IDX_DDT]) * cosmo.MPC_KM / cosmo.C_KMS * cosmo.ARCSEC ** 2 / cosmo.DAY_S
    return cosmo.delay_days_per_arcsec2(sysd["z_d"], sysd["z_s"], float(th[IDX_H0]),
                                        sysd["omega_m"], sysd["kappa_ext"])


def v2_unit(th, sysd):
    """km^2/s^2 per (kappa x arcsec) of the dynamics (see the module docstring)."""
    if int(sysd.get("distance_mode", 0)) == 1:
        D_d, D_dt_int = float(th[IDX_DD]), float(th[IDX_DDT])
        return cosmo.C_KMS ** 2 / (4 * math.pi) * D_dt_int / ((1 + sysd["z_d"]) * D_d) * cosmo.ARCSEC
    return cosmo.v2_unit(sysd["z_d"], sysd["z_s"], sysd["omega_m"], sysd["kappa_ext"])


def sheet_mass(th, sysd):
    """Round mass Gaussians (kap0, sig, qp) of the sheet for the dynamics (the dPIE's 1-D MGE
    of Sect. 3.2 on the system's sheet range), or None."""
    sh = sheet_of(th, sysd)
    if sh is None:
        return None
    return mass_sheet.sheet_mge(sh["lam"], n=int(sysd.get("sheet_n", 40)),
                                P=int(sysd["mge_P"]), rmin=float(sysd.get("sheet_rmin", 0.1)),
                                rmax=float(sysd.get("sheet_rmax", 1000.0)), rc=sh["rc"], rt=sh["rt"])


def solve_images(beta, th, sysd, guesses, tol=1e-13, iters=100):
    """Newton solution of beta = theta - alpha(theta) for the class's lens model from each
    starting guess (as lens.solve_images for the bare EPL model)."""
    out = []
    for g0 in guesses:
        p = np.array(g0, np.float64)
        for _ in range(iters):
            ax, ay = alpha(np.array([p[0]]), np.array([p[1]]), th, sysd)
            a11, a12, a21, a22 = jac(np.array([p[0]]), np.array([p[1]]), th, sysd)
            F = np.array([p[0] - ax[0] - beta[0], p[1] - ay[0] - beta[1]])
            A = np.array([[1 - a11[0], -a12[0]], [-a21[0], 1 - a22[0]]])
            step = np.linalg.solve(A, F)
            p = p - step
            if np.max(np.abs(step)) < tol:
                break
        out.append(p)
    return np.array(out)
