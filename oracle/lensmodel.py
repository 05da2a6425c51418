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

Pins: tests/test_oracle_lensmodel.py (the sheet's Jacobian by differences of its deflection,
the model's psi <-> alpha <-> Jacobian by differences, the ideal-sheet transform leaving the
images and beta_hat-mapped images unchanged and scaling delays by lambda, distance mode 1
reproducing mode 0 at the distances of the same H0).
"""
import math

import numpy as np

from . import cosmo, lens, mass_sheet

IDX_LAM, IDX_DD, IDX_DDT, IDX_H0 = 20, 21, 22, 19


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
    ax, ay = lens.alpha_total(x, y, th, sysd["sis"])
    sh = sheet_of(th, sysd)
    if sh is None:
        return ax, ay
    sx, sy = mass_sheet.sheet_alpha(x - th[4], y - th[5], sh)
    return sh["lam"] * ax + sx, sh["lam"] * ay + sy


def psi(x, y, th, sysd):
    p = lens.psi_total(x, y, th, sysd["sis"])
    sh = sheet_of(th, sysd)
    if sh is None:
        return p
    return sh["lam"] * p + mass_sheet.sheet_psi(x - th[4], y - th[5], sh)


def jac(x, y, th, sysd):
    a = lens.jac_total(x, y, th, sysd["sis"])
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
