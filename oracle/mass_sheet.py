"""Internal mass sheet of the EPL mass class (oracle, FP64; test infrastructure).

Sect. 3.3 (joint modelling): the EPL class is kappa_int = (1 - lambda_int) + lambda_int kappa_epl,
with the constant sheet (1 - lambda_int) represented by a dual pseudo-isothermal profile
(dPIE, Eq. dpie_kappa) of core r_core = 45" and truncation r_tr = 45.09":
    kappa_dPIE(R) = (a0/2) f (1/sqrt(R^2 + r_core^2) - 1/sqrt(R^2 + r_tr^2)),
    f = r_tr^2/(r_tr^2 - r_core^2),
flat out to ~20" and vanishing far out; a0 is set here from lambda_int so that the sheet's
central value is 1 - lambda_int (the paper's small-R form of lambda_int = 1 - kappa_dPIE).
The sheet is centred on the lens centre.

For this circular profile the mean convergence inside R gives the deflection (Gauss):
    alpha(R) = a0 f R [1/(r_core + sqrt(R^2 + r_core^2)) - 1/(r_tr + sqrt(R^2 + r_tr^2))]
along (theta - c)/R, and the potential (up to a constant)
    psi(R) = a0 f [sqrt(R^2 + r_core^2) - r_core ln(r_core + sqrt(R^2 + r_core^2))
                   - sqrt(R^2 + r_tr^2) + r_tr ln(r_tr + sqrt(R^2 + r_tr^2))],
evaluated as psi(R) - psi(0) in a form free of cancelling constants (dpie_psi).
The ideal sheet (kappa = 1 - lambda_int everywhere) has alpha = (1 - lambda) (theta - c) and
psi = (1 - lambda) |theta - c|^2 / 2.

The lens model of the class scales every deflection of the galaxy model (EPL, shear, SIS
perturbers) by lambda_int and adds the sheet.  Under the ideal sheet this is the
mass-sheet transform (Sect. 2.2, the MSD): beta -> lambda beta + (1 - lambda) c, so a
source moved and resized accordingly gives the same images, and Fermat-potential
differences (time delays) scale by lambda.

For the dynamics the sheet joins the galaxy's mass Gaussians through its own 1-D MGE
(class_mass); Sigma v_los^2 is linear in the mass Gaussians' amplitudes, so the sheet adds
its own term to lambda times the galaxy's.

Pins (tests/test_oracle_mass_sheet.py): the deflection against Gauss's theorem by
quadrature of kappa; the potential's gradient against the deflection; the central
convergence 1 - lambda; exact invariance of the model image and image positions, and
lambda-scaled delays, under the ideal sheet; the dPIE sheet's departure from that inside
the arcs; the MGE of the dPIE convergence; the linearity of Sigma v^2 in the class's mass
model, and the change of v_rms between two lensing-equivalent models (Sect. 2.2: the
kinematics break the mass-sheet degeneracy).
"""
import numpy as np

from . import lens, mge

R_CORE = 45.0
R_TR = 45.09


def dpie_a0(lam, rc=R_CORE, rt=R_TR):
    """Normalisation a0 with central convergence 1 - lam."""
    f = rt * rt / (rt * rt - rc * rc)
    return 2.0 * (1.0 - lam) / (f * (1.0 / rc - 1.0 / rt))


def dpie_kappa(R, a0, rc=R_CORE, rt=R_TR):
    """Convergence at radius R (real or complex)."""
    f = rt * rt / (rt * rt - rc * rc)
    R2 = R * R
    return 0.5 * a0 * f * (1.0 / np.sqrt(R2 + rc * rc) - 1.0 / np.sqrt(R2 + rt * rt))


def dpie_alpha(dx, dy, a0, rc=R_CORE, rt=R_TR):
    f = rt * rt / (rt * rt - rc * rc)
    R2 = dx * dx + dy * dy
    s = a0 * f * (1.0 / (rc + np.sqrt(R2 + rc * rc)) - 1.0 / (rt + np.sqrt(R2 + rt * rt)))
    return s * dx, s * dy


def dpie_psi(dx, dy, a0, rc=R_CORE, rt=R_TR):
    """psi(R) - psi(0) = a0 f [g(R; r_core) - g(R; r_tr)],
    g(R; r) = sqrt(R^2 + r^2) - r - r ln((r + sqrt(R^2 + r^2))/(2 r)), written without the
    large constants that cancel (r_tr is close to r_core)."""
    f = rt * rt / (rt * rt - rc * rc)
    R2 = dx * dx + dy * dy

    def g(r):
        qr = np.sqrt(R2 + r * r) + r
        return R2 / qr - r * np.log1p(R2 / (2.0 * r * qr))
    return a0 * f * (g(rc) - g(rt))


def sheet_alpha(dx, dy, sheet):
    lam = sheet["lam"]
    if sheet.get("kind", "dpie") == "ideal":
        return (1.0 - lam) * dx, (1.0 - lam) * dy
    return dpie_alpha(dx, dy, dpie_a0(lam, sheet.get("rc", R_CORE), sheet.get("rt", R_TR)),
                      sheet.get("rc", R_CORE), sheet.get("rt", R_TR))


def sheet_psi(dx, dy, sheet):
    lam = sheet["lam"]
    if sheet.get("kind", "dpie") == "ideal":
        return 0.5 * (1.0 - lam) * (dx * dx + dy * dy)
    return dpie_psi(dx, dy, dpie_a0(lam, sheet.get("rc", R_CORE), sheet.get("rt", R_TR)),
                    sheet.get("rc", R_CORE), sheet.get("rt", R_TR))


def alpha_fn(sheet):
    """Deflection of the class's lens model, lambda x (EPL + shear + SIS) + sheet, with the
    signature of lens.alpha_total."""
    def alpha(x, y, th, sis):
        ax, ay = lens.alpha_total(x, y, th, sis)
        sx, sy = sheet_alpha(x - th[4], y - th[5], sheet)
        return sheet["lam"] * ax + sx, sheet["lam"] * ay + sy
    return alpha


def psi_fn(sheet):
    def psi(x, y, th, sis):
        return sheet["lam"] * lens.psi_total(x, y, th, sis) + sheet_psi(x - th[4], y - th[5], sheet)
    return psi


def sheet_mge(lam, n=40, P=10, rmin=0.1, rmax=1000.0, rc=R_CORE, rt=R_TR):
    """Round mass Gaussians (kap0, sig, qp) of the dPIE sheet by the 1-D MGE of Sect. 3.2,
    to join the galaxy's (scaled by lam) as the dynamics' mass model."""
    a0 = dpie_a0(lam, rc, rt)
    sig, A = mge.mge_1d(lambda z: dpie_kappa(z, a0, rc, rt), rmin, rmax, n, P)
    return dict(kap0=A, sig=sig, qp=np.ones_like(sig))


def class_mass(ms_gal, lam, **kw):
    """Mass Gaussians of kappa_int = lam kappa_gal + kappa_dPIE."""
    sh = sheet_mge(lam, **kw)
    return dict(kap0=np.concatenate([lam * ms_gal["kap0"], sh["kap0"]]),
                sig=np.concatenate([ms_gal["sig"], sh["sig"]]),
                qp=np.concatenate([ms_gal["qp"], sh["qp"]]))
