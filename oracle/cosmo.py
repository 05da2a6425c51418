"""Cosmological distances and unit constants (oracle, FP64).

Eq. time delay distance (Sect. 2.1): D_dt = (1+z_d) D_d D_s / D_ds, proportional
to 1/H0.  Flat LambdaCDM as in Table 2 (H0=82.5, Om=0.27).  Critical density
(Eq. critical_sfd, Sect. 2.3): Sigma_crit = c^2/(4 pi G) D_dt / ((1+z_d) D_d^2).
The external-convergence rescaling D_dt,int = (1-kappa_ext) D_dt follows
Eq. Dt external internal.

Pins: D_d and D_dt printed in Table 2 and its footnote; D_dt proportional to 1/H0;
v2_unit by the singular isothermal sphere's sigma^2 = theta_E c^2 D_s/(4 pi D_ds) reached
through the MGE and the Jeans solution; delay_days_per_arcsec2 by the SIS two-image delay
D_dt (theta_A^2 - theta_B^2)/(2c) in SI units.
"""
import math

from scipy.integrate import quad

C_KMS = 299792.458                 # speed of light [km/s]
ARCSEC = math.pi / 648000.0        # 1 arcsec in radians
MPC_KM = 3.0856775814913673e19     # 1 Mpc in km
DAY_S = 86400.0


def comoving(z, H0, om):
    """Line-of-sight comoving distance [Mpc] in flat LambdaCDM."""
    val, _ = quad(lambda zz: 1.0 / math.sqrt(om * (1 + zz) ** 3 + 1.0 - om), 0.0, z,
                  epsabs=0.0, epsrel=1e-13, limit=200)
    return C_KMS / H0 * val


def distances(z_d, z_s, H0, om):
    """Angular-diameter distances D_d, D_s, D_ds and the time-delay distance D_dt [Mpc]."""
    cd, cs = comoving(z_d, H0, om), comoving(z_s, H0, om)
    D_d = cd / (1 + z_d)
    D_s = cs / (1 + z_s)
    D_ds = (cs - cd) / (1 + z_s)
    D_dt = (1 + z_d) * D_d * D_s / D_ds
    return D_d, D_s, D_ds, D_dt


def v2_unit(z_d, z_s, om, kappa_ext=0.0):
    """Velocity^2 [km^2/s^2] carried by G * Sigma_crit * (1 arcsec at D_d) for a
    surface density of kappa = 1 and a length of 1 arcsec.

    G Sigma_crit D_d arcsec = c^2/(4 pi) * D_dt,int / ((1+z_d) D_d) * arcsec
    (Eq. critical_sfd with the internal distance of Eq. sfd final).  The ratio
    D_dt/D_d does not depend on H0, so neither does the dynamics."""
    D_d, _, _, D_dt = distances(z_d, z_s, 70.0, om)
    D_dt_int = (1.0 - kappa_ext) * D_dt
    return C_KMS ** 2 / (4 * math.pi) * D_dt_int / ((1 + z_d) * D_d) * ARCSEC


def delay_days_per_arcsec2(z_d, z_s, H0, om, kappa_ext=0.0):
    """Days of delay per arcsec^2 of Fermat-potential difference (Eq. time delay
    between multiple images) with the modelled distance D_dt,int = (1-kappa_ext) D_dt."""
    _, _, _, D_dt = distances(z_d, z_s, H0, om)
    D_dt_int = (1.0 - kappa_ext) * D_dt
    return D_dt_int * MPC_KM / C_KMS * ARCSEC ** 2 / DAY_S
