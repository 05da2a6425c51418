"""Post-processing of finished chains (host side, NumPy/SciPy): model weights from the
Bayesian information criterion and H0 from the joint distance posterior.

BIC (Eqs. BIC and BIC2).  BIC = k ln n - 2 ln L_max, with the dynamics-only likelihood the
paper uses for the weighting (ln L = -chi^2_dyn/2, n = number of kinematic data points,
k = number of model parameters).  Model i gets
    f_BIC,i = exp(-(BIC_i - BIC_min)/2) / sum_j exp(-(BIC_j - BIC_min)/2).
With a scatter sigma_BIC of the BIC across source grids, the weight as a function of
Delta = BIC_i - BIC_min (1 for Delta <= 0, exp(-Delta/2) above, the paper requiring
Delta >= 0) is convolved with a Gaussian of variance sigma_BIC^2, which has the closed form
    f*(Delta) = Phi(-Delta/s) + exp(s^2/8 - Delta/2) Phi((Delta - s^2/2)/s),   s = sigma_BIC,
and the results are normalised over the models.

H0 (Sect. 5 of the results): draws of H0 ~ U[50, 120] and Omega_m ~ U[0.05, 0.5] in flat
LambdaCDM give D_d and D_dt; each D_dt is scaled by (1 - kappa_ext) with kappa_ext drawn
from the external-convergence distribution supplied by the caller (Eq. Dt external
internal); each draw is weighted by a Gaussian kernel density estimate of the chain's
joint posterior P(D_dt,int, D_d | d) (or of one of the two marginals), and H0 is
summarised by weighted percentiles.
"""
import math

import numpy as np
from scipy.special import ndtr
from scipy.stats import gaussian_kde

C_KMS = 299792.458


def bic(chi2_min, n_params, n_data):
    """BIC = k ln n - 2 ln L_max with ln L_max = -chi2_min / 2."""
    return n_params * math.log(n_data) + float(chi2_min)


def bic_weights(bics, sigma_bic=0.0):
    """Normalised model weights f_BIC (sigma_bic = 0) or f*_BIC (sigma_bic > 0)."""
    b = np.asarray(bics, np.float64)
    d = b - b.min()
    if sigma_bic <= 0.0:
        f = np.exp(-0.5 * d)
    else:
        s = float(sigma_bic)
        f = ndtr(-d / s) + np.exp(s * s / 8.0 - 0.5 * d) * ndtr((d - 0.5 * s * s) / s)
    return f / f.sum()


_GL_X, _GL_W = np.polynomial.legendre.leggauss(48)


def flat_lcdm_distances(z_d, z_s, H0, om):
    """D_d and D_dt [Mpc] for arrays of H0 [km/s/Mpc] and Omega_m in flat LambdaCDM
    (48-point Gauss-Legendre in redshift for each comoving distance)."""
    H0 = np.asarray(H0, np.float64)
    om = np.asarray(om, np.float64)

    def chi(z):
        zz = 0.5 * z * (_GL_X + 1.0)
        E = np.sqrt(om[..., None] * (1.0 + zz) ** 3 + 1.0 - om[..., None])
        return 0.5 * z * np.sum(_GL_W / E, axis=-1)

    cd, cs = chi(z_d), chi(z_s)
    D_d = C_KMS / H0 * cd / (1.0 + z_d)
    D_s = C_KMS / H0 * cs / (1.0 + z_s)
    D_ds = C_KMS / H0 * (cs - cd) / (1.0 + z_s)
    return D_d, (1.0 + z_d) * D_d * D_s / D_ds


def weighted_percentiles(x, w, q):
    o = np.argsort(x)
    c = np.cumsum(w[o])
    c /= c[-1]
    return np.interp(np.asarray(q, np.float64) / 100.0, c, x[o])


def h0_posterior(ddt_int, dd, z_d, z_s, kappa_ext_draws=None, use="both", n=500000, seed=0,
                 chain_weights=None, h0_range=(50.0, 120.0), om_range=(0.05, 0.5)):
    """H0 from a chain of (D_dt,int, D_d) [Mpc].  use: "both" (the joint posterior),
    "ddt" or "dd" (one marginal).  kappa_ext_draws: samples of kappa_ext to draw from (None:
    kappa_ext = 0).  Returns dict(h0, weight, median, lo, hi) with lo/hi the 16th/84th
    weighted percentiles."""
    rng = np.random.Generator(np.random.PCG64(seed))
    H0 = rng.uniform(*h0_range, n)
    om = rng.uniform(*om_range, n)
    D_d, D_dt = flat_lcdm_distances(z_d, z_s, H0, om)
    if kappa_ext_draws is not None:
        k = np.asarray(kappa_ext_draws, np.float64)
        D_dt = (1.0 - k[rng.integers(0, k.size, n)]) * D_dt
    chain = {"both": np.vstack([ddt_int, dd]), "ddt": np.asarray(ddt_int)[None, :],
             "dd": np.asarray(dd)[None, :]}[use]
    at = {"both": np.vstack([D_dt, D_d]), "ddt": D_dt[None, :], "dd": D_d[None, :]}[use]
    kde = gaussian_kde(chain, weights=chain_weights)
    w = kde(at)
    med, lo, hi = weighted_percentiles(H0, w, [50.0, 16.0, 84.0])
    return dict(h0=H0, weight=w, median=med, lo=lo, hi=hi)
