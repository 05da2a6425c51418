"""Kinematic PSF, aperture binning and chi^2_dyn (oracle, FP64).

Eq. binned (Sect. 2.4): [v_los^2]_l = sum_bin (I v_los^2) (x) PSF_kin / sum_bin I (x) PSF_kin,
with I v_los^2 = Sigma v_los^2 (the numerator of Eq. VLos) and I the tracer surface
brightness; Eq. Vrms: v_rms,l = sqrt([v_los^2]_l); Eq. chi2_dyn with a diagonal
covariance.  The maps live on the sub-sampled sky grid (each spaxel split into
kss x kss sub-samples that inherit the spaxel's bin); the convolution is the
discrete 'same' convolution with zero outside the grid, and bins only hold
spaxels at least the kernel radius from the grid edge.

Pins: brute-force convolution; a delta kernel is the identity.
"""
import numpy as np

from .imaging import convolve_same


def sky_subsamples(kx, ky, kss, kpix):
    """Sub-sample centres on the sky, shape (ky*kss, kx*kss)."""
    d = kpix / kss
    nx, ny = kx * kss, ky * kss
    x = (np.arange(nx) - 0.5 * (nx - 1)) * d
    y = (np.arange(ny) - 0.5 * (ny - 1)) * d
    return np.meshgrid(x, y)


def subsample_bins(bins, kss):
    return np.repeat(np.repeat(np.asarray(bins), kss, axis=0), kss, axis=1)


def bin_moments(sv2, sb, sysd):
    """Convolve both maps with PSF_kin and sum them per bin."""
    k = np.asarray(sysd["kpsf"], np.float64)
    c_num = convolve_same(sv2, k)
    c_den = convolve_same(sb, k)
    lab = subsample_bins(sysd["bins"], sysd["kss"])
    nb = sysd["n_bins"]
    num = np.zeros(nb)
    den = np.zeros(nb)
    for l in range(nb):
        m = lab == l
        num[l] = c_num[m].sum()
        den[l] = c_den[m].sum()
    return num, den


def chi2_dyn(v_pre, sysd):
    v = np.asarray(sysd["v_obs"], np.float64)
    s = np.asarray(sysd["v_sig"], np.float64)
    return float(np.sum(((v - v_pre) / s) ** 2))
