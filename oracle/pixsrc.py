"""Pixelated source reconstruction (oracle, FP64; test infrastructure).

Sect. 3.1.1, Eqs. dpre, bayes1, s_MP, evi_ext: the source is a vector s of N_s pixel
intensities on a regular grid; the image-plane prediction is d_pre = f s with f = B L, where
L maps source pixels to image pixels through the lens equation (each image pixel averages
its ss x ss sub-pixel rays, each ray taking the bilinear interpolation of the four source
pixels around beta = theta - alpha(theta); rays outside the grid take zero) and B is the PSF
blurring ('same' convolution, zero outside the image).  Only the pixels of the arc mask
enter the fit (f is restricted to those rows after the blurring).

With a diagonal data covariance C_D, F = f^T C_D^-1 f and D = f^T C_D^-1 d, the most probable
source for regularisation strength lambda is s_MP = (F + lambda C)^-1 D (Eq. s_MP), where
C = H^T H is the curvature regularisation: H stacks, at every source pixel, the second
differences along x and along y, s(i, j-1) - 2 s(i, j) + s(i, j+1), with pixels outside the
grid taken as zero (so C is positive definite).

Evidence (Eq. evi_ext; its explicit form is cited, not printed): the marginal likelihood of the
linear Gaussian model, likelihood exp(-E_D)/Z_D with E_D = (f s - d)^T C_D^-1 (f s - d)/2,
prior exp(-lambda E_S)/Z_S with E_S = s^T C s/2, integrated over s:
    ln P(d | lambda) = -E_D(s_MP) - lambda E_S(s_MP) - ln det(F + lambda C)/2
                       + (N_s/2) ln lambda + ln det C/2 - (N_d/2) ln 2 pi - ln det C_D/2,
maximised over lambda (the delta-function approximation of Eq. evi_ext).  Its derivative in
lambda is -E_S(s_MP) - Tr[(F + lambda C)^-1 C]/2 + N_s/(2 lambda) (s_MP extremises the
exponent), so the optimum satisfies 2 lambda E_S = N_s - lambda Tr[(F + lambda C)^-1 C].

Pins (tests/test_oracle_pixsrc.py): the evidence against the direct Gaussian marginal
N(d; 0, C_D + f (lambda C)^-1 f^T); its lambda-derivative against the closed form above; the
exact recovery of a source that lies in the pixel basis from noiseless data as lambda -> 0;
the curvature operator annihilating straight lines away from the grid edge; the response f
against a direct ray-traced image of the same pixelated source.
"""
import math

import numpy as np
from scipy.optimize import minimize_scalar

from . import imaging, lens, lensmodel


class SourceGrid:
    """n_x x n_y pixel centres on [x0, x1] x [y0, y1] (pixel i, j at x0 + (j + 1/2) dx)."""

    def __init__(self, x0, x1, y0, y1, nx, ny):
        self.x0, self.y0, self.nx, self.ny = x0, y0, nx, ny
        self.dx, self.dy = (x1 - x0) / nx, (y1 - y0) / ny

    @property
    def n(self):
        return self.nx * self.ny

    def bilinear(self, bx, by):
        """(indices [..., 4], weights [..., 4]) of the bilinear interpolation at (bx, by);
        points outside the span of the pixel centres get zero weights."""
        u = (bx - self.x0) / self.dx - 0.5
        v = (by - self.y0) / self.dy - 0.5
        i0, j0 = np.floor(v).astype(np.int64), np.floor(u).astype(np.int64)
        tu, tv = u - j0, v - i0
        inside = (j0 >= 0) & (j0 + 1 < self.nx) & (i0 >= 0) & (i0 + 1 < self.ny)
        j0c, i0c = np.clip(j0, 0, self.nx - 2), np.clip(i0, 0, self.ny - 2)
        idx = np.stack([i0c * self.nx + j0c, i0c * self.nx + j0c + 1,
                        (i0c + 1) * self.nx + j0c, (i0c + 1) * self.nx + j0c + 1], -1)
        w = np.stack([(1 - tu) * (1 - tv), tu * (1 - tv), (1 - tu) * tv, tu * tv], -1)
        return idx, w * inside[..., None]


def lens_matrix(th, sysd, grid, alpha=None):
    """L [ny*nx, N_s]: each image pixel's mean over its sub-pixel rays of the bilinear weights
    (alpha(x, y, th, sis) if given, else the system's mass class)."""
    X, Y = imaging.subpixel_grid(sysd["nx"], sysd["ny"], sysd["ss"], sysd["pix"])
    ax, ay = alpha(X, Y, th, sysd["sis"]) if alpha else lensmodel.alpha(X, Y, th, sysd)
    idx, w = grid.bilinear(X - ax, Y - ay)            # [ny, nx, ss^2, 4]
    npix = sysd["nx"] * sysd["ny"]
    rows = np.broadcast_to(np.arange(npix).reshape(sysd["ny"], sysd["nx"], 1, 1), idx.shape)
    L = np.zeros((npix, grid.n))
    np.add.at(L, (rows.ravel(), idx.ravel()), w.ravel() / (sysd["ss"] ** 2))
    return L


def response(th, sysd, grid, alpha=None):
    """f = B L restricted to the mask's pixels: [N_d, N_s]."""
    L = lens_matrix(th, sysd, grid, alpha)
    psf = np.asarray(sysd["psf"], np.float64)
    ny, nx = sysd["ny"], sysd["nx"]
    f = np.stack([imaging.convolve_same(L[:, j].reshape(ny, nx), psf).ravel()
                  for j in range(grid.n)], axis=1)
    m = np.asarray(sysd["mask"]).ravel() != 0
    return f[m]


def curvature(grid):
    """C = H^T H, H the second differences along x and y with zero outside the grid."""
    H = curvature_operator(grid)
    return H.T @ H


def curvature_operator(grid):
    """H [2 N_s, N_s]: rows N_s x-differences, then N_s y-differences."""
    n, nx, ny = grid.n, grid.nx, grid.ny
    H = np.zeros((2 * n, n))
    for i in range(ny):
        for j in range(nx):
            p = i * nx + j
            H[p, p] = -2.0
            if j > 0:
                H[p, p - 1] = 1.0
            if j + 1 < nx:
                H[p, p + 1] = 1.0
            H[n + p, p] = -2.0
            if i > 0:
                H[n + p, p - nx] = 1.0
            if i + 1 < ny:
                H[n + p, p + nx] = 1.0
    return H


def solve(f, d, sig, C, lam):
    """(s_MP, ln evidence) for data d with per-pixel sigma (diagonal C_D)."""
    wi = 1.0 / (sig * sig)
    F = f.T @ (wi[:, None] * f)
    D = f.T @ (wi * d)
    A = F + lam * C
    cA = np.linalg.cholesky(A)
    s = np.linalg.solve(A, D)
    r = f @ s - d
    E_D = 0.5 * np.sum(wi * r * r)
    E_S = 0.5 * s @ (C @ s)
    logdetA = 2.0 * np.sum(np.log(np.diag(cA)))
    logdetC = 2.0 * np.sum(np.log(np.diag(np.linalg.cholesky(C))))
    Nd, Ns = len(d), len(s)
    lnP = (-E_D - lam * E_S - 0.5 * logdetA + 0.5 * Ns * math.log(lam) + 0.5 * logdetC
           - 0.5 * Nd * math.log(2 * math.pi) + np.sum(np.log(np.sqrt(wi))))
    return s, lnP


def best_lambda(f, d, sig, C, lo=1e-6, hi=1e6):
    """lambda maximising the evidence (search in ln lambda); returns (lambda, s_MP, ln P)."""
    res = minimize_scalar(lambda t: -solve(f, d, sig, C, math.exp(t))[1],
                          bounds=(math.log(lo), math.log(hi)), method="bounded",
                          options={"xatol": 1e-8})
    lam = math.exp(res.x)
    s, lnP = solve(f, d, sig, C, lam)
    return lam, s, lnP


def grid_of(sysd):
    """The system's source grid (descriptor entries spx_box = (x0, x1, y0, y1), spx_n = (nx, ny))."""
    x0, x1, y0, y1 = sysd["spx_box"]
    return SourceGrid(x0, x1, y0, y1, int(sysd["spx_n"][0]), int(sysd["spx_n"][1]))


def evidence_term(th, sysd):
    """The extended-image term of a pixelated-source system (Sect. 3.1.1): the arcs
    d_esr = data - B (lens light) on the mask's pixels are reconstructed on the system's source
    grid and scored by the evidence at the optimal regularisation (Eq. evi_ext); returns
    (ln P, lambda_hat, s_MP)."""
    grid = grid_of(sysd)
    m = np.asarray(sysd["mask"]).ravel() != 0
    ll = imaging.model_image(th, sysd, source=False).ravel()
    d = np.asarray(sysd["data"], np.float64).ravel()[m] - ll[m]
    sig = np.asarray(sysd["sigma"], np.float64).ravel()[m]
    f = response(th, sysd, grid)
    lo, hi = sysd.get("spx_lam", (1e-6, 1e6))
    lam, s, lnP = best_lambda(f, d, sig, curvature(grid), lo, hi)
    return lnP, lam, s