"""Pins of the pixelated source reconstruction (oracle/pixsrc.py), Sect. 3.1.1.

* the evidence of the regularised inversion against the direct Gaussian marginal
  ln N(d; 0, C_D + f (lambda C)^-1 f^T), computed from the dense data covariance;
* its derivative in lambda against -E_S(s_MP) - Tr[(F + lambda C)^-1 C]/2 + N_s/(2 lambda);
* a source in the pixel basis is recovered from noiseless data as lambda -> 0;
* the curvature operator annihilates a straight line away from the grid edge;
* the response f = B L against an image ray-traced through SciPy's linear grid interpolator
  of the same pixelated source (independent of the operator's own bilinear weights)."""
import math

import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

from oracle import imaging, lens, model, pixsrc
from paper_2504_01302_b300 import synth


I = synth.IDX


@pytest.fixture(scope="module")
def setup():
    # the 64^2 correctness system, whose Einstein ring lies inside the image: every pixel of a
    # 10 x 10 grid over the source region is reached by rays, so F is non-singular
    sys_list, ths, _ = model.workload(0)
    s, th = sys_list[0], ths[0].copy()
    c = (th[I["x_src"]], th[I["y_src"]])
    grid = pixsrc.SourceGrid(c[0] - 0.4, c[0] + 0.4, c[1] - 0.4, c[1] + 0.4, 10, 10)
    f = pixsrc.response(th, s, grid)
    m = np.asarray(s["mask"]).ravel() != 0
    sig = np.asarray(s["sigma"], np.float64).ravel()[m]
    C = pixsrc.curvature(grid)
    rng = np.random.Generator(np.random.PCG64(5))
    s_true = np.exp(-((np.arange(100) % 10 - 4.5) ** 2 + (np.arange(100) // 10 - 4.5) ** 2) / 8.0)
    d = f @ s_true + sig * rng.standard_normal(len(sig))
    return s, th, grid, f, sig, C, s_true, d


def test_evidence_is_the_gaussian_marginal(setup):
    s, th, grid, f, sig, C, s_true, d = setup
    for lam in (0.1, 10.0):
        _, lnP = pixsrc.solve(f, d, sig, C, lam)
        cov = np.diag(sig * sig) + f @ np.linalg.solve(lam * C, f.T)
        cl = np.linalg.cholesky(cov)
        z = np.linalg.solve(cl, d)
        ref = -0.5 * z @ z - np.sum(np.log(np.diag(cl))) - 0.5 * len(d) * math.log(2 * math.pi)
        assert abs(lnP - ref) < 1e-8 * abs(ref), (lam, lnP, ref)


def test_evidence_lambda_derivative(setup):
    s, th, grid, f, sig, C, s_true, d = setup
    lam = 3.0
    h = 1e-4 * lam
    fd = (pixsrc.solve(f, d, sig, C, lam + h)[1] - pixsrc.solve(f, d, sig, C, lam - h)[1]) / (2 * h)
    sMP, _ = pixsrc.solve(f, d, sig, C, lam)
    wi = 1.0 / (sig * sig)
    A = f.T @ (wi[:, None] * f) + lam * C
    ana = -0.5 * sMP @ (C @ sMP) - 0.5 * np.trace(np.linalg.solve(A, C)) + 0.5 * grid.n / lam
    assert abs(fd - ana) < 1e-6 * max(abs(ana), 1.0), (fd, ana)
    # and the optimum satisfies 2 lambda E_S = N_s - lambda Tr[A^-1 C]
    lam_b, sb, _ = pixsrc.best_lambda(f, d, sig, C)
    Ab = f.T @ (wi[:, None] * f) + lam_b * C
    lhs = lam_b * sb @ (C @ sb)
    rhs = grid.n - lam_b * np.trace(np.linalg.solve(Ab, C))
    assert abs(lhs - rhs) < 1e-4 * grid.n, (lam_b, lhs, rhs)


def test_noiseless_pixel_source_recovered(setup):
    s, th, grid, f, sig, C, s_true, d = setup
    sMP, _ = pixsrc.solve(f, f @ s_true, sig, C, 1e-9)
    assert np.max(np.abs(sMP - s_true)) < 1e-5 * np.max(s_true)


def test_curvature_annihilates_lines():
    grid = pixsrc.SourceGrid(0.0, 1.0, 0.0, 1.0, 7, 6)
    H = pixsrc.curvature_operator(grid)
    j, i = np.meshgrid(np.arange(7), np.arange(6))
    line = (0.3 + 1.7 * j - 0.9 * i).ravel()
    r = H @ line
    interior_x = ((j > 0) & (j < 6)).ravel()
    interior_y = ((i > 0) & (i < 5)).ravel()
    assert np.max(np.abs(r[:grid.n][interior_x])) < 1e-12
    assert np.max(np.abs(r[grid.n:][interior_y])) < 1e-12
    assert np.all(np.linalg.eigvalsh(pixsrc.curvature(grid)) > 0)


def test_response_matches_ray_traced_image(setup):
    s, th, grid, f, sig, C, s_true, d = setup
    xs = grid.x0 + (np.arange(grid.nx) + 0.5) * grid.dx
    ys = grid.y0 + (np.arange(grid.ny) + 0.5) * grid.dy
    interp = RegularGridInterpolator((ys, xs), s_true.reshape(grid.ny, grid.nx), method="linear",
                                     bounds_error=False, fill_value=0.0)
    X, Y = imaging.subpixel_grid(s["nx"], s["ny"], s["ss"], s["pix"])
    ax, ay = lens.alpha_total(X, Y, th, s["sis"])
    img = interp(np.stack([(Y - ay).ravel(), (X - ax).ravel()], -1)).reshape(X.shape).mean(-1)
    ref = imaging.convolve_same(img, np.asarray(s["psf"], np.float64)).ravel()
    m = np.asarray(s["mask"]).ravel() != 0
    assert np.max(np.abs(f @ s_true - ref[m])) < 1e-12 * np.max(np.abs(ref))


def test_evidence_term_recovers_a_pixel_source_under_the_lens_light():
    # the composition used as the image term of a pixelated-source system: noiseless data =
    # blurred lens light + (B L s_true) over the whole image; the arcs after subtracting the
    # model's own lens light are reconstructed on the system's grid, and at the optimal
    # regularisation of noiseless data s_MP returns s_true (lens light not subtracted, or the
    # mask mishandled, would leave the lens light in the source)
    sys_list, ths, _ = model.workload(0)
    s, th = dict(sys_list[0]), ths[0].copy()
    c = (th[I["x_src"]], th[I["y_src"]])
    s.update(src_pix=1, spx_box=(c[0] - 0.4, c[0] + 0.4, c[1] - 0.4, c[1] + 0.4), spx_n=(10, 10),
             spx_lam=(1e-8, 1e4))
    grid = pixsrc.grid_of(s)
    s_true = np.exp(-((np.arange(100) % 10 - 4.5) ** 2 + (np.arange(100) // 10 - 4.5) ** 2) / 8.0)
    L = pixsrc.lens_matrix(th, s, grid)
    arcs = imaging.convolve_same((L @ s_true).reshape(s["ny"], s["nx"]), np.asarray(s["psf"], np.float64))
    s["data"] = imaging.model_image(th, s, source=False) + arcs
    lnP, lam, s_mp = pixsrc.evidence_term(th, s)
    assert np.max(np.abs(s_mp - s_true)) < 2e-3 * np.max(s_true), np.max(np.abs(s_mp - s_true))
    ev = model.evaluate(th, s)
    assert ev["status"] == 0 and ev["chi2_pix"] == -2 * lnP and ev["image"] is None
