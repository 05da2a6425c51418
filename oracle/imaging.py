"""Extended-image model, PSF blurring and pixel chi^2 (oracle, FP64).

* Each pixel is split into s x s sub-pixels; every sub-pixel is ray-shot through
  the lens equation (Eq. lens_equation), the Sersic source is evaluated at beta
  and the lens light at theta; the s^2 values are averaged (the blurring matrix
  B of Table 1 acts at data resolution, N_d x N_d).
* Blurring by the PSF (Eq. dpre: f = B L): discrete 2-D convolution
  m[i,j] = sum_{a,b} P[a,b] img[i-(a-h), j-(b-h)], h = (K-1)/2, zero outside the grid.
* chi^2 (Eq. chi2 of lens_light): sum over unmasked pixels of ((d - m)/sigma)^2.

Pixel (i, j) centre: x = (j - (Nx-1)/2) p, y = (i - (Ny-1)/2) p.
Sub-pixel offsets ((m + 1/2)/s - 1/2) p.

Pins: a delta PSF is the identity; PSF flux conservation for a compact image;
brute-force 2-D convolution.
"""
import numpy as np

from . import chameleon, lens, lensmodel, light


def subpixel_grid(nx, ny, ss, pix):
    """Sub-pixel centre coordinates, shape (ny, nx, ss*ss)."""
    xc = (np.arange(nx) - 0.5 * (nx - 1)) * pix
    yc = (np.arange(ny) - 0.5 * (ny - 1)) * pix
    off = ((np.arange(ss) + 0.5) / ss - 0.5) * pix
    X = xc[None, :, None, None] + off[None, None, None, :]
    Y = yc[:, None, None, None] + off[None, None, :, None]
    X = np.broadcast_to(X, (ny, nx, ss, ss)).reshape(ny, nx, ss * ss)
    Y = np.broadcast_to(Y, (ny, nx, ss, ss)).reshape(ny, nx, ss * ss)
    return X, Y


def surface_brightness(x, y, th, sysd, alpha=None, source=True):
    """Source (through the lens) + lens light at sky points (x, y); alpha: a deflection
    function alpha(x, y, th, sis) (default: the system's mass class, lensmodel.alpha);
    source=False: the lens light alone."""
    from paper_2504_01302_b300.synth import IDX
    src = 0.0
    if source:
        ax, ay = (alpha(x, y, th, sysd["sis"]) if alpha else lensmodel.alpha(x, y, th, sysd))
        bx, by = x - ax, y - ay
        src = light.sersic_xy(bx, by, th[IDX["I_e_src"]], th[IDX["R_e_src"]], th[IDX["n_src"]],
                              sysd["src_q"], th[IDX["x_src"]], th[IDX["y_src"]], sysd["src_phi"])
    xc, yc, phi = th[IDX["x_c"]], th[IDX["y_c"]], th[IDX["phi"]]
    if lensmodel.is_composite(sysd):
        # the composite class's lens light: Chameleon profiles (Eq. Chameleon) in the galaxy frame
        xp, yp = lens.frame(x, y, xc, yc, phi)
        ll = 0.0
        for I0, wc, wt, q in lensmodel.chameleons(th, sysd):
            ll = ll + chameleon.kappa(xp, yp, I0, wc, wt, q)
        return src + ll
    ll = light.sersic_xy(x, y, th[IDX["I_e_ll"]], th[IDX["R_e_ll"]], sysd["ll_n"], sysd["ll_q"],
                         xc, yc, phi)
    for I_e, R_e, n, q in sysd["ll2"]:
        ll = ll + light.sersic_xy(x, y, I_e, R_e, n, q, xc, yc, phi)
    return src + ll


def unblurred_image(th, sysd, alpha=None, source=True):
    X, Y = subpixel_grid(sysd["nx"], sysd["ny"], sysd["ss"], sysd["pix"])
    return surface_brightness(X, Y, th, sysd, alpha, source).mean(axis=-1)


def convolve_same(img, psf):
    """True 2-D convolution, output the size of img, zero outside the grid."""
    K = psf.shape[0]
    h = (K - 1) // 2
    ny, nx = img.shape
    pad = np.zeros((ny + 2 * h, nx + 2 * h))
    pad[h:h + ny, h:h + nx] = img
    out = np.zeros((ny, nx))
    for a in range(K):
        for b in range(K):
            # m[i,j] += P[a,b] * img[i - (a-h), j - (b-h)]
            out += psf[a, b] * pad[2 * h - a:2 * h - a + ny, 2 * h - b:2 * h - b + nx]
    return out


def model_image(th, sysd, alpha=None, source=True):
    return convolve_same(unblurred_image(th, sysd, alpha, source),
                         np.asarray(sysd["psf"], np.float64))


def chi2_pix(model, sysd):
    d = np.asarray(sysd["data"], np.float64)
    s = np.asarray(sysd["sigma"], np.float64)
    m = np.asarray(sysd["mask"]) != 0
    r = (d - model) / s
    return float(np.sum(r[m] ** 2))
