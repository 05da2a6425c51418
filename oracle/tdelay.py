"""Time delays from the Fermat potential (oracle, FP64).

Eq. fermat potential: phi(theta, beta) = |theta - beta|^2/2 - psi(theta).
Eq. time delay between multiple images: Delta t_ij = D_dt/c [phi_i - phi_j], here
with the modelled distance D_dt,int = (1 - kappa_ext) D_dt (Eq. Dt external internal).
The source position is the magnification-weighted mean of the images mapped to
the source plane (Sect. 3.1.1, around Eq. chi2_img), weights |mu_j| = 1/|det(I - d alpha/d theta)|,
and phi is evaluated at the observed image positions.  Image 0 is the reference:
Eq. chi2_tmd sums the N_img - 1 delays Delta t_i0.

Image positions (Eq. chi2_img, Sect. 3.1.1): the observed images are mapped to the
source plane, their magnification-weighted mean beta_hat is mapped back to the image
plane, giving theta_pre, and chi^2_img = sum_j |theta_j - theta_pre_j|^2 / sigma_j^2.  The
paper does not say how the mapping back is solved; here each theta_pre_j is the root of
the lens equation theta - alpha(theta) = beta_hat reached by Newton iterations started at
the observed theta_j (the image the observed one stands for).

Pins: Delta t proportional to 1/H0; a constant added to psi cancels; at exact
images (Newton-solved) beta_hat equals the true source and grad phi = 0; chi^2_img is zero
at exact images, theta_pre solves the lens equation, and chi^2_img grows as the square of a
small displacement of one image.
"""
import numpy as np

from . import lensmodel


def beta_hat(th, sysd, img):
    x, y = img[:, 0], img[:, 1]
    ax, ay = lensmodel.alpha(x, y, th, sysd)
    a11, a12, a21, a22 = lensmodel.jac(x, y, th, sysd)
    det = (1 - a11) * (1 - a22) - a12 * a21
    w = 1.0 / np.abs(det)
    bx, by = x - ax, y - ay
    return np.array([np.sum(w * bx) / w.sum(), np.sum(w * by) / w.sum()])


def fermat(th, sysd, img, bh):
    x, y = img[:, 0], img[:, 1]
    return 0.5 * ((x - bh[0]) ** 2 + (y - bh[1]) ** 2) - lensmodel.psi(x, y, th, sysd)


def delays(th, sysd):
    """Model delays Delta t_i0 [days], i = 1..N_img-1 (the lens model and distances of the
    system's mass class and distance mode, oracle/lensmodel.py)."""
    img = np.asarray(sysd["img_xy"], np.float64)
    bh = beta_hat(th, sysd, img)
    ph = fermat(th, sysd, img, bh)
    return lensmodel.delay_unit(th, sysd) * (ph[1:] - ph[0])


def chi2_tmd(dt, sysd):
    o = np.asarray(sysd["dt_obs"], np.float64)
    s = np.asarray(sysd["dt_sig"], np.float64)
    return float(np.sum(((o - dt) / s) ** 2))


def predicted_images(th, sysd, tol=1e-14, iters=50):
    """theta_pre: beta_hat of the observed images mapped back to the image plane by Newton
    iterations on theta - alpha(theta) = beta_hat started at each observed image."""
    img = np.asarray(sysd["img_xy"], np.float64)
    bh = beta_hat(th, sysd, img)
    out = np.empty_like(img)
    for j, t0 in enumerate(img):
        t = t0.copy()
        for _ in range(iters):
            ax, ay = lensmodel.alpha(np.array([t[0]]), np.array([t[1]]), th, sysd)
            a11, a12, a21, a22 = lensmodel.jac(np.array([t[0]]), np.array([t[1]]), th, sysd)
            f = np.array([t[0] - ax[0] - bh[0], t[1] - ay[0] - bh[1]])
            A = np.array([[1 - a11[0], -a12[0]], [-a21[0], 1 - a22[0]]])
            step = np.linalg.solve(A, f)
            t = t - step
            if np.max(np.abs(step)) < tol:
                break
        out[j] = t
    return out


def chi2_img(th, sysd):
    img = np.asarray(sysd["img_xy"], np.float64)
    sig = np.asarray(sysd["img_sig"], np.float64)
    pre = predicted_images(th, sysd)
    return float(np.sum(np.sum((img - pre) ** 2, axis=1) / sig ** 2))
