// Lens-model arithmetic of the quasar images (FP64), templated on the scalar type so the
// gradient kernel can run it on dual numbers.  Formulas:
//  * EPL deflection: Tessore & Metcalf (2015) series for the App. C convergence,
//    alpha' = 2 b_TM/(1+q) (b_TM/R)^(t-1) sum_n Omega_n, b_TM = q b, R = sqrt(q^2 x^2 + y^2),
//    Omega_0 = e^{i ph}, Omega_n = -f (2n-(2-t))/(2n+(2-t)) e^{2 i ph} Omega_{n-1}.
//  * EPL potential psi = (x alpha_x + y alpha_y)/(2-t) and Jacobian from homogeneity,
//    complex shear = ((1-t) alpha - kappa z)/conj(z).
//  * External shear psi = gamma/2 R^2 cos(2 phi - 2 phi_ext) about the lens centre (Sect. 3.3).
//  * SIS perturber psi = theta_E |theta - theta_s|.
//  * Delays (Eqs. fermat potential, time delay between multiple images, chi2_tmd): source
//    at the |mu|-weighted mean of the images mapped back (Sect. 3.1.1), image 0 the reference.
#pragma once
#include <math.h>

#include "dual.cuh"

template <class T>
struct LensEvalT {
  T ax, ay;              // deflection (sky)
  T a11, a12, a21, a22;  // d alpha / d theta (sky)
  T psi;                 // potential
};

// EPL + shear + SIS at sky point (x, y); th = parameter vector (entries 0..7 used).  The
// position may be a plain double or of the parameter type (Newton iterates on positions).
template <class T, class P = double>
__device__ inline LensEvalT<T> lens_eval_t(P x, P y, const T *th, const double *sis, int n_sis) {
  const T tE = th[0], g = th[1], q = th[2], phi = th[3], xc = th[4], yc = th[5];
  const T gext = th[6], pext = th[7];
  const T t = g - 1.0;
  const T cphi = dcos(phi), sphi = dsin(phi);
  const T dx = x - xc, dy = y - yc;
  const T xp = cphi * dx + sphi * dy, yp = -sphi * dx + cphi * dy;
  const T b = dpow(2.0 / (1.0 + q), 1.0 / t) * tE;
  const T bt = q * b;
  const T R = dsqrt(q * q * xp * xp + yp * yp);
  const T wr = q * xp / R, wi = yp / R;
  const T w2r = wr * wr - wi * wi, w2i = 2.0 * wr * wi;
  const T f = (1.0 - q) / (1.0 + q);
  int nt = 0;
  if (dval(f) > 0.0) nt = (int)ceil(log(1e-16) / log(dval(f)));
  if (nt > 200) nt = 200;
  T omr = wr, omi = wi, Sr = wr, Si = wi;
  for (int n = 1; n <= nt; ++n) {
    const T rho = -f * (2.0 * n - (2.0 - t)) / (2.0 * n + (2.0 - t));
    const T nr = rho * (w2r * omr - w2i * omi);
    const T ni = rho * (w2r * omi + w2i * omr);
    omr = nr;
    omi = ni;
    Sr = Sr + omr;
    Si = Si + omi;
  }
  const T pref = 2.0 * bt / (1.0 + q) * dpow(bt / R, t - 1.0);
  const T apx = pref * Sr, apy = pref * Si;
  // potential (frame dot product is rotation invariant)
  const T psi_epl = (xp * apx + yp * apy) / (2.0 - t);
  // Jacobian in the frame
  const T Rp = dsqrt(xp * xp + yp * yp / (q * q));
  const T kap = (2.0 - t) / 2.0 * dpow(b / Rp, t);
  // gamma = ((1-t) alpha - kappa z) / conj(z)
  const T nr = (1.0 - t) * apx - kap * xp, ni = (1.0 - t) * apy - kap * yp;
  const T zz = xp * xp + yp * yp;  // divide by conj(z): multiply by z / |z|^2
  const T g1 = (nr * xp - ni * yp) / zz, g2 = (nr * yp + ni * xp) / zz;
  const T j11 = kap + g1, j12 = g2, j21 = g2, j22 = kap - g1;
  LensEvalT<T> e;
  e.ax = cphi * apx - sphi * apy;
  e.ay = sphi * apx + cphi * apy;
  const T c = cphi, s = sphi;
  e.a11 = c * c * j11 - c * s * (j12 + j21) + s * s * j22;
  e.a12 = c * s * (j11 - j22) + c * c * j12 - s * s * j21;
  e.a21 = c * s * (j11 - j22) + c * c * j21 - s * s * j12;
  e.a22 = s * s * j11 + c * s * (j12 + j21) + c * c * j22;
  e.psi = psi_epl;
  // external shear
  const T g1e = gext * dcos(2.0 * pext), g2e = gext * dsin(2.0 * pext);
  e.ax = e.ax + g1e * dx + g2e * dy;
  e.ay = e.ay + g2e * dx - g1e * dy;
  e.a11 = e.a11 + g1e;
  e.a12 = e.a12 + g2e;
  e.a21 = e.a21 + g2e;
  e.a22 = e.a22 - g1e;
  e.psi = e.psi + 0.5 * (g1e * (dx * dx - dy * dy) + 2.0 * g2e * dx * dy);
  // SIS perturbers (fixed)
  for (int i = 0; i < n_sis; ++i) {
    const double te = sis[3 * i];
    const P sx = x - sis[3 * i + 1], sy = y - sis[3 * i + 2];
    const P r = dsqrt(sx * sx + sy * sy), r3 = r * r * r;
    e.ax = e.ax + te * sx / r;
    e.ay = e.ay + te * sy / r;
    e.a11 = e.a11 + te * sy * sy / r3;
    e.a12 = e.a12 - te * sx * sy / r3;
    e.a21 = e.a21 - te * sx * sy / r3;
    e.a22 = e.a22 + te * sx * sx / r3;
    e.psi = e.psi + te * r;
  }
  return e;
}

// chi^2 of the delays; h0 is the Hubble constant (theta[19]).
template <class T>
__device__ inline T chi2_tmd_t(const T *th, T h0, const double *img_xy, int n_img,
                               const double *dt_obs, const double *dt_sig, double dt_per_arcsec2_H0,
                               const double *sis, int n_sis) {
  T w[8], bx[8], by[8], psi[8];
  T wsum(0.0), bhx(0.0), bhy(0.0);
  for (int i = 0; i < n_img; ++i) {
    const double x = img_xy[2 * i], y = img_xy[2 * i + 1];
    LensEvalT<T> e = lens_eval_t<T>(x, y, th, sis, n_sis);
    const T det = (1.0 - e.a11) * (1.0 - e.a22) - e.a12 * e.a21;
    w[i] = 1.0 / dfabs(det);
    bx[i] = x - e.ax;
    by[i] = y - e.ay;
    psi[i] = e.psi;
    wsum = wsum + w[i];
    bhx = bhx + w[i] * bx[i];
    bhy = bhy + w[i] * by[i];
  }
  bhx = bhx / wsum;
  bhy = bhy / wsum;
  const T kdt = dt_per_arcsec2_H0 / h0;
  T phi0(0.0), chi2(0.0);
  for (int i = 0; i < n_img; ++i) {
    const double x = img_xy[2 * i], y = img_xy[2 * i + 1];
    const T ph = 0.5 * ((x - bhx) * (x - bhx) + (y - bhy) * (y - bhy)) - psi[i];
    if (i == 0) {
      phi0 = ph;
    } else {
      const T dt = kdt * (ph - phi0);
      const T r = (dt_obs[i - 1] - dt) / dt_sig[i - 1];
      chi2 = chi2 + r * r;
    }
  }
  return chi2;
}

// beta_hat: the |mu|-weighted mean of the observed images mapped to the source plane.
template <class T>
__device__ inline void beta_hat_t(const T *th, const double *img_xy, int n_img, const double *sis,
                                  int n_sis, T &bhx, T &bhy) {
  T wsum(0.0);
  bhx = T(0.0);
  bhy = T(0.0);
  for (int i = 0; i < n_img; ++i) {
    const double x = img_xy[2 * i], y = img_xy[2 * i + 1];
    LensEvalT<T> e = lens_eval_t<T>(x, y, th, sis, n_sis);
    const T det = (1.0 - e.a11) * (1.0 - e.a22) - e.a12 * e.a21;
    const T w = 1.0 / dfabs(det);
    wsum = wsum + w;
    bhx = bhx + w * (x - e.ax);
    bhy = bhy + w * (y - e.ay);
  }
  bhx = bhx / wsum;
  bhy = bhy / wsum;
}

// chi^2 of the image positions (Eq. chi2_img): beta_hat mapped back to the image plane by
// Newton iterations on theta - alpha(theta) = beta_hat from each observed image (fixed
// count: quadratic convergence from a start within ~0.01" of the root; the tangents of a
// dual type converge with the values).
#define GLAD_NEWTON_IT 12
template <class T>
__device__ inline T chi2_img_t(const T *th, const double *img_xy, int n_img, const double *img_sig,
                               const double *sis, int n_sis) {
  T bhx, bhy;
  beta_hat_t<T>(th, img_xy, n_img, sis, n_sis, bhx, bhy);
  T chi2(0.0);
  for (int i = 0; i < n_img; ++i) {
    const double x = img_xy[2 * i], y = img_xy[2 * i + 1];
    T tx(x), ty(y);
    for (int it = 0; it < GLAD_NEWTON_IT; ++it) {
      LensEvalT<T> e = lens_eval_t<T, T>(tx, ty, th, sis, n_sis);
      const T fx = tx - e.ax - bhx, fy = ty - e.ay - bhy;
      const T m11 = 1.0 - e.a11, m12 = -e.a12, m21 = -e.a21, m22 = 1.0 - e.a22;
      const T det = m11 * m22 - m12 * m21;
      tx = tx - (m22 * fx - m12 * fy) / det;
      ty = ty - (m11 * fy - m21 * fx) / det;
    }
    const T rx = x - tx, ry = y - ty;
    chi2 = chi2 + (rx * rx + ry * ry) / (img_sig[i] * img_sig[i]);
  }
  return chi2;
}
