// Lens-model arithmetic of the quasar images (FP64), templated on the scalar type so the
// gradient kernel can run it on dual numbers.  Formulas:
//  * EPL deflection: Tessore & Metcalf (2015) series for the App. C convergence,
//    alpha' = 2 b_TM/(1+q) (b_TM/R)^(t-1) sum_n Omega_n, b_TM = q b, R = sqrt(q^2 x^2 + y^2),
//    Omega_0 = e^{i ph}, Omega_n = -f (2n-(2-t))/(2n+(2-t)) e^{2 i ph} Omega_{n-1}.
//  * EPL potential psi = (x alpha_x + y alpha_y)/(2-t) and Jacobian from homogeneity,
//    complex shear = ((1-t) alpha - kappa z)/conj(z).
//  * External shear psi = gamma/2 R^2 cos(2 phi - 2 phi_ext) about the lens centre (Sect. 3.3).
//  * SIS perturber psi = theta_E |theta - theta_s|.
//  * Internal mass sheet (Sect. 3.3, Eqs. kappa int, dpie_kappa): the galaxy terms above are
//    scaled by lambda_int = theta[20] and the sheet centred on the lens added: the dPIE with
//    central convergence 1 - lambda_int, a0 f = 2 (1 - lambda)/(1/r_c - 1/r_t),
//      alpha = a0 f [1/(r_c + Q_c) - 1/(r_t + Q_t)] (x - x_c), Q = sqrt(R^2 + r^2)
//            = (1 - lambda) 2 r_c r_t [1 + (r_c + r_t)/(Q_c + Q_t)] / ((r_c + Q_c)(r_t + Q_t)) (x - x_c),
//      psi   = a0 f [g(r_c) - g(r_t)],  g(r) = R^2/(Q + r) - r ln(1 + R^2/(2 r (Q + r))),
//      d alpha_i / d x_j = s delta_ij + 2 s' x_i x_j with s' = d s / d(R^2);
//    or the ideal sheet alpha = (1 - lambda)(x - x_c), psi = (1 - lambda) R^2 / 2.
//  * Delays (Eqs. fermat potential, time delay between multiple images, chi2_tmd): source
//    at the |mu|-weighted mean of the images mapped back (Sect. 3.1.1), image 0 the reference;
//    days per arcsec^2 of Fermat potential D_dt,int / c from H0 (distance mode 0) or from
//    D_dt,int = theta[22] (mode 1).
#pragma once
#include <math.h>

#include "dual.cuh"
#include "glad_internal.cuh"

template <class T>
struct LensEvalT {
  T ax, ay;              // deflection (sky)
  T a11, a12, a21, a22;  // d alpha / d theta (sky)
  T psi;                 // potential
};

// EPL + shear + SIS (and the system's internal sheet) at sky point (x, y); th = the full
// parameter vector (entries 0..7 and, with a sheet, 20 used).  The position may be a plain
// double or of the parameter type (Newton iterates on positions).
template <class T, class P = double>
__device__ inline LensEvalT<T> lens_eval_t(P x, P y, const T *th, const SysDev &S) {
  const double *sis = S.sis;
  const int n_sis = S.n_sis;
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
  if (S.sheet) {
    const T lam = th[20], om = 1.0 - lam;
    e.ax = lam * e.ax;
    e.ay = lam * e.ay;
    e.a11 = lam * e.a11;
    e.a12 = lam * e.a12;
    e.a21 = lam * e.a21;
    e.a22 = lam * e.a22;
    e.psi = lam * e.psi;
    const T R2 = dx * dx + dy * dy;
    if (S.sheet == 2) {
      e.ax = e.ax + om * dx;
      e.ay = e.ay + om * dy;
      e.a11 = e.a11 + om;
      e.a22 = e.a22 + om;
      e.psi = e.psi + 0.5 * om * R2;
    } else {
      const double rc = S.sh_rc, rt = S.sh_rt;
      const T Qc = dsqrt(R2 + rc * rc), Qt = dsqrt(R2 + rt * rt);
      const T sv = om * (2.0 * rc * rt) * (1.0 + (rc + rt) / (Qc + Qt)) / ((rc + Qc) * (rt + Qt));
      const T a0f = om * (2.0 * rc * rt / (rt - rc));
      const T sp = a0f * (1.0 / (2.0 * Qt * (rt + Qt) * (rt + Qt)) - 1.0 / (2.0 * Qc * (rc + Qc) * (rc + Qc)));
      e.ax = e.ax + sv * dx;
      e.ay = e.ay + sv * dy;
      e.a11 = e.a11 + sv + 2.0 * sp * dx * dx;
      e.a12 = e.a12 + 2.0 * sp * dx * dy;
      e.a21 = e.a21 + 2.0 * sp * dx * dy;
      e.a22 = e.a22 + sv + 2.0 * sp * dy * dy;
      const T gc = R2 / (Qc + rc) - rc * dlog1p(R2 / (2.0 * rc * (Qc + rc)));
      const T gt = R2 / (Qt + rt) - rt * dlog1p(R2 / (2.0 * rt * (Qt + rt)));
      e.psi = e.psi + a0f * (gc - gt);
    }
  }
  return e;
}

// Days of delay per arcsec^2 of Fermat potential: D_dt,int / c from H0 = theta[19] (distance
// mode 0) or D_dt,int = theta[22] (mode 1).
template <class T>
__device__ inline T delay_unit_t(const T *th, const SysDev &S) {
  if (S.distance_mode == 1) return S.dt_per_arcsec2_Mpc * th[22];
  return S.dt_per_arcsec2_H0 / th[19];
}

// chi^2 of the delays (th: the full parameter vector).
template <class T>
__device__ inline T chi2_tmd_t(const T *th, const SysDev &S) {
  const double *img_xy = S.img_xy;
  const int n_img = S.n_img;
  T w[GLAD_MAX_IMG], bx[GLAD_MAX_IMG], by[GLAD_MAX_IMG], psi[GLAD_MAX_IMG];
  T wsum(0.0), bhx(0.0), bhy(0.0);
  for (int i = 0; i < n_img; ++i) {
    const double x = img_xy[2 * i], y = img_xy[2 * i + 1];
    LensEvalT<T> e = lens_eval_t<T>(x, y, th, S);
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
  const T kdt = delay_unit_t<T>(th, S);
  T phi0(0.0), chi2(0.0);
  for (int i = 0; i < n_img; ++i) {
    const double x = img_xy[2 * i], y = img_xy[2 * i + 1];
    const T ph = 0.5 * ((x - bhx) * (x - bhx) + (y - bhy) * (y - bhy)) - psi[i];
    if (i == 0) {
      phi0 = ph;
    } else {
      const T dt = kdt * (ph - phi0);
      const T r = (S.dt_obs[i - 1] - dt) / S.dt_sig[i - 1];
      chi2 = chi2 + r * r;
    }
  }
  return chi2;
}

// beta_hat: the |mu|-weighted mean of the observed images mapped to the source plane.
template <class T>
__device__ inline void beta_hat_t(const T *th, const SysDev &S, T &bhx, T &bhy) {
  const double *img_xy = S.img_xy;
  const int n_img = S.n_img;
  T wsum(0.0);
  bhx = T(0.0);
  bhy = T(0.0);
  for (int i = 0; i < n_img; ++i) {
    const double x = img_xy[2 * i], y = img_xy[2 * i + 1];
    LensEvalT<T> e = lens_eval_t<T>(x, y, th, S);
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
__device__ inline T chi2_img_t(const T *th, const SysDev &S) {
  const double *img_xy = S.img_xy, *img_sig = S.img_sig;
  const int n_img = S.n_img;
  T bhx, bhy;
  beta_hat_t<T>(th, S, bhx, bhy);
  T chi2(0.0);
  for (int i = 0; i < n_img; ++i) {
    const double x = img_xy[2 * i], y = img_xy[2 * i + 1];
    T tx(x), ty(y);
    for (int it = 0; it < GLAD_NEWTON_IT; ++it) {
      LensEvalT<T> e = lens_eval_t<T, T>(tx, ty, th, S);
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
