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

// ---- composite class (Sect. 3.3): the pieces below, in the galaxy frame or round ----------
// Round Gaussian lens of mass M, t = R^2 / (2 sigma^2): h1(t) = (1 - e^-t)/t sets the
// deflection M h1 / (2 pi sigma^2) (dx, dy); G(t) = ln t + E1(t) (G' = h1) its potential
// M G / (2 pi); h1'(t) its Jacobian.  Small t: Taylor series; large t: E1 by its continued
// fraction (Lentz), E1 < 1e-23 beyond t = 50.
__device__ inline double h1_val(double t) { return t < 1e-4 ? 1.0 - t / 2 + t * t / 6 : -expm1(-t) / t; }
__device__ inline double h1_der(double t) {
  return t < 1e-4 ? -0.5 + t / 3 - t * t / 8 : (exp(-t) * (t + 1.0) - 1.0) / (t * t);
}
__device__ inline double G_val(double t) {
  if (t < 2.0) {
    // G = -gamma + sum_{k>=1} (-1)^(k+1) t^k / (k k!)
    double s = 0.0, term = 1.0;
    for (int k = 1; k < 40; ++k) {
      term *= t / k;
      s += (k & 1 ? 1.0 : -1.0) * term / k;
    }
    return -0.57721566490153286 + s;
  }
  if (t > 50.0) return log(t);
  // E1(t) = e^-t / (t + 1 - 1^2/(t + 3 - 2^2/(t + 5 - ...))) by the modified Lentz method
  double b = t + 1.0, c = 1e300, d = 1.0 / b, h = d;
  for (int i = 1; i < 200; ++i) {
    const double a = -(double)i * i;
    b += 2.0;
    d = 1.0 / (a * d + b);
    c = b + a / c;
    const double del = c * d;
    h *= del;
    if (fabs(del - 1.0) < 1e-16) break;
  }
  return log(t) + h * exp(-t);
}
__device__ inline double dh1(double t) { return h1_val(t); }
__device__ inline double dh1p(double t) { return h1_der(t); }
__device__ inline double dG(double t) { return G_val(t); }
template <int N>
__device__ inline Dual<N, double> dh1(const Dual<N, double> &t) { return dual_apply(t, h1_val(t.v), h1_der(t.v)); }
template <int N>
__device__ inline Dual<N, double> dh1p(const Dual<N, double> &t) {
  // d h1' / dt = (2 - e^-t (t^2 + 2 t + 2)) / t^3, series 1/3 - t/4 near 0
  const double v = t.v, d2 = v < 1e-3 ? 1.0 / 3 - v / 4 : (2.0 - exp(-v) * (v * v + 2 * v + 2)) / (v * v * v);
  return dual_apply(t, h1_der(v), d2);
}
template <int N>
__device__ inline Dual<N, double> dG(const Dual<N, double> &t) { return dual_apply(t, G_val(t.v), h1_val(t.v)); }

// Softened isothermal ellipsoid A / sqrt(x^2 + y^2/q^2 + s^2) (frame; q fixed): deflection,
// potential x a_x + y a_y - b s ln sqrt(D) and Jacobian, b = 2 q A, D = (psi + s)^2 + e^2 x^2
template <class T>
__device__ inline void nie_add(const T &x, const T &y, const T &A, const T &s, double q, LensEvalT<T> &f) {
  const double e = sqrt(1.0 - q * q);
  const T b = 2.0 * q * A;
  const T ps = dsqrt(q * q * (s * s + x * x) + y * y);
  const T D = (ps + s) * (ps + s) + (e * e) * x * x;
  T ax, ay;
  if (e > 1e-7) {
    ax = (b / e) * datan(e * x / (ps + s));
    ay = (b / e) * datanh(e * y / (ps + (q * q) * s));
  } else {
    const T fac = 2.0 * A / (dsqrt(x * x + y * y + s * s) + s);
    ax = fac * x;
    ay = fac * y;
  }
  f.ax = f.ax + ax;
  f.ay = f.ay + ay;
  f.psi = f.psi + x * ax + y * ay - b * s * 0.5 * dlog(D);
  f.a11 = f.a11 + b * ((ps + s) - (q * q) * x * x / ps) / D;
  const T a12 = -b * x * y / (ps * D);
  f.a12 = f.a12 + a12;
  f.a21 = f.a21 + a12;
  f.a22 = f.a22 + b * ((ps + (q * q) * s) - y * y / ps) / ((q * q) * D);
}

// Cored steep ellipsoid amp / (x^2 + y^2/q^2 + s^2)^(3/2) (frame), as -(1/s) d/ds of the
// softened isothermal one with A = 1: deflection 2 q amp (x (psi + q^2 s), y (psi + s)) / (s psi D),
// potential, and Jacobian -(1/s) d/ds of the isothermal Jacobian (d psi / ds = q^2 s / psi)
template <class T>
__device__ inline void cse_add(const T &x, const T &y, const T &amp, const T &s, const T &q, LensEvalT<T> &f) {
  const T q2 = q * q, e2 = 1.0 - q2, b = 2.0 * q;
  const T ps = dsqrt(q2 * (s * s + x * x) + y * y);
  const T D = (ps + s) * (ps + s) + e2 * x * x;
  const T inv = 1.0 / (s * ps * D);
  const T ax = b * x * (ps + q2 * s) * inv, ay = b * y * (ps + s) * inv;
  f.ax = f.ax + amp * ax;
  f.ay = f.ay + amp * ay;
  f.psi = f.psi + amp * (x * ax + y * ay + b / s * 0.5 * dlog(D) + b * (ps + s) * (q2 * s / ps + 1.0) / D);
  const T pss = q2 * s / ps;
  const T Ds = 2.0 * (ps + s) * (pss + 1.0);
  const T N1 = ps + s - q2 * x * x / ps, N1s = pss + 1.0 + q2 * x * x * pss / (ps * ps);
  const T N2 = ps + q2 * s - y * y / ps, N2s = pss + q2 + y * y * pss / (ps * ps);
  const T d11 = b * (N1s * D - N1 * Ds) / (D * D);
  const T d12 = b * x * y * (pss * D + ps * Ds) / ((ps * D) * (ps * D));
  const T d22 = b * (N2s * D - N2 * Ds) / (q2 * D * D);
  f.a11 = f.a11 - amp * d11 / s;
  f.a12 = f.a12 - amp * d12 / s;
  f.a21 = f.a21 - amp * d12 / s;
  f.a22 = f.a22 - amp * d22 / s;
}

// EPL galaxy (Tessore & Metcalf series) in the sky frame, before shear and perturbers
template <class T, class P>
__device__ inline LensEvalT<T> epl_eval_t(P x, P y, const T *th) {
  const T tE = th[0], g = th[1], q = th[2], phi = th[3], xc = th[4], yc = th[5];
  LensEvalT<T> e;
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
  e.ax = cphi * apx - sphi * apy;
  e.ay = sphi * apx + cphi * apy;
  const T c = cphi, s = sphi;
  e.a11 = c * c * j11 - c * s * (j12 + j21) + s * s * j22;
  e.a12 = c * s * (j11 - j22) + c * c * j12 - s * s * j21;
  e.a21 = c * s * (j11 - j22) + c * c * j21 - s * s * j12;
  e.a22 = s * s * j11 + c * s * (j12 + j21) + c * c * j22;
  e.psi = psi_epl;
  return e;
}

// EPL + shear + SIS (and the system's internal sheet) at sky point (x, y); th = the full
// parameter vector (entries 0..7 and, with a sheet, 20 used).  The position may be a plain
// double or of the parameter type (Newton iterates on positions).
template <class T, class P = double>
__device__ inline LensEvalT<T> lens_eval_t(P x, P y, const T *th, const SysDev &S, T mbh = T(0.0)) {
  const double *sis = S.sis;
  const int n_sis = S.n_sis;
  const T q = th[2], phi = th[3], xc = th[4], yc = th[5];
  const T gext = th[6], pext = th[7];
  const T dx = x - xc, dy = y - yc;
  LensEvalT<T> e;
  if (S.mass_class == 1) {
    // composite galaxy: Upsilon L_scale x Chameleons + halo CSEs in the frame, black hole round
    const T cphi = dcos(phi), sphi = dsin(phi);
    const T xp = cphi * dx + sphi * dy, yp = -sphi * dx + cphi * dy;
    LensEvalT<T> f;
    f.ax = f.ay = f.a11 = f.a12 = f.a21 = f.a22 = f.psi = T(0.0);
    const T ups = th[17] * S.L_scale;
    for (int c = 0; c < S.n_lcomp; ++c) {
      const double qc = S.lcomp[4 * c + 3];
      const T I0 = c == 0 ? th[13] : T(S.lcomp[4 * c]);
      const T wt = c == 0 ? th[14] : T(S.lcomp[4 * c + 2]);
      const T A = ups * I0 / (1.0 + qc);
      const T sc = T(2.0 * S.lcomp[4 * c + 1] / (1.0 + qc)), st = 2.0 * wt / (1.0 + qc);
      LensEvalT<T> g2;
      g2.ax = g2.ay = g2.a11 = g2.a12 = g2.a21 = g2.a22 = g2.psi = T(0.0);
      nie_add<T>(xp, yp, A, sc, qc, f);
      nie_add<T>(xp, yp, A, st, qc, g2);
      f.ax = f.ax - g2.ax;
      f.ay = f.ay - g2.ay;
      f.psi = f.psi - g2.psi;
      f.a11 = f.a11 - g2.a11;
      f.a12 = f.a12 - g2.a12;
      f.a21 = f.a21 - g2.a21;
      f.a22 = f.a22 - g2.a22;
    }
    const T ks = th[0], rs = th[1];
    const T rs3 = rs * rs * rs;
    for (int i = 0; i < GLAD_N_CSE; ++i) {
      if (S.cse_a[i] == 0.0) continue;
      cse_add<T>(xp, yp, ks * S.cse_a[i] * rs3, S.cse_s[i] * rs, q, f);
    }
    const T c = cphi, s = sphi;
    e.ax = c * f.ax - s * f.ay;
    e.ay = s * f.ax + c * f.ay;
    e.a11 = c * c * f.a11 - c * s * (f.a12 + f.a21) + s * s * f.a22;
    e.a12 = c * s * (f.a11 - f.a22) + c * c * f.a12 - s * s * f.a21;
    e.a21 = c * s * (f.a11 - f.a22) + c * c * f.a21 - s * s * f.a12;
    e.a22 = s * s * f.a11 + c * s * (f.a12 + f.a21) + c * c * f.a22;
    e.psi = f.psi;
    if (S.has_bh) {
      const double s2x2 = 2.0 * S.bh_sigma * S.bh_sigma;
      const T R2 = dx * dx + dy * dy, t = R2 / s2x2;
      const T S0 = mbh / (PI_D * s2x2);
      const T gv = S0 * dh1(t), gp = S0 * dh1p(t) / s2x2;
      e.ax = e.ax + gv * dx;
      e.ay = e.ay + gv * dy;
      e.a11 = e.a11 + gv + 2.0 * gp * dx * dx;
      e.a12 = e.a12 + 2.0 * gp * dx * dy;
      e.a21 = e.a21 + 2.0 * gp * dx * dy;
      e.a22 = e.a22 + gv + 2.0 * gp * dy * dy;
      e.psi = e.psi + mbh / (2.0 * PI_D) * dG(t);
    }
  } else {
    e = epl_eval_t<T, P>(x, y, th);
  }
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
__device__ inline T chi2_tmd_t(const T *th, const SysDev &S, T mbh = T(0.0)) {
  const double *img_xy = S.img_xy;
  const int n_img = S.n_img;
  T w[GLAD_MAX_IMG], bx[GLAD_MAX_IMG], by[GLAD_MAX_IMG], psi[GLAD_MAX_IMG];
  T wsum(0.0), bhx(0.0), bhy(0.0);
  for (int i = 0; i < n_img; ++i) {
    const double x = img_xy[2 * i], y = img_xy[2 * i + 1];
    LensEvalT<T> e = lens_eval_t<T>(x, y, th, S, mbh);
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
__device__ inline void beta_hat_t(const T *th, const SysDev &S, T &bhx, T &bhy, T mbh = T(0.0)) {
  const double *img_xy = S.img_xy;
  const int n_img = S.n_img;
  T wsum(0.0);
  bhx = T(0.0);
  bhy = T(0.0);
  for (int i = 0; i < n_img; ++i) {
    const double x = img_xy[2 * i], y = img_xy[2 * i + 1];
    LensEvalT<T> e = lens_eval_t<T>(x, y, th, S, mbh);
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
__device__ inline T chi2_img_t(const T *th, const SysDev &S, T mbh = T(0.0)) {
  const double *img_xy = S.img_xy, *img_sig = S.img_sig;
  const int n_img = S.n_img;
  T bhx, bhy;
  beta_hat_t<T>(th, S, bhx, bhy, mbh);
  T chi2(0.0);
  for (int i = 0; i < n_img; ++i) {
    const double x = img_xy[2 * i], y = img_xy[2 * i + 1];
    T tx(x), ty(y);
    for (int it = 0; it < GLAD_NEWTON_IT; ++it) {
      LensEvalT<T> e = lens_eval_t<T, T>(tx, ty, th, S, mbh);
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
