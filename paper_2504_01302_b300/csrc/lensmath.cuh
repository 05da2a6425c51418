// Lens-model arithmetic of the prep kernel (FP64, quasar images).  Formulas:
//  * EPL deflection: Tessore & Metcalf (2015) series for the App. C convergence,
//    alpha' = 2 b_TM/(1+q) (b_TM/R)^(t-1) sum_n Omega_n, b_TM = q b, R = sqrt(q^2 x^2 + y^2),
//    Omega_0 = e^{i ph}, Omega_n = -f (2n-(2-t))/(2n+(2-t)) e^{2 i ph} Omega_{n-1}.
//  * EPL potential psi = (x alpha_x + y alpha_y)/(2-t) and Jacobian from homogeneity,
//    complex shear = ((1-t) alpha - kappa z)/conj(z).
//  * External shear psi = gamma/2 R^2 cos(2 phi - 2 phi_ext) about the lens centre (Sect. 3.3).
//  * SIS perturber psi = theta_E |theta - theta_s|.
#pragma once
#include <math.h>

struct LensEval {
  double ax, ay;              // deflection (sky)
  double a11, a12, a21, a22;  // d alpha / d theta (sky)
  double psi;                 // potential
};

// EPL + shear + SIS at sky point (x, y) in FP64; th = parameter vector.
__device__ inline LensEval lens_eval_d(double x, double y, const double *th,
                                       const double *sis, int n_sis) {
  const double tE = th[0], g = th[1], q = th[2], phi = th[3], xc = th[4], yc = th[5];
  const double gext = th[6], pext = th[7];
  const double t = g - 1.0;
  double cphi, sphi;
  sincos(phi, &sphi, &cphi);
  const double dx = x - xc, dy = y - yc;
  const double xp = cphi * dx + sphi * dy, yp = -sphi * dx + cphi * dy;
  const double b = pow(2.0 / (1.0 + q), 1.0 / t) * tE;
  const double bt = q * b;
  const double R = sqrt(q * q * xp * xp + yp * yp);
  const double wr = q * xp / R, wi = yp / R;
  const double w2r = wr * wr - wi * wi, w2i = 2.0 * wr * wi;
  const double f = (1.0 - q) / (1.0 + q);
  int nt = 0;
  if (f > 0.0) nt = (int)ceil(log(1e-16) / log(f));
  if (nt > 200) nt = 200;
  double omr = wr, omi = wi, Sr = wr, Si = wi;
  for (int n = 1; n <= nt; ++n) {
    const double rho = -f * (2.0 * n - (2.0 - t)) / (2.0 * n + (2.0 - t));
    const double nr = rho * (w2r * omr - w2i * omi);
    const double ni = rho * (w2r * omi + w2i * omr);
    omr = nr;
    omi = ni;
    Sr += omr;
    Si += omi;
  }
  const double pref = 2.0 * bt / (1.0 + q) * pow(bt / R, t - 1.0);
  const double apx = pref * Sr, apy = pref * Si;
  // potential (frame dot product is rotation invariant)
  const double psi_epl = (xp * apx + yp * apy) / (2.0 - t);
  // Jacobian in the frame
  const double Rp = sqrt(xp * xp + yp * yp / (q * q));
  const double kap = (2.0 - t) / 2.0 * pow(b / Rp, t);
  // gamma = ((1-t) alpha - kappa z) / conj(z)
  const double nr = (1.0 - t) * apx - kap * xp, ni = (1.0 - t) * apy - kap * yp;
  const double zz = xp * xp + yp * yp;   // divide by conj(z): multiply by z / |z|^2
  const double g1 = (nr * xp - ni * yp) / zz, g2 = (nr * yp + ni * xp) / zz;
  const double j11 = kap + g1, j12 = g2, j21 = g2, j22 = kap - g1;
  LensEval e;
  e.ax = cphi * apx - sphi * apy;
  e.ay = sphi * apx + cphi * apy;
  const double c = cphi, s = sphi;
  e.a11 = c * c * j11 - c * s * (j12 + j21) + s * s * j22;
  e.a12 = c * s * (j11 - j22) + c * c * j12 - s * s * j21;
  e.a21 = c * s * (j11 - j22) + c * c * j21 - s * s * j12;
  e.a22 = s * s * j11 + c * s * (j12 + j21) + c * c * j22;
  e.psi = psi_epl;
  // external shear
  double s2p, c2p;
  sincos(2.0 * pext, &s2p, &c2p);
  const double g1e = gext * c2p, g2e = gext * s2p;
  e.ax += g1e * dx + g2e * dy;
  e.ay += g2e * dx - g1e * dy;
  e.a11 += g1e;
  e.a12 += g2e;
  e.a21 += g2e;
  e.a22 -= g1e;
  e.psi += 0.5 * (g1e * (dx * dx - dy * dy) + 2.0 * g2e * dx * dy);
  // SIS perturbers
  for (int i = 0; i < n_sis; ++i) {
    const double te = sis[3 * i], sx = x - sis[3 * i + 1], sy = y - sis[3 * i + 2];
    const double r = sqrt(sx * sx + sy * sy), r3 = r * r * r;
    e.ax += te * sx / r;
    e.ay += te * sy / r;
    e.a11 += te * sy * sy / r3;
    e.a12 -= te * sx * sy / r3;
    e.a21 -= te * sx * sy / r3;
    e.a22 += te * sx * sx / r3;
    e.psi += te * r;
  }
  return e;
}
