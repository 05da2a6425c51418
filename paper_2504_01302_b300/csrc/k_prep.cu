// Per-sample preparation (one CTA per sample, FP64):
//  * domain checks of the parameter vector;
//  * 1-D MGE of each lens-light Sersic and of the App. C convergence by the Euler
//    inversion of Sect. 3.2:  A_n = w_n dln(sigma) / sqrt(2 pi) * sum_m eta_m Re F(sigma_n chi_m);
//  * black-hole Gaussian, M_BH = f_BH * Upsilon * L_tot * L_scale;
//  * deprojection (App. A): q = sqrt(q'^2 - cos^2 i)/sin i, needs cos^2 i < q'^2,
//    and a positivity check of both densities at probe radii (Sect. 3.3);
//  * per-Gaussian JAM inputs nu_k, 1/(2 s_k^2 q_k^2), C_j = 4 pi G rho_j q_j s_j^2, e_j^2;
//  * FP32 lensing parameter block (EPL series coefficients, shear, light);
//  * time delays (Eqs. fermat potential, time delay between multiple images, chi2_tmd)
//    with the magnification-weighted source estimate of Sect. 3.1.1, and the
//    image-position term (Eq. chi2_img) for systems that give image-position errors.
// A second kernel expands the (tracer k, mass j, node g) JAM coefficient table.
#include <type_traits>

#include "cplx.cuh"
#include "glad_internal.cuh"
#include "lensmath.cuh"

namespace {

// Sersic profile at complex radius z
__device__ inline double sersic_re(cplx z, double Ie, double Re, double n, double bn) {
  cplx l = clog_({z.r / Re, z.i / Re});
  cplx w = cexp_({l.r / n, l.i / n});
  cplx F = cexp_({-bn * (w.r - 1.0), -bn * w.i});
  return Ie * F.r;
}

// App. C convergence at complex radius z: coef * (z^2 + rs^2)^(-(g-1)/2)
__device__ inline double epl_kappa_re(cplx z, double coef, double g, double rs2) {
  cplx z2 = cmul(z, z);
  z2.r += rs2;
  cplx l = clog_(z2);
  const double e = -0.5 * (g - 1.0);
  cplx F = cexp_({e * l.r, e * l.i});
  return coef * F.r;
}

// Parameters inside their domain; entries the system does not use (lambda_int without a
// sheet, H0 in distance mode 1, D_d and D_dt,int in mode 0) are not looked at.
__device__ inline int domain_ok(const double *th, const SysDev &S) {
  bool ok = true;
  const bool mode1 = S.distance_mode == 1;
  for (int i = 0; i < 19; ++i) ok = ok && isfinite(th[i]);
  const double g = th[1], q = th[2], inc = th[15];
  if (S.mass_class == 1)  // kappa_s >= 0, r_s > 0, halo q in (0, 1], I0 > 0, w_t > w_c
    ok = ok && th[0] >= 0.0 && th[1] > 0.0 && q > 0.0 && q <= 1.0 && th[13] > 0.0 && th[14] > S.lcomp[1];
  else
    ok = ok && th[0] > 0.0 && g > 1.0 && g < 3.0 && q > 0.0 && q <= 1.0 && th[14] > 0.0 && th[13] > 0.0;
  ok = ok && th[9] > 0.0 && th[10] > 0.0 && inc > 0.0 &&
       inc <= 1.5707963267948966 + 1e-12 && th[16] < 1.0 && th[17] >= 0.0 && th[18] >= 0.0;
  if (mode1)
    ok = ok && isfinite(th[21]) && isfinite(th[22]) && th[21] > 0.0 && th[22] > 0.0;
  else
    ok = ok && isfinite(th[19]) && th[19] > 0.0;
  if (S.sheet) ok = ok && isfinite(th[20]) && th[20] > 0.0;
  return ok ? 1 : 0;
}

__global__ void __launch_bounds__(128) k_prep(const SysDev *__restrict__ sysv,
                                              const int *__restrict__ sys_id,
                                              const double *__restrict__ theta, WsDev ws,
                                              int max_light, int max_mass) {
  const int b = blockIdx.x;
  const int tid = threadIdx.x;
  const SysDev &S = sysv[sys_id[b]];
  const double *th = theta + (size_t)GLAD_NTHETA * b;
  __shared__ double sh_A[GLAD_MAX_LIGHT + GLAD_MAX_MASS + 1];
  __shared__ double sh_rho[GLAD_MAX_LIGHT + GLAD_MAX_MASS + 1];
  __shared__ double sh_q[GLAD_MAX_LIGHT + GLAD_MAX_MASS + 1];
  __shared__ int sh_flag;
  __shared__ double sh_mbh;  // black-hole mass before lambda_int (the composite lens uses it)
  __shared__ double sh_dm[4];  // its derivatives by theta 13, 14, 17, 18 (composite class)

  const int ok = domain_ok(th, S);
  if (!ok) {
    if (tid == 0) {
      ws.status[b] = GLAD_SAMPLE_DOMAIN;
      ws.lp[b].valid = 0;
    }
    return;
  }
  const double tE = th[0], g = th[1], q = th[2], inc = th[15];
  double si, ci;
  sincos(inc, &si, &ci);
  const double s2 = si * si, c2 = ci * ci;
  const int nL = S.n_light, nM = S.n_mass, nMt = S.n_mass_tot;
  const int P2 = 2 * S.mge_P + 1;

  // ---- 1-D MGE (Euler inversion), FP64: the (Gaussian, Euler node) terms are spread over
  // the block and summed per Gaussian in shared memory
  const double coef_m = (3.0 - g) / (1.0 + q) * pow(tE, g - 1.0);
  // Gaussians expanded here: the tracer's, then the EPL's (or, composite class, the halo's
  // n_halo, whose mass index is nL + h after the nL copies of the tracer)
  const bool comp = S.mass_class == 1;
  const int off = comp ? nL : 0;
  const int nE = nL + (comp ? S.n_halo : nM);
  __shared__ double sh_dAw[GLAD_MAX_LIGHT];  // composite: d A_k / d w_t of the first Chameleon
  for (int k = tid; k < nL + nM; k += blockDim.x) {
    sh_A[k] = 0.0;
    sh_q[k] = k < nL ? S.qp_light[k] : (comp && k < 2 * nL ? S.qp_light[k - nL] : q);
    if (k < nL) sh_dAw[k] = 0.0;
  }
  __syncthreads();
  for (int it = tid; it < nE * P2; it += blockDim.x) {
    const int k = it / P2, m = it - k * P2;
    const double2 ch = S.chi[m];
    double v;
    int dst = k;
    if (k < nL) {
      const int c = S.lcomp_of[k];
      const double sg = S.sig_light[k];
      if (comp) {
        const double qc = S.lcomp[4 * c + 3];
        const double I0 = c == 0 ? th[13] : S.lcomp[4 * c];
        const double wt = c == 0 ? th[14] : S.lcomp[4 * c + 2];
        const double st = 2.0 * wt / (1.0 + qc);
        const cplx z = {sg * ch.x, sg * ch.y};
        v = S.mw_light[k] * S.eta[m] *
            chameleon_c(z, I0 / (1.0 + qc), 2.0 * S.lcomp[4 * c + 1] / (1.0 + qc), st).r;
        if (c == 0) {
          // d/dw_t: A st (z^2 + st^2)^(-3/2) 2/(1+q)
          const cplx z2 = cmul(z, z);
          const cplx p = cpow_({z2.r + st * st, z2.i}, -1.5);
          atomicAdd(&sh_dAw[k], S.mw_light[k] * S.eta[m] * I0 / (1.0 + qc) * st * 2.0 / (1.0 + qc) * p.r);
        }
      } else {
        const double Ie = c == 0 ? th[13] : S.lcomp[4 * c];
        const double Re = c == 0 ? th[14] : S.lcomp[4 * c + 1];
        const double n = S.lcomp[4 * c + 2];
        v = S.mw_light[k] * S.eta[m] * sersic_re({sg * ch.x, sg * ch.y}, Ie, Re, n, sersic_bn_d(n));
      }
    } else if (comp) {
      // halo: kappa_s k(z / r_s), the exact profile
      const int j = off + (k - nL);
      const double sg = S.sig_mass[j];
      v = th[0] * S.mw_mass[j] * S.eta[m] * nfw_k_c({sg * ch.x / th[1], sg * ch.y / th[1]}, nullptr).r;
      dst = nL + j;
    } else {
      // (3-g)/2 b^(g-1) with b = (2/(1+q))^(1/(g-1)) theta_E
      const double sg = S.sig_mass[k - nL];
      v = S.mw_mass[k - nL] * S.eta[m] *
          epl_kappa_re({sg * ch.x, sg * ch.y}, coef_m, g, S.r_soft * S.r_soft);
    }
    atomicAdd(&sh_A[dst], v);
  }
  if (tid == 0) sh_flag = 0;
  __syncthreads();
  if (comp) {
    // baryons: Upsilon_* L_scale times the tracer Gaussians
    const double ups = th[17] * S.L_scale;
    for (int k = tid; k < nL; k += blockDim.x) sh_A[nL + k] = ups * sh_A[k];
    __syncthreads();
  }
  // internal mass sheet (Sect. 3.3, Eq. kappa int): the galaxy's Gaussians scaled by lambda,
  // then the sheet's round Gaussians, (1 - lambda) times their unit amplitudes
  const int nS = S.n_sheet;
  const double lam = S.sheet ? th[20] : 1.0;
  for (int j = tid; j < nM + nS; j += blockDim.x) {
    if (j < nM) {
      sh_A[nL + j] *= lam;
    } else {
      sh_A[nL + j] = (1.0 - lam) * S.sheet_A1[j - nM];
      sh_q[nL + j] = 1.0;
    }
  }
  __syncthreads();
  if (tid == 0) {
    double L = 0.0;
    for (int k = 0; k < nL; ++k) L += 2.0 * PI_D * sh_A[k] * S.sig_light[k] * S.sig_light[k] * sh_q[k];
    sh_mbh = S.has_bh ? th[18] * th[17] * L * S.L_scale : 0.0;  // before lambda (lensing)
    if (comp) {
      // d M_BH / d(I0, w_t, Upsilon, f_BH) for the lensing gradient: L_tot's parts
      double L0 = 0.0, Lw = 0.0;
      for (int k = 0; k < nL; ++k)
        if (S.lcomp_of[k] == 0) {
          const double w = 2.0 * PI_D * S.sig_light[k] * S.sig_light[k] * sh_q[k];
          L0 += w * sh_A[k];
          Lw += w * sh_dAw[k];
        }
      const double f = S.has_bh ? th[18] * th[17] * S.L_scale : 0.0;
      sh_dm[0] = f * L0 / th[13];
      sh_dm[1] = f * Lw;
      sh_dm[2] = S.has_bh ? th[18] * L * S.L_scale : 0.0;
      sh_dm[3] = S.has_bh ? th[17] * L * S.L_scale : 0.0;
    }
    if (S.has_bh) {
      sh_A[nL + nM + nS] = lam * sh_mbh / (2.0 * PI_D * S.bh_sigma * S.bh_sigma);
      sh_q[nL + nM + nS] = 1.0;
    }
    // deprojection needs cos^2 i < q'^2 for every Gaussian (App. A)
    double qmin = q;
    for (int k = 0; k < nL; ++k) qmin = fmin(qmin, sh_q[k]);
    if (c2 >= qmin * qmin) sh_flag = GLAD_SAMPLE_DEPROJ;
  }
  __syncthreads();
  if (sh_flag) {
    if (tid == 0) {
      ws.status[b] = sh_flag;
      ws.lp[b].valid = 0;
    }
    return;
  }
  const int nG = nL + nMt;
  // velocity^2 unit of the dynamics: fixed (distance mode 0) or times D_dt,int / D_d (mode 1)
  const double v2u = S.distance_mode == 1 ? S.v2unit * th[22] / th[21] : S.v2unit;
  // ---- deprojection; densities rho0 (tracer nu0 and mass rho0) and intrinsic q
  for (int k = tid; k < nG; k += blockDim.x) {
    const double sg = k < nL ? S.sig_light[k] : S.sig_mass[k - nL];
    const double qp = sh_q[k];
    const double qi = sqrt(qp * qp - c2) / si;
    sh_rho[k] = qp * sh_A[k] / (SQRT2PI_D * sg * qi);
    const size_t bl = (size_t)b * max_light, bm = (size_t)b * max_mass;
    if (k < nL) {
      ws.nu0[bl + k] = sh_rho[k];
      ws.c0[bl + k] = 1.0 / (2.0 * sg * sg * qi * qi);
      ws.I0f[bl + k] = (float)sh_A[k];
      if (ws.prec == 2) ws.I0d[bl + k] = sh_A[k];
    } else {
      const int j = k - nL;
      ws.Cj[bm + j] = 2.0 * SQRT2PI_D * v2u * qp * sh_A[k] * sg;
      ws.e2[bm + j] = 1.0 - qi * qi;
    }
  }
  __syncthreads();
  // ---- positivity at probe radii: equatorial R = sigma_n and on the axis z = sigma_n
  for (int k = tid; k < nG; k += blockDim.x) {
    const bool light = k < nL;
    const double s = light ? S.sig_light[k] : S.sig_mass[k - nL];
    const int lo = light ? 0 : nL, hi = light ? nL : nG;
    double eq = 0.0, ax = 0.0;
    for (int m = lo; m < hi; ++m) {
      const double sg = m < nL ? S.sig_light[m] : S.sig_mass[m - nL];
      const double qp = sh_q[m];
      const double qi2 = (qp * qp - c2) / s2;
      eq += sh_rho[m] * exp(-s * s / (2.0 * sg * sg));
      ax += sh_rho[m] * exp(-s * s / (2.0 * sg * sg * qi2));
    }
    if (!(eq > 0.0) || !(ax > 0.0)) atomicOr(&sh_flag, 1);
  }
  __syncthreads();
  if (sh_flag) {
    if (tid == 0) {
      ws.status[b] = GLAD_SAMPLE_NEGDENS;
      ws.lp[b].valid = 0;
    }
    return;
  }

  // ---- lens model at the observed images (FP64), one image per thread of the second warp
  __shared__ double im_ax[GLAD_MAX_IMG], im_ay[GLAD_MAX_IMG], im_w[GLAD_MAX_IMG], im_psi[GLAD_MAX_IMG];
  if (tid >= 32 && tid < 32 + S.n_img) {
    const int i = tid - 32;
    LensEvalT<double> e = lens_eval_t<double>(S.img_xy[2 * i], S.img_xy[2 * i + 1], th, S, sh_mbh);
    im_ax[i] = e.ax;
    im_ay[i] = e.ay;
    im_psi[i] = e.psi;
    im_w[i] = 1.0 / fabs((1.0 - e.a11) * (1.0 - e.a22) - e.a12 * e.a21);
  }
  // ---- EPL series coefficients of the FP32 lensing block, one per thread
  const double tq = g - 1.0;
  const double fq = (1.0 - q) / (1.0 + q);
  int nt = 0;
  if (fq > 0.0 && !comp) nt = (int)ceil(log(1e-9) / log(fq));
  if (nt > GLAD_MAX_TM) nt = GLAD_MAX_TM;
  // the lensing block in FP32 and, for the FP64 lensing modes, in FP64 (same values)
  auto fill_rho = [&](auto &L) {
    using T = std::remove_reference_t<decltype(L.q)>;
    for (int n = 1 + tid; n <= nt; n += blockDim.x) {
      const double num = 2.0 * n - (2.0 - tq), den = 2.0 * n + (2.0 - tq);
      L.rho[n - 1] = (T)(-fq * num / den);
      L.drho_t[n - 1] = (T)(-fq * 4.0 * n / (den * den));
      L.drho_q[n - 1] = (T)(2.0 * num / (den * (1.0 + q) * (1.0 + q)));
    }
  };
  fill_rho(ws.lp[b]);
  if (ws.prec > 0) fill_rho(ws.lp64[b]);
  __syncthreads();
  if (tid == 0) {
    ws.status[b] = GLAD_SAMPLE_OK;
    // ---- dynamics scalars
    DynP dp;
    dp.s2 = s2;
    dp.c2 = c2;
    dp.b = 1.0 / (1.0 - th[16]);
    dp.xc = th[4];
    dp.yc = th[5];
    sincos(th[3], &dp.sphi, &dp.cphi);
    ws.dp[b] = dp;
    // ---- lensing block (FP32; FP64 too for the FP64 lensing modes)
    auto fill = [&](auto &L) {
      using T = std::remove_reference_t<decltype(L.q)>;
      const double bb = pow(2.0 / (1.0 + q), 1.0 / tq) * tE;
      const double bt = q * bb;
      L.xc = (T)th[4];
      L.yc = (T)th[5];
      L.cphi = (T)dp.cphi;
      L.sphi = (T)dp.sphi;
      L.q = (T)q;
      L.t = (T)tq;
      // ln pref = ln 2 + t ln b_TM - ln(1+q), b_TM = q (2/(1+q))^(1/t) theta_E
      const double pref = 2.0 * bt / (1.0 + q) * pow(bt, tq - 1.0);
      L.pref = (T)pref;
      L.nterms = nt;
      L.pref_d[0] = (T)(pref * tq / tE);
      L.pref_d[1] = (T)(pref * (log(bt) - log(2.0 / (1.0 + q)) / tq));
      L.pref_d[2] = (T)(pref * (tq / q - 2.0 / (1.0 + q)));
      double s2p, c2p;
      sincos(2.0 * th[7], &s2p, &c2p);
      L.g1 = (T)(th[6] * c2p);
      L.g2 = (T)(th[6] * s2p);
      L.gext = (T)th[6];
      L.c2pe = (T)c2p;
      L.s2pe = (T)s2p;
      {
        const double n = th[10];
        L.src_bnp = (T)(2.0 - 4.0 / (405.0 * n * n) - 92.0 / (25515.0 * n * n * n) -
                            393.0 / (1148175.0 * n * n * n * n) +
                            4.0 * 2194697.0 / (30690717750.0 * n * n * n * n * n));
      }
      L.src_Ie = (T)th[8];
      L.src_Rei = (T)(1.0 / th[9]);
      L.src_ninv = (T)(1.0 / th[10]);
      L.src_bn = (T)sersic_bn_d(th[10]);
      L.src_x = (T)th[11];
      L.src_y = (T)th[12];
      L.sheet = S.sheet;
      L.lam = (T)lam;
      L.sh_rc = (T)S.sh_rc;
      L.sh_rt = (T)S.sh_rt;
      L.sh_rc2 = (T)(S.sh_rc * S.sh_rc);
      L.sh_rt2 = (T)(S.sh_rt * S.sh_rt);
      L.mclass = S.mass_class;
      if (comp) {
        const double ups = th[17] * S.L_scale;
        for (int c = 0; c < S.n_lcomp && c < 4; ++c) {
          const double qc = S.lcomp[4 * c + 3];
          const double I0 = c == 0 ? th[13] : S.lcomp[4 * c];
          const double wt = c == 0 ? th[14] : S.lcomp[4 * c + 2];
          L.li_A[c] = (T)(I0 / (1.0 + qc));
          L.ch_A[c] = (T)(ups * I0 / (1.0 + qc));
          L.ch_sc[c] = (T)(2.0 * S.lcomp[4 * c + 1] / (1.0 + qc));
          L.ch_st[c] = (T)(2.0 * wt / (1.0 + qc));
          L.ch_q[c] = (T)qc;
          L.ch_e[c] = (T)sqrt(1.0 - qc * qc);
        }
        L.ups = (T)ups;
        L.h_ks = (T)th[0];
        L.h_rs = (T)th[1];
        L.h_q = (T)q;
        L.h_e2 = (T)(1.0 - q * q);
        L.bh_M = (T)sh_mbh;
        L.bh_2s2 = (T)(2.0 * S.bh_sigma * S.bh_sigma);
        for (int i = 0; i < 4; ++i) L.bh_dM[i] = (T)sh_dm[i];
        const double rs3 = th[1] * th[1] * th[1];
        for (int i = 0; i < GLAD_N_CSE; ++i) {
          L.cse_amp[i] = (T)(th[0] * S.cse_a[i] * rs3);
          L.cse_sc[i] = (T)(S.cse_s[i] * th[1]);
          L.cse_a3[i] = (T)(S.cse_a[i] * rs3);
        }
      }
      for (int c = 0; c < S.n_lcomp && c < 4 && !comp; ++c) {  // Sersic lens light (class 0)
        const double Ie = c == 0 ? th[13] : S.lcomp[4 * c];
        const double Re = c == 0 ? th[14] : S.lcomp[4 * c + 1];
        const double n = S.lcomp[4 * c + 2], ql = S.lcomp[4 * c + 3];
        L.ll_Ie[c] = (T)Ie;
        L.ll_Rei[c] = (T)(1.0 / Re);
        L.ll_ninv[c] = (T)(1.0 / n);
        L.ll_bn[c] = (T)sersic_bn_d(n);
        L.ll_qi2[c] = (T)(1.0 / (ql * ql));
      }
      L.valid = 1;
    };
    fill(ws.lp[b]);
    if (ws.prec > 0) fill(ws.lp64[b]);
  }
  if (tid == 32) {
    // ---- time delays (FP64): beta_hat, Fermat potentials, chi^2_tmd from the images
    double wsum = 0.0, bhx = 0.0, bhy = 0.0;
    for (int i = 0; i < S.n_img; ++i) {
      wsum += im_w[i];
      bhx += im_w[i] * (S.img_xy[2 * i] - im_ax[i]);
      bhy += im_w[i] * (S.img_xy[2 * i + 1] - im_ay[i]);
    }
    bhx /= wsum;
    bhy /= wsum;
    const double kdt = delay_unit_t<double>(th, S);
    double phi0 = 0.0, chi2 = 0.0;
    for (int i = 0; i < S.n_img; ++i) {
      const double x = S.img_xy[2 * i], y = S.img_xy[2 * i + 1];
      const double ph = 0.5 * ((x - bhx) * (x - bhx) + (y - bhy) * (y - bhy)) - im_psi[i];
      if (i == 0) {
        phi0 = ph;
      } else {
        const double r = (S.dt_obs[i - 1] - kdt * (ph - phi0)) / S.dt_sig[i - 1];
        chi2 += r * r;
      }
    }
    ws.terms[4 * (size_t)b + 2] = chi2;
  }
  if (tid == 64 && S.img_sig) {
    // ---- image positions (FP64), beside the delays
    ws.terms[4 * (size_t)b + 3] = chi2_img_t<double>(th, S, sh_mbh);
  }
}

// (k, j, g) coefficient table: exponent coefficients in log2 units and the two
// prefactor terms of the pair form of the cylindrically aligned JAM integral.
__global__ void __launch_bounds__(TAB_THREADS) k_table(const SysDev *__restrict__ sysv,
                                                       const int *__restrict__ sys_id, WsDev ws,
                                                       int max_light, int max_mass, int max_ent) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  const int e = blockIdx.x * TAB_THREADS + threadIdx.x;
  if (e >= S.n_ent || S.jam_align != 0) return;  // the spherically aligned model has no table
  const int kj = e / S.n_gl;
  const int j = kj % S.n_mass_tot;
  const int k = kj / S.n_mass_tot;
  const DynP dp = ws.dp[b];
  // a = u^2/(2 s_j^2), p = 1/(2 s_k^2) + a and u^2 are per-entry constants of the system
  const double a = S.gl_a[e], p = S.gl_p[e], wu = S.gl_wu[e];
  const double e2 = ws.e2[(size_t)b * max_mass + j];
  const double h = 1.0 - e2 * S.gl_u2[e];
  const double ih = 1.0 / h, rsh = rsqrt(h);
  const double c = ws.c0[(size_t)b * max_light + k] + a * ih;
  const double ic = 1.0 / c;
  const double al = p * dp.s2 + c * dp.c2;
  const double ial = 1.0 / al;
  const double A = a * ih * rsh * ic;  // a / (h^(3/2) c)
  const double P0 = A * (dp.b * dp.s2 + dp.c2);
  const double P1 = dp.s2 * (2.0 * a * rsh - 2.0 * p * dp.b * A);
  const double T = ws.nu0[(size_t)b * max_light + k] * ws.Cj[(size_t)b * max_mass + j] * wu *
                   sqrt(PI_D * ial);
  ws.tab[(size_t)b * max_ent + e] =
      make_float4((float)(-p * LOG2E_D), (float)(-p * c * ial * LOG2E_D), (float)(T * P0),
                  (float)(T * P1));
  if (ws.prec == 2) {
    // FP64 pair sum: natural-log exponent coefficients
    double4_16a t64;
    t64.x = -p;
    t64.y = -p * c * ial;
    t64.z = T * P0;
    t64.w = T * P1;
    ws.tab64[(size_t)b * max_ent + e] = t64;
  }
}

}  // namespace

cudaError_t launch_prep(glad_ctx *c, const int *sys_id, const double *theta, int B,
                        cudaStream_t st) {
  k_prep<<<B, 128, 0, st>>>(c->d_sys, sys_id, theta, c->ws.d, c->max_light, c->max_mass_tot);
  return cudaGetLastError();
}

cudaError_t launch_table(glad_ctx *c, const int *sys_id, int B, cudaStream_t st) {
  dim3 grid(c->max_tab_blocks, B);
  k_table<<<grid, TAB_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d, c->max_light, c->max_mass_tot,
                                        c->max_ent);
  return cudaGetLastError();
}
