// C ABI of libglad: context creation (host-side FP64 precomputation and staging),
// workspace management and the launch sequences of the likelihood calls.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <complex>
#include <cstdarg>
#include <string>
#include <vector>

#include "glad_internal.cuh"

cudaError_t grad_ws_ensure(glad_ctx *c, int B);
void grad_ws_free(glad_ctx *c);
float *grad_resid_buffer(glad_ctx *c);
cudaError_t launch_jam_fg(glad_ctx *c, const int *sys_id, int B, cudaStream_t st);
void set_grad_smem_limit();

namespace {

thread_local std::string g_err;

glad_status fail(glad_status s, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

const double C_KMS = 299792.458;
const double ARCSEC = PI_D / 648000.0;
const double MPC_KM = 3.0856775814913673e19;
const double DAY_S = 86400.0;

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n (n >= 2).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  auto legendre = [n](double z, double &p_n, double &p_nm1) {
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    p_n = p1;
    p_nm1 = p0;
  };
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(PI_D * (i + 0.75) / (n + 0.5));
    double pn, pm, dp;
    for (int it = 0; it < 100; ++it) {
      legendre(z, pn, pm);
      dp = n * (z * pn - pm) / (z * z - 1.0);
      const double dz = pn / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) break;
    }
    legendre(z, pn, pm);
    dp = n * (z * pn - pm) / (z * z - 1.0);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// flat LambdaCDM comoving distance [Mpc] by 96-point Gauss-Legendre (smooth integrand)
double comoving(double z, double H0, double om) {
  std::vector<double> x, w;
  gauss_legendre(96, x, w);
  double s = 0.0;
  for (size_t i = 0; i < x.size(); ++i) {
    const double zz = 0.5 * z * (x[i] + 1.0);
    s += w[i] / sqrt(om * pow(1.0 + zz, 3) + 1.0 - om);
  }
  return C_KMS / H0 * 0.5 * z * s;
}

// Euler coefficients (Abate & Whitt 2006) in the Gaussian-mixture scaling of Sect. 3.2:
// eta_m = (-1)^m 2 sqrt(2 pi) 10^(P/3) xi_m and chi_m = sqrt(2 P ln10 / 3 + 2 pi i m)
void euler_coefficients(int P, std::vector<double> &eta, std::vector<std::complex<double>> &chi) {
  std::vector<double> xi(2 * P + 1, 0.0);
  eta.assign(2 * P + 1, 0.0);
  chi.assign(2 * P + 1, 0.0);
  xi[0] = 0.5;
  for (int m = 1; m <= P; ++m) xi[m] = 1.0;
  xi[2 * P] = pow(2.0, -P);
  double binom = 1.0;  // C(P, k)
  for (int k = 1; k < P; ++k) {
    binom = binom * (P - k + 1) / k;
    xi[2 * P - k] = xi[2 * P - k + 1] + pow(2.0, -P) * binom;
  }
  const double A = 2.0 * P * log(10.0) / 3.0;
  for (int m = 0; m <= 2 * P; ++m) {
    eta[m] = (m % 2 ? -1.0 : 1.0) * 2.0 * SQRT2PI_D * pow(10.0, P / 3.0) * xi[m];
    // principal square root of A + 2 pi i m
    const double re = A, im = 2.0 * PI_D * m;
    const double r = sqrt(hypot(re, im));
    const double th = 0.5 * atan2(im, re);
    chi[m] = std::complex<double>(r * cos(th), r * sin(th));
  }
}

template <class T>
T *upload(SysHost &sh, const T *src, size_t n) {
  T *d = nullptr;
  if (n == 0) n = 1;
  if (cudaMalloc(&d, n * sizeof(T)) != cudaSuccess) {
    sh.allocs.push_back(nullptr);
    return nullptr;
  }
  sh.allocs.push_back(d);
  if (src && cudaMemcpy(d, src, n * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return nullptr;
  return d;
}

glad_status validate(const glad_system_desc &d, int idx) {
#define REQ(cond, ...) \
  if (!(cond)) return fail(GLAD_EINVAL, "system %d: " __VA_ARGS__)
  REQ(d.nx > 0 && d.ny > 0 && d.ss > 0 && d.pix > 0, "bad image geometry", idx);
  REQ(d.data && d.sigma && d.mask && d.psf, "missing image arrays", idx);
  REQ(d.psf_k > 0 && d.psf_k % 2 == 1, "psf_k must be odd", idx);
  REQ(d.kx > 0 && d.ky > 0 && d.kss > 0 && d.kpix > 0, "bad sky geometry", idx);
  REQ(d.kpsf && d.kpsf_k > 0 && d.kpsf_k % 2 == 1, "kpsf_k must be odd", idx);
  REQ(d.bins && d.v_obs && d.v_sig && d.n_bins > 0, "missing kinematic arrays", idx);
  REQ(d.n_mge_mass >= 2 && d.n_mge_light, "bad MGE sizes", idx);
  REQ(d.mge_P > 0 && d.n_gl >= 2, "bad MGE order or quadrature order", idx);
  REQ(d.mass_rmin > 0 && d.mass_rmax > d.mass_rmin && d.light_rmin > 0 &&
          d.light_rmax > d.light_rmin, "bad MGE ranges", idx);
  REQ(d.n_img >= 2 && d.img_xy && d.dt_obs && d.dt_sig, "need >= 2 images with delays", idx);
  if (d.img_sig)
    for (int i = 0; i < d.n_img; ++i) REQ(d.img_sig[i] > 0, "img_sig must be positive", idx);
  REQ(d.n_ll2 >= 0 && (d.n_ll2 == 0 || d.ll2), "bad extra lens lights", idx);
  REQ(d.n_sis >= 0 && (d.n_sis == 0 || d.sis), "bad SIS list", idx);
  REQ(d.z_s > d.z_d && d.z_d > 0 && d.omega_m > 0 && d.omega_m < 1, "bad cosmology", idx);
  REQ(d.jam_align == 0 || d.jam_align == 1, "jam_align must be 0 or 1", idx);
  REQ(d.sph_nr == 0 || d.sph_nr >= 4, "sph_nr must be 0 (default) or >= 4", idx);
  REQ(d.sph_nw == 0 || d.sph_nw >= 2, "sph_nw must be 0 (default) or >= 2", idx);
  REQ(d.sph_nlos >= 0, "sph_nlos must be >= 0", idx);
  REQ(d.sheet >= 0 && d.sheet <= 2, "sheet must be 0, 1 or 2", idx);
  REQ(d.distance_mode == 0 || d.distance_mode == 1, "distance_mode must be 0 or 1", idx);
  REQ(d.mass_class == 0 || d.mass_class == 1, "mass_class must be 0 or 1", idx);
  if (d.mass_class == 1) {
    REQ(d.ll_wc > 0 && d.ll_q > 0 && d.ll_q <= 1, "composite class needs ll_wc > 0, 0 < ll_q <= 1", idx);
    for (int k = 0; k < d.n_ll2; ++k)
      REQ(d.ll2[4 * k] > 0 && d.ll2[4 * k + 1] > 0 && d.ll2[4 * k + 2] > d.ll2[4 * k + 1] &&
              d.ll2[4 * k + 3] > 0 && d.ll2[4 * k + 3] <= 1,
          "Chameleon rows need I0 > 0, 0 < w_c < w_t, 0 < q <= 1", idx);
  }
  if (d.sheet) {
    const double rc = d.sheet_rc > 0 ? d.sheet_rc : 45.0, rt = d.sheet_rt > 0 ? d.sheet_rt : 45.09;
    REQ(d.sheet_rc >= 0 && d.sheet_rt >= 0 && rt > rc, "sheet radii need 0 < rc < rt", idx);
    REQ(d.sheet_n == 0 || d.sheet_n >= 2, "sheet_n must be 0 (default) or >= 2", idx);
    const double lo = d.sheet_rmin > 0 ? d.sheet_rmin : 0.1, hi = d.sheet_rmax > 0 ? d.sheet_rmax : 1000.0;
    REQ(d.sheet_rmin >= 0 && d.sheet_rmax >= 0 && hi > lo, "bad sheet MGE range", idx);
  }
  REQ(d.src_pix == 0 || d.src_pix == 1, "src_pix must be 0 or 1", idx);
  if (d.src_pix) {
    REQ(d.spx_nx >= 3 && d.spx_ny >= 3, "source grid needs >= 3 pixels along x and y", idx);
    REQ(d.spx_x1 > d.spx_x0 && d.spx_y1 > d.spx_y0, "bad source grid extent", idx);
    REQ((d.spx_lam_lo == 0 && d.spx_lam_hi == 0) || (d.spx_lam_lo > 0 && d.spx_lam_hi > d.spx_lam_lo),
        "regularisation range needs 0 < spx_lam_lo < spx_lam_hi (or both 0)", idx);
    REQ(d.spx_iters >= 0 && d.spx_iters <= SPX_MAX_ITERS, "spx_iters must be in [0, 200]", idx);
    int nm = 0;
    for (int i = 0; i < d.nx * d.ny; ++i) nm += d.mask[i] != 0;
    REQ(nm > 0, "pixelated source needs a non-empty mask", idx);
  }
#undef REQ
#define SUP(cond, ...) \
  if (!(cond)) return fail(GLAD_EUNSUPPORTED, "system %d: " __VA_ARGS__)
  SUP(d.psf_k <= GLAD_MAX_PSF, "psf_k > %d", idx, GLAD_MAX_PSF);
  SUP(d.n_bins <= GLAD_MAX_BINS, "n_bins > %d", idx, GLAD_MAX_BINS);
  const int n_sheet = d.sheet ? (d.sheet_n ? d.sheet_n : 40) : 0;
  int nl_all = 0;
  for (int c = 0; c < 1 + d.n_ll2 && d.n_mge_light; ++c) nl_all += d.n_mge_light[c];
  // galaxy mass Gaussians: the EPL's, or (composite) the tracer's copies and the halo's
  const int n_gal = d.n_mge_mass + (d.mass_class == 1 ? nl_all : 0);
  SUP(n_gal + n_sheet <= GLAD_MAX_MASS, "n_mge_mass + sheet Gaussians > %d", idx, GLAD_MAX_MASS);
  SUP(d.mge_P <= GLAD_MAX_P, "mge_P > %d", idx, GLAD_MAX_P);
  SUP(d.n_img <= GLAD_MAX_IMG, "n_img > %d", idx, GLAD_MAX_IMG);
  SUP(1 + d.n_ll2 <= 4, "more than 4 lens-light components", idx);
  int nl = 0;
  for (int c = 0; c < 1 + d.n_ll2; ++c) {
    if (d.n_mge_light[c] < 2) return fail(GLAD_EINVAL, "system %d: n_mge_light < 2", idx);
    nl += d.n_mge_light[c];
  }
  SUP(nl <= GLAD_MAX_LIGHT, "tracer Gaussians > %d", idx, GLAD_MAX_LIGHT);
  for (int i = 0; i < d.kx * d.ky; ++i)
    if (d.bins[i] >= d.n_bins) return fail(GLAD_EINVAL, "system %d: bin index >= n_bins", idx);
  if (d.src_pix) {
    SUP((long long)d.spx_nx * d.spx_ny <= GLAD_MAX_SRCPIX, "source grid > %d pixels", idx,
        GLAD_MAX_SRCPIX);
    SUP(d.ss <= 4, "pixelated source with more than 4 x 4 rays per pixel", idx);
  }
  if (d.jam_align == 1) {
    const int nr = d.sph_nr ? d.sph_nr : SPH_DEFAULT_NR, nw = d.sph_nw ? d.sph_nw : SPH_DEFAULT_NW;
    SUP(nr * nw <= GLAD_SPH_MAX_GRID, "sph_nr * sph_nw > %d", idx, GLAD_SPH_MAX_GRID);
    SUP((n_gal + n_sheet + (d.has_bh ? 1 : 0)) * d.n_gl <= GLAD_SPH_MAX_MG,
        "mass Gaussians x n_gl > %d for the spherically aligned model", idx, GLAD_SPH_MAX_MG);
    SUP(d.sph_nlos <= 4096, "sph_nlos > 4096", idx);
    // shared memory of the gradient kernels (grid adjoint: coefficients and their accumulators;
    // line-of-sight adjoint: grid, grid adjoint and per-thread tracer accumulators)
    const size_t mg = (size_t)(n_gal + n_sheet + (d.has_bh ? 1 : 0)) * d.n_gl;
    const size_t ladj = (size_t)nr * (nw - 1) * 16 + (size_t)nr * (nw | 1) * 8 + (size_t)nl * (16 + 128 * 8);
    const size_t gadj = mg * 40 + 8 * 64 * 16 + (size_t)nl * 24 + 16;
    SUP(ladj <= 226 * 1024 && gadj <= 226 * 1024,
        "spherically aligned model too large for the gradient kernels' shared memory", idx);
  }
#undef SUP
  return GLAD_OK;
}

glad_status build_system(int idx, const glad_system_desc &d, SysHost &sh, SysDev &sd) {
  memset(&sd, 0, sizeof sd);
  sh.d = d;
  const int npix = d.nx * d.ny;
  sh.npix = npix;
  sd.nx = d.nx;
  sd.ny = d.ny;
  sd.ss = d.ss;
  sd.npix = npix;
  sd.pix = (float)d.pix;
  // 1/sigma in FP64: its float32 rounding would scale chi^2_pix coherently by up to ~1e-7
  std::vector<double> wgt(npix);
  for (int i = 0; i < npix; ++i) wgt[i] = d.mask[i] ? 1.0 / (double)d.sigma[i] : 0.0;
  sd.data = upload(sh, d.data, npix);
  sd.wgt = upload(sh, wgt.data(), npix);
  sd.psf_k = d.psf_k;
  sd.psf = upload(sh, d.psf, (size_t)d.psf_k * d.psf_k);
  // the blocked convolution's copy: centred in the next supported side, transposed
  sd.psf_km = d.psf_k <= 11 ? 11 : d.psf_k <= 21 ? 21 : d.psf_k <= 31 ? 31 : 0;
  sd.psf_t = nullptr;
  if (sd.psf_km) {
    const int km = sd.psf_km, pt = CONV_PT(km), off = (km - d.psf_k) / 2;
    std::vector<float> t((size_t)km * pt, 0.0f);
    for (int a = 0; a < d.psf_k; ++a)
      for (int cc = 0; cc < d.psf_k; ++cc) t[(size_t)(cc + off) * pt + (a + off)] = d.psf[a * d.psf_k + cc];
    sd.psf_t = upload(sh, t.data(), t.size());
  }
  sd.src_q = (float)d.src_q;
  sd.src_cphi = (float)cos(d.src_phi);
  sd.src_sphi = (float)sin(d.src_phi);
  sd.pix64 = d.pix;
  sd.src_q64 = d.src_q;
  sd.src_cphi64 = cos(d.src_phi);
  sd.src_sphi64 = sin(d.src_phi);
  sd.n_lcomp = 1 + d.n_ll2;
  // lens-light rows: Sersic (I_e, R_e, n, q) or, in the composite class, Chameleon
  // (I0, w_c, w_t, q); row 0's I_e, R_e (or I0, w_t) come from theta
  std::vector<double> lcomp(4 * sd.n_lcomp);
  lcomp[0] = 0.0;
  lcomp[1] = d.mass_class == 1 ? d.ll_wc : 0.0;
  lcomp[2] = d.mass_class == 1 ? 0.0 : d.ll_n;
  lcomp[3] = d.ll_q;
  for (int k = 0; k < d.n_ll2; ++k)
    for (int m = 0; m < 4; ++m) lcomp[4 * (k + 1) + m] = d.ll2[4 * k + m];
  sd.lcomp = upload(sh, lcomp.data(), lcomp.size());
  sd.n_sis = d.n_sis;
  sd.sis = upload(sh, d.sis, (size_t)3 * d.n_sis);
  sd.r_soft = d.r_soft;
  // sky sub-grid
  sd.nsx = d.kx * d.kss;
  sd.nsy = d.ky * d.kss;
  sd.n_sub = sd.nsx * sd.nsy;
  sh.n_sub = sd.n_sub;
  sd.dsub = (float)(d.kpix / d.kss);
  sd.dsub64 = d.kpix / d.kss;
  // binning-after-PSF operator: W_l(s') = sum_{s in bin l} P(s - s')
  {
    const int K = d.kpsf_k, h = (K - 1) / 2, nsx = sd.nsx, nsy = sd.nsy;
    std::vector<int> off(sd.n_sub + 1, 0);
    std::vector<int> wb;
    std::vector<float> wv;
    std::vector<int> taps_a, taps_b;
    std::vector<double> taps_v;
    for (int a = 0; a < K; ++a)
      for (int bb = 0; bb < K; ++bb)
        if (d.kpsf[a * K + bb] != 0.0f) {
          taps_a.push_back(a - h);
          taps_b.push_back(bb - h);
          taps_v.push_back(d.kpsf[a * K + bb]);
        }
    std::vector<double> accw(d.n_bins, 0.0);
    std::vector<int> touched;
    for (int I = 0; I < nsy; ++I)
      for (int J = 0; J < nsx; ++J) {
        touched.clear();
        for (size_t t = 0; t < taps_v.size(); ++t) {
          // s = s' + (a-h, b-h) receives P[a,b] * m(s')
          const int si = I + taps_a[t], sj = J + taps_b[t];
          if (si < 0 || si >= nsy || sj < 0 || sj >= nsx) continue;
          const int l = d.bins[(si / d.kss) * d.kx + (sj / d.kss)];
          if (l < 0) continue;
          if (accw[l] == 0.0) touched.push_back(l);
          accw[l] += taps_v[t];
        }
        std::sort(touched.begin(), touched.end());
        for (int l : touched) {
          wb.push_back(l);
          wv.push_back((float)accw[l]);
          accw[l] = 0.0;
        }
        off[I * nsx + J + 1] = (int)wb.size();
      }
    sd.w_off = upload(sh, off.data(), off.size());
    sd.w_bin = upload(sh, wb.data(), wb.size());
    sd.w_val = upload(sh, wv.data(), wv.size());
  }
  sd.n_bins = d.n_bins;
  sd.v_obs = upload(sh, d.v_obs, d.n_bins);
  sd.v_sig = upload(sh, d.v_sig, d.n_bins);
  std::vector<double> sig_l, mw_l, qp_l;
  std::vector<int> comp_of;
  for (int cc = 0; cc < 1 + d.n_ll2; ++cc) {
    const int N = d.n_mge_light[cc];
    const double lo = log(d.light_rmin), hi = log(d.light_rmax), dl = (hi - lo) / (N - 1);
    const double q = cc == 0 ? d.ll_q : d.ll2[4 * (cc - 1) + 3];
    for (int k = 0; k < N; ++k) {
      sig_l.push_back(exp(lo + dl * k));
      mw_l.push_back((k == 0 || k == N - 1 ? 0.5 : 1.0) * dl / SQRT2PI_D);
      qp_l.push_back(q);
      comp_of.push_back(cc);
    }
  }
  const int nL = (int)sig_l.size();
  // MGE Gaussians: mass [galaxy nM][internal sheet nS][black hole]
  // (composite class: the galaxy's Gaussians are the nL tracer Gaussians, scaled per sample by
  // Upsilon L_scale, and then the halo's n_mge_mass on the mass range)
  const int nH = d.n_mge_mass;
  const int off = d.mass_class == 1 ? nL : 0;
  const int nM = off + nH;
  const int nS = d.sheet ? (d.sheet_n ? d.sheet_n : 40) : 0;
  const int nMt = nM + nS + (d.has_bh ? 1 : 0);
  std::vector<double> sig_m(nMt), mw_m(nM, 0.0), sheet_a1(std::max(nS, 1), 0.0);
  {
    for (int j = 0; j < off; ++j) sig_m[j] = sig_l[j];
    const double lo = log(d.mass_rmin), hi = log(d.mass_rmax), dl = (hi - lo) / (nH - 1);
    for (int j = 0; j < nH; ++j) {
      sig_m[off + j] = exp(lo + dl * j);
      mw_m[off + j] = (j == 0 || j == nH - 1 ? 0.5 : 1.0) * dl / SQRT2PI_D;
    }
    if (d.has_bh) sig_m[nM + nS] = d.bh_sigma;
  }
  sd.mass_class = d.mass_class;
  sd.n_halo = d.mass_class == 1 ? nH : 0;
  {
    const double *ca = nullptr, *cs = nullptr;
    if (d.mass_class == 1) cse_table(&ca, &cs);
    sd.cse_a = upload(sh, ca, GLAD_N_CSE);
    sd.cse_s = upload(sh, cs, GLAD_N_CSE);
  }
  sd.sheet = d.sheet;
  sd.sh_rc = d.sheet_rc > 0 ? d.sheet_rc : 45.0;
  sd.sh_rt = d.sheet_rt > 0 ? d.sheet_rt : 45.09;
  if (nS) {
    // the dPIE sheet's 1-D MGE (Sect. 3.2, Euler inversion) at 1 - lambda_int = 1, in FP64 once:
    // kappa(R) = [1/sqrt(R^2 + rc^2) - 1/sqrt(R^2 + rt^2)] / (1/rc - 1/rt) (Eq. dpie_kappa with
    // central value 1); per sample the amplitudes are scaled by 1 - lambda_int
    const double rc = sd.sh_rc, rt = sd.sh_rt;
    const double lo = log(d.sheet_rmin > 0 ? d.sheet_rmin : 0.1);
    const double hi = log(d.sheet_rmax > 0 ? d.sheet_rmax : 1000.0);
    const double dl = (hi - lo) / (nS - 1);
    const int P = d.mge_P;
    std::vector<double> eta;
    std::vector<std::complex<double>> chi;
    euler_coefficients(P, eta, chi);
    const double norm = 1.0 / ((rt - rc) / (rc * rt));
    for (int j = 0; j < nS; ++j) {
      const double sg = exp(lo + dl * j);
      double f = 0.0;
      for (int m = 0; m <= 2 * P; ++m) {
        const std::complex<double> z = sg * chi[m], z2 = z * z;
        const std::complex<double> F = norm * (1.0 / std::sqrt(z2 + rc * rc) - 1.0 / std::sqrt(z2 + rt * rt));
        f += eta[m] * F.real();
      }
      sig_m[nM + j] = sg;
      sheet_a1[j] = (j == 0 || j == nS - 1 ? 0.5 : 1.0) * dl / SQRT2PI_D * f;
    }
  }
  sd.n_sheet = nS;
  sd.sheet_A1 = upload(sh, sheet_a1.data(), sheet_a1.size());
  sd.n_mass = nM;
  sd.n_mass_tot = nMt;
  sd.n_light = nL;
  sh.n_mass_tot = nMt;
  sh.n_light = nL;
  sd.lcomp_of = upload(sh, comp_of.data(), nL);
  sd.sig_mass = upload(sh, sig_m.data(), nMt);
  sd.sig_light = upload(sh, sig_l.data(), nL);
  sd.mw_mass = upload(sh, mw_m.data(), nM);
  sd.mw_light = upload(sh, mw_l.data(), nL);
  sd.qp_light = upload(sh, qp_l.data(), nL);
  // Euler coefficients (Abate & Whitt 2006) in the Gaussian-mixture scaling of Sect. 3.2
  {
    const int P = d.mge_P;
    std::vector<double> eta;
    std::vector<std::complex<double>> chic;
    euler_coefficients(P, eta, chic);
    std::vector<double2> chi(2 * P + 1);
    for (int m = 0; m <= 2 * P; ++m) chi[m] = make_double2(chic[m].real(), chic[m].imag());
    sd.mge_P = P;
    sd.eta = upload(sh, eta.data(), eta.size());
    sd.chi = upload(sh, chi.data(), chi.size());
  }
  // JAM u nodes with the per-pair map u = u_s (exp(lam t) - 1), lam = ln(1 + 1/u_s),
  // u_s = min(1, sigma_j / max(r_max, sigma_k))
  {
    const int G = d.n_gl;
    std::vector<double> x, w;
    gauss_legendre(G, x, w);
    double r_max = 0.0;
    for (int I = 0; I < sd.nsy; ++I)
      for (int J = 0; J < sd.nsx; ++J) {
        const double xx = (J - 0.5 * (sd.nsx - 1)) * (d.kpix / d.kss);
        const double yy = (I - 0.5 * (sd.nsy - 1)) * (d.kpix / d.kss);
        r_max = std::max(r_max, hypot(xx, yy));
      }
    const int n_ent = nL * nMt * G;
    std::vector<double> gu(n_ent), gw(n_ent);
    for (int k = 0; k < nL; ++k)
      for (int j = 0; j < nMt; ++j) {
        const double us = std::min(1.0, sig_m[j] / std::max(r_max, sig_l[k]));
        const double lam = log1p(1.0 / us);
        for (int g = 0; g < G; ++g) {
          const double t = 0.5 * (x[g] + 1.0), wt = 0.5 * w[g];
          const double e = exp(lam * t);
          gu[(k * nMt + j) * G + g] = us * (e - 1.0);
          gw[(k * nMt + j) * G + g] = wt * us * lam * e;
        }
      }
    sd.n_gl = G;
    sd.n_ent = n_ent;
    sh.n_ent = n_ent;
    sd.gl_u = upload(sh, gu.data(), n_ent);
    sd.gl_wu = upload(sh, gw.data(), n_ent);
    // entry order for the adjoint: ascending p = 1/(2 s_k^2) + u^2/(2 s_j^2)
    std::vector<double> pe(n_ent);
    for (int k = 0; k < nL; ++k)
      for (int j = 0; j < nMt; ++j)
        for (int g = 0; g < G; ++g) {
          const int e = (k * nMt + j) * G + g;
          pe[e] = 1.0 / (2.0 * sig_l[k] * sig_l[k]) + gu[e] * gu[e] / (2.0 * sig_m[j] * sig_m[j]);
        }
    // per-entry constants of the table formula: a = u^2/(2 s_j^2), p = 1/(2 s_k^2) + a, u^2
    std::vector<double> ga(n_ent), gp(n_ent), gu2(n_ent);
    for (int k = 0; k < nL; ++k)
      for (int j = 0; j < nMt; ++j)
        for (int g = 0; g < G; ++g) {
          const int e = (k * nMt + j) * G + g;
          gu2[e] = gu[e] * gu[e];
          ga[e] = gu2[e] / (2.0 * sig_m[j] * sig_m[j]);
          gp[e] = 1.0 / (2.0 * sig_l[k] * sig_l[k]) + ga[e];
        }
    sd.gl_a = upload(sh, ga.data(), n_ent);
    sd.gl_p = upload(sh, gp.data(), n_ent);
    sd.gl_u2 = upload(sh, gu2.data(), n_ent);
    std::vector<int> perm(n_ent);
    for (int e = 0; e < n_ent; ++e) perm[e] = e;
    std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return pe[a] < pe[b]; });
    sd.adj_perm = upload(sh, perm.data(), n_ent);
  }
  {
    std::vector<float> cx(nL), cy(nL);
    for (int k = 0; k < nL; ++k) {
      cx[k] = (float)(LOG2E_D / (2.0 * sig_l[k] * sig_l[k]));
      cy[k] = (float)(LOG2E_D / (2.0 * sig_l[k] * sig_l[k] * qp_l[k] * qp_l[k]));
    }
    sd.sb_cx = upload(sh, cx.data(), nL);
    sd.sb_cy = upload(sh, cy.data(), nL);
  }
  // spherically aligned model: polar grid r in [r_lo, r_end] (r_lo = d_sub/4, r_end = 9 x the
  // largest tracer sigma) and the u rule of mass Gaussian j: u = u_s (exp(lam t) - 1),
  // lam = ln(1 + 1/u_s), u_s = min(1, sigma_j / r_end), n_gl-point Gauss-Legendre in t
  sd.jam_align = d.jam_align;
  if (d.jam_align == 1) {
    sd.sph_nr = d.sph_nr ? d.sph_nr : SPH_DEFAULT_NR;
    sd.sph_nw = d.sph_nw ? d.sph_nw : SPH_DEFAULT_NW;
    sd.sph_nlos = d.sph_nlos ? d.sph_nlos : SPH_DEFAULT_NLOS;
    double smax = 0.0;
    for (int k = 0; k < nL; ++k) smax = std::max(smax, sig_l[k]);
    sd.sph_r_lo = 0.25 * d.kpix / d.kss;
    sd.sph_r_end = 9.0 * smax;
    if (!(sd.sph_r_end > sd.sph_r_lo))
      return fail(GLAD_EINVAL, "system %d: tracer too compact for the sky sampling", idx);
    sd.sph_lr0 = log(sd.sph_r_lo);
    sd.sph_dlr = (log(sd.sph_r_end) - sd.sph_lr0) / (sd.sph_nr - 1);
    const int G = d.n_gl;
    std::vector<double> x, w, su(nMt * G), sw(nMt * G);
    gauss_legendre(G, x, w);
    for (int j = 0; j < nMt; ++j) {
      const double us = std::min(1.0, sig_m[j] / sd.sph_r_end);
      const double lam = log1p(1.0 / us);
      for (int g = 0; g < G; ++g) {
        const double t = 0.5 * (x[g] + 1.0), e = exp(lam * t);
        su[j * G + g] = us * (e - 1.0);
        sw[j * G + g] = 0.5 * w[g] * us * lam * e;
      }
    }
    sd.sph_u = upload(sh, su.data(), su.size());
    sd.sph_wu = upload(sh, sw.data(), sw.size());
  }
  // pixelated source: the mask's pixel list, C = H^T H (H: second differences along x and y,
  // zero outside the grid) and ln det C by a banded Cholesky (half-bandwidth 2 nx), and the
  // evidence's lambda-free constant
  sd.src_pix = d.src_pix;
  if (d.src_pix) {
    const int gx = d.spx_nx, gy = d.spx_ny, ns = gx * gy;
    sd.spx_nx = gx;
    sd.spx_ny = gy;
    sd.spx_ns = ns;
    sd.spx_x0 = (float)d.spx_x0;
    sd.spx_y0 = (float)d.spx_y0;
    sd.spx_idx = (float)(gx / (d.spx_x1 - d.spx_x0));
    sd.spx_idy = (float)(gy / (d.spx_y1 - d.spx_y0));
    sd.spx_iters = d.spx_iters ? d.spx_iters : SPX_DEFAULT_ITERS;
    sd.spx_tlo = log(d.spx_lam_lo > 0 ? d.spx_lam_lo : 1e-6);
    sd.spx_thi = log(d.spx_lam_hi > 0 ? d.spx_lam_hi : 1e6);
    std::vector<int> ml;
    double sum_lninv = 0.0;
    for (int i = 0; i < npix; ++i)
      if (d.mask[i]) {
        ml.push_back(i);
        sum_lninv -= log((double)d.sigma[i]);
      }
    sd.n_mask = (int)ml.size();
    sd.mask_list = upload(sh, ml.data(), ml.size());
    // C = H^T H (for ln det C; the kernels form its entries themselves) in band storage: its
    // entries lie within 2 gx of the diagonal, and so do its Cholesky factor's
    const int bw = 2 * gx;
    std::vector<double> Cb((size_t)ns * (bw + 1), 0.0), Lb((size_t)ns * (bw + 1), 0.0);
    auto band = [&](std::vector<double> &m, int r, int c) -> double & {
      return m[(size_t)r * (bw + 1) + (r - c)];
    };
    for (int i = 0; i < gy; ++i)
      for (int j = 0; j < gx; ++j) {
        const int p = i * gx + j;
        for (int dir = 0; dir < 2; ++dir) {
          // one row of H: -2 at p, +1 at the neighbours along the direction inside the grid
          int idx3[3] = {p, -1, -1};
          double h3[3] = {-2.0, 1.0, 1.0};
          if (dir == 0) {
            if (j > 0) idx3[1] = p - 1;
            if (j + 1 < gx) idx3[2] = p + 1;
          } else {
            if (i > 0) idx3[1] = p - gx;
            if (i + 1 < gy) idx3[2] = p + gx;
          }
          for (int u = 0; u < 3; ++u)
            for (int v = 0; v < 3; ++v)
              if (idx3[u] >= 0 && idx3[v] >= 0 && idx3[u] >= idx3[v])
                band(Cb, idx3[u], idx3[v]) += h3[u] * h3[v];
        }
      }
    double logdetC = 0.0;
    for (int jj = 0; jj < ns; ++jj) {
      double dsum = band(Cb, jj, jj);
      for (int k = std::max(0, jj - bw); k < jj; ++k) dsum -= band(Lb, jj, k) * band(Lb, jj, k);
      if (!(dsum > 0.0)) return fail(GLAD_EINVAL, "system %d: curvature matrix not positive definite", idx);
      const double ljj = sqrt(dsum);
      band(Lb, jj, jj) = ljj;
      logdetC += 2.0 * log(ljj);
      for (int ii = jj + 1; ii < std::min(ns, jj + bw + 1); ++ii) {
        double t = band(Cb, ii, jj);
        for (int k = std::max(0, ii - bw); k < jj; ++k) t -= band(Lb, ii, k) * band(Lb, jj, k);
        band(Lb, ii, jj) = t / ljj;
      }
    }
    sd.spx_const = 0.5 * logdetC - 0.5 * sd.n_mask * log(2.0 * PI_D) + sum_lninv;
  }
  sd.has_bh = d.has_bh;
  sd.bh_sigma = d.bh_sigma;
  sd.L_scale = d.L_scale;
  // distances: v^2 unit = c^2/(4 pi) D_dt,int / ((1+z_d) D_d) arcsec (independent of H0);
  // delay per arcsec^2 of Fermat potential = D_dt,int / c * arcsec^2 (proportional to 1/H0)
  {
    const double H = 70.0;
    const double cd = comoving(d.z_d, H, d.omega_m), cs = comoving(d.z_s, H, d.omega_m);
    const double D_d = cd / (1 + d.z_d), D_s = cs / (1 + d.z_s), D_ds = (cs - cd) / (1 + d.z_s);
    const double D_dt = (1 + d.z_d) * D_d * D_s / D_ds;
    const double D_int = (1.0 - d.kappa_ext) * D_dt;
    sd.distance_mode = d.distance_mode;
    // mode 1 scales these per sample: v^2 unit by D_dt,int / D_d, delays by D_dt,int [Mpc]
    sd.v2unit = d.distance_mode == 1 ? C_KMS * C_KMS / (4.0 * PI_D) / (1 + d.z_d) * ARCSEC
                                     : C_KMS * C_KMS / (4.0 * PI_D) * D_int / ((1 + d.z_d) * D_d) * ARCSEC;
    sd.dt_per_arcsec2_H0 = D_int * H * MPC_KM / C_KMS * ARCSEC * ARCSEC / DAY_S;
    sd.dt_per_arcsec2_Mpc = MPC_KM / C_KMS * ARCSEC * ARCSEC / DAY_S;
  }
  sd.n_img = d.n_img;
  sd.img_xy = upload(sh, d.img_xy, 2 * (size_t)d.n_img);
  sd.dt_obs = upload(sh, d.dt_obs, d.n_img - 1);
  sd.dt_sig = upload(sh, d.dt_sig, d.n_img - 1);
  sd.img_sig = d.img_sig ? upload(sh, d.img_sig, d.n_img) : nullptr;
  sd.atx = (sd.nsx + 15) / 16;
  sd.n_atile = sd.atx * ((sd.nsy + 15) / 16);
  sd.n_img_tiles = (npix + LENS_THREADS - 1) / LENS_THREADS;
  sd.n_sky_tiles = (sd.n_sub + JAM_TILE - 1) / JAM_TILE;
  sd.n_tab_blocks = (sd.n_ent + TAB_THREADS - 1) / TAB_THREADS;
  for (void *p : sh.allocs)
    if (!p) return fail(GLAD_ENOMEM, "system %d: device allocation failed", idx);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GLAD_ECUDA, "system %d: upload failed: %s", idx, cudaGetErrorString(e));
  return GLAD_OK;
}

void ws_free(Workspace &w) {
  for (void *p : w.allocs) cudaFree(p);
  w.allocs.clear();
  w.d = WsDev{};
  w.B = 0;
  w.prec = 0;
}

template <class T>
bool ws_alloc(Workspace &w, T *&p, size_t n) {
  void *d = nullptr;
  if (cudaMalloc(&d, std::max<size_t>(n, 1) * sizeof(T)) != cudaSuccess) return false;
  w.allocs.push_back(d);
  p = (T *)d;
  return true;
}

glad_status ws_ensure(glad_ctx *c, int B) {
  if (c->ws.B >= B && c->ws.prec >= c->tune.prec) return GLAD_OK;
  B = std::max(B, c->ws.B);
  cudaDeviceSynchronize();
  ws_free(c->ws);
  Workspace &w = c->ws;
  const size_t b = B;
  bool ok = ws_alloc(w, w.d.lp, b) && ws_alloc(w, w.d.dp, b) &&
            ws_alloc(w, w.d.nu0, b * c->max_light) && ws_alloc(w, w.d.c0, b * c->max_light) &&
            ws_alloc(w, w.d.Cj, b * c->max_mass_tot) && ws_alloc(w, w.d.e2, b * c->max_mass_tot) &&
            ws_alloc(w, w.d.I0f, b * c->max_light) && ws_alloc(w, w.d.tab, b * c->max_ent) &&
            ws_alloc(w, w.d.img, b * c->max_pix) && ws_alloc(w, w.d.binacc, b * c->max_bins * 2) &&
            ws_alloc(w, w.d.terms, b * 4) && ws_alloc(w, w.d.status, b) &&
            ws_alloc(w, w.d.wl_off, b + 1) && ws_alloc(w, w.d.wl_counter, 1) &&
            ws_alloc(w, w.d.evals, 2) && ws_alloc(w, w.d.sph_mt, b * c->max_smg) &&
            ws_alloc(w, w.d.sph_mrz, b * c->max_smg) && ws_alloc(w, w.d.sph_tr, b * c->max_light) &&
            ws_alloc(w, w.d.sgrid, b * c->max_sgrid);
  // the pixelated source's ray entries and arcs, for contexts with such systems
  if (ok && c->n_pix)
    ok = ws_alloc(w, w.d.pix_Li, b * c->max_lpix) && ws_alloc(w, w.d.pix_Lw, b * c->max_lpix) &&
         ws_alloc(w, w.d.pix_dres, b * c->max_pix);
  w.d.max_lpix = c->max_lpix;
  // the FP64 forward modes' arrays, only once such a mode has been asked for
  if (ok && c->tune.prec > 0)
    ok = ws_alloc(w, w.d.lp64, b) && ws_alloc(w, w.d.img64, b * c->max_pix) &&
         ws_alloc(w, w.d.tab64, b * c->max_ent) && ws_alloc(w, w.d.I0d, b * c->max_light);
  if (!ok) {
    ws_free(w);
    return fail(GLAD_ENOMEM, "workspace for B=%d does not fit on the device", B);
  }
  w.B = B;
  w.prec = c->tune.prec;
  return GLAD_OK;
}

// One sample's model image (image_out) or binned v_rms (vrms_out): the part of the forward
// sequence that output needs, on the caller's stream.
glad_status forward(glad_ctx *c, const int *sys_id, const double *theta, int B, cudaStream_t st,
                    float *image_out, float *vrms_out) {
  glad_status s = ws_ensure(c, B);
  if (s != GLAD_OK) return s;
  cudaError_t e;
  c->ws.d.neg_mode = c->tune.neg_mode;
  c->ws.d.prec = c->tune.prec;
  e = cudaMemsetAsync(c->ws.d.terms, 0, sizeof(double) * 4 * B, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ws.d.evals, 0, 2 * sizeof(unsigned long long), st);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(c->ws.d.binacc, 0, sizeof(double) * 2 * c->max_bins * (size_t)B, st);
  if (e == cudaSuccess) e = GLAD_PROF(c, st, KID_PREP, launch_prep(c, sys_id, theta, B, st));
  if (e == cudaSuccess && image_out)
    e = GLAD_PROF(c, st, KID_IMAGE_CONV, launch_lens(c, sys_id, B, image_out, st, nullptr));
  if (e == cudaSuccess && vrms_out) {
    e = launch_dyn_tables(c, sys_id, B, st);
    if (e == cudaSuccess) e = launch_dyn_sums(c, sys_id, B, st);
    if (e == cudaSuccess) e = GLAD_PROF(c, st, KID_KIN, launch_kin_finalize(c, sys_id, B, vrms_out, st));
  }
  if (e != cudaSuccess) return fail(GLAD_ECUDA, "launch failed: %s", cudaGetErrorString(e));
  return GLAD_OK;
}

// The full likelihood (and with `grad` its gradient): after k_prep the lensing branch
// (k_image, k_conv and, for the gradient, its adjoint) runs on the context's low-priority
// stream and the dynamics branch (table, JAM pair sum, v_rms, dynamics adjoint) on its
// high-priority stream; events fork both from the caller's stream and join them back before
// the combination.
glad_status full_path(glad_ctx *c, const int *sys_id, const double *theta, int B, cudaStream_t st,
                      double *logL, int *sample_status, double *terms, double *grad) {
  if (grad && c->n_pix)
    return fail(GLAD_EUNSUPPORTED, "glad_loglike_grad: no gradient for pixelated-source systems");
  glad_status s = ws_ensure(c, B);
  if (s == GLAD_OK && c->n_pix && pixsrc_ws_ensure(c, B) != cudaSuccess)
    s = fail(GLAD_ENOMEM, "pixelated-source workspace for B=%d does not fit on the device", B);
  if (s != GLAD_OK) return s;
  cudaError_t e;
  c->ws.d.neg_mode = c->tune.neg_mode;
  c->ws.d.prec = grad ? 0 : c->tune.prec;  // the gradient runs in the default precision
  e = cudaMemsetAsync(c->ws.d.terms, 0, sizeof(double) * 4 * B, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->ws.d.evals, 0, 2 * sizeof(unsigned long long), st);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(c->ws.d.binacc, 0, sizeof(double) * 2 * c->max_bins * (size_t)B, st);
  if (e == cudaSuccess && grad) e = grad_prepare(c, B, grad, st);
  if (e == cudaSuccess) e = GLAD_PROF(c, st, KID_PREP, launch_prep(c, sys_id, theta, B, st));
  // fork (profiling mode 2 runs both branches on the caller's stream, one after the other,
  // so that each kernel's event pair times it alone)
  const bool serial = c->prof == 2;
  cudaStream_t dy = serial ? st : c->dyn, side = serial ? st : c->side;
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_fork, st);
  if (e == cudaSuccess && !serial) e = cudaStreamWaitEvent(side, c->ev_fork, 0);
  if (e == cudaSuccess && !serial) e = cudaStreamWaitEvent(dy, c->ev_fork, 0);
  // lensing, low priority
  if (e == cudaSuccess)
    e = GLAD_PROF(c, side, KID_IMAGE_CONV,
                  launch_lens(c, sys_id, B, nullptr, side, grad ? grad_resid_buffer(c) : nullptr));
  if (e == cudaSuccess && grad) e = launch_grad_lens(c, sys_id, B, grad, side);
  // dynamics, high priority
  if (e == cudaSuccess) e = launch_dyn_tables(c, sys_id, B, dy);
  if (e == cudaSuccess) {
    if (!grad) {
      e = launch_dyn_sums(c, sys_id, B, dy);
    } else {
      // the pair sum with its derivative moments; the spherically aligned model's forward sums
      // (its adjoint recomputes what it needs)
      if (c->n_cyl) e = GLAD_PROF(c, dy, KID_GRAD_JAM_FWD, launch_jam_fg(c, sys_id, B, dy));
      if (e == cudaSuccess && c->n_sph)
        e = GLAD_PROF(c, dy, KID_SPH_LOS, launch_sph_los(c, sys_id, B, dy));
    }
  }
  if (e == cudaSuccess) e = GLAD_PROF(c, dy, KID_KIN, launch_kin_finalize(c, sys_id, B, nullptr, dy));
  if (e == cudaSuccess && grad) e = launch_grad_dyn(c, sys_id, theta, B, grad, dy);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_join_dyn, dy);
  // the pixelated source's evidence search last on the lensing stream: enqueueing it waits on
  // the device for the search to converge, by which time the dynamics are queued beside it
  if (e == cudaSuccess && c->n_pix && !grad)
    e = launch_pixsrc(c, sys_id, B, side, nullptr, nullptr, nullptr);
  if (e == cudaSuccess) e = cudaEventRecord(c->ev_join, side);
  // join
  if (e == cudaSuccess && !serial) e = cudaStreamWaitEvent(st, c->ev_join, 0);
  if (e == cudaSuccess && !serial) e = cudaStreamWaitEvent(st, c->ev_join_dyn, 0);
  if (e == cudaSuccess && grad) e = launch_grad_finish(c, B, grad, st);
  if (e == cudaSuccess)
    e = GLAD_PROF(c, st, KID_COMBINE, launch_combine(c, B, logL, sample_status, terms, st));
  if (e != cudaSuccess) return fail(GLAD_ECUDA, "launch failed: %s", cudaGetErrorString(e));
  return GLAD_OK;
}

const char *kKernelNames[KID_N] = {
    "k_prep", "k_table", "k_image+k_conv", "k_jam", "k_kin_finalize", "k_combine",
    "k_grad_lens", "k_jam_fwd_grad", "k_jam_adjoint", "k_grad_chain", "k_sph_coef+k_sph_grid",
    "k_sph_los", "k_sph_adjoint", "k_pix_operator", "k_pix_evidence"};

}  // namespace

cudaError_t launch_dyn_tables(glad_ctx *c, const int *sys_id, int B, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (c->n_cyl) e = GLAD_PROF(c, st, KID_TABLE, launch_table(c, sys_id, B, st));
  if (e == cudaSuccess && c->n_sph) e = GLAD_PROF(c, st, KID_SPH_GRID, launch_sph_grid(c, sys_id, B, st));
  return e;
}

cudaError_t launch_dyn_sums(glad_ctx *c, const int *sys_id, int B, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (c->n_cyl)
    e = GLAD_PROF(c, st, KID_JAM, c->ws.d.prec == 2 ? launch_jam64(c, sys_id, B, st)
                                                     : launch_jam(c, sys_id, B, st));
  if (e == cudaSuccess && c->n_sph) e = GLAD_PROF(c, st, KID_SPH_LOS, launch_sph_los(c, sys_id, B, st));
  return e;
}

// error reporting for entry points defined in other files
glad_status glad_set_error(glad_status s, const char *msg) { return fail(s, "%s", msg); }

cudaError_t prof_begin(glad_ctx *c, cudaStream_t st, cudaEvent_t *a) {
  *a = nullptr;
  if (!c->prof) return cudaSuccess;
  if (c->ev_pool.empty()) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    c->ev_pool.push_back(e);
  }
  *a = c->ev_pool.back();
  c->ev_pool.pop_back();
  return cudaEventRecord(*a, st);
}

cudaError_t prof_end(glad_ctx *c, cudaStream_t st, int id, cudaEvent_t a) {
  if (!c->prof || !a) return cudaSuccess;
  cudaEvent_t b;
  if (c->ev_pool.empty()) {
    cudaError_t r = cudaEventCreate(&b);
    if (r != cudaSuccess) return r;
  } else {
    b = c->ev_pool.back();
    c->ev_pool.pop_back();
  }
  c->recs.push_back({id, a, b});
  return cudaEventRecord(b, st);
}

extern "C" {

const char *glad_last_error(void) { return g_err.c_str(); }

glad_status glad_set_precision(glad_ctx *c, int mode) {
  if (!c || mode < 0 || mode > 2) return fail(GLAD_EINVAL, "glad_set_precision: mode %d", mode);
  c->tune.prec = mode;
  return GLAD_OK;
}

glad_status glad_set_negligible(glad_ctx *c, int mode) {
  if (!c || mode < 0 || mode > 2) return fail(GLAD_EINVAL, "glad_set_negligible: mode %d", mode);
  c->tune.neg_mode = mode;
  return GLAD_OK;
}

glad_status glad_jam_evaluations(glad_ctx *c, unsigned long long *count,
                                 unsigned long long *count_adjoint) {
  if (!c || !count) return fail(GLAD_EINVAL, "glad_jam_evaluations: bad arguments");
  *count = 0;
  if (count_adjoint) *count_adjoint = 0;
  if (!c->ws.d.evals) return GLAD_OK;
  unsigned long long n[2] = {0, 0};
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpy(n, c->ws.d.evals, sizeof(n), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail(GLAD_ECUDA, "glad_jam_evaluations: %s", cudaGetErrorString(e));
  *count = n[0];
  if (count_adjoint) *count_adjoint = n[1];
  return GLAD_OK;
}

int glad_profile(glad_ctx *c, int enable) {
  if (!c) return -1;
  if (enable < 0 || enable > 2) return -1;
  c->prof = enable;
  return 0;
}

int glad_kernel_times(glad_ctx *c, int n, double *ms, int *launches) {
  if (!c) return -1;
  if (n <= 0 || !ms || !launches) return KID_N;  // count query: keep the recorded pairs
  {
    for (auto &r : c->recs) {
      cudaEventSynchronize(r.b);
      float t = 0.0f;
      cudaEventElapsedTime(&t, r.a, r.b);
      if (r.id < n) {
        ms[r.id] += t;
        launches[r.id] += 1;
      }
    }
  }
  for (auto &r : c->recs) {
    c->ev_pool.push_back(r.a);
    c->ev_pool.push_back(r.b);
  }
  c->recs.clear();
  return KID_N;
}

const char *glad_kernel_name(int k) { return (k >= 0 && k < KID_N) ? kKernelNames[k] : ""; }

glad_status glad_create(const glad_system_desc *sys, int n_sys, glad_ctx **out) {
  g_err.clear();
  if (!sys || n_sys < 1 || !out) return fail(GLAD_EINVAL, "glad_create: bad arguments");
  *out = nullptr;
  for (int i = 0; i < n_sys; ++i) {
    glad_status s = validate(sys[i], i);
    if (s != GLAD_OK) return s;
  }
  glad_ctx *c = new glad_ctx();
  c->n_sys = n_sys;
  c->sys.resize(n_sys);
  c->h_sysdev.resize(n_sys);
  for (int i = 0; i < n_sys; ++i) {
    glad_status s = build_system(i, sys[i], c->sys[i], c->h_sysdev[i]);
    if (s != GLAD_OK) {
      glad_destroy(c);
      return s;
    }
    const SysDev &d = c->h_sysdev[i];
    c->max_light = std::max(c->max_light, d.n_light);
    c->max_mass_tot = std::max(c->max_mass_tot, d.n_mass_tot);
    c->max_ent = std::max(c->max_ent, d.n_ent);
    c->max_pix = std::max(c->max_pix, d.npix);
    c->max_bins = std::max(c->max_bins, d.n_bins);
    c->max_sub = std::max(c->max_sub, d.n_sub);
    c->max_img_tiles = std::max(c->max_img_tiles, d.n_img_tiles);
    c->max_sky_tiles = std::max(c->max_sky_tiles, d.n_sky_tiles);
    c->max_tab_blocks = std::max(c->max_tab_blocks, d.n_tab_blocks);
    c->max_apts = std::max(c->max_apts, d.n_atile * 256);
    if (d.jam_align == 1) {
      ++c->n_sph;
      c->max_sgrid = std::max(c->max_sgrid, d.sph_nr * d.sph_nw);
      c->max_smg = std::max(c->max_smg, d.n_mass_tot * d.n_gl);
    } else {
      ++c->n_cyl;
    }
    if (d.src_pix) {
      ++c->n_pix;
      c->max_ns = std::max(c->max_ns, d.spx_ns);
      c->max_nd = std::max(c->max_nd, d.n_mask);
      c->max_lpix = std::max(c->max_lpix, d.npix * 4 * d.ss * d.ss);
    }
  }
  if (cudaMalloc(&c->d_sys, sizeof(SysDev) * n_sys) != cudaSuccess ||
      cudaMemcpy(c->d_sys, c->h_sysdev.data(), sizeof(SysDev) * n_sys, cudaMemcpyHostToDevice) !=
          cudaSuccess ||
      cudaMalloc(&c->d_one_sys, sizeof(int) * n_sys) != cudaSuccess) {
    glad_destroy(c);
    return fail(GLAD_ENOMEM, "glad_create: device allocation failed");
  }
  std::vector<int> ids(n_sys);
  for (int i = 0; i < n_sys; ++i) ids[i] = i;
  cudaMemcpy(c->d_one_sys, ids.data(), sizeof(int) * n_sys, cudaMemcpyHostToDevice);
  set_conv_smem_limit();
  set_grad_smem_limit();
  if (set_sph_smem_limit() != cudaSuccess || set_sph_grad_smem_limit() != cudaSuccess) {
    glad_destroy(c);
    return fail(GLAD_ECUDA, "glad_create: shared-memory limits of the spherical kernels not set");
  }
  int prio_lo = 0, prio_hi = 0;
  cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  if (cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
      cudaStreamCreateWithPriority(&c->dyn, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&c->ev_join_dyn, cudaEventDisableTiming) != cudaSuccess) {
    glad_destroy(c);
    return fail(GLAD_ECUDA, "glad_create: stream or event creation failed");
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    glad_destroy(c);
    return fail(GLAD_ECUDA, "glad_create: %s", cudaGetErrorString(e));
  }
  *out = c;
  return GLAD_OK;
}

void glad_destroy(glad_ctx *c) {
  if (!c) return;
  cudaDeviceSynchronize();
  ws_free(c->ws);
  grad_ws_free(c);
  pixsrc_ws_free(c);
  for (auto &s : c->sys)
    for (void *p : s.allocs)
      if (p) cudaFree(p);
  cudaFree(c->d_sys);
  cudaFree(c->d_one_sys);
  for (auto &r : c->recs) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (auto e : c->ev_pool) cudaEventDestroy(e);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->ev_join_dyn) cudaEventDestroy(c->ev_join_dyn);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->dyn) cudaStreamDestroy(c->dyn);
  delete c;
}

glad_status glad_loglike(glad_ctx *c, const int *sys_id, const double *theta, int B, double *logL,
                         int *sample_status, double *terms, void *stream) {
  g_err.clear();
  if (!c || !sys_id || !theta || !logL || !sample_status || B < 1)
    return fail(GLAD_EINVAL, "glad_loglike: bad arguments");
  return full_path(c, sys_id, theta, B, (cudaStream_t)stream, logL, sample_status, terms, nullptr);
}

glad_status glad_loglike_grad(glad_ctx *c, const int *sys_id, const double *theta, int B,
                              double *logL, double *grad, int *sample_status, double *terms,
                              void *stream) {
  g_err.clear();
  if (!c || !sys_id || !theta || !logL || !grad || !sample_status || B < 1)
    return fail(GLAD_EINVAL, "glad_loglike_grad: bad arguments");
  if (grad_ws_ensure(c, B) != cudaSuccess)
    return fail(GLAD_ENOMEM, "gradient workspace for B=%d does not fit", B);
  return full_path(c, sys_id, theta, B, (cudaStream_t)stream, logL, sample_status, terms, grad);
}

glad_status glad_model_image(glad_ctx *c, int sys, const double *theta, float *image,
                             void *stream) {
  g_err.clear();
  if (!c || !theta || !image || sys < 0 || sys >= c->n_sys)
    return fail(GLAD_EINVAL, "glad_model_image: bad arguments");
  if (c->h_sysdev[sys].src_pix)
    return fail(GLAD_EUNSUPPORTED, "glad_model_image: system %d has a pixelated source", sys);
  return forward(c, c->d_one_sys + sys, theta, 1, (cudaStream_t)stream, image, nullptr);
}

glad_status glad_pixsrc(glad_ctx *c, const int *sys_id, const double *theta, int B, double *lam,
                        double *lnP, double *s_out, void *stream) {
  g_err.clear();
  if (!c || !sys_id || !theta || B < 1) return fail(GLAD_EINVAL, "glad_pixsrc: bad arguments");
  if (!c->n_pix) return fail(GLAD_EINVAL, "glad_pixsrc: no system with a pixelated source");
  cudaStream_t st = (cudaStream_t)stream;
  glad_status s = ws_ensure(c, B);
  if (s != GLAD_OK) return s;
  if (pixsrc_ws_ensure(c, B) != cudaSuccess)
    return fail(GLAD_ENOMEM, "pixelated-source workspace for B=%d does not fit on the device", B);
  c->ws.d.neg_mode = c->tune.neg_mode;
  c->ws.d.prec = c->tune.prec;
  cudaError_t e = cudaMemsetAsync(c->ws.d.terms, 0, sizeof(double) * 4 * B, st);
  if (e == cudaSuccess) e = GLAD_PROF(c, st, KID_PREP, launch_prep(c, sys_id, theta, B, st));
  if (e == cudaSuccess) e = GLAD_PROF(c, st, KID_IMAGE_CONV, launch_lens(c, sys_id, B, nullptr, st, nullptr));
  if (e == cudaSuccess) e = launch_pixsrc(c, sys_id, B, st, lam, lnP, s_out);
  if (e != cudaSuccess) return fail(GLAD_ECUDA, "launch failed: %s", cudaGetErrorString(e));
  return GLAD_OK;
}

unsigned long long glad_pix_factorizations(glad_ctx *c) { return c ? pixsrc_factorizations(c) : 0; }

unsigned long long glad_pix_launches(glad_ctx *c) { return c ? pixsrc_launches(c) : 0; }

glad_status glad_set_pix_path(glad_ctx *c, int mode) {
  if (!c || mode < 0 || mode > 2) return fail(GLAD_EINVAL, "glad_set_pix_path: mode %d", mode);
  c->tune.pix_path = mode;
  return GLAD_OK;
}

glad_status glad_vrms(glad_ctx *c, int sys, const double *theta, float *vrms, void *stream) {
  g_err.clear();
  if (!c || !theta || !vrms || sys < 0 || sys >= c->n_sys)
    return fail(GLAD_EINVAL, "glad_vrms: bad arguments");
  return forward(c, c->d_one_sys + sys, theta, 1, (cudaStream_t)stream, nullptr, vrms);
}

}  // extern "C"
