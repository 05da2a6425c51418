// Internal declarations of libglad: device-side system layout, per-sample
// workspace, small math helpers and the kernel launchers of each .cu file.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/glad.h"

#define GLAD_MAX_TM 64        // EPL series terms kept in the per-sample block
#define GLAD_MAX_BINS 1024    // kinematic bins per system (shared-memory bin accumulators)
#define GLAD_MAX_LIGHT 128    // tracer Gaussians per system
#define GLAD_MAX_MASS 127     // mass Gaussians per system (without the black hole)
#define GLAD_MAX_PSF 63       // imaging PSF side
#define GLAD_MAX_P 20         // Euler order
#define GLAD_MAX_IMG 8        // quasar images
#define GLAD_SPH_MAX_GRID 4096  // polar grid points of the spherically aligned model
#define GLAD_SPH_MAX_MG 4096    // (mass Gaussian, u node) pairs of the spherically aligned model
#define GLAD_N_CSE 44           // cored steep ellipsoids of the composite class's halo
#define SPH_DEFAULT_NR 128      // default polar grid and line-of-sight rule of that model
#define SPH_DEFAULT_NW 8
#define SPH_DEFAULT_NLOS 32
#define GLAD_MAX_SRCPIX 4624    // source pixels of a pixelated-source grid (68 x 68)
#define SPX_DEFAULT_ITERS 40    // evidence evaluations of the regularisation search
#define SPX_MAX_ITERS 200       // the largest spx_iters taken

// ---------------------------------------------------------------------------
// device-resident description of one system (all pointers are device memory)
// ---------------------------------------------------------------------------
struct SysDev {
  // imaging
  int nx, ny, ss, npix;
  float pix;
  const float *data;     // [npix]
  const double *wgt;     // [npix] mask / sigma
  int psf_k;
  const float *psf;      // [psf_k^2]
  int psf_km;            // padded side of psf_t (11, 21 or 31; 0 above 31)
  const float *psf_t;    // [psf_km * CONV_PT(psf_km)]: psf centred in psf_km^2 zeros,
                         // transposed (column c of the PSF is row c here), rows padded to 4
  float src_q, src_cphi, src_sphi;
  double pix64, src_q64, src_cphi64, src_sphi64;  // the same in FP64 (FP64 lensing modes)
  int n_lcomp;           // lens-light components (1 + n_ll2)
  const double *lcomp;   // [n_lcomp*4]: I_e, R_e, n, q (row 0: I_e, R_e from theta)
  int n_sis;
  const double *sis;     // [n_sis*3]
  double r_soft;
  // kinematics: sub-sampled sky grid and the binning-after-PSF operator (CSR by sub-sample)
  int nsx, nsy, n_sub;
  float dsub;
  double dsub64;         // the same in FP64 (the FP64 pair sum)
  const int *w_off;      // [n_sub+1]
  const int *w_bin;      // [nnz]
  const float *w_val;    // [nnz]
  int n_bins;
  const float *v_obs, *v_sig;
  // mass class: 0 EPL, 1 composite (Chameleon baryons x Upsilon, elliptical NFW halo, black hole)
  int mass_class;
  int n_halo;                              // composite: halo Gaussians (after the nL light copies)
  const double *cse_a, *cse_s;             // composite: the halo's CSEs, units of r_s [GLAD_N_CSE]
  // MGE: mass Gaussians are ordered [galaxy n_mass][sheet n_sheet][black hole]; the composite
  // class's galaxy part is [Upsilon x the n_light tracer Gaussians][halo n_halo]
  int n_mass, n_mass_tot, n_light;
  int n_sheet;                             // round Gaussians of the internal sheet (0: none)
  const double *sheet_A1;                  // [n_sheet] their amplitudes at 1 - lambda_int = 1
  const int *lcomp_of;   // [n_light]
  const double *sig_mass, *sig_light;      // [n_mass_tot], [n_light]
  const double *mw_mass, *mw_light;        // w_n * dln(sigma) / sqrt(2 pi)
  const double *qp_light;                  // [n_light]
  int mge_P;
  const double *eta;                        // [2P+1]
  const double2 *chi;                       // [2P+1]
  // JAM pair table geometry
  int n_gl, n_ent;                          // n_ent = n_light * n_mass_tot * n_gl
  const double *gl_u, *gl_wu;               // [n_ent]: u node, weight * du/dt
  const double *gl_a, *gl_p, *gl_u2;        // [n_ent]: u^2/(2 s_j^2), 1/(2 s_k^2) + a, u^2
  const float *sb_cx, *sb_cy;               // [n_light]: log2(e)/(2 s^2), log2(e)/(2 s^2 q'^2)
  int has_bh;
  double bh_sigma, L_scale;
  double v2unit;                            // km^2/s^2 per (kappa * arcsec); distance mode 1:
                                            // per (kappa * arcsec) and unit D_dt,int / D_d
  double dt_per_arcsec2_H0;                 // days per arcsec^2 times H0 (distance mode 0)
  double dt_per_arcsec2_Mpc;                // days per arcsec^2 per Mpc of D_dt,int (mode 1)
  int distance_mode;                        // 0: H0 = theta[19]; 1: theta[21], theta[22]
  // internal mass sheet: 0 none, 1 dPIE (core sh_rc, truncation sh_rt), 2 ideal (uniform)
  int sheet;
  double sh_rc, sh_rt;
  int n_img;
  const double *img_xy, *dt_obs, *dt_sig;
  const double *img_sig;                    // [n_img] or null: no image-position term
  // tile counts
  int n_img_tiles, n_sky_tiles, n_tab_blocks;
  // gradient adjoint: table entries in ascending order of their x exponent p (fixed per
  // system) and the sky grid in 16 x 16 point tiles (atx across, n_atile in all)
  const int *adj_perm;                      // [n_ent]
  int atx, n_atile;
  // spherically aligned JAM (jam_align 1): polar grid of sph_nr radii log-spaced on
  // [sph_r_lo, sph_r_end] (ln r = sph_lr0 + a sph_dlr) x sph_nw values of sin^2 theta,
  // sph_nlos line-of-sight nodes, and the u rule of each mass Gaussian
  int jam_align, sph_nr, sph_nw, sph_nlos;
  double sph_r_lo, sph_r_end, sph_lr0, sph_dlr;
  const double *sph_u, *sph_wu;             // [n_mass_tot * n_gl]
  // pixelated source (src_pix 1, Sect. 3.1.1): spx_nx x spx_ny pixels of size spx_dx x spx_dy
  // from (spx_x0, spx_y0) on the source plane; the fit runs over the n_mask pixels listed in
  // mask_list; the curvature regularisation C = H^T H is formed where it is needed; the evidence's
  // lambda-free constant spx_const = ln det C / 2 - (N_d / 2) ln 2 pi + sum ln(1 / sigma);
  // the search over ln lambda in [spx_tlo, spx_thi] takes at most spx_iters evaluations
  int src_pix, spx_nx, spx_ny, spx_ns, n_mask, spx_iters;
  float spx_x0, spx_y0, spx_idx, spx_idy;   // origin and inverse pixel sizes
  const int *mask_list;                     // [n_mask] pixel indices, ascending
  double spx_const, spx_tlo, spx_thi;
};

// per-sample lensing parameters, written by the prep kernel: FP32 (LensP) for the default
// precision and the gradient kernels, FP64 (LensPT<double>) for the FP64 lensing modes
template <class T>
struct LensPT {
  T xc, yc, cphi, sphi;
  T q, t, pref, pad0;        // alpha' = pref * R^(1-t) * sum Omega_n
  T g1, g2;                  // external shear
  int nterms, valid;
  T src_Ie, src_Rei, src_ninv, src_bn, src_x, src_y;
  T ll_Ie[4], ll_Rei[4], ll_ninv[4], ll_bn[4], ll_qi2[4];
  T rho[GLAD_MAX_TM];        // Omega_n = rho_n e^{2 i ph} Omega_{n-1}
  // derivatives used by the gradient kernels
  T drho_t[GLAD_MAX_TM], drho_q[GLAD_MAX_TM];  // d rho_n / d t, d rho_n / d q
  T pref_d[3];               // d pref / d (theta_E, t, q)
  T gext, c2pe, s2pe;        // shear strength and cos/sin(2 phi_ext)
  T src_bnp;                 // d b_n / d n of the source
  // internal mass sheet: the galaxy's deflection is scaled by lam and the sheet's added,
  // alpha_sheet = (1 - lam) u(R^2) (x - x_c, y - y_c) with u = 1 (ideal) or, for the dPIE,
  // u = 2 rc rt [1 + (rc + rt)/(Q_c + Q_t)] / ((rc + Q_c)(rt + Q_t)), Q = sqrt(R^2 + r^2)
  // (the difference of the two cored terms written without cancellation)
  T lam;
  int sheet;
  T sh_rc2, sh_rt2, sh_rc, sh_rt;
  // composite class (mclass 1): Chameleon c of the lens light is li_A[c] [(m^2 + sc^2)^-1/2 -
  // (m^2 + st^2)^-1/2], m^2 = x'^2 + y'^2/q^2, li_A = I0/(1+q), s = 2w/(1+q); its baryonic
  // deflection is that of two softened isothermal ellipsoids of amplitude ch_A = Upsilon L_scale
  // li_A (b = 2 q ch_A), e = sqrt(1 - q^2); the halo's CSE i has amplitude cse_amp = kappa_s a_i
  // r_s^3 and core cse_sc = s_i r_s (axis ratio h_q); the black hole is a round Gaussian of mass
  // bh_M (convergence x arcsec^2) and 2 sigma^2 = bh_2s2
  // (for the gradient: ups = Upsilon L_scale, h_ks = kappa_s, h_rs = r_s, cse_a3 = a_i r_s^3,
  // bh_dM = d bh_M / d(theta 13, 14, 17, 18))
  int mclass;
  T li_A[4], ch_A[4], ch_sc[4], ch_st[4], ch_q[4], ch_e[4];
  T ups, h_ks, h_rs, h_q, h_e2;
  T bh_M, bh_2s2, bh_dM[4];
  T cse_amp[GLAD_N_CSE], cse_sc[GLAD_N_CSE], cse_a3[GLAD_N_CSE];
};
typedef LensPT<float> LensP;

// per-sample dynamics scalars (FP64)
struct DynP {
  double s2, c2, b;      // sin^2 i, cos^2 i, 1/(1-beta)
  double xc, yc, cphi, sphi;
};

// ---------------------------------------------------------------------------
// host-side context
// ---------------------------------------------------------------------------
struct SysHost {
  glad_system_desc d;      // scalars (pointer fields are not kept)
  int n_mass_tot, n_light, n_ent, n_sub, npix;
  std::vector<void *> allocs;
};

struct WsDev {
  LensP *lp;
  DynP *dp;
  double *nu0, *c0, *Cj, *e2;  // [B*max_light] / [B*max_mass_tot]
  float *I0f;                  // [B*max_light]
  float4 *tab;                 // [B*max_ent]
  float *img;                  // [B*max_pix]
  double *binacc;              // [B*max_bins*2]
  double *terms;               // [B*4]: chi2_pix, chi2_dyn, chi2_tmd, chi2_img
  int *status;                 // [B]
  int *wl_off;                 // [B+1] persistent JAM work list (first item of each sample)
  int *wl_counter;             // [1]   next work item
  unsigned long long *evals;   // [2]   JAM integrand evaluations executed: pair sum (forward or
                               //       derivative pass), table adjoint (null: not counted)
  float4 *sph_mt;              // [B*max_smg] spherical model: (mass Gaussian, u node) coefficients
  float *sph_mrz;              // [B*max_smg] their F_R - F_z weights
  float4 *sph_tr;              // [B*max_light] tracer Gaussians (nu0, exponent coefficients, dnu factor)
  float2 *sgrid;               // [B*max_sgrid] (v_r^2, d) on the polar grid
  int neg_mode;                // negligible-term skipping in the forward JAM pass: 0 off,
                               // 1 on, 2 on with every tile's check failed (summed again)
  // FP64 forward modes (glad_set_precision; null in the default precision): the FP64 lensing
  // block, unblurred image, pair-form table (ax, ay, Q0, Q1) and projected tracer amplitudes
  LensPT<double> *lp64;        // [B]
  double *img64;               // [B*max_pix]
  double4_16a *tab64;          // [B*max_ent]
  double *I0d;                 // [B*max_light]
  int prec;                    // 0 default, 1 FP64 lensing, 2 FP64 lensing and pair sum
  // pixelated source (null without such systems): each image pixel's 4 ss^2 bilinear source
  // entries (index, weight / ss^2) written by k_image, and the arcs data - B (lens light)
  // written by the PSF kernels
  int *pix_Li;                 // [B*max_lpix]
  float *pix_Lw;               // [B*max_lpix]
  float *pix_dres;             // [B*max_pix]
  int max_lpix;                // npix * 4 ss^2 of the largest pixelated-source system
};

struct Workspace {
  int B = 0;
  int prec = 0;  // precision mode whose FP64 arrays are allocated (0: none)
  WsDev d{};
  std::vector<void *> allocs;
};

struct GradWs;  // gradient workspace (k_grad.cu)
struct PixWs;   // pixelated-source workspace (k_pixsrc.cu)

struct glad_ctx {
  int n_sys = 0;
  std::vector<SysHost> sys;
  SysDev *d_sys = nullptr;       // [n_sys]
  std::vector<SysDev> h_sysdev;  // host copy of the device descriptors
  int max_light = 0, max_mass_tot = 0, max_ent = 0, max_pix = 0, max_bins = 0, max_sub = 0;
  int max_apts = 0;  // largest 16 x 16-tiled sky grid (points, padded)
  int max_img_tiles = 0, max_sky_tiles = 0, max_tab_blocks = 0;
  int n_cyl = 0, n_sph = 0;        // systems with the cylindrically / spherically aligned model
  int max_sgrid = 0, max_smg = 0;  // largest polar grid and (mass Gaussian, u node) count
  int n_pix = 0;                    // systems with a pixelated source
  int max_ns = 0, max_nd = 0;       // their largest source grid and mask
  int max_lpix = 0;                 // their largest npix * 4 ss^2 (bilinear ray entries)
  Workspace ws;
  PixWs *pws = nullptr;             // pixelated-source workspace (k_pixsrc.cu)
  GradWs *gws = nullptr;
  // launch shapes chosen by glad_autotune (defaults until it runs)
  struct Tune {
    int prec = 0;         // precision mode of the forward pass (glad_set_precision)
    int neg_mode = 1;     // negligible-term skipping of the forward JAM pass (see WsDev)
    int jam_pts = 8;      // sky points per thread in the JAM pair-sum kernels
    int jam_minb = 4;     // minimum resident CTAs per SM requested from the register allocator
    int jam_unroll = 2;   // unroll of the table-entry loop
    int jam_persistent = 0;  // 1: one persistent launch over a (sample, tile) work list
    int jam_form = 0;        // form of the pair sum (k_jam.cu): 0 .. 3
    int adj_ept = 4;      // table entries per thread in the JAM adjoint
    int pix_path = 0;     // evidence evaluation (k_pixsrc.cu): 0 by batch size, 1 one CTA per
                          // sample, 2 multi-launch
  } tune;
  int *d_one_sys = nullptr;      // scratch sys id for single-sample calls
  // after k_prep the dynamics branch runs on a high-priority stream and the lensing branch
  // on a low-priority one, both forked from and joined back into the caller's stream by
  // events (capturable into a CUDA graph): the lensing work fills the dynamics kernels'
  // tails without delaying the next kernel of the dynamics chain
  cudaStream_t side = nullptr, dyn = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_join_dyn = nullptr;
  // kernel timing (glad_profile)
  int prof = 0;
  struct Rec {
    int id;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
  std::vector<cudaEvent_t> ev_pool;
};

// kernel ids for glad_kernel_times
enum {
  KID_PREP = 0, KID_TABLE, KID_IMAGE_CONV, KID_JAM, KID_KIN, KID_COMBINE,
  KID_GRAD_LENS, KID_GRAD_JAM_FWD, KID_GRAD_JAM_ADJ, KID_GRAD_CHAIN, KID_SPH_GRID, KID_SPH_LOS,
  KID_GRAD_SPH, KID_PIX_OP, KID_PIX_EV, KID_N
};

// record an event pair around `call` when profiling is on
cudaError_t prof_begin(glad_ctx *c, cudaStream_t st, cudaEvent_t *a);
cudaError_t prof_end(glad_ctx *c, cudaStream_t st, int id, cudaEvent_t a);
#define GLAD_PROF(c, st, id, call)               \
  [&]() -> cudaError_t {                         \
    cudaEvent_t _a = nullptr;                    \
    cudaError_t _e = prof_begin((c), (st), &_a); \
    if (_e != cudaSuccess) return _e;            \
    _e = (call);                                 \
    if (_e != cudaSuccess) return _e;            \
    return prof_end((c), (st), (id), _a);        \
  }()

// ---------------------------------------------------------------------------
// launchers (one per kernel file)
// ---------------------------------------------------------------------------
cudaError_t launch_prep(glad_ctx *c, const int *sys_id, const double *theta, int B,
                        cudaStream_t st);
cudaError_t launch_table(glad_ctx *c, const int *sys_id, int B, cudaStream_t st);
cudaError_t launch_lens(glad_ctx *c, const int *sys_id, int B, float *image_out,
                        cudaStream_t st, float *resid_out = nullptr);
cudaError_t launch_jam(glad_ctx *c, const int *sys_id, int B, cudaStream_t st);
cudaError_t launch_jam64(glad_ctx *c, const int *sys_id, int B, cudaStream_t st);
// gradient pieces (k_grad.cu): zeroing, lensing adjoint, dynamics adjoint + chain, final fix-up
cudaError_t grad_prepare(glad_ctx *c, int B, double *grad, cudaStream_t st);
cudaError_t launch_grad_lens(glad_ctx *c, const int *sys_id, int B, double *grad, cudaStream_t st);
cudaError_t launch_grad_dyn(glad_ctx *c, const int *sys_id, const double *theta, int B,
                            double *grad, cudaStream_t st);
cudaError_t launch_grad_finish(glad_ctx *c, int B, double *grad, cudaStream_t st);
cudaError_t launch_kin_finalize(glad_ctx *c, const int *sys_id, int B, float *vrms_out,
                                cudaStream_t st);
cudaError_t launch_combine(glad_ctx *c, int B, double *logL, int *status, double *terms,
                           cudaStream_t st);
// spherically aligned model (k_sph.cu): coefficients + polar grid, then the line-of-sight sums
cudaError_t launch_sph_grid(glad_ctx *c, const int *sys_id, int B, cudaStream_t st);
cudaError_t launch_sph_los(glad_ctx *c, const int *sys_id, int B, cudaStream_t st);
cudaError_t set_sph_smem_limit();
// its adjoint (k_sph_grad.cu): line-of-sight and grid adjoints, carried to the JAM inputs
cudaError_t launch_grad_sph(glad_ctx *c, const int *sys_id, int B, double *grad, cudaStream_t st);
cudaError_t set_sph_grad_smem_limit();
// the halo's CSE decomposition (glad_cse.cu): amplitudes and cores in units of r_s, fitted once
void cse_table(const double **a, const double **s);
// the dynamics sum of either model for the systems of the context (glad_host.cu): the
// table/grid stage and the sky-point stage, each recorded under its kernel id
cudaError_t launch_dyn_tables(glad_ctx *c, const int *sys_id, int B, cudaStream_t st);
cudaError_t launch_dyn_sums(glad_ctx *c, const int *sys_id, int B, cudaStream_t st);
void set_conv_smem_limit();
// pixelated source (k_pixsrc.cu): response rows, Gram matrix, then the evidence search over
// the regularisation; lam/lnP/s outputs (any may be null) for glad_pixsrc
cudaError_t launch_pixsrc(glad_ctx *c, const int *sys_id, int B, cudaStream_t st,
                          double *lam_out, double *lnP_out, double *s_out);
cudaError_t pixsrc_ws_ensure(glad_ctx *c, int B);
void pixsrc_ws_free(glad_ctx *c);
unsigned long long pixsrc_factorizations(glad_ctx *c);
unsigned long long pixsrc_launches(glad_ctx *c);
bool pixsrc_multi_launch(glad_ctx *c, int B);
bool jam_shape_supported(int pts, int minb, int unr, int form);
int jam_shape_list(int (*out)[4], int cap);

// tile shapes (shared by launchers and the workspace sizing)
#define JAM_THREADS 256
#define JAM_PTS 4
#define JAM_TILE (JAM_THREADS * JAM_PTS)
#define JAM_CHUNK 512
#define LENS_THREADS 256
#define TAB_THREADS 256
#define CONV_TX 32
#define CONV_TY 8
#define CONV_PT(km) (((km) + 3) / 4 * 4)  // row stride of the transposed padded PSF
#define CONV_R 8                          // output rows per thread in the blocked convolution

// ---------------------------------------------------------------------------
// math helpers usable from host and device
// ---------------------------------------------------------------------------
#define LOG2E_D 1.4426950408889634
#define SQRT2PI_D 2.5066282746310002
#define PI_D 3.141592653589793

__host__ __device__ inline double sersic_bn_d(double n) {
  // Ciotti & Bertin (1999) asymptotic series, 4th order in 1/n
  double i1 = 1.0 / n;
  return 2.0 * n - 1.0 / 3.0 + i1 * (4.0 / 405.0 + i1 * (46.0 / 25515.0 +
         i1 * (131.0 / 1148175.0 - i1 * (2194697.0 / 30690717750.0))));
}
