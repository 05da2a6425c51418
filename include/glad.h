/*
 * glad.h -- C ABI of libglad.so: the batched joint lensing + dynamics
 * log-likelihood of GLaD (arXiv:2504.01302) and its gradient, on one NVIDIA
 * B300 (sm_103a).
 *
 * Conventions shared by every entry point
 *  - Pointers marked [host] are read during the call and may be freed after it.
 *    Pointers marked [dev] are CUDA device memory owned by the caller; the library
 *    never frees them.  A context owns every array it stages on the device.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls enqueue work on it and return without synchronising; the return code
 *    reports argument and launch errors only.  Kernel-time problems of one sample
 *    (invalid parameters) are NOT errors: that sample gets logL = -inf,
 *    gradient 0 and a non-zero status.
 *  - One context is not thread-safe: serialise calls that use it.
 *  - On a non-zero return, glad_last_error() holds a message (thread-local).
 *
 * Parameter vector theta (23 float64 per sample, angles in radians):
 *   0 theta_E  1 gamma'  2 q  3 phi (PA, counter-clockwise from +x)  4 x_c  5 y_c
 *   6 gamma_ext  7 phi_ext  8 I_e,src  9 R_e,src  10 n_src  11 x_src  12 y_src
 *   13 I_e,ll  14 R_e,ll  15 inclination i  16 beta (= beta_z)  17 Upsilon (M/L)
 *   18 f_BH = M_BH/M_*  19 H0 [km/s/Mpc]  20 lambda_int (internal mass sheet)
 *   21 D_d [Mpc]  22 D_dt,int [Mpc]
 * An entry a system does not use is ignored (it may hold anything, NaN included) and its
 * gradient is 0: lambda_int without a sheet; H0 in distance mode 1; D_d and D_dt,int in
 * distance mode 0.
 * In the composite mass class (mass_class 1) five entries take that class's parameters:
 *   0 kappa_s (halo convergence scale, >= 0)  1 r_s (halo scale radius, arcsec)  2 q of the halo
 *   13 I0 and 14 w_t (arcsec) of the first Chameleon of the lens light; 17 is Upsilon_*.
 */
#ifndef GLAD_H
#define GLAD_H

#ifdef __cplusplus
extern "C" {
#endif

#define GLAD_NTHETA 23

typedef enum {
  GLAD_OK = 0,
  GLAD_EINVAL = 1,      /* bad argument or system descriptor */
  GLAD_ENOMEM = 2,      /* device allocation failed */
  GLAD_ECUDA = 3,       /* a CUDA call or kernel launch failed */
  GLAD_ETIMEOUT = 4,    /* a bounded device-side wait gave up */
  GLAD_EUNSUPPORTED = 5 /* size outside what the kernels support */
} glad_status;

/* Per-sample status written by the likelihood calls. */
enum {
  GLAD_SAMPLE_OK = 0,
  GLAD_SAMPLE_DOMAIN = 1,     /* parameter outside its domain (q not in (0,1], gamma' not in (1,3), ...) */
  GLAD_SAMPLE_DEPROJ = 2,     /* cos^2 i >= q'^2 of some Gaussian: no oblate deprojection (App. A) */
  GLAD_SAMPLE_NEGDENS = 3,    /* deprojected density <= 0 at a probe radius (Sect. 3.3) */
  GLAD_SAMPLE_NONFINITE = 4   /* a chi^2 term came out NaN or infinite */
};

/*
 * One mock or observed system, read at glad_create (all pointers [host]).
 *
 * Imaging (Sect. 3.1.1, Table 1): an ny x nx image (row-major, pixel (i,j) centred at
 * x = (j-(nx-1)/2) pix, y = (i-(ny-1)/2) pix arcsec), each pixel split into ss x ss
 * sub-pixels that are ray-shot and averaged, then blurred by the psf_k x psf_k PSF
 * (odd size, unit sum, discrete convolution, zero outside the image).  chi^2_pix runs
 * over mask != 0 (Eq. chi2 of lens_light).
 *
 * Dynamics (Sect. 2.4, Eqs. binned, Vrms, chi2_dyn): a ky x kx spaxel grid of kpix
 * arcsec centred on the origin, each spaxel split into kss x kss sub-samples at which
 * the JAM moment is evaluated; kpsf (kpsf_k^2, odd, unit sum) blurs the two sub-sample
 * maps; bins[ky*kx] gives each spaxel's bin (0..n_bins-1, -1 = unused).  Bins must hold
 * only spaxels whose sub-samples lie at least (kpsf_k-1)/2 sub-samples from the edge.
 *
 * MGE (Sect. 3.2): the App. C convergence is expanded into n_mge_mass Gaussians
 * log-spaced on [mass_rmin, mass_rmax]; lens-light component c into n_mge_light[c]
 * Gaussians on [light_rmin, light_rmax]; Euler order mge_P.  has_bh adds a spherical
 * black-hole Gaussian of dispersion bh_sigma and mass f_BH * Upsilon * L_tot * L_scale
 * (L_tot = total light of the tracer MGE).  n_gl: Gauss-Legendre order of the JAM u
 * integral.
 *
 * Delays (Eqs. fermat potential, chi2_tmd): n_img observed image positions
 * (img_xy[n_img*2]) and n_img-1 delays relative to image 0 (dt_obs, dt_sig, days).
 * Image positions (Eq. chi2_img): with img_sig[n_img] (arcsec) given, chi^2_img of the
 * observed images against beta_hat mapped back to the image plane (Newton iterations on
 * the lens equation from each observed image) joins the likelihood; NULL leaves it out.
 *
 * Mass class (Sect. 3.3): mass_class 0 is the EPL class above (theta_E, gamma', q; Sersic lens
 * light).  mass_class 1 is the composite class kappa = Upsilon_* L_scale I_light + kappa_enfw +
 * kappa_BH: the lens light is Chameleon profiles (Eq. Chameleon) I0/(1+q) [(m^2 + 4 w_c^2/(1+q)^2)^(-1/2)
 * - (m^2 + 4 w_t^2/(1+q)^2)^(-1/2)], m^2 = x'^2 + y'^2/q^2 in the galaxy frame (the first with
 * I0 = theta[13], w_t = theta[14], w_c = ll_wc and q = ll_q; ll2 rows are further Chameleons
 * (I0, w_c, w_t, q)); the baryons are Upsilon_* L_scale times that light; the halo is the
 * elliptical NFW kappa_s k(m_h / r_s), m_h^2 = x'^2 + y'^2/q_h^2 (Eq. kappa_enfw), deflected as 44
 * cored steep ellipsoids (App. B, glad_enfw_cse) and expanded for the dynamics by the 1-D MGE of
 * the exact profile (n_mge_mass Gaussians on [mass_rmin, mass_rmax]); the black hole (mass
 * f_BH Upsilon_* L_tot L_scale) is the round Gaussian of dispersion bh_sigma in the lensing as in
 * the dynamics.  The mass Gaussians are then Upsilon_* L_scale times the tracer Gaussians, the
 * halo's, the sheet's and the black hole.  External shear and SIS perturbers as in class 0.
 *
 * Internal mass sheet (Sect. 3.3, Eqs. kappa int and dpie_kappa): with sheet != 0 the mass
 * class becomes kappa_int = (1 - lambda_int) + lambda_int kappa_gal: every deflection of the
 * galaxy model (EPL, external shear, SIS perturbers) and its mass Gaussians (black hole
 * included) are scaled by lambda_int = theta[20], and a sheet centred on the lens is added:
 * sheet 1 the dPIE profile with core sheet_rc and truncation sheet_rt arcsec (0: the paper's
 * 45 and 45.09) normalised to a central convergence 1 - lambda_int; sheet 2 an ideal uniform
 * sheet kappa = 1 - lambda_int in the lensing (exactly the mass-sheet transform), with the
 * dPIE standing in for it in the dynamics.  For the dynamics the dPIE goes through a 1-D MGE
 * of sheet_n round Gaussians log-spaced on [sheet_rmin, sheet_rmax] (0: 40 on [0.1, 1000]),
 * computed once at glad_create for 1 - lambda_int = 1 and scaled per sample.  lambda_int must
 * be > 0; a sheet with lambda_int > 1 is negative and, once the total density turns negative
 * at a probe radius, the sample gets GLAD_SAMPLE_NEGDENS (Sect. 3.3).
 *
 * Distances (Sect. 2.3, Eqs. critical_sfd, sfd final): distance_mode 0 derives them from
 * H0 = theta[19] in flat LambdaCDM (z_d, z_s, omega_m) with D_dt,int = (1 - kappa_ext) D_dt;
 * distance_mode 1 takes D_d = theta[21] and D_dt,int = theta[22] (Mpc, both > 0) as sampled
 * parameters (Table 2).  Delays are D_dt,int / c times Fermat-potential differences; the
 * dynamics scale as D_dt,int / D_d (G Sigma_crit D_d arcsec = c^2/(4 pi) D_dt,int /
 * ((1 + z_d) D_d) arcsec).
 *
 * Jeans model (Sect. 3.2): jam_align 0 takes the cylindrically aligned velocity ellipsoid
 * (constant beta_z, the pair form over (tracer, mass, u node) terms); jam_align 1 the
 * spherically aligned one of Eqs. J1/J2 (constant beta = 1 - v_theta^2/v_r^2), solved
 * along the characteristics of J1/J2 on a polar grid of sph_nr radii (log-spaced from a
 * quarter sky sub-sample to 9 x the largest tracer sigma) x sph_nw values of sin^2 theta,
 * and projected with sph_nlos nodes per line of sight; 0 selects the defaults 128, 8, 32.
 * Limits: sph_nr * sph_nw <= 4096 and (mass Gaussians incl. sheet and black hole) x n_gl <= 4096
 * (GLAD_EUNSUPPORTED beyond, as for sizes whose gradient kernels would need more than
 * 226 KB of shared memory per block).  glad_loglike_grad differentiates both models.
 *
 * Source (Sect. 3.1.1): src_pix 0 takes the Sersic source of theta[8..12]; src_pix 1
 * reconstructs the source on a grid of spx_nx x spx_ny pixels (3 <= each, product <= 4624)
 * covering [spx_x0, spx_x1] x [spx_y0, spx_y1] of the source plane: the response
 * f = B L maps the grid to the masked image pixels (each image pixel averages its ss^2 rays,
 * each ray the bilinear interpolation of the four grid pixels around beta; rays outside the
 * grid contribute nothing; B the PSF blurring), the arcs d_esr = data - B (lens light) are
 * fitted by s_MP = (F + lambda C)^-1 D (Eq. s_MP; F = f^T C_D^-1 f, D = f^T C_D^-1 d_esr,
 * C = H^T H the curvature regularisation, second differences along x and y with zero outside
 * the grid), and the image term is the log-evidence at the lambda that maximises it (Eq.
 * evi_ext, the marginal likelihood of the linear Gaussian model):
 *   ln P = -E_D - lambda E_S - ln det(F + lambda C)/2 + (N_s/2) ln lambda
 *          + ln det C / 2 - (N_d/2) ln 2 pi - ln det C_D / 2,
 * E_D = (f s_MP - d)^T C_D^-1 (f s_MP - d) / 2 and E_S = s_MP^T C s_MP / 2,
 * maximised over ln lambda in [ln spx_lam_lo, ln spx_lam_hi] by Brent's method to 1e-3 in
 * ln lambda or spx_iters evaluations.  terms[0] then holds -2 ln P (so that logL is still
 * -(sum of terms)/2) and theta[8..12] are not used.  Arithmetic: rays and the response in
 * FP32; the Gram matrix [F D; D^T d^T C_D^-1 d] from FP32 products summed in FP32 over 256
 * rows and in FP64 across them, its data row (D, d^T C_D^-1 d) summed in FP64; the
 * factorisation in double-float (the matrix held as pairs of floats, ~48 bits; every
 * multiply-add exact to that precision on the FP32 pipes) with FP64 pivots and triangular
 * solves; E_D (from the residuals of the masked pixels) by double-float dot products, E_S in
 * FP64.
 * glad_loglike_grad, glad_model_image and glad_loglike_static refuse contexts or systems with
 * a pixelated source (GLAD_EUNSUPPORTED); glad_pixsrc returns the search's result.
 */
typedef struct glad_system_desc {
  int nx, ny, ss;
  double pix;
  const float *data, *sigma;       /* [ny*nx] */
  const unsigned char *mask;       /* [ny*nx], 0 = excluded */
  int psf_k;
  const float *psf;                /* [psf_k*psf_k] */
  double src_q, src_phi;           /* Sersic source axis ratio and PA */
  double ll_n, ll_q;               /* first lens light: Sersic index and axis ratio */
  int n_ll2;
  const double *ll2;               /* [n_ll2*4]: I_e, R_e, n, q of further lens lights */
  int n_sis;
  const double *sis;               /* [n_sis*3]: theta_E, x, y of SIS perturbers */
  double r_soft;                   /* App. C softening radius of the MGE'd convergence */
  int kx, ky, kss;
  double kpix;
  int kpsf_k;
  const float *kpsf;               /* [kpsf_k*kpsf_k] */
  const int *bins;                 /* [ky*kx] */
  int n_bins;
  const float *v_obs, *v_sig;      /* [n_bins] km/s */
  int n_mge_mass;
  const int *n_mge_light;          /* [1 + n_ll2] */
  int mge_P, n_gl;
  double mass_rmin, mass_rmax, light_rmin, light_rmax;
  int has_bh;
  double bh_sigma, L_scale;
  int n_img;
  const double *img_xy, *dt_obs, *dt_sig;
  const double *img_sig;           /* [n_img] or NULL: no image-position term */
  double z_d, z_s, omega_m, kappa_ext;
  int jam_align;                   /* 0 cylindrically, 1 spherically aligned Jeans model */
  int sph_nr, sph_nw, sph_nlos;    /* rule of the spherically aligned model (0: defaults) */
  int sheet;                       /* 0 none, 1 dPIE, 2 ideal uniform sheet (see above) */
  double sheet_rc, sheet_rt;       /* dPIE core and truncation radii [arcsec] (0: 45, 45.09) */
  int sheet_n;                     /* Gaussians of the sheet's MGE (0: 40) */
  double sheet_rmin, sheet_rmax;   /* their sigma range [arcsec] (0: 0.1, 1000) */
  int distance_mode;               /* 0: H0 = theta[19]; 1: D_d = theta[21], D_dt,int = theta[22] */
  int mass_class;                  /* 0 EPL, 1 composite (see above) */
  double ll_wc;                    /* composite class: w_c of the first Chameleon [arcsec] */
  int src_pix;                     /* 0 Sersic source, 1 pixelated source (see above) */
  int spx_nx, spx_ny;              /* pixelated source: grid pixels along x and y */
  double spx_x0, spx_x1, spx_y0, spx_y1;  /* its extent on the source plane [arcsec] */
  double spx_lam_lo, spx_lam_hi;   /* regularisation search range (0, 0: 1e-6, 1e6) */
  int spx_iters;                   /* at most this many evidence evaluations (0: 40) */
} glad_system_desc;

typedef struct glad_ctx glad_ctx;

/* Validate n_sys descriptors, precompute per-system constants (distances, Gauss-Legendre
 * nodes, Euler coefficients, the binning-after-PSF operator) and stage them on the current
 * device.  *out receives the context.  Errors: GLAD_EINVAL, GLAD_ENOMEM, GLAD_ECUDA,
 * GLAD_EUNSUPPORTED (a size above the kernels' limits). */
glad_status glad_create(const glad_system_desc *sys, int n_sys, glad_ctx **out);

/* Free everything the context staged (synchronises the device first). */
void glad_destroy(glad_ctx *ctx);

/* Batched joint log-likelihood, Eq. chi_general / Eq. Posterior_LD:
 *   logL[b] = -(chi2_pix + chi2_dyn + chi2_tmd + chi2_img)/2   for sample b in [0, B)
 * (chi2_img = 0 for systems without img_sig).
 * sys_id [dev, int32 B], theta [dev, float64 B*23], logL [dev, float64 B],
 * sample_status [dev, int32 B], terms [dev, float64 B*4] or NULL: the four chi^2 terms in
 * that order.
 * The per-sample workspace is allocated (cudaMalloc) the first time a batch of this
 * size is seen and kept by the context.
 * Errors: GLAD_EINVAL (B < 1, NULL output), GLAD_ENOMEM (workspace), GLAD_ECUDA. */
glad_status glad_loglike(glad_ctx *ctx, const int *sys_id, const double *theta, int B,
                         double *logL, int *sample_status, double *terms, void *stream);

/* As glad_loglike, plus the gradient grad [dev, float64 B*23] = d logL / d theta from
 * hand-written adjoint kernels.  Invalid samples get grad = 0. */
glad_status glad_loglike_grad(glad_ctx *ctx, const int *sys_id, const double *theta, int B,
                              double *logL, double *grad, int *sample_status, double *terms,
                              void *stream);

/* PSF-blurred model image (Eq. dpre with the parametric source) of one sample of
 * system `sys`: theta [dev, 23 float64], image [dev, float32 ny*nx]. */
glad_status glad_model_image(glad_ctx *ctx, int sys, const double *theta, float *image,
                             void *stream);

/* Binned model v_rms (Eqs. binned and Vrms) of one sample of system `sys`:
 * theta [dev, 23 float64], vrms [dev, float32 n_bins] km/s. */
glad_status glad_vrms(glad_ctx *ctx, int sys, const double *theta, float *vrms, void *stream);

/* Kernel-level timing, for benchmarks.  glad_profile(ctx, 1) makes every later call
 * record a CUDA event pair on its stream around each kernel it launches (0 stops it).
 * In mode 1 the lensing and dynamics branches of glad_loglike / glad_loglike_grad still
 * run concurrently on the context's two streams, so a branch's event time includes the
 * time it waited for SMs held by the other; mode 2 runs both branches on the caller's
 * stream, one after the other, so each event pair times its kernel alone.  Returns 0, or
 * -1 for a null context or another mode.
 * glad_kernel_times(ctx, n, ms, launches) waits for those events, adds the elapsed
 * milliseconds and the launch count of kernel id k (0 <= k < n) into ms[k] and
 * launches[k] [host arrays of n], and forgets the recorded pairs.  Returns the number
 * of kernel ids; with n = 0 (or NULL arrays) it only returns that number and keeps the
 * recorded pairs.  glad_kernel_name(k) names id k. */
int glad_profile(glad_ctx *ctx, int enable);
int glad_kernel_times(glad_ctx *ctx, int n, double *ms, int *launches);
const char *glad_kernel_name(int k);

/* glad_loglike without any device allocation (the paper has no counterpart: this is a
 * service to callers that cannot call cudaMalloc while they run, e.g. code inside a CUDA
 * graph capture someone else owns, or a sampler loop under a fixed device-memory budget).
 * Same arguments, kernels and results as glad_loglike, but the per-sample scratch lives in
 * one 64 MiB file-scope device array instead of the context's workspace, so this call
 * allocates nothing (the context itself must already exist).  Every GPU that loads the
 * library holds that array until the process exits.  The first call on a device looks up
 * the array's device address (cudaGetSymbolAddress), so make it before any stream capture.
 * All calls share the one array and each clears the accumulators it needs: calls that
 * overlap on the GPU (different streams, threads or contexts) race and must be serialised.
 * A batch whose scratch exceeds 64 MiB (about 170 samples of the 200x200 RXJ1131-scale
 * system) returns GLAD_EUNSUPPORTED with the limit in glad_last_error().  It uses the
 * context's launch shape (glad_autotune / glad_set_tuning, grid or persistent form) and
 * negligible-term mode, but its integrand evaluations are not counted by
 * glad_jam_evaluations.  For the length of the call it points the context's workspace view
 * at the static array: no other host thread may use the same context meanwhile (the
 * general rule that one context is not thread-safe). */
glad_status glad_loglike_static(glad_ctx *ctx, const int *sys_id, const double *theta, int B,
                                double *logL, int *sample_status, double *terms, void *stream);

/* Autotuner (the project's own, no counterpart in the paper): times the candidate
 * launch shapes of the JAM kernels on this batch (arguments as glad_loglike) -- for the
 * pair sum: points per thread, minimum resident CTAs per SM asked of the register
 * allocator, unroll of the table-entry loop, form of the sum, grid or persistent form; with
 * with_grad, table entries per thread of its adjoint (2 or 4) -- and keeps the fastest in
 * the context for later calls.  Forms: 0 direct, two sky points per packed f32x2 operation;
 * 2 direct, two table entries per packed operation; 1 and 3 the recurrence forms of 0 and 2,
 * which write an entry's exponent at the i-th of 4 consecutive sky rows as
 * a(i) = a(0) + i B + i^2 C (log2 units) and sum 2^a(i) = 2^a(0) (2^B)^i 2^(C i^2) with two
 * ex2 per chain, the last factor folded into the entry's prefactors; they take the entries
 * with |C| <= 1 (the rest are summed directly), can lose terms below 2^-67 of their
 * prefactor (counted in the negligible-term check) and round differently from the direct
 * forms (~1e-6 relative per term).  When the environment variable GLAD_TUNE_CACHE names a file,
 * the choice is appended there keyed by device name and batch shape, and later calls
 * with the same key read it back and skip the timing.  Synchronises the stream and
 * allocates a few small scratch arrays.  glad_tuning reports the current choice:
 * *jam_code = 1000000 * form + 100000 * persistent + 1000 * points + 10 * min CTAs
 * + unroll,
 * *adj_ept = entries per thread. */
glad_status glad_autotune(glad_ctx *ctx, const int *sys_id, const double *theta, int B,
                          int with_grad, void *stream);
int glad_tuning(glad_ctx *ctx, int *jam_code, int *adj_ept);
/* Pin a launch shape instead of tuning (codes as reported by glad_tuning: 4052, 4054, 4064,
 * 8032, 8042, 8044, 16021 (form 0); 1008032, 1008041, 1008042, 1016021 (form 1); 2004042,
 * 2004052, 2004051, 2008031 (form 2); 3004042, 3004041, 3004051, 3008031 (form 3); each
 * optionally + 100000 for the persistent form; adj_ept 2 or 4).  GLAD_EINVAL for other
 * values. */
glad_status glad_set_tuning(glad_ctx *ctx, int jam_code, int adj_ept);

/* The pixelated-source reconstruction of a batch (the systems with src_pix 1; other samples
 * are left untouched): lam [dev, float64 B] the regularisation that maximises the evidence,
 * lnP [dev, float64 B] the log-evidence there, s [dev, float64 B * 4624] (row b holds sample
 * b's s_MP, spx_nx * spx_ny values, grid row-major from (spx_x0, spx_y0)) or NULL.
 * Arguments and errors as glad_loglike; the arrays of invalid samples are not written. */
glad_status glad_pixsrc(glad_ctx *ctx, const int *sys_id, const double *theta, int B,
                        double *lam, double *lnP, double *s, void *stream);
/* Cholesky factorisations of F + lambda C run since the last call (each evidence evaluation
 * of the regularisation search is one), and reset the count. */
unsigned long long glad_pix_factorizations(glad_ctx *ctx);
/* Kernel launches the pixelated-source stage enqueued since the last call (the response, the
 * Gram matrix and every pass of the search; their number varies with the passes the search
 * needed, see glad_set_pix_path), and reset the count.  0 for a NULL context. */
unsigned long long glad_pix_launches(glad_ctx *ctx);
/* How each evidence evaluation of the pixelated source runs (the results agree to rounding):
 * mode 1: one CTA per sample does the whole evaluation in one launch; mode 2: a sequence of
 * launches per evaluation, each 32-column panel step of the factorisation spread over many CTAs
 * per sample (one sample alone then uses the whole GPU); mode 0 (the default): mode 2, the
 * faster at every batch size measured (16 to 1,184 samples).  GLAD_EINVAL for other modes.
 * Outside graph capture the search's passes are enqueued in groups and the call waits on the
 * device for each group before the next but one, ending as soon as every search has converged
 * (so the call returns when the search is nearly done); under capture the full fixed pass
 * count is recorded.  This applies to glad_pixsrc and to glad_loglike on such systems. */
glad_status glad_set_pix_path(glad_ctx *ctx, int mode);

/* Precision of the forward pass (Sect. 3: the paper computes in FP64 throughout).
 * mode 0 (the default): FP32 bulk -- ray shooting, light, PSF blurring, the Jeans sums -- with
 * the MGE, deprojection, pair table, delays and every chi^2 reduction in FP64.
 * mode 1: as 0, but the ray shooting, source and lens light and the PSF blurring in FP64.
 * mode 2: as 1, and the cylindrically aligned pair sum, the tracer surface brightness and the
 * binning in FP64 too (every table entry, no skipping): the whole forward pass in FP64 (the
 * spherically aligned model's grid and line-of-sight sums stay FP32).
 * The inputs given as float32 (image data, noise, PSFs, kinematic data) are used as given.
 * Applies to glad_loglike, glad_model_image and glad_vrms; glad_loglike_grad (its logL too) and
 * glad_loglike_static always run in mode 0.  The FP64 modes allocate their own arrays at the next
 * call (an FP64 copy of the lensing block, image and table per sample) and cost far more time
 * (FP64 runs at 1/64 of the FP32 rate on this GPU).  GLAD_EINVAL for other modes. */
glad_status glad_set_precision(glad_ctx *ctx, int mode);

/* Negligible terms in the forward JAM pair sum (the project's own, no counterpart in the
 * paper).  For every sky tile the full sum at the tile's four corners gives a reference
 * value; a table entry whose term stays below 2^-(22 + log2 n_entries) of that reference
 * (2^-(30 + log2 n_entries) in the derivative pass) over the whole tile is not evaluated
 * there, and the summed bound of everything left out
 * must come to at most 2^-26 of the smallest |Sigma v^2| in the tile (below the FP32
 * rounding of each sum), else the tile is summed again with only the exact skipping of
 * entries that underflow to zero.  mode 0: exact skipping only; 1 (the default): with
 * negligible terms left out; 2: as 1 but every tile's check is failed (for tests: the
 * tiles are summed twice and the results equal mode 0).  Applies to glad_loglike,
 * glad_loglike_static, glad_vrms and the derivative pass of glad_loglike_grad (there the
 * check also covers d(Sigma v^2)/d(x'^2) and d(Sigma v^2)/d(y'^2), each against 2^-26 of
 * its largest magnitude in the tile: below the FP32 rounding of those sums).
 * GLAD_EINVAL for other modes. */
glad_status glad_set_negligible(glad_ctx *ctx, int mode);

/* Integrand evaluations executed in the last glad_loglike, glad_loglike_grad or glad_vrms
 * call on this context (skipped terms excluded): *count by the JAM pair sum (forward or
 * derivative pass), *count_adjoint (may be NULL) by the table adjoint of the gradient, as
 * (entry, sky point) pairs.  Synchronises the device. */
glad_status glad_jam_evaluations(glad_ctx *ctx, unsigned long long *count,
                                 unsigned long long *count_adjoint);

/* The composite class's halo decomposition (App. B: the elliptical NFW convergence
 * kappa_s k(xi / r_s) as 44 cored steep ellipsoids, kappa_s sum_i a_i r_s^3 (xi^2 + (s_i r_s)^2)^(-3/2)).
 * The paper takes it from the literature without printing it; the library fits it once per
 * process (cores log-spaced on [1e-5, 1e4] r_s, amplitudes >= 0 by non-negative least squares
 * of the relative error on xi / r_s in [1e-4, 1e3]).  Writes a[i], s[i] (i < 44, [host]) and,
 * if max_rel_err is not NULL, the fit's largest relative error on that range; returns 44
 * (and writes nothing when n < 44).  Needs no GPU. */
int glad_enfw_cse(int n, double *a, double *s, double *max_rel_err);

/* Message of the last failing call on this thread ("" if none). */
const char *glad_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GLAD_H */
