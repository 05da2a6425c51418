// Gradient workspace shared by the adjoint kernels (k_grad.cu, k_sph_grad.cu).
#pragma once
#include <vector>

#include "glad_internal.cuh"

#define SPH_GADJ_PTS 32  // polar grid points per CTA of the spherically aligned grid adjoint
#define SPH_GADJ_NQ 5    // coefficient adjoints per (mass Gaussian, u node): A1, A2, cz, cG, mrz

struct GradWs {
  int B = 0;
  float *resid = nullptr;    // [B*max_pix]  d logL / d m (blurred model)
  float *gpix = nullptr;     // [B*max_pix]  d logL / d img (unblurred)
  float4 *pt = nullptr;      // [B*max_sub]  V, dV/dX, dV/dY (X = x'^2, Y = y'^2)
  float4 *adjpt = nullptr;   // [B*max_apts*2] (X, X, Y, Y), (XY, XY, g_N, g_N), 16x16-tile order
  double *entadj = nullptr;  // [B*max_ent*3] d logL / d (Q0, Q1, a_y)
  double *adjI0 = nullptr;   // [B*max_light] d logL / d I0_k (tracer amplitudes)
  // per sample, the JAM adjoint carried to the per-Gaussian JAM inputs: d logL / d nu0_k,
  // c0_k [max_light each], C_j, e2_j [max_mass_tot each], sin^2 i, cos^2 i, b, and the
  // inclination directly [4]
  double *tadj = nullptr;    // [B*tstride]
  int tstride = 0;
  // spherically aligned model: adjoint of the polar grid (v_r^2, d), and per grid-adjoint
  // CTA the partial sums of the coefficient, tracer and beta adjoints
  float2 *sgadj = nullptr;   // [B*max_sgrid]
  float *scoef = nullptr;    // [B*sph_cta*max_smg*SPH_GADJ_NQ]
  float *strc = nullptr;     // [B*sph_cta*max_light*2]: d/d nu0_k, d/d c0_k
  float *sbeta = nullptr;    // [B*sph_cta]
  int sph_cta = 0;
  std::vector<void *> allocs;
};

