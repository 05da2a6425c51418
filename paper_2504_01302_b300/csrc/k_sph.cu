// Spherically aligned JAM (Sect. 3.2, Eqs. J1/J2 with constant anisotropy beta).
//
// With P = nu v_r^2 and V = nu v_phi^2, eliminating V from J1/J2 leaves one first-order
// equation for P whose characteristics through (r, theta) are r' = r e^s, R' = R e^{beta s}
// (R = r sin theta).  With P -> 0 at infinity
//   P(r, theta)  = int_0^inf e^{2 beta s} r'^2 nu F_z ds,                      F_z = Phi_z / z,
//   Dt(r, theta) = (1 - beta) int_0^inf e^{4 beta s} r'^2 (F_z dnu + nu G) ds + nu (F_R - F_z),
// where V = (1 - beta) P + R^2 Dt, dnu = nu_R/R - nu_z/z, G = F_{z,R}/R - F_{z,z}/z and
// F_R = Phi_R / R.  For a mass Gaussian j (the Emsellem et al. 1994 potential), with
// h = exp(-u^2 (R^2 + z^2 w^2)/(2 sigma_j^2)), w = (1 - e_j^2 u^2)^(-1/2), K_j = 4 pi G rho_j q_j:
//   F_z = K_j int u^2 w^3 h du,  G = K_j/sigma_j^2 int u^6 e_j^2 w^5 h du,
//   F_R - F_z = -K_j int u^4 e_j^2 w^3 h du            (cancellation-free forms).
// With the velocity ellipsoid along (r, theta, phi) the line-of-sight moment is
//   nu v_los^2 = P [(1 - beta) + beta mu^2] + Dt sin^2 i x^2,   mu = (z cos i - y sin i)/r.
//
//  k_sph_coef: per sample, the (mass Gaussian, u node) coefficients and the tracer
//    Gaussians' exponent coefficients, FP64 arithmetic stored as FP32.
//  k_sph_grid: v_r^2 = P/nu and d = Dt/nu on the polar grid (n_r radii log-spaced on
//    [r_lo, r_end], n_w values of w = sin^2 theta linear on [0, 1]); the characteristic's
//    s range [0, ln(r_end/r)] in 16 pieces of 4-point Gauss-Legendre (64 nodes): one warp
//    per grid point, two nodes per lane, packed FP32 pairs.
//  k_sph_los: Sigma v_los^2 at every sky sub-sample: n_los midpoint nodes in tau with
//    z' = c sinh(tau), c = max(rho, r_lo), tau in [-asinh(r_end/c), asinh(r_end/c)]; the grid
//    values cubic (4-point Lagrange) in ln r and linear in w; nu exact at each node.  Then
//    the tracer surface brightness and the binning-after-PSF scatter into the per-bin
//    accumulators, as in the cylindrical kernel.
#include <algorithm>

#include "glad_internal.cuh"

namespace {

#define SPH_THREADS 256
#define SPH_WARPS (SPH_THREADS / 32)
#define SPH_PIECES 16
#define SPH_LOS_BLK 8  // blocks of SPH_THREADS sky sub-samples per line-of-sight CTA
#ifndef SPH_LOS_MINB
#define SPH_LOS_MINB 4  // resident CTAs per SM asked of the register allocator (line of sight)
#endif

__device__ __forceinline__ float sph_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 4-point Gauss-Legendre rule mapped to [0, 1]
__constant__ float kGL4x[4] = {0.069431844202973712f, 0.33000947820757187f,
                               0.66999052179242813f, 0.93056815579702629f};
__constant__ float kGL4w[4] = {0.17392742256872693f, 0.32607257743127307f,
                               0.32607257743127307f, 0.17392742256872693f};

__global__ void k_sph_coef(const SysDev *__restrict__ sysv, const int *__restrict__ sys_id,
                           WsDev ws, int max_light, int max_mass, int max_mg) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (S.jam_align != 1) return;
  const int G = S.n_gl, NMG = S.n_mass_tot * G;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < NMG) {
    const int j = e / G;
    const double u = S.sph_u[e], wu = S.sph_wu[e];
    const double sj = S.sig_mass[j];
    const double e2 = ws.e2[(size_t)b * max_mass + j];
    const double K = ws.Cj[(size_t)b * max_mass + j] / (sj * sj);  // 4 pi G rho_j q_j
    const double u2 = u * u;
    const double w2 = 1.0 / (1.0 - e2 * u2);
    const double w = sqrt(w2);
    const double a = u2 / (2.0 * sj * sj);
    const double c = K * wu * u2;
    ws.sph_mt[(size_t)b * max_mg + e] =
        make_float4((float)(-a * LOG2E_D), (float)(-a * w2 * LOG2E_D), (float)(c * w * w2),
                    (float)(c * u2 * u2 * e2 * w * w2 * w2 / (sj * sj)));
    ws.sph_mrz[(size_t)b * max_mg + e] = (float)(-c * u2 * e2 * w * w2);
  }
  if (blockIdx.x == 0)
    for (int k = threadIdx.x; k < S.n_light; k += blockDim.x) {
      const double sk = S.sig_light[k];
      const double c1 = 1.0 / (2.0 * sk * sk);
      const double c0 = ws.c0[(size_t)b * max_light + k];  // 1/(2 s_k^2 p_k^2)
      ws.sph_tr[(size_t)b * max_light + k] =
          make_float4((float)ws.nu0[(size_t)b * max_light + k], (float)(-c1 * LOG2E_D),
                      (float)(-c0 * LOG2E_D), (float)(2.0 * (c0 - c1)));
    }
}

__global__ void __launch_bounds__(SPH_THREADS) k_sph_grid(const SysDev *__restrict__ sysv,
                                                          const int *__restrict__ sys_id, WsDev ws,
                                                          int max_light, int max_mg, int max_sgrid) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (S.jam_align != 1) return;
  const int nw = S.sph_nw, n_pts = S.sph_nr * nw;
  if ((int)blockIdx.x * SPH_WARPS >= n_pts) return;
  extern __shared__ float4 sph_smem[];
  const int NMG = S.n_mass_tot * S.n_gl, nL = S.n_light;
  float4 *mt = sph_smem;             // [NMG]
  float4 *trc = mt + NMG;            // [nL]
  float *mrz = (float *)(trc + nL);  // [NMG]
  for (int e = threadIdx.x; e < NMG; e += SPH_THREADS) {
    mt[e] = ws.sph_mt[(size_t)b * max_mg + e];
    mrz[e] = ws.sph_mrz[(size_t)b * max_mg + e];
  }
  for (int k = threadIdx.x; k < nL; k += SPH_THREADS) trc[k] = ws.sph_tr[(size_t)b * max_light + k];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pt = blockIdx.x * SPH_WARPS + warp;
  if (pt >= n_pts) return;  // no block-wide barrier below
  const float beta = (float)(1.0 - 1.0 / ws.dp[b].b);
  const int ia = pt / nw, ic = pt - ia * nw;
  const float r = expf((float)(S.sph_lr0 + ia * S.sph_dlr));
  const float wc = (float)ic / (float)(nw - 1);
  const float ds = (float)((S.sph_nr - 1 - ia) * S.sph_dlr / SPH_PIECES);
  float2 R2v, Z2v;
  float pw[2], dw[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int i = lane + 32 * h;
    const int g = i & 3;
    const float s = ((float)(i >> 2) + kGL4x[g]) * ds;
    const float W = kGL4w[g] * ds;
    const float rp2 = r * r * expf(2.0f * s);
    const float x = -2.0f * (1.0f - beta) * s;
    // R'^2 = r'^2 w e^x, z'^2 = r'^2 (1 - w e^x) = r'^2 [(1 - w) - w expm1(x)]
    const float R2 = rp2 * wc * expf(x);
    const float Z2 = rp2 * ((1.0f - wc) - wc * expm1f(x));
    if (h == 0) {
      R2v.x = R2;
      Z2v.x = Z2;
    } else {
      R2v.y = R2;
      Z2v.y = Z2;
    }
    pw[h] = W * expf(2.0f * beta * s) * rp2;
    dw[h] = (1.0f - beta) * W * expf(4.0f * beta * s) * rp2;
  }
  float2 Fz = make_float2(0.f, 0.f), Gs = make_float2(0.f, 0.f);
#pragma unroll 4
  for (int e = 0; e < NMG; ++e) {
    const float4 q = mt[e];
    const float2 arg = __ffma2_rn(make_float2(q.y, q.y), Z2v, __fmul2_rn(make_float2(q.x, q.x), R2v));
    const float2 hv = make_float2(sph_ex2(arg.x), sph_ex2(arg.y));
    Fz = __ffma2_rn(make_float2(q.z, q.z), hv, Fz);
    Gs = __ffma2_rn(make_float2(q.w, q.w), hv, Gs);
  }
  float2 nu = make_float2(0.f, 0.f), dnu = make_float2(0.f, 0.f);
  for (int k = 0; k < nL; ++k) {
    const float4 t = trc[k];
    const float2 arg = __ffma2_rn(make_float2(t.z, t.z), Z2v, __fmul2_rn(make_float2(t.y, t.y), R2v));
    const float2 E = __fmul2_rn(make_float2(t.x, t.x), make_float2(sph_ex2(arg.x), sph_ex2(arg.y)));
    nu = __fadd2_rn(nu, E);
    dnu = __ffma2_rn(make_float2(t.w, t.w), E, dnu);
  }
  float P = pw[0] * nu.x * Fz.x + pw[1] * nu.y * Fz.y;
  float D = dw[0] * (Fz.x * dnu.x + nu.x * Gs.x) + dw[1] * (Fz.y * dnu.y + nu.y * Gs.y);
  // the grid point itself: nu and F_R - F_z
  const float R2b = r * r * wc, Z2b = r * r * (1.0f - wc);
  float frz = 0.f, nub = 0.f;
  for (int e = lane; e < NMG; e += 32) {
    const float4 q = mt[e];
    frz = fmaf(mrz[e], sph_ex2(fmaf(q.y, Z2b, q.x * R2b)), frz);
  }
  for (int k = lane; k < nL; k += 32) {
    const float4 t = trc[k];
    nub = fmaf(t.x, sph_ex2(fmaf(t.z, Z2b, t.y * R2b)), nub);
  }
  for (int off = 16; off > 0; off >>= 1) {
    P += __shfl_xor_sync(0xffffffffu, P, off);
    D += __shfl_xor_sync(0xffffffffu, D, off);
    frz += __shfl_xor_sync(0xffffffffu, frz, off);
    nub += __shfl_xor_sync(0xffffffffu, nub, off);
  }
  if (lane == 0) {
    // nu underflows only where the line-of-sight weight nu is zero as well
    const float inv = nub > 0.f ? 1.0f / nub : 0.f;
    ws.sgrid[(size_t)b * max_sgrid + pt] = make_float2(P * inv, D * inv + frz);
  }
}

// (v_r^2, d) of grid radius a at w columns c and c+1, for one node's interpolation
__device__ __forceinline__ float2 sph_interp(const float4 *g4, int nr, int nwm, float lr0,
                                             float idlr, float r2, float ir2, float R2) {
  const float fa = fminf(fmaxf((0.5f * 0.69314718055994531f * __log2f(r2) - lr0) * idlr, 0.f),
                         (float)(nr - 1));
  const float fc = fminf(fmaxf(R2 * ir2 * (float)nwm, 0.f), (float)nwm);
  const int i0 = min(max((int)floorf(fa) - 1, 0), nr - 4);
  const int c0 = min((int)fc, nwm - 1);
  const float t = fa - (float)i0, tc = fc - (float)c0, uc = 1.f - tc;
  // 4-point Lagrange weights on the stencil nodes 0..3
  const float t1 = t - 1.f, t2 = t - 2.f, t3 = t - 3.f;
  const float L0 = -t1 * t2 * t3 * (1.f / 6.f), L1 = 0.5f * t * t2 * t3;
  const float L2 = -0.5f * t * t1 * t3, L3 = t * t1 * t2 * (1.f / 6.f);
  const float4 *gp = g4 + i0 * nwm + c0;
  const float4 a0 = gp[0], a1 = gp[nwm], a2 = gp[2 * nwm], a3 = gp[3 * nwm];
  float2 g;
  g.x = L0 * (uc * a0.x + tc * a0.z) + L1 * (uc * a1.x + tc * a1.z) +
        L2 * (uc * a2.x + tc * a2.z) + L3 * (uc * a3.x + tc * a3.z);
  g.y = L0 * (uc * a0.y + tc * a0.w) + L1 * (uc * a1.y + tc * a1.w) +
        L2 * (uc * a2.y + tc * a2.w) + L3 * (uc * a3.y + tc * a3.w);
  return g;
}

// The two nodes of a mirrored pair (+z', -z') lie at the same radius (r^2 = rho^2 + z'^2): one
// radial stencil and one set of Lagrange weights serve both; only their w columns differ.
__device__ __forceinline__ void sph_interp_pair(const float4 *g4, int nr, int nwm, float lr0,
                                                float idlr, float r2, float ir2, float R2a,
                                                float R2b, float2 &ga, float2 &gb) {
  const float fa = fminf(fmaxf((0.5f * 0.69314718055994531f * __log2f(r2) - lr0) * idlr, 0.f),
                         (float)(nr - 1));
  const int i0 = min(max((int)floorf(fa) - 1, 0), nr - 4);
  const float t = fa - (float)i0;
  const float t1 = t - 1.f, t2 = t - 2.f, t3 = t - 3.f;
  const float L[4] = {-t1 * t2 * t3 * (1.f / 6.f), 0.5f * t * t2 * t3, -0.5f * t * t1 * t3,
                      t * t1 * t2 * (1.f / 6.f)};
  const float fca = fminf(fmaxf(R2a * ir2 * (float)nwm, 0.f), (float)nwm);
  const float fcb = fminf(fmaxf(R2b * ir2 * (float)nwm, 0.f), (float)nwm);
  const int ca = min((int)fca, nwm - 1), cb = min((int)fcb, nwm - 1);
  const float ta = fca - (float)ca, tb = fcb - (float)cb;
  const float4 *pa = g4 + i0 * nwm + ca, *pb = g4 + i0 * nwm + cb;
  ga = make_float2(0.f, 0.f);
  gb = ga;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const float4 A = pa[o * nwm], Bq = pb[o * nwm];
    ga.x = fmaf(L[o], fmaf(ta, A.z - A.x, A.x), ga.x);
    ga.y = fmaf(L[o], fmaf(ta, A.w - A.y, A.y), ga.y);
    gb.x = fmaf(L[o], fmaf(tb, Bq.z - Bq.x, Bq.x), gb.x);
    gb.y = fmaf(L[o], fmaf(tb, Bq.w - Bq.y, Bq.y), gb.y);
  }
}

// The midpoint nodes come in pairs tau_i, tau_{n-1-i} = -tau_i that share e^tau and
// e^-tau; each pair is one packed FP32 step (the middle node of an odd n is done alone).
__global__ void __launch_bounds__(SPH_THREADS, SPH_LOS_MINB) k_sph_los(const SysDev *__restrict__ sysv,
                                                         const int *__restrict__ sys_id, WsDev ws,
                                                         int max_light, int max_sgrid, int max_bins) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (S.jam_align != 1) return;
  if ((int)blockIdx.x * SPH_THREADS * SPH_LOS_BLK >= S.n_sub) return;
  extern __shared__ float4 sph_smem[];
  const int tid = threadIdx.x;
  const int nr = S.sph_nr, nw = S.sph_nw, nwm = nw - 1, nL = S.n_light;
  float4 *g4 = sph_smem;                 // [nr * (nw - 1)]: (v, d) at columns c and c + 1
  float4 *trc = g4 + nr * nwm;           // [nL]
  float4 *sbc = trc + nL;                // [nL]
  float *bnum = (float *)(sbc + nL);     // [n_bins]
  float *bden = bnum + S.n_bins;         // [n_bins]
  const float2 *gsrc = ws.sgrid + (size_t)b * max_sgrid;
  for (int i = tid; i < nr * nwm; i += SPH_THREADS) {
    const int a = i / nwm, c = i - a * nwm;
    const float2 u = gsrc[a * nw + c], v = gsrc[a * nw + c + 1];
    g4[i] = make_float4(u.x, u.y, v.x, v.y);
  }
  for (int k = tid; k < nL; k += SPH_THREADS) {
    trc[k] = ws.sph_tr[(size_t)b * max_light + k];
    sbc[k] = make_float4(ws.I0f[(size_t)b * max_light + k], S.sb_cx[k], S.sb_cy[k], 0.f);
  }
  for (int l = tid; l < S.n_bins; l += SPH_THREADS) {
    bnum[l] = 0.f;
    bden[l] = 0.f;
  }
  __syncthreads();
  const DynP dp = ws.dp[b];
  // SPH_LOS_BLK consecutive blocks of sky sub-samples per CTA: one grid load and one bin flush
  for (int blk = 0; blk < SPH_LOS_BLK; ++blk) {
  const int s = (blockIdx.x * SPH_LOS_BLK + blk) * SPH_THREADS + tid;
  if (s < S.n_sub) {
    const float beta = (float)(1.0 - 1.0 / dp.b);
    const float si = (float)sqrt(dp.s2), ci = (float)sqrt(dp.c2), s2 = (float)dp.s2;
    const float cphi = (float)dp.cphi, sphi = (float)dp.sphi;
    const float hx = 0.5f * (S.nsx - 1), hy = 0.5f * (S.nsy - 1);
    const int I = s / S.nsx, J = s - I * S.nsx;
    const float x = (J - hx) * S.dsub - (float)dp.xc;
    const float y = (I - hy) * S.dsub - (float)dp.yc;
    const float xp = cphi * x + sphi * y, yp = -sphi * x + cphi * y;
    const float r_lo = (float)S.sph_r_lo, r_end = (float)S.sph_r_end;
    const float lr0 = (float)S.sph_lr0, idlr = (float)(1.0 / S.sph_dlr);
    const float c = fmaxf(sqrtf(xp * xp + yp * yp), r_lo);
    const float tm = asinhf(r_end / c);
    const int n = S.sph_nlos;
    const float dtau = 2.0f * tm / (float)n;
    const float X2 = xp * xp, omb = 1.0f - beta, dX = s2 * X2;
    const float ya = yp * ci, za = yp * si;
    const float rho2 = fmaf(yp, yp, X2);  // r^2 of a node = rho^2 + z'^2
    float acc = 0.f;
    for (int i = 0; i < (n >> 1); ++i) {
      const float tau = ((float)i + 0.5f) * dtau - tm;
      const float et = sph_ex2(tau * (float)LOG2E_D), eti = __fdividef(1.0f, et);
      const float zp = 0.5f * c * (et - eti), wt = 0.5f * dtau * c * (et + eti);
      // nodes +z' and -z'
      const float2 yy = make_float2(ya - zp * si, ya + zp * si);
      const float2 zz = make_float2(za + zp * ci, za - zp * ci);
      const float2 R2 = make_float2(fmaf(yy.x, yy.x, X2), fmaf(yy.y, yy.y, X2));
      const float2 Z2 = make_float2(zz.x * zz.x, zz.y * zz.y);
      const float r2 = fmaxf(fmaf(zp, zp, rho2), 1e-30f), ir2 = __fdividef(1.0f, r2);
      float2 ga, gb;
      sph_interp_pair(g4, nr, nwm, lr0, idlr, r2, ir2, R2.x, R2.y, ga, gb);
      float2 nu = make_float2(0.f, 0.f);
#pragma unroll 4
      for (int k = 0; k < nL; ++k) {
        const float4 q = trc[k];
        const float2 arg = __ffma2_rn(make_float2(q.z, q.z), Z2, __fmul2_rn(make_float2(q.y, q.y), R2));
        nu = __ffma2_rn(make_float2(q.x, q.x), make_float2(sph_ex2(arg.x), sph_ex2(arg.y)), nu);
      }
      const float mua = zz.x * ci - yy.x * si, mub = zz.y * ci - yy.y * si;
      const float fa = nu.x * (ga.x * fmaf(beta * mua * mua, ir2, omb) + ga.y * dX);
      const float fb = nu.y * (gb.x * fmaf(beta * mub * mub, ir2, omb) + gb.y * dX);
      acc = fmaf(wt, fa + fb, acc);
    }
    if (n & 1) {  // middle node, z' = 0
      const float R2 = fmaf(ya, ya, X2), Z2 = za * za;
      const float r2 = fmaxf(R2 + Z2, 1e-30f), ir2 = __fdividef(1.0f, r2);
      const float2 g = sph_interp(g4, nr, nwm, lr0, idlr, r2, ir2, R2);
      float nu = 0.f;
      for (int k = 0; k < nL; ++k) {
        const float4 q = trc[k];
        nu = fmaf(q.x, sph_ex2(fmaf(q.z, Z2, q.y * R2)), nu);
      }
      const float mu = za * ci - ya * si;
      acc = fmaf(dtau * c, nu * (g.x * fmaf(beta * mu * mu, ir2, omb) + g.y * dX), acc);
    }
    // tracer surface brightness and the binning-after-PSF scatter
    const float Y2 = yp * yp;
    float sb = 0.f;
    for (int k = 0; k < nL; ++k) sb = fmaf(sbc[k].x, sph_ex2(-fmaf(sbc[k].z, Y2, sbc[k].y * X2)), sb);
    for (int e = S.w_off[s]; e < S.w_off[s + 1]; ++e) {
      const int l = S.w_bin[e];
      const float w = S.w_val[e];
      atomicAdd(&bnum[l], w * acc);
      atomicAdd(&bden[l], w * sb);
    }
  }
  }
  __syncthreads();
  double *acc_g = ws.binacc + (size_t)b * max_bins * 2;
  for (int l = tid; l < S.n_bins; l += SPH_THREADS) {
    if (bnum[l] != 0.0f) atomicAdd(&acc_g[2 * l], (double)bnum[l]);
    if (bden[l] != 0.0f) atomicAdd(&acc_g[2 * l + 1], (double)bden[l]);
  }
}

size_t sph_grid_smem(int mg, int nl) { return (size_t)mg * (sizeof(float4) + sizeof(float)) + (size_t)nl * sizeof(float4); }

// paired grid, tracer and surface-brightness coefficients, bin accumulators
size_t sph_los_smem(int g4, int nl, int nb) {
  return (size_t)(g4 + 2 * nl) * sizeof(float4) + (size_t)2 * nb * sizeof(float);
}

}  // namespace

cudaError_t set_sph_smem_limit() {
  cudaError_t e = cudaFuncSetAttribute(k_sph_grid, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sph_grid_smem(GLAD_SPH_MAX_MG, GLAD_MAX_LIGHT));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_sph_los, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)sph_los_smem(GLAD_SPH_MAX_GRID, GLAD_MAX_LIGHT, GLAD_MAX_BINS));
  return e;
}

cudaError_t launch_sph_grid(glad_ctx *c, const int *sys_id, int B, cudaStream_t st) {
  int pts = 0, mg = 0;
  for (auto &sd : c->h_sysdev)
    if (sd.jam_align == 1) {
      pts = std::max(pts, sd.sph_nr * sd.sph_nw);
      mg = std::max(mg, sd.n_mass_tot * sd.n_gl);
    }
  if (pts == 0) return cudaSuccess;
  k_sph_coef<<<dim3((mg + 255) / 256, B), 256, 0, st>>>(c->d_sys, sys_id, c->ws.d, c->max_light,
                                                         c->max_mass_tot, c->max_smg);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sph_grid<<<dim3((pts + SPH_WARPS - 1) / SPH_WARPS, B), SPH_THREADS, sph_grid_smem(mg, c->max_light),
               st>>>(c->d_sys, sys_id, c->ws.d, c->max_light, c->max_smg, c->max_sgrid);
  return cudaGetLastError();
}

cudaError_t launch_sph_los(glad_ctx *c, const int *sys_id, int B, cudaStream_t st) {
  int sub = 0, g4 = 0, nb = 0;
  for (auto &sd : c->h_sysdev)
    if (sd.jam_align == 1) {
      sub = std::max(sub, sd.n_sub);
      g4 = std::max(g4, sd.sph_nr * (sd.sph_nw - 1));
      nb = std::max(nb, sd.n_bins);
    }
  if (sub == 0) return cudaSuccess;
  k_sph_los<<<dim3((sub + SPH_THREADS * SPH_LOS_BLK - 1) / (SPH_THREADS * SPH_LOS_BLK), B), SPH_THREADS,
              sph_los_smem(g4, c->max_light, nb), st>>>(
      c->d_sys, sys_id, c->ws.d, c->max_light, c->max_sgrid, c->max_bins);
  return cudaGetLastError();
}
