// Gradient of the spherically aligned JAM (Sect. 3.2, Eqs. J1/J2): the hand-written
// adjoint of k_sph_coef, k_sph_grid and k_sph_los, ending in the same per-Gaussian JAM
// inputs (nu0_k, c0_k, C_j, e2_j) that k_grad_chain carries to theta, plus beta (as
// b = 1/(1 - beta)), the inclination (directly) and the sky-frame terms (x_c, y_c, phi).
//
//  k_sph_los_adj: per sky sub-sample (one warp, lanes over its nodes), with g_N = d logL /
//    d(Sigma v^2) from k_kin_adj, the line-of-sight rule again: reverse mode into the grid values (v_r^2, d) of the stencil
//    cells and into the tracer inputs nu0_k, c0_k; forward mode (3 tangents) through the
//    node geometry for x', y' (then x_c, y_c, phi) and the inclination; beta explicitly.
//  k_sph_grid_adj: per polar grid point (one warp), with the grid adjoint: phase 1 (lanes
//    over the 64 characteristic nodes) recomputes the node sums and turns the adjoints of
//    v_r^2 = P/nu and d = D/nu + (F_R - F_z) into adjoints of each node's F_z, G, nu, dnu,
//    the tracer inputs and beta; phase 2 (lanes over (mass Gaussian, u node) entries) sums
//    each entry's coefficient adjoints over the warp's nodes.  Per CTA partial sums, no
//    global atomics.
//  k_sph_coef_adj: per (mass Gaussian, u node) entry, the partial sums carried through the
//    coefficient formulas to C_j and e2_j; the tracer and beta partials added up.
#include <algorithm>

#include "glad_internal.cuh"
#include "grad_ws.cuh"

namespace {

#define SPH_LADJ_THREADS 128
#define SPH_LADJ_PPW 16  // consecutive sky sub-samples per warp in the line-of-sight adjoint
#ifndef SPH_LADJ_MINB
#define SPH_LADJ_MINB 5  // resident CTAs per SM asked of the register allocator
#endif
#define SPH_PIECES 16
constexpr float LN2F = 0.6931471805599453f;

__device__ __forceinline__ float ex2f_(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 4-point Gauss-Legendre rule mapped to [0, 1] (as the forward kernel)
__constant__ float kAdjGLx[4] = {0.069431844202973712f, 0.33000947820757187f,
                                 0.66999052179242813f, 0.93056815579702629f};
__constant__ float kAdjGLw[4] = {0.17392742256872693f, 0.32607257743127307f,
                                 0.32607257743127307f, 0.17392742256872693f};

// a lane's pending grid-adjoint contributions for one stencil position (cell = i0 * gst + c0):
// v[4 o + {0, 1, 2, 3}] = (v_r^2 at c0, d at c0, v_r^2 at c0 + 1, d at c0 + 1) of row i0 + o
struct GRun {
  int cell;
  float v[16];
};

__device__ __forceinline__ void grun_flush(GRun &r, float *gax, float *gay, int gst) {
  if (r.cell < 0) return;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const int cell = r.cell + o * gst;
    if (r.v[4 * o] != 0.f) atomicAdd(&gax[cell], r.v[4 * o]);
    if (r.v[4 * o + 1] != 0.f) atomicAdd(&gay[cell], r.v[4 * o + 1]);
    if (r.v[4 * o + 2] != 0.f) atomicAdd(&gax[cell + 1], r.v[4 * o + 2]);
    if (r.v[4 * o + 3] != 0.f) atomicAdd(&gay[cell + 1], r.v[4 * o + 3]);
  }
}

struct LosPt {
  float xp, yp, X2, si, ci, s2, beta, omb, lr0, idlr, gN;
  int nr, nw, nwm, nL;
};

// one line-of-sight node z' = zs (derivative dzs_dc with respect to the node scale c, which
// depends on x', y' through dc_dxp, dc_dyp) of weight wt (dwt_dc): adds the tangents
// A[0..2] = d/d(x', y', i) and A[3] = d/d beta of g_N wt f, and adds the
// reverse-mode adjoints of the grid cells to the lane's pending run (flushed into gax, gay,
// rows of gst words with gst odd so that different rows fall in different banks, whenever
// the stencil moves) and those of the tracer inputs into shared memory
__device__ __forceinline__ void los_node_adj(const LosPt &q, const float4 *g4, float *gax,
                                             float *gay, int gst, GRun &run, const float4 *trc,
                                             float2 *tacc, int tid, float zs,
                                             float dzs_dc, float wt, float dwt_dc, float dc_dxp,
                                             float dc_dyp, float *A) {
  const float dzx = dzs_dc * dc_dxp, dzy = dzs_dc * dc_dyp;
  const float yy = q.yp * q.ci - zs * q.si, zz = q.yp * q.si + zs * q.ci;
  // tangents x', y', i (z' does not depend on i; d sin i/di = cos i, d cos i/di = -sin i)
  const float dyy[3] = {-q.si * dzx, q.ci - q.si * dzy, -q.yp * q.si - zs * q.ci};
  const float dzz[3] = {q.ci * dzx, q.si + q.ci * dzy, yy};
  const float R2 = fmaf(yy, yy, q.X2), Z2 = zz * zz;
  float dR2[3], dZ2[3], dr2[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    dR2[i] = 2.f * yy * dyy[i] + (i == 0 ? 2.f * q.xp : 0.f);
    dZ2[i] = 2.f * zz * dzz[i];
    dr2[i] = dR2[i] + dZ2[i];
  }
  const float r2raw = R2 + Z2;
  const bool fl = !(r2raw >= 1e-30f);
  const float r2 = fl ? 1e-30f : r2raw, ir2 = __fdividef(1.0f, r2);
  const float fa_raw = (0.5f * LN2F * __log2f(r2) - q.lr0) * q.idlr;
  const float fa = fminf(fmaxf(fa_raw, 0.f), (float)(q.nr - 1));
  const bool fa_in = !fl && fa_raw > 0.f && fa_raw < (float)(q.nr - 1);
  const float fc_raw = R2 * ir2 * (float)q.nwm;
  const float fc = fminf(fmaxf(fc_raw, 0.f), (float)q.nwm);
  const bool fc_in = !fl && fc_raw > 0.f && fc_raw < (float)q.nwm;
  const int i0 = min(max((int)floorf(fa) - 1, 0), q.nr - 4);
  const int c0 = min((int)fc, q.nwm - 1);
  const float t = fa - (float)i0, tc = fc - (float)c0, uc = 1.f - tc;
  const float t1 = t - 1.f, t2 = t - 2.f, t3 = t - 3.f;
  const float L[4] = {-t1 * t2 * t3 * (1.f / 6.f), 0.5f * t * t2 * t3, -0.5f * t * t1 * t3,
                      t * t1 * t2 * (1.f / 6.f)};
  const float dL[4] = {-(t2 * t3 + t1 * t3 + t1 * t2) * (1.f / 6.f), 0.5f * (t2 * t3 + t * t3 + t * t2),
                       -0.5f * (t1 * t3 + t * t3 + t * t1), (t1 * t2 + t * t2 + t * t1) * (1.f / 6.f)};
  float2 g = make_float2(0.f, 0.f), gt = g, gc = g;
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const float4 a = g4[(i0 + o) * q.nwm + c0];
    const float cx = uc * a.x + tc * a.z, cy = uc * a.y + tc * a.w;
    g.x = fmaf(L[o], cx, g.x);
    g.y = fmaf(L[o], cy, g.y);
    gt.x = fmaf(dL[o], cx, gt.x);
    gt.y = fmaf(dL[o], cy, gt.y);
    gc.x = fmaf(L[o], a.z - a.x, gc.x);
    gc.y = fmaf(L[o], a.w - a.y, gc.y);
  }
  const float mu = zz * q.ci - yy * q.si;
  const float m2 = mu * mu * ir2;
  const float Bk = g.x * fmaf(q.beta, m2, q.omb) + g.y * q.s2 * q.X2;
  const float w_g = q.gN * wt;
  const float om = w_g * Bk;  // d(g_N wt f)/d nu
  // tracer sums and the tracer adjoints
  float nu = 0.f, nua = 0.f, nub = 0.f;
  for (int k = 0; k < q.nL; ++k) {
    const float4 c = trc[k];
    const float E = ex2f_(fmaf(c.z, Z2, c.y * R2));
    const float nE = c.x * E;
    nu += nE;
    nua = fmaf(c.y, nE, nua);
    nub = fmaf(c.z, nE, nub);
    float2 &ta = tacc[k * SPH_LADJ_THREADS + tid];
    ta.x = fmaf(om, E, ta.x);
    ta.y = fmaf(-om * Z2, nE, ta.y);
  }
  // reverse: the 8 stencil cells
  const float av = w_g * nu * fmaf(q.beta, m2, q.omb), ad = w_g * nu * q.s2 * q.X2;
  const int base = i0 * gst + c0;
  if (base != run.cell) {
    grun_flush(run, gax, gay, gst);
    run.cell = base;
#pragma unroll
    for (int i = 0; i < 16; ++i) run.v[i] = 0.f;
  }
#pragma unroll
  for (int o = 0; o < 4; ++o) {
    const float lu = L[o] * uc, lt = L[o] * tc;
    run.v[4 * o] = fmaf(lu, av, run.v[4 * o]);
    run.v[4 * o + 1] = fmaf(lu, ad, run.v[4 * o + 1]);
    run.v[4 * o + 2] = fmaf(lt, av, run.v[4 * o + 2]);
    run.v[4 * o + 3] = fmaf(lt, ad, run.v[4 * o + 3]);
  }
  // forward tangents
  const float f = nu * Bk;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float dfa = fa_in ? 0.5f * q.idlr * ir2 * dr2[i] : 0.f;
    const float dfc = fc_in ? (float)q.nwm * ir2 * (dR2[i] - R2 * ir2 * dr2[i]) : 0.f;
    const float dgx = gt.x * dfa + gc.x * dfc, dgy = gt.y * dfa + gc.y * dfc;
    const float dnu = LN2F * (nua * dR2[i] + nub * dZ2[i]);
    const float dmu = q.ci * dzz[i] - q.si * dyy[i] + (i == 2 ? -zz * q.si - yy * q.ci : 0.f);
    const float dm2 = fl ? 0.f : 2.f * mu * ir2 * dmu - m2 * ir2 * dr2[i];
    const float dB = dgx * fmaf(q.beta, m2, q.omb) + g.x * q.beta * dm2 + dgy * q.s2 * q.X2 +
                     g.y * (i == 0 ? 2.f * q.s2 * q.xp : (i == 2 ? 2.f * q.si * q.ci * q.X2 : 0.f));
    const float dwt = i == 0 ? dwt_dc * dc_dxp : (i == 1 ? dwt_dc * dc_dyp : 0.f);
    A[i] = fmaf(q.gN, dwt * f + wt * (dnu * Bk + nu * dB), A[i]);
  }
  A[3] = fmaf(w_g * nu, g.x * (m2 - 1.f), A[3]);
}

// One warp per sky sub-sample (lanes over its line-of-sight nodes, so that a warp's grid
// cells differ: the nodes lie at different radii), SPH_LADJ_PPW consecutive sub-samples per
// warp: a lane's node keeps its stencil cells from one sub-sample to the next, so its grid
// adjoint is summed in registers and reaches shared memory only when the stencil moves.
__global__ void __launch_bounds__(SPH_LADJ_THREADS, SPH_LADJ_MINB) k_sph_los_adj(
    const SysDev *__restrict__ sysv, const int *__restrict__ sys_id, WsDev ws, GradWs gw,
    int max_light, int max_mass, int max_sgrid, int max_apts, double *grad) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (S.jam_align != 1) return;
  constexpr int PPC = SPH_LADJ_PPW * (SPH_LADJ_THREADS / 32);  // sub-samples per CTA
  if ((int)blockIdx.x * PPC >= S.n_sub) return;
  extern __shared__ float4 ladj_smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nr = S.sph_nr, nw = S.sph_nw, nwm = nw - 1, nL = S.n_light, ng = nr * nw;
  const int gst = nw | 1;                     // odd row stride of the grid adjoint
  float4 *g4 = ladj_smem;                     // [nr * nwm]
  float4 *trc = g4 + nr * nwm;                // [nL]
  float2 *tacc = (float2 *)(trc + nL);        // [nL * SPH_LADJ_THREADS]
  float *gax = (float *)(tacc + nL * SPH_LADJ_THREADS);  // [nr * gst]: d/d v_r^2
  float *gay = gax + nr * gst;                // [nr * gst]: d/d d
  __shared__ double red[SPH_LADJ_THREADS / 32][6];
  const float2 *gsrc = ws.sgrid + (size_t)b * max_sgrid;
  for (int i = tid; i < nr * nwm; i += SPH_LADJ_THREADS) {
    const int a = i / nwm, c = i - a * nwm;
    const float2 u = gsrc[a * nw + c], v = gsrc[a * nw + c + 1];
    g4[i] = make_float4(u.x, u.y, v.x, v.y);
  }
  for (int i = tid; i < 2 * nr * gst; i += SPH_LADJ_THREADS) gax[i] = 0.f;
  for (int k = tid; k < nL; k += SPH_LADJ_THREADS) trc[k] = ws.sph_tr[(size_t)b * max_light + k];
  for (int i = tid; i < nL * SPH_LADJ_THREADS; i += SPH_LADJ_THREADS) tacc[i] = make_float2(0.f, 0.f);
  __syncthreads();
  const DynP dp = ws.dp[b];
  const float cphi = (float)dp.cphi, sphi = (float)dp.sphi;
  LosPt q;
  q.si = (float)sqrt(dp.s2);
  q.ci = (float)sqrt(dp.c2);
  q.s2 = (float)dp.s2;
  q.beta = (float)(1.0 - 1.0 / dp.b);
  q.omb = 1.f - q.beta;
  q.lr0 = (float)S.sph_lr0;
  q.idlr = (float)(1.0 / S.sph_dlr);
  q.nr = nr;
  q.nw = nw;
  q.nwm = nwm;
  q.nL = nL;
  const float r_lo = (float)S.sph_r_lo, r_end = (float)S.sph_r_end;
  const int n = S.sph_nlos;
  const float inv_n = 1.0f / (float)n;
  // per-warp sums (lane 0 keeps them): d/d inc, d/d beta, phi, x_c, y_c
  double wsum[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  // the warp's g_N, loaded up front (lane p holds point p's)
  float gN_l = 0.f;
  {
    const int s = blockIdx.x * PPC + warp * SPH_LADJ_PPW + lane;
    if (lane < SPH_LADJ_PPW && s < S.n_sub) {
      const int I = s / S.nsx, J = s - I * S.nsx;
      const size_t pos = (size_t)b * max_apts + (size_t)((I >> 4) * S.atx + (J >> 4)) * 256 +
                         (I & 15) * 16 + (J & 15);
      gN_l = gw.adjpt[2 * pos + 1].z;
    }
  }
  // the pending run of the lane's first node slot (node = lane); further slots (n_los > 32)
  // scatter at once
  GRun run0, runx;
  run0.cell = runx.cell = -1;
  for (int p = 0; p < SPH_LADJ_PPW; ++p) {
    const int s = blockIdx.x * PPC + warp * SPH_LADJ_PPW + p;
    if (s >= S.n_sub) break;  // warp-uniform
    const int I = s / S.nsx, J = s - I * S.nsx;
    q.gN = __shfl_sync(0xffffffffu, gN_l, p);
    if (q.gN == 0.f) continue;
    const float x = (J - 0.5f * (S.nsx - 1)) * S.dsub - (float)dp.xc;
    const float y = (I - 0.5f * (S.nsy - 1)) * S.dsub - (float)dp.yc;
    q.xp = cphi * x + sphi * y;
    q.yp = -sphi * x + cphi * y;
    q.X2 = q.xp * q.xp;
    const float rho = sqrtf(q.X2 + q.yp * q.yp);
    const bool act = rho > r_lo;
    const float c = act ? rho : r_lo;
    const float dc_dxp = act ? q.xp / rho : 0.f, dc_dyp = act ? q.yp / rho : 0.f;
    const float qq = r_end / c;
    const float tm = asinhf(qq);
    const float dtm_dc = -qq / (c * sqrtf(1.f + qq * qq));
    float A[4] = {0.f, 0.f, 0.f, 0.f};
    for (int j = lane; j < n; j += 32) {
      const float kap = (float)(2 * j + 1 - n) * inv_n;
      const float tau = kap * tm;
      const float et = ex2f_(tau * 1.4426950408889634f), eti = __fdividef(1.0f, et);
      const float sh = 0.5f * (et - eti), ch = 0.5f * (et + eti);
      const float wt = 2.f * tm * inv_n * c * ch;
      const float dzp_dc = sh + c * ch * kap * dtm_dc;
      const float dwt_dc = 2.f * inv_n * (dtm_dc * c * ch + tm * ch + tm * c * sh * kap * dtm_dc);
      if (j < 32) {
        los_node_adj(q, g4, gax, gay, gst, run0, trc, tacc, tid, c * sh, dzp_dc, wt, dwt_dc, dc_dxp,
                     dc_dyp, A);
      } else {
        los_node_adj(q, g4, gax, gay, gst, runx, trc, tacc, tid, c * sh, dzp_dc, wt, dwt_dc, dc_dxp,
                     dc_dyp, A);
        grun_flush(runx, gax, gay, gst);
        runx.cell = -1;
      }
    }
    for (int i = 0; i < 4; ++i)
      for (int off = 16; off > 0; off >>= 1) A[i] += __shfl_xor_sync(0xffffffffu, A[i], off);
    if (lane == 0) {
      // x' = c x + s y, y' = -s x + c y with (x, y) = sky - centre
      wsum[0] += A[2];
      wsum[1] += A[3];
      wsum[2] += A[0] * q.yp - A[1] * q.xp;
      wsum[3] += -A[0] * cphi + A[1] * sphi;
      wsum[4] += -A[0] * sphi - A[1] * cphi;
    }
  }
  grun_flush(run0, gax, gay, gst);
  if (lane == 0)
    for (int i = 0; i < 5; ++i) red[warp][i] = wsum[i];
  __syncthreads();
  // grid adjoint to global, tracer adjoints summed over the CTA's threads
  float2 *gg = gw.sgadj + (size_t)b * max_sgrid;
  for (int i = tid; i < ng; i += SPH_LADJ_THREADS) {
    const int a = i / nw, cell = a * gst + (i - a * nw);
    const float vx = gax[cell], vy = gay[cell];
    if (vx != 0.f) atomicAdd(&gg[i].x, vx);
    if (vy != 0.f) atomicAdd(&gg[i].y, vy);
  }
  double *t = gw.tadj + (size_t)b * gw.tstride;
  for (int k = tid; k < nL; k += SPH_LADJ_THREADS) {
    double a0 = 0.0, a1 = 0.0;
    for (int j = 0; j < SPH_LADJ_THREADS; ++j) {
      const float2 v = tacc[k * SPH_LADJ_THREADS + j];
      a0 += v.x;
      a1 += v.y;
    }
    if (a0 != 0.0) atomicAdd(&t[k], a0);
    if (a1 != 0.0) atomicAdd(&t[max_light + k], a1);
  }
  if (tid < 5) {
    double sum = 0.0;
    for (int w = 0; w < SPH_LADJ_THREADS / 32; ++w) sum += red[w][tid];
    if (sum != 0.0) {
      const int base = 2 * max_light + 2 * max_mass;
      if (tid == 0) atomicAdd(&t[base + 3], sum);                        // inclination
      if (tid == 1) atomicAdd(&t[base + 2], sum / (dp.b * dp.b));       // b = 1/(1-beta)
      if (tid == 2) atomicAdd(&grad[(size_t)GLAD_NTHETA * b + 3], sum);  // phi
      if (tid == 3) atomicAdd(&grad[(size_t)GLAD_NTHETA * b + 4], sum);  // x_c
      if (tid == 4) atomicAdd(&grad[(size_t)GLAD_NTHETA * b + 5], sum);  // y_c
    }
  }
}

// shared memory of the grid adjoint: coefficients, F_R - F_z weights, tracer, the CTA's
// coefficient accumulators, one 64-node buffer per warp, tracer accumulators
size_t sph_gadj_smem(int mg, int nl) {
  return (size_t)mg * sizeof(float4) + (size_t)nl * sizeof(float4) + (size_t)mg * sizeof(float) +
         (size_t)mg * SPH_GADJ_NQ * sizeof(float) + (size_t)8 * 64 * sizeof(float4) +
         (size_t)nl * 2 * sizeof(float) + 16;
}

__global__ void __launch_bounds__(256) k_sph_grid_adj(const SysDev *__restrict__ sysv,
                                                      const int *__restrict__ sys_id, WsDev ws,
                                                      GradWs gw, int max_light, int max_mg,
                                                      int max_sgrid) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (S.jam_align != 1) return;
  const int nw = S.sph_nw, n_pts = S.sph_nr * nw;
  const int ncta = (n_pts + SPH_GADJ_PTS - 1) / SPH_GADJ_PTS;
  if ((int)blockIdx.x >= ncta) return;
  extern __shared__ float4 gadj_smem[];
  const int NMG = S.n_mass_tot * S.n_gl, nL = S.n_light;
  float4 *mt = gadj_smem;                          // [NMG]
  float4 *trc = mt + NMG;                          // [nL]
  float4 *nodes = trc + nL;                        // [8][64]: R'^2, z'^2, A_Fz, A_G
  float *mrz = (float *)(nodes + 8 * 64);          // [NMG]
  float *acc = mrz + NMG;                          // [NMG][5]: A1, A2, cz, cG, mrz
  float *tac = acc + NMG * SPH_GADJ_NQ;            // [nL][2]: nu0, c0
  float *bac = tac + 2 * nL;                       // [1]
  const int tid = threadIdx.x;
  for (int e = tid; e < NMG; e += 256) {
    mt[e] = ws.sph_mt[(size_t)b * max_mg + e];
    mrz[e] = ws.sph_mrz[(size_t)b * max_mg + e];
  }
  for (int i = tid; i < NMG * SPH_GADJ_NQ; i += 256) acc[i] = 0.f;
  for (int k = tid; k < nL; k += 256) {
    trc[k] = ws.sph_tr[(size_t)b * max_light + k];
    tac[2 * k] = 0.f;
    tac[2 * k + 1] = 0.f;
  }
  if (tid == 0) bac[0] = 0.f;
  __syncthreads();
  const int warp = tid >> 5, lane = tid & 31;
  float4 *nb = nodes + warp * 64;
  const float beta = (float)(1.0 - 1.0 / ws.dp[b].b);
  const float2 *gadj = gw.sgadj + (size_t)b * max_sgrid;
  float bsum = 0.f;
  for (int rep = 0; rep < SPH_GADJ_PTS / 8; ++rep) {
    const int pt = blockIdx.x * SPH_GADJ_PTS + rep * 8 + warp;
    if (pt >= n_pts) break;  // warp-uniform; no block barrier until the end
    const float2 Ag = gadj[pt];
    if (Ag.x == 0.f && Ag.y == 0.f) continue;
    const int ia = pt / nw, ic = pt - ia * nw;
    const float r = expf((float)(S.sph_lr0 + ia * S.sph_dlr));
    const float wc = (float)ic / (float)(nw - 1);
    const float ds = (float)((S.sph_nr - 1 - ia) * S.sph_dlr / SPH_PIECES);
    // ---- phase 1: lanes over nodes (lane and lane + 32)
    float R2[2], Z2[2], sv[2], pw[2], dw[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int i = lane + 32 * h, g = i & 3;
      const float s = ((float)(i >> 2) + kAdjGLx[g]) * ds;
      const float W = kAdjGLw[g] * ds;
      const float rp2 = r * r * expf(2.0f * s);
      const float x = -2.0f * (1.0f - beta) * s;
      R2[h] = rp2 * wc * expf(x);
      Z2[h] = rp2 * ((1.0f - wc) - wc * expm1f(x));
      sv[h] = s;
      pw[h] = W * expf(2.0f * beta * s) * rp2;
      dw[h] = (1.0f - beta) * W * expf(4.0f * beta * s) * rp2;
    }
    float Fz[2] = {0.f, 0.f}, Gs[2] = {0.f, 0.f}, zA1[2] = {0.f, 0.f}, zA2[2] = {0.f, 0.f};
    float gA1[2] = {0.f, 0.f}, gA2[2] = {0.f, 0.f};
    for (int e = 0; e < NMG; ++e) {
      const float4 c = mt[e];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float hv = ex2f_(fmaf(c.y, Z2[h], c.x * R2[h]));
        const float hz = c.z * hv, hg = c.w * hv;
        Fz[h] += hz;
        Gs[h] += hg;
        zA1[h] = fmaf(c.x, hz, zA1[h]);
        zA2[h] = fmaf(c.y, hz, zA2[h]);
        gA1[h] = fmaf(c.x, hg, gA1[h]);
        gA2[h] = fmaf(c.y, hg, gA2[h]);
      }
    }
    float nu[2] = {0.f, 0.f}, dnu[2] = {0.f, 0.f}, na[2] = {0.f, 0.f}, nbz[2] = {0.f, 0.f};
    float dna[2] = {0.f, 0.f}, dnb[2] = {0.f, 0.f};
    for (int k = 0; k < nL; ++k) {
      const float4 c = trc[k];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float E = c.x * ex2f_(fmaf(c.z, Z2[h], c.y * R2[h]));
        nu[h] += E;
        dnu[h] = fmaf(c.w, E, dnu[h]);
        na[h] = fmaf(c.y, E, na[h]);
        nbz[h] = fmaf(c.z, E, nbz[h]);
        dna[h] = fmaf(c.w * c.y, E, dna[h]);
        dnb[h] = fmaf(c.w * c.z, E, dnb[h]);
      }
    }
    float P = pw[0] * nu[0] * Fz[0] + pw[1] * nu[1] * Fz[1];
    float D = dw[0] * (Fz[0] * dnu[0] + nu[0] * Gs[0]) + dw[1] * (Fz[1] * dnu[1] + nu[1] * Gs[1]);
    // the grid point itself
    const float R2b = r * r * wc, Z2b = r * r * (1.0f - wc);
    float frz = 0.f, nub = 0.f;
    for (int e = lane; e < NMG; e += 32) {
      const float4 c = mt[e];
      frz = fmaf(mrz[e], ex2f_(fmaf(c.y, Z2b, c.x * R2b)), frz);
    }
    for (int k = lane; k < nL; k += 32) {
      const float4 c = trc[k];
      nub = fmaf(c.x, ex2f_(fmaf(c.z, Z2b, c.y * R2b)), nub);
    }
    for (int off = 16; off > 0; off >>= 1) {
      P += __shfl_xor_sync(0xffffffffu, P, off);
      D += __shfl_xor_sync(0xffffffffu, D, off);
      nub += __shfl_xor_sync(0xffffffffu, nub, off);
    }
    // v = P/nu_b, d = D/nu_b + frz (v = 0, d = frz where nu_b underflows)
    const float inv = nub > 0.f ? 1.0f / nub : 0.f;
    const float AP = Ag.x * inv, AD = Ag.y * inv;
    const float Anb = -(Ag.x * P + Ag.y * D) * inv * inv;
    const float Afrz = Ag.y;
    float bl = 0.f;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float AFz = AP * pw[h] * nu[h] + AD * dw[h] * dnu[h];
      const float AG = AD * dw[h] * nu[h];
      const float Anu = AP * pw[h] * Fz[h] + AD * dw[h] * Gs[h];
      const float Adnu = AD * dw[h] * Fz[h];
      const float AR2 = LN2F * (AFz * zA1[h] + AG * gA1[h] + Anu * na[h] + Adnu * dna[h]);
      const float AZ2 = LN2F * (AFz * zA2[h] + AG * gA2[h] + Anu * nbz[h] + Adnu * dnb[h]);
      const float s = sv[h];
      // d/d beta: R'^2 and z'^2 (d/d beta = +-2 s R'^2), pw (2 s pw), dw (4 s - 1/(1-beta))
      bl += (AR2 - AZ2) * 2.f * s * R2[h] + AP * 2.f * s * pw[h] * nu[h] * Fz[h] +
            AD * (4.f * s - 1.f / (1.f - beta)) * dw[h] * (Fz[h] * dnu[h] + nu[h] * Gs[h]);
      nb[lane + 32 * h] = make_float4(R2[h], Z2[h], AFz, AG);
      // tracer inputs: d/d nu0_k and d/d c0_k (c0 enters the z'^2 coefficient and dnu's 2(c0 - c1))
      Fz[h] = Anu;   // reuse as (A_nu, A_dnu) for the tracer pass
      Gs[h] = Adnu;
    }
    bsum += bl;
    for (int k = 0; k < nL; ++k) {
      const float4 c = trc[k];
      float a0 = 0.f, a1 = 0.f;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float E = ex2f_(fmaf(c.z, Z2[h], c.y * R2[h]));
        const float an = Fz[h] + Gs[h] * c.w;
        a0 = fmaf(an, E, a0);
        a1 += c.x * E * (2.f * Gs[h] - an * Z2[h]);
      }
      for (int off = 16; off > 0; off >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, off);
        a1 += __shfl_xor_sync(0xffffffffu, a1, off);
      }
      if (lane == 0) {
        atomicAdd(&tac[2 * k], a0);
        atomicAdd(&tac[2 * k + 1], a1);
      }
    }
    // nu at the grid point
    for (int k = lane; k < nL; k += 32) {
      const float4 c = trc[k];
      const float E = ex2f_(fmaf(c.z, Z2b, c.y * R2b));
      atomicAdd(&tac[2 * k], Anb * E);
      atomicAdd(&tac[2 * k + 1], -Anb * c.x * E * Z2b);
    }
    __syncwarp();
    // ---- phase 2: lanes over entries, the warp's 64 nodes from shared memory
    for (int e = lane; e < NMG; e += 32) {
      const float4 c = mt[e];
      float s_cz = 0.f, s_cg = 0.f, s_a1 = 0.f, s_a2 = 0.f;
      for (int i = 0; i < 64; ++i) {
        const float4 nd = nb[i];
        const float hv = ex2f_(fmaf(c.y, nd.y, c.x * nd.x));
        s_cz = fmaf(nd.z, hv, s_cz);
        s_cg = fmaf(nd.w, hv, s_cg);
        const float tt = fmaf(nd.z, c.z, nd.w * c.w) * hv;
        s_a1 = fmaf(tt, nd.x, s_a1);
        s_a2 = fmaf(tt, nd.y, s_a2);
      }
      const float hb = ex2f_(fmaf(c.y, Z2b, c.x * R2b));
      const float tb = Afrz * mrz[e] * hb;
      float *a = acc + e * SPH_GADJ_NQ;
      atomicAdd(&a[0], LN2F * fmaf(tb, R2b, s_a1));
      atomicAdd(&a[1], LN2F * fmaf(tb, Z2b, s_a2));
      atomicAdd(&a[2], s_cz);
      atomicAdd(&a[3], s_cg);
      atomicAdd(&a[4], Afrz * hb);
    }
    __syncwarp();
  }
  for (int off = 16; off > 0; off >>= 1) bsum += __shfl_xor_sync(0xffffffffu, bsum, off);
  if (lane == 0 && bsum != 0.f) atomicAdd(bac, bsum);
  __syncthreads();
  const size_t cta = (size_t)b * gw.sph_cta + blockIdx.x;
  for (int i = tid; i < NMG * SPH_GADJ_NQ; i += 256) gw.scoef[cta * max_mg * SPH_GADJ_NQ + i] = acc[i];
  for (int i = tid; i < 2 * nL; i += 256) gw.strc[cta * max_light * 2 + i] = tac[i];
  if (tid == 0) gw.sbeta[cta] = bac[0];
}

__global__ void k_sph_coef_adj(const SysDev *__restrict__ sysv, const int *__restrict__ sys_id,
                               WsDev ws, GradWs gw, int max_light, int max_mass, int max_mg) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (S.jam_align != 1) return;
  const int G = S.n_gl, NMG = S.n_mass_tot * G, nL = S.n_light;
  const int ncta = (S.sph_nr * S.sph_nw + SPH_GADJ_PTS - 1) / SPH_GADJ_PTS;
  double *t = gw.tadj + (size_t)b * gw.tstride;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < NMG) {
    double A[SPH_GADJ_NQ] = {0, 0, 0, 0, 0};
    for (int c = 0; c < ncta; ++c) {
      const float *p = gw.scoef + (((size_t)b * gw.sph_cta + c) * max_mg + e) * SPH_GADJ_NQ;
      for (int q = 0; q < SPH_GADJ_NQ; ++q) A[q] += p[q];
    }
    const int j = e / G;
    const double u = S.sph_u[e], wu = S.sph_wu[e];
    const double sj = S.sig_mass[j];
    const double e2 = ws.e2[(size_t)b * max_mass + j];
    const double K = ws.Cj[(size_t)b * max_mass + j] / (sj * sj);
    const double u2 = u * u, u4 = u2 * u2;
    const double w2 = 1.0 / (1.0 - e2 * u2), w = sqrt(w2), w3 = w * w2, w5 = w3 * w2;
    const double a = u2 / (2.0 * sj * sj);
    // A1 = -a log2e (fixed), A2 = -a w2 log2e, cz = K wu u^2 w^3, cG = K/s^2 wu u^6 e2 w^5,
    // mrz = -K wu u^4 e2 w^3; d w2 / d e2 = u^2 w2^2
    const double dA2 = -a * LOG2E_D * u2 * w2 * w2;
    const double dcz_K = wu * u2 * w3, dcz_e = K * wu * u2 * 1.5 * u2 * w * w2 * w2;
    const double dcg_K = wu * u4 * u2 * e2 * w5 / (sj * sj);
    const double dcg_e = K / (sj * sj) * wu * u4 * u2 * w5 * (1.0 + 2.5 * e2 * u2 * w2);
    const double dmr_K = -wu * u4 * e2 * w3;
    const double dmr_e = -K * wu * u4 * w3 * (1.0 + 1.5 * e2 * u2 * w2);
    const double aK = A[2] * dcz_K + A[3] * dcg_K + A[4] * dmr_K;
    const double ae2 = A[1] * dA2 + A[2] * dcz_e + A[3] * dcg_e + A[4] * dmr_e;
    // C_j = K sigma_j^2
    if (aK != 0.0) atomicAdd(&t[2 * max_light + j], aK / (sj * sj));
    if (ae2 != 0.0) atomicAdd(&t[2 * max_light + max_mass + j], ae2);
  }
  if (blockIdx.x == 0) {
    for (int k = threadIdx.x; k < nL; k += blockDim.x) {
      double a0 = 0.0, a1 = 0.0;
      for (int c = 0; c < ncta; ++c) {
        const float *p = gw.strc + (((size_t)b * gw.sph_cta + c) * max_light + k) * 2;
        a0 += p[0];
        a1 += p[1];
      }
      if (a0 != 0.0) atomicAdd(&t[k], a0);
      if (a1 != 0.0) atomicAdd(&t[max_light + k], a1);
    }
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int c = 0; c < ncta; ++c) s += gw.sbeta[(size_t)b * gw.sph_cta + c];
      const double bb = ws.dp[b].b;
      if (s != 0.0) atomicAdd(&t[2 * max_light + 2 * max_mass + 2], s / (bb * bb));
    }
  }
}

size_t sph_ladj_smem(int g4, int g, int nl) {
  return (size_t)(g4 + nl) * sizeof(float4) + (size_t)2 * g * sizeof(float) +
         (size_t)nl * SPH_LADJ_THREADS * sizeof(float2);
}

}  // namespace

// the largest dynamic shared memory each kernel may take: the device's opt-in limit less the
// kernel's static shared memory (descriptors needing more are refused at glad_create)
template <class K>
cudaError_t allow_dynamic_smem(K kernel) {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa{};
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, kernel);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             optin - (int)fa.sharedSizeBytes);
  return e;
}

cudaError_t set_sph_grad_smem_limit() {
  cudaError_t e = allow_dynamic_smem(k_sph_los_adj);
  if (e == cudaSuccess) e = allow_dynamic_smem(k_sph_grid_adj);
  return e;
}

cudaError_t launch_grad_sph(glad_ctx *c, const int *sys_id, int B, double *grad, cudaStream_t st) {
  GradWs &g = *c->gws;
  int blk = 0, g4 = 0, gp = 0, ga = 0, mg = 0;
  for (auto &sd : c->h_sysdev)
    if (sd.jam_align == 1) {
      const int ppc = SPH_LADJ_PPW * (SPH_LADJ_THREADS / 32);
      blk = std::max(blk, (sd.n_sub + ppc - 1) / ppc);
      g4 = std::max(g4, sd.sph_nr * (sd.sph_nw - 1));
      gp = std::max(gp, sd.sph_nr * sd.sph_nw);
      ga = std::max(ga, sd.sph_nr * (sd.sph_nw | 1));
      mg = std::max(mg, sd.n_mass_tot * sd.n_gl);
    }
  if (blk == 0) return cudaSuccess;
  k_sph_los_adj<<<dim3(blk, B), SPH_LADJ_THREADS, sph_ladj_smem(g4, ga, c->max_light), st>>>(
      c->d_sys, sys_id, c->ws.d, g, c->max_light, c->max_mass_tot, c->max_sgrid, c->max_apts, grad);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sph_grid_adj<<<dim3((gp + SPH_GADJ_PTS - 1) / SPH_GADJ_PTS, B), 256, sph_gadj_smem(mg, c->max_light),
                   st>>>(c->d_sys, sys_id, c->ws.d, g, c->max_light, c->max_smg, c->max_sgrid);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_sph_coef_adj<<<dim3((mg + 255) / 256, B), 256, 0, st>>>(c->d_sys, sys_id, c->ws.d, g, c->max_light,
                                                            c->max_mass_tot, c->max_smg);
  return cudaGetLastError();
}
