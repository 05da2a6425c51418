// Pixelated source reconstruction (Sect. 3.1.1, Eqs. dpre, s_MP, evi_ext; Table 1).
//  k_image (k_lens.cu) leaves, for every image pixel of a pixelated-source system, the
//    bilinear grid entries of its ss^2 rays (the lensing operator L), and the PSF kernels the
//    arcs d_esr = data - B (lens light).
//  k_pix_f: one warp per masked pixel q builds row q of the response f = B L (the PSF taps
//    around q gather their pixels' ray entries into a shared row of N_s) and stores
//    g_q = [f_q, d_q] / sigma_q in FP32.
//  k_pix_gram: [F D; D^T d^T C_D^-1 d] = g^T g, lower triangle, 64 x 64 tiles: FP32 products
//    summed in FP32 over 256 rows and in double-float across them; k_pix_dcol then redoes the data
//    row (D and d^T C_D^-1 d) with double-float sums of the exact products.
//  the k_pixm_* sequence (the default), which spreads each panel step over many CTAs per
//    sample, or k_pix_eval, one CTA per sample: M = [F + lambda C; D^T], blocked Cholesky
//    (32-wide panels, 64 x 64 trailing tiles) whose last row is y = L^-1 D, s_MP by the
//    backward solve L^T s = y, and the log-evidence
//      ln P = -E_D - lambda E_S - sum ln L_ii + (N_s/2) ln lambda + const,
//    E_D = |f s_MP - d|^2 / 2 (units of sigma) from the residuals of the masked pixels,
//    E_S = |H s_MP|^2 / 2, then one step of Brent's minimisation of -ln P over ln lambda; its
//    last pass writes s_MP for the caller.  E_D + lambda E_S is stationary at s_MP, so an
//    error in s_MP moves it only at second order; written as the difference
//    d^T C_D^-1 d - D^T s_MP it would lose ~1e-8 of two sums that reach N_d (S/N)^2.
// The factorisation keeps ~FP64 accuracy because the evidence needs ln det(F + lambda C) to
// ~1e-2 absolute over N_s ~ 1e3 pivots of a matrix whose conditioning grows as lambda falls.
// It runs in double-float (~48 bits) on the FP32 pipes throughout, since this GPU's FP64
// rate is 1/73 of its FP32 rate with or without tensor cores; FP64 is left to the Gram
// matrix's sums, the assembly, the energies and one logarithm per evaluation.
#include <math.h>

#include <algorithm>

#include "glad_internal.cuh"

// state of Brent's minimisation (golden section with parabolic steps) of phi(t) = -ln P(e^t)
// over t = ln lambda in [a, b]: x the best point, w the second best, v the previous w, d the
// last step, e the one before, u the pending trial; phase 0 evaluates x first, 1 evaluates u,
// 2 stops
struct PixSearch {
  double a, b, x, w, v, fx, fw, fv, d, e, u;
  int phase, it;
};

struct PixDev {
  float *g;             // [B * max_nd * ldg] rows [f_q / sigma_q, d_q / sigma_q]
  double *F;            // [B * ldg * ldg] Gram matrix, lower triangle
  float2 *A;            // [B * (max_ns + 1)^2] M = [F + lambda C; D^T] (row stride N_s + 1) and
                        // its factor, lower triangle, double-float (hi, lo) pairs of floats
  float2 *s;            // [B * max_ns] s_MP
  float2 *rd;           // [B * max_ns] 1 / L_ii, for the backward solve
  PixSearch *srch;      // [B]
  unsigned long long *nfac;  // [1] factorisations run
  // the multi-launch form's per-sample state
  float2 *pm;           // [B] product of the pivots so far, pm * 2^pe
  int *pe;              // [B]
  int *bad;             // [B] a pivot was not positive
  double *es;           // [B] |H s_MP|^2
  double *edp;          // [B * ed_chunks] partial sums of the squared residuals
  float2 *dgf;          // [B * 32 * 32] the factored diagonal block of the current panel step
  int ldg, max_ns, max_nd, ed_chunks;
};

struct PixWs {
  int B = 0;
  PixDev d{};
  std::vector<void *> allocs;
  // the multi-launch form's streams: hi (the critical path: panels, tile column 0, solves) at
  // the greatest priority, aux (the other trailing tiles) at the least, so that a panel's CTAs
  // take the first SMs that the tiles free; forked from and joined back into the caller's
  // stream by events
  cudaStream_t hi = nullptr, aux = nullptr;
  cudaEvent_t ev_p = nullptr, ev_r = nullptr, ev_in = nullptr, ev_out = nullptr;
  // the search's early end (not under graph capture): per pass the count of samples still
  // searching, copied to pinned host memory, and two events for the groups of passes
  int *d_open = nullptr, *h_open = nullptr;
  cudaEvent_t ev_grp[2] = {nullptr, nullptr};
  unsigned long long launches = 0;  // kernels enqueued (glad_pix_launches)
  int slots = 444;                  // resident k_pixm_rest CTAs on the GPU (three per SM)
};

namespace {

constexpr double GOLD = 0.3819660112501051;  // (3 - sqrt 5) / 2
constexpr double TTOL = 1e-3;                // tolerance in ln lambda (ln P moves by ~P"/2 TTOL^2)

#define PIX_F_WARPS 8
#define PIX_THREADS 256
#define PIXM_ED_ROWS 64
#define PIXM_PANEL_THREADS 128
#define PIX_GROUP 2          // search passes per group between the host's convergence checks
#define PIXM_REST_SMEM (2 * 2 * 64 * 33 * (int)sizeof(float2))
#define PIXM_REST_TPC 8      // most tiles per CTA of k_pixm_rest

// ---------------------------------------------------------------------------------------
// Brent's method (Brent 1973, "Algorithms for Minimization without Derivatives", ch. 5):
// golden-section steps, replaced by the vertex of the parabola through x, w, v when that
// vertex falls inside the interval and moves by less than half of the step before last.
__device__ void brent_start(PixSearch &s, double lo, double hi) {
  s.a = lo;
  s.b = hi;
  s.x = s.w = s.v = s.u = lo + GOLD * (hi - lo);
  s.fx = s.fw = s.fv = 0.0;
  s.d = s.e = 0.0;
  s.phase = 0;
  s.it = 0;
}

// takes phi at the pending point and chooses the next one (or stops)
__device__ void brent_step(PixSearch &s, double f, int max_it) {
  s.it += 1;
  if (s.phase == 0) {
    s.fx = s.fw = s.fv = f;
    s.phase = 1;
  } else {
    const double u = s.u;
    if (f <= s.fx) {
      if (u < s.x) s.b = s.x;
      else s.a = s.x;
      s.v = s.w;
      s.fv = s.fw;
      s.w = s.x;
      s.fw = s.fx;
      s.x = u;
      s.fx = f;
    } else {
      if (u < s.x) s.a = u;
      else s.b = u;
      if (f <= s.fw || s.w == s.x) {
        s.v = s.w;
        s.fv = s.fw;
        s.w = u;
        s.fw = f;
      } else if (f <= s.fv || s.v == s.x || s.v == s.w) {
        s.v = u;
        s.fv = f;
      }
    }
  }
  const double m = 0.5 * (s.a + s.b);
  const double tol1 = 1e-10 * fabs(s.x) + TTOL / 3.0, tol2 = 2.0 * tol1;
  if (fabs(s.x - m) <= tol2 - 0.5 * (s.b - s.a) || s.it >= max_it) {
    s.phase = 2;
    return;
  }
  bool golden = true;
  if (fabs(s.e) > tol1) {
    // parabola through (x, fx), (w, fw), (v, fv): vertex at x + p/q
    double r = (s.x - s.w) * (s.fx - s.fv);
    double q = (s.x - s.v) * (s.fx - s.fw);
    double p = (s.x - s.v) * q - (s.x - s.w) * r;
    q = 2.0 * (q - r);
    if (q > 0.0) p = -p;
    else q = -q;
    const double e_prev = s.e;
    s.e = s.d;
    if (fabs(p) < fabs(0.5 * q * e_prev) && p > q * (s.a - s.x) && p < q * (s.b - s.x)) {
      s.d = p / q;
      const double uu = s.x + s.d;
      if (uu - s.a < tol2 || s.b - uu < tol2) s.d = s.x < m ? tol1 : -tol1;
      golden = false;
    }
  }
  if (golden) {
    s.e = (s.x < m ? s.b : s.a) - s.x;
    s.d = GOLD * s.e;
  }
  s.u = s.x + (fabs(s.d) >= tol1 ? s.d : (s.d > 0.0 ? tol1 : -tol1));
}

// ---------------------------------------------------------------------------------------
// Double-float arithmetic for the trailing update of the factorisation (an unevaluated sum
// hi + lo of two FP32 numbers carries ~48 bits): B300 runs FP32 at 73x its FP64 rate, so a
// multiply-add in ~12 FP32 operations is ~6x faster than a DFMA.  The product's rounding
// error comes exactly from an FMA (TwoProduct), the sum's from Knuth's TwoSum; the low parts
// are summed plainly (their rounding is ~2^-48 of the result over 32 terms).
__device__ __forceinline__ float2 df_split(double x) {
  const float h = __double2float_rn(x);
  return make_float2(h, __double2float_rn(x - (double)h));
}

__device__ __forceinline__ double df_val(float2 v) { return (double)v.x + (double)v.y; }

// (a.x + a.y) - (hi + lo), renormalised
__device__ __forceinline__ float2 df_sub(float2 a, float hi, float lo) {
  const float s = __fsub_rn(a.x, hi);
  const float v = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, v)), __fsub_rn(-hi, v));
  const float l = __fadd_rn(__fsub_rn(a.y, lo), e);
  const float h = __fadd_rn(s, l);
  return make_float2(h, __fsub_rn(l, __fsub_rn(h, s)));
}

// (hi, lo) += a * b
__device__ __forceinline__ void df_fma(float &hi, float &lo, float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float pe = __fmaf_rn(a.x, b.x, -p);
  pe = __fmaf_rn(a.x, b.y, pe);
  pe = __fmaf_rn(a.y, b.x, pe);
  const float s = __fadd_rn(hi, p);
  const float v = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, v)), __fsub_rn(p, v));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(pe, e));
}

// (a.x + a.y) * (b.x + b.y), renormalised (the product's error by FMA, the cross terms added)
__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  float e = __fmaf_rn(a.x, b.x, -p);
  e = __fmaf_rn(a.x, b.y, e);
  e = __fmaf_rn(a.y, b.x, e);
  const float h = __fadd_rn(p, e);
  return make_float2(h, __fsub_rn(e, __fsub_rn(h, p)));
}

// ---------------------------------------------------------------------------------------
// rows of the response: f_q = sum over the PSF taps (a, c) of P[a][c] L_p, p = q - (a - h, c - h)
__global__ void __launch_bounds__(PIX_F_WARPS * 32) k_pix_f(const SysDev *__restrict__ sysv,
                                                            const int *__restrict__ sys_id, WsDev ws,
                                                            PixDev pd, int max_pix) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (!S.src_pix) return;
  extern __shared__ float frow[];  // [PIX_F_WARPS][ldg]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int qr = blockIdx.x * PIX_F_WARPS + warp;
  if (qr >= S.n_mask) return;
  const int ns = S.spx_ns;
  float *row = frow + warp * pd.ldg;
  for (int k = lane; k <= ns; k += 32) row[k] = 0.0f;
  __syncwarp();
  const int q = S.mask_list[qr];
  const int qi = q / S.nx, qj = q - qi * S.nx;
  const int K = S.psf_k, h = (K - 1) / 2, nr = 4 * S.ss * S.ss;
  const int *Li = ws.pix_Li + (size_t)b * ws.max_lpix;
  const float *Lw = ws.pix_Lw + (size_t)b * ws.max_lpix;
  // the lanes take taps 32 apart in the K^2 window (32 is coprime to the odd K^2, so t0 -> t
  // is a permutation): neighbouring taps land on neighbouring rays and the same grid pixels,
  // and would collide in the shared row's atomics
  const int KK = K * K;
  for (int t0 = lane; t0 < KK; t0 += 32) {
    const int t = (int)(((long long)t0 * 32) % KK);
    const int a = t / K, c = t - a * K;
    const int pi = qi - (a - h), pj = qj - (c - h);
    if (pi < 0 || pi >= S.ny || pj < 0 || pj >= S.nx) continue;
    const float P = S.psf[t];
    // a pixel's entries: ss^2 rays x 4, 16-byte aligned (nr is a multiple of 4)
    const int4 *li = reinterpret_cast<const int4 *>(Li + (size_t)(pi * S.nx + pj) * nr);
    const float4 *lw = reinterpret_cast<const float4 *>(Lw + (size_t)(pi * S.nx + pj) * nr);
    for (int r = 0; r < nr / 4; ++r) {
      const float4 w = lw[r];
      if (w.x == 0.0f && w.y == 0.0f && w.z == 0.0f && w.w == 0.0f) continue;
      const int4 ix = li[r];
      atomicAdd(&row[ix.x], P * w.x);
      atomicAdd(&row[ix.y], P * w.y);
      atomicAdd(&row[ix.z], P * w.z);
      atomicAdd(&row[ix.w], P * w.w);
    }
  }
  __syncwarp();
  const float wq = (float)S.wgt[q];
  float *gq = pd.g + ((size_t)b * pd.max_nd + qr) * pd.ldg;
  for (int k = lane; k < ns; k += 32) gq[k] = row[k] * wq;
  if (lane == 0) gq[ns] = ws.pix_dres[(size_t)b * max_pix + q] * wq;
}

// lower triangle of g^T g over the (N_s + 1) columns: tile (ti, tj), tj <= ti
__global__ void __launch_bounds__(PIX_THREADS, 3) k_pix_gram(const SysDev *__restrict__ sysv,
                                                          const int *__restrict__ sys_id, WsDev ws,
                                                          PixDev pd) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (!S.src_pix) return;
  const int n1 = S.spx_ns + 1, nt = (n1 + 63) / 64;
  int ti = 0, rest = blockIdx.x;
  while (rest > ti) {
    rest -= ti + 1;
    ++ti;
  }
  const int tj = rest;
  if (ti >= nt) return;
  __shared__ __align__(16) float As[16][64], Bs[16][64];
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  const int nd = S.n_mask;
  const float *g = pd.g + (size_t)b * pd.max_nd * pd.ldg;
  // FP32 sums over 256 rows, carried across them in double-float (hi, lo) pairs (FP32
  // TwoSum: FP64 adds would hold the FP64 unit ~64 cycles per warp instruction, all warps at
  // once at every flush)
  float acc[4][4], sh[4][4], sl[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[u][v] = sh[u][v] = sl[u][v] = 0.0f;
  const int lr = tid >> 4, lc = (tid & 15) * 4;  // loader: row lr, columns lc .. lc + 3
  const float4 z4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  for (int q0 = 0, ch = 0; q0 < nd; q0 += 16, ++ch) {
    const int qq = q0 + lr;
    // g's rows start on 16-byte boundaries (ldg a multiple of 4) and lc is a multiple of 4:
    // one float4 per matrix where the four columns exist, else element by element
    const int ca = ti * 64 + lc, cb = tj * 64 + lc;
    const float *ga = g + (size_t)qq * pd.ldg + ca, *gb = g + (size_t)qq * pd.ldg + cb;
    float4 a4 = z4, b4 = z4;
    if (qq < nd) {
      if (ca + 3 < n1) a4 = *reinterpret_cast<const float4 *>(ga);
      else {
        a4.x = ca < n1 ? ga[0] : 0.0f;
        a4.y = ca + 1 < n1 ? ga[1] : 0.0f;
        a4.z = ca + 2 < n1 ? ga[2] : 0.0f;
      }
      if (cb + 3 < n1) b4 = *reinterpret_cast<const float4 *>(gb);
      else {
        b4.x = cb < n1 ? gb[0] : 0.0f;
        b4.y = cb + 1 < n1 ? gb[1] : 0.0f;
        b4.z = cb + 2 < n1 ? gb[2] : 0.0f;
      }
    }
    *reinterpret_cast<float4 *>(&As[lr][lc]) = a4;
    *reinterpret_cast<float4 *>(&Bs[lr][lc]) = b4;
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      const float4 a4 = *reinterpret_cast<const float4 *>(&As[r][ty * 4]);
      const float4 b4 = *reinterpret_cast<const float4 *>(&Bs[r][tx * 4]);
      const float av[4] = {a4.x, a4.y, a4.z, a4.w}, bv[4] = {b4.x, b4.y, b4.z, b4.w};
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
    }
    __syncthreads();
    if ((ch & 15) == 15) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          // (sh, sl) += acc: TwoSum of sh and acc, the error into sl
          const float t = __fadd_rn(sh[u][v], acc[u][v]);
          const float w = __fsub_rn(t, sh[u][v]);
          const float e = __fadd_rn(__fsub_rn(sh[u][v], __fsub_rn(t, w)), __fsub_rn(acc[u][v], w));
          sh[u][v] = t;
          sl[u][v] = __fadd_rn(sl[u][v], e);
          acc[u][v] = 0.0f;
        }
    }
  }
  double *F = pd.F + (size_t)b * pd.ldg * pd.ldg;
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int i = ti * 64 + ty * 4 + u, j = tj * 64 + tx * 4 + v;
      if (i < n1 && j <= i)
        F[(size_t)i * pd.ldg + j] = ((double)sh[u][v] + (double)sl[u][v]) + (double)acc[u][v];
    }
}

// the data row of the Gram matrix again, to ~48 bits: D_j = sum_q g_qj g_qn and d^T C_D^-1 d
// (the data term -(d^T C_D^-1 d - D^T s_MP)/2 of ln P is a difference of sums that each reach
// ~N_d times the noise level: their FP32 rounding would move ln P by ~1e-6 of them)
__global__ void __launch_bounds__(PIX_THREADS) k_pix_dcol(const SysDev *__restrict__ sysv,
                                                          const int *__restrict__ sys_id, WsDev ws,
                                                          PixDev pd) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (!S.src_pix) return;
  const int n = S.spx_ns, j = blockIdx.x * PIX_THREADS + threadIdx.x;
  if (j > n) return;
  const float *g = pd.g + (size_t)b * pd.max_nd * pd.ldg;
  // each product of two floats is exact as p + pe (FMA); the sum runs in double-float (Knuth's
  // TwoSum, errors gathered in lo) on the FP32 pipe rather than as FP64 multiply-adds
  float hi = 0.0f, lo = 0.0f;
  for (int q = 0; q < S.n_mask; ++q) {
    const float *gq = g + (size_t)q * pd.ldg;
    const float a = gq[j], c = gq[n];
    const float p = __fmul_rn(a, c), pe = __fmaf_rn(a, c, -p);
    const float t = __fadd_rn(hi, p), w = __fsub_rn(t, hi);
    const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, w)), __fsub_rn(p, w));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(pe, e));
  }
  pd.F[(size_t)b * pd.ldg * pd.ldg + (size_t)n * pd.ldg + j] = (double)hi + (double)lo;
}

__global__ void k_pix_init(const SysDev *__restrict__ sysv, const int *__restrict__ sys_id,
                           WsDev ws, PixDev pd, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (!S.src_pix) return;
  brent_start(pd.srch[b], S.spx_tlo, S.spx_thi);
}

// ---------------------------------------------------------------------------------------
// The evidence evaluation.  The factorisation runs on the augmented matrix
//     M = [ F + lambda C    . ]     (N_s + 1 rows, row stride N_s + 1, lower triangle)
//         [ D^T             . ]
// whose Cholesky factor's last row is y^T = (L^-1 D)^T: row N_s is one more panel row of
// every step (its pivot is never taken), so the forward solve comes out of the factorisation.
// Everything on a step's critical path is double-float on the FP32 pipes (a warp's FP64
// instruction holds this GPU's FP64 unit for ~64 cycles, and these paths are sequential): the
// pivots' square roots and reciprocals (FP32 seeds refined by one Newton step in double-float,
// doubling their 24 bits), the pivots' log-product (mantissas multiplied in double-float,
// binary exponents summed, one FP64 log per evaluation), the panels and the backward solve.

// sqrt(d) for d > 0: s0 = sqrt(d.hi) in FP32, then s0 + (d - s0^2) / (2 s0) (Newton's step for
// s^2 = d), the residual exact to its last bits: s0^2 = p + pe exactly (FMA), and d.hi - p is
// exact because p lies within an ulp or two of d.hi (Sterbenz)
__device__ __forceinline__ float2 df_sqrt(float2 d) {
  const float s0 = sqrtf(d.x);
  const float p = __fmul_rn(s0, s0);
  const float pe = __fmaf_rn(s0, s0, -p);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(d.x, p), pe), d.y);
  const float c = __fmul_rn(r, __frcp_rn(__fmul_rn(2.0f, s0)));
  const float h = __fadd_rn(s0, c);
  return make_float2(h, __fsub_rn(c, __fsub_rn(h, s0)));
}

// 1 / l: r0 = 1 / l.hi in FP32, then r0 + r0 (1 - l r0) (Newton's step for 1/x), the residual
// 1 - l.hi r0 exact by FMA
__device__ __forceinline__ float2 df_rcp(float2 l) {
  const float r0 = __frcp_rn(l.x);
  float e = __fmaf_rn(-l.x, r0, 1.0f);
  e = __fmaf_rn(-l.y, r0, e);
  const float c = __fmul_rn(r0, e);
  const float h = __fadd_rn(r0, c);
  return make_float2(h, __fsub_rn(c, __fsub_rn(h, r0)));
}

__device__ __forceinline__ float2 shfl_f2(float2 v, int src) {
  return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}

// is sample b evaluated in this pass, and at which ln lambda
__device__ __forceinline__ bool pix_active(const SysDev &S, const WsDev &ws, const PixDev &pd,
                                          int b, int final_pass, double &t) {
  if (ws.status[b] != GLAD_SAMPLE_OK || !S.src_pix) return false;
  const PixSearch *sp = pd.srch + b;
  const int phase = sp->phase;
  if (!final_pass && phase == 2) return false;
  t = (final_pass || phase == 0) ? sp->x : sp->u;
  return true;
}

__device__ __forceinline__ float2 *pix_A(const PixDev &pd, int b) {
  return pd.A + (size_t)b * (pd.max_ns + 1) * (pd.max_ns + 1);
}

// C = H^T H entry (p, q): H stacks the second differences along x and along y (zero outside
// the grid), so C = I (x) Dx^T Dx + Dy^T Dy (x) I with D the 1-D second difference, whose
// D^T D has 6 on the diagonal (5 at the two ends), -4 one off it and 1 two off it
__device__ __forceinline__ double pix_curv(const SysDev &S, int p, int q) {
  const int nx = S.spx_nx, pi = p / nx, pj = p - pi * nx, qi = q / nx, qj = q - qi * nx;
  auto dtd = [](int a, int b, int m) {
    const int k = abs(a - b);
    return k == 0 ? 4 + (a > 0) + (a + 1 < m) : k == 1 ? -4 : k == 2 ? 1 : 0;
  };
  return (double)((pi == qi ? dtd(pj, qj, nx) : 0) + (pj == qj ? dtd(pi, qi, S.spx_ny) : 0));
}

// M: rows i < N_s get F + lambda C, row N_s gets D (row N_s of the Gram matrix), lower
// triangle without column N_s, over the elements first, first + step, ...
__device__ __forceinline__ void pix_assemble(const SysDev &S, const PixDev &pd, int b, double lam,
                                             size_t first, size_t step) {
  const int n = S.spx_ns, ldg = pd.ldg, lda = n + 1;
  const double *F = pd.F + (size_t)b * ldg * ldg;
  float2 *A = pix_A(pd, b);
  for (size_t e = first; e < (size_t)(n + 1) * n; e += step) {
    const int i = (int)(e / n), j = (int)(e - (size_t)i * n);
    if (j > i) continue;
    const double v = i < n ? F[(size_t)i * ldg + j] + lam * pix_curv(S, i, j) : F[(size_t)n * ldg + j];
    A[(size_t)i * lda + j] = df_split(v);
  }
}

// the diagonal block at (k0, k0) (kb <= 32 pivots) factored in shared memory by the whole CTA
// in double-float, right-looking with one barrier per pivot: every thread computes pivot j
// itself (sqrt and reciprocal of the updated diagonal entry, which step j does not write) and
// updates its elements (i, c), j < c <= i, by L_ij L_cj with L_xj = a_xj / L_jj formed on the
// fly; the columns are scaled at the end.  Ds holds the block's factor on return (identity
// beyond kb), Rs the pivots' reciprocals; *bad is set on a pivot that is not positive (taken
// as 1).
template <int NT>
__device__ __forceinline__ void pix_diag(const float2 *A, int lda, int k0, int kb, float2 (*Ds)[33],
                                         float2 *Rs, int *bad) {
  static_assert(NT % 32 == 0 && 1024 % NT == 0, "CTA size");
  constexpr int EPT = 1024 / NT;  // block elements per thread
  const int tid = threadIdx.x;
  __shared__ float2 Ls[32];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = tid + q * NT, i = e >> 5, j = e & 31;
    Ds[i][j] = (i < kb && j <= i) ? A[(size_t)(k0 + i) * lda + k0 + j]
                                  : make_float2(i == j ? 1.0f : 0.0f, 0.0f);
  }
  __syncthreads();
  for (int j = 0; j < kb; ++j) {
    float2 d = Ds[j][j];
    if (!(d.x > 0.0f)) d = make_float2(1.0f, 0.0f);
    const float2 l = df_sqrt(d);
    const float2 r = df_rcp(l);
    if (tid == 0) {
      if (!(Ds[j][j].x > 0.0f)) *bad = 1;
      Ls[j] = l;
      Rs[j] = r;
    }
    // warp w takes rows i > j with i = w mod (NT / 32), lane c column c (active for c in (j, i])
    constexpr int NW = NT / 32;
    const int w = tid >> 5, c = tid & 31;
    const float2 lcj = df_mul(Ds[c][j], r);
    for (int i = j + 1 + ((w - (j + 1)) % NW + NW) % NW; i < kb; i += NW) {
      if (c > j && c <= i) {
        const float2 lij = df_mul(Ds[i][j], r);
        float hi = 0.0f, lo = 0.0f;
        df_fma(hi, lo, lij, lcj);
        Ds[i][c] = df_sub(Ds[i][c], hi, lo);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = tid + q * NT, i = e >> 5, j = e & 31;
    if (j < kb && i < kb) {
      if (i == j) Ds[i][j] = Ls[j];
      else if (i > j) Ds[i][j] = df_mul(Ds[i][j], Rs[j]);
    }
  }
  __syncthreads();
}

// warp 0: the product of the block's pivots folded into (pm, pe) = pm * 2^pe held by lane 0
// (each pivot's mantissa in [1/2, 1) and exponent apart, a product tree over the lanes)
__device__ __forceinline__ void pix_pivot_product(const float2 (*Ds)[33], int kb, float2 &pm, int &pe) {
  const int lane = threadIdx.x & 31;
  float2 v = make_float2(1.0f, 0.0f);
  int e = 0;
  if (lane < kb) {
    const float2 l = Ds[lane][lane];
    const float f = frexpf(l.x, &e);
    v = make_float2(f, ldexpf(l.y, -e));
  }
  for (int off = 16; off > 0; off >>= 1) {
    v = df_mul(v, make_float2(__shfl_xor_sync(0xffffffffu, v.x, off),
                              __shfl_xor_sync(0xffffffffu, v.y, off)));
    e += __shfl_xor_sync(0xffffffffu, e, off);
  }
  if (lane == 0) {
    pm = df_mul(pm, v);
    int e2;
    const float f = frexpf(pm.x, &e2);
    pm = make_float2(f, ldexpf(pm.y, -e2));
    pe += e + e2;
  }
}

// sum ln L_ii from the pivots' product pm * 2^pe
__device__ __forceinline__ double pix_half_logdet(float2 pm, int pe) {
  return log((double)pm.x + (double)pm.y) + pe * M_LN2;
}

// panel rows i = first, first + step, ... below last: x L11^T = a, in double-float (the
// divisions as products with the pivots' reciprocals), each thread's row staged in its column
// of X[32][NT] in shared memory: the loops stay rolled (a fully unrolled 32-column triangle in
// registers is ~7k instructions, which the instruction cache does not hold)
template <int NT>
__device__ __forceinline__ void pix_panel_rows_smem(float2 *A, int lda, int k0, int kb,
                                                    const float2 (*Ds)[33], const float2 *Rs,
                                                    float2 (*X)[NT], int first, int last, int step) {
  const int t = threadIdx.x;
  for (int i = first; i < last; i += step) {
    float2 *ai = A + (size_t)i * lda + k0;
#pragma unroll
    for (int m = 0; m < 32; ++m)
      if (m < kb) X[m][t] = ai[m];
    for (int m = 0; m < kb; ++m) {
      float hi = 0.0f, lo = 0.0f;
#pragma unroll 4
      for (int q = 0; q < m; ++q) df_fma(hi, lo, X[q][t], Ds[m][q]);
      X[m][t] = df_mul(df_sub(X[m][t], hi, lo), Rs[m]);
    }
#pragma unroll
    for (int m = 0; m < 32; ++m)
      if (m < kb) ai[m] = X[m][t];
  }
}

// the same with the row in registers (fully unrolled; the one-CTA-per-sample kernel, which has
// no room for X, and whose other CTA on the SM covers the instruction fetches)
__device__ __forceinline__ void pix_panel_rows(float2 *A, int lda, int k0, int kb,
                                               const float2 (*Ds)[33], const float2 *Rs, int first,
                                               int last, int step) {
  for (int i = first; i < last; i += step) {
    float2 xs[32];
    float2 *ai = A + (size_t)i * lda + k0;
#pragma unroll
    for (int m = 0; m < 32; ++m) {
      xs[m] = make_float2(0.0f, 0.0f);
      if (m < kb) {
        float hi = 0.0f, lo = 0.0f;
#pragma unroll
        for (int qd = 0; qd < m; ++qd) df_fma(hi, lo, xs[qd], Ds[m][qd]);
        xs[m] = df_mul(df_sub(ai[m], hi, lo), Rs[m]);
      }
    }
#pragma unroll
    for (int m = 0; m < 32; ++m)
      if (m < kb) ai[m] = xs[m];
  }
}

// trailing tile (ti, tj) of the panel step at k0, rows from r0 = k0 + kb below nr = N_s + 1,
// columns below N_s: M[gi][gj] -= sum_m L[gi][k0 + m] L[gj][k0 + m], in double-float
template <int NT>
__device__ __forceinline__ void pix_tile_compute(float2 *A, int lda, int n, int r0, int ti, int tj,
                                                 const float2 (*Pi)[33], const float2 (*Pj)[33]);

template <int NT>
__device__ __forceinline__ void pix_tile(float2 *A, int lda, int n, int k0, int kb, int r0, int ti,
                                         int tj, float2 (*Pi)[33], float2 (*Pj)[33]) {
  static_assert(NT == 256, "16 x 16 threads, 4 x 4 outputs each");
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < 64 * 32 / NT; ++q) {
    const int e = tid + q * NT, r = e >> 5, m = e & 31;
    const int gi = r0 + ti * 64 + r, gj = r0 + tj * 64 + r;
    const float2 z = make_float2(0.0f, 0.0f);
    Pi[r][m] = (gi <= n && m < kb) ? A[(size_t)gi * lda + k0 + m] : z;
    Pj[r][m] = (gj < n && m < kb) ? A[(size_t)gj * lda + k0 + m] : z;
  }
  __syncthreads();
  pix_tile_compute<NT>(A, lda, n, r0, ti, tj, Pi, Pj);
  __syncthreads();
}

// 8-byte asynchronous copies global -> shared (cp.async; zero-filled when !pred, the source
// address then only has to be valid), their commit and wait
__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, bool pred) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(pred ? 8 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// the panel rows of tile (ti, tj) into Pi, Pj by asynchronous copies (one commit group)
template <int NT>
__device__ __forceinline__ void pix_tile_fetch(const float2 *A, int lda, int n, int k0, int kb, int r0,
                                               int ti, int tj, float2 (*Pi)[33], float2 (*Pj)[33]) {
  const int tid = threadIdx.x;
#pragma unroll
  for (int q = 0; q < 64 * 32 / NT; ++q) {
    const int e = tid + q * NT, r = e >> 5, m = e & 31;
    const int gi = r0 + ti * 64 + r, gj = r0 + tj * 64 + r;
    const bool pi = gi <= n && m < kb, pj = gj < n && m < kb;
    cp_async8(&Pi[r][m], pi ? A + (size_t)gi * lda + k0 + m : A, pi);
    cp_async8(&Pj[r][m], pj ? A + (size_t)gj * lda + k0 + m : A, pj);
  }
  cp_async_commit();
}

// tile idx of the lower triangle with tj >= 1, row-major over (ti - 1, tj - 1)
__device__ __forceinline__ void pix_rest_tile(int idx, int &ti, int &tj) {
  int u = (int)((sqrt(8.0 * idx + 1.0) - 1.0) * 0.5);
  while (u * (u + 1) / 2 > idx) --u;
  while ((u + 1) * (u + 2) / 2 <= idx) ++u;
  ti = u + 1;
  tj = idx - u * (u + 1) / 2 + 1;
}

template <int NT>
__device__ __forceinline__ void pix_tile_compute(float2 *A, int lda, int n, int r0, int ti, int tj,
                                                 const float2 (*Pi)[33], const float2 (*Pj)[33]) {
  const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
  float ah[4][4], al[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) ah[u][v] = al[u][v] = 0.0f;
  // thread (ty, tx) owns rows ty + 16u and columns tx + 16v: a warp's Pj reads then fall on
  // consecutive rows (row stride 33 pairs: distinct banks) and its stores on consecutive columns
#pragma unroll 4
  for (int m = 0; m < 32; ++m) {
    float2 av[4], bv[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      av[u] = Pi[ty + 16 * u][m];
      bv[u] = Pj[tx + 16 * u][m];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) df_fma(ah[u][v], al[u][v], av[u], bv[v]);
  }
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const int gi = r0 + ti * 64 + ty + 16 * u, gj = r0 + tj * 64 + tx + 16 * v;
      if (gi <= n && gj <= gi && gj < n)
        A[(size_t)gi * lda + gj] = df_sub(A[(size_t)gi * lda + gj], ah[u][v], al[u][v]);
    }
}

// one block of the backward solve L^T s = y (y in row N_s of M, updated in place): warp 0
// solves the block's kb unknowns into sb (and into s when s is given), then rows i = first,
// first + step, ... below k0 take y_i -= sum_m L[k0 + m][i] s[k0 + m]; all in double-float
template <int NT>
__device__ __forceinline__ void pix_bsolve_block(const float2 *A, int lda, int n, const float2 *rd,
                                                 float2 *s, int k0, int kb, int first, int step,
                                                 float2 (*Lb)[33], float2 *rb, float2 *sb) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float2 *y = const_cast<float2 *>(A) + (size_t)n * lda;
  // the block's factor and reciprocals staged first (Lb[32][33], rb[32] in shared memory): no
  // global load inside the sequential loop
#pragma unroll
  for (int q = 0; q < 32 * 32 / NT; ++q) {
    const int e = threadIdx.x + q * NT, i = e >> 5, c = e & 31;
    if (i < kb && c <= i) Lb[i][c] = A[(size_t)(k0 + i) * lda + k0 + c];
  }
  if (threadIdx.x < kb) rb[threadIdx.x] = rd[k0 + threadIdx.x];
  __syncthreads();
  if (warp == 0) {
    float2 v = lane < kb ? y[k0 + lane] : make_float2(0.0f, 0.0f);
    for (int j = kb - 1; j >= 0; --j) {
      const float2 sj = df_mul(shfl_f2(v, j), rb[j]);
      if (lane == j) v = sj;
      if (lane < j) {
        float hi = 0.0f, lo = 0.0f;
        df_fma(hi, lo, Lb[j][lane], sj);
        v = df_sub(v, hi, lo);
      }
    }
    sb[lane] = lane < kb ? v : make_float2(0.0f, 0.0f);
    if (s && lane < kb) s[k0 + lane] = v;
  }
  __syncthreads();
  for (int i = first; i < k0; i += step) {
    float hi = 0.0f, lo = 0.0f;
#pragma unroll
    for (int m = 0; m < 32; ++m)
      if (m < kb) df_fma(hi, lo, A[(size_t)(k0 + m) * lda + i], sb[m]);
    y[i] = df_sub(y[i], hi, lo);
  }
  __syncthreads();
}

// this thread's share of |H s|^2 (C = H^T H: second differences along x and y, zero outside
// the grid) over the pixels first, first + step, ...
__device__ __forceinline__ double pix_es_part(const SysDev &S, const float2 *s, int first, int step) {
  double es = 0.0;
  auto sv = [&](int p) { return df_val(s[p]); };
  for (int p = first; p < S.spx_ns; p += step) {
    const int i = p / S.spx_nx, j = p - i * S.spx_nx;
    const double c2 = -2.0 * sv(p);
    const double hx = c2 + (j > 0 ? sv(p - 1) : 0.0) + (j + 1 < S.spx_nx ? sv(p + 1) : 0.0);
    const double hy = c2 + (i > 0 ? sv(p - S.spx_nx) : 0.0) + (i + 1 < S.spx_ny ? sv(p + S.spx_nx) : 0.0);
    es = fma(hx, hx, fma(hy, hy, es));
  }
  return es;
}

// the sum of squared residuals (f_q s - d_q)^2 / sigma_q^2 over the masked rows q0, q0 + qstep,
// ... below q1, one warp per row (lane 0 holds the warp's share): the dot products in
// double-float against s_MP
__device__ __forceinline__ double pix_ed_rows(const SysDev &S, const PixDev &pd, int b,
                                              const float2 *ys, int q0, int q1, int qstep) {
  const int lane = threadIdx.x & 31, n = S.spx_ns, ldg = pd.ldg;
  const float *g = pd.g + (size_t)b * pd.max_nd * ldg;
  double ed = 0.0;
  for (int q = q0; q < q1; q += qstep) {
    const float *gq = g + (size_t)q * ldg;
    float hi = 0.0f, lo = 0.0f;
    for (int k = lane; k < n; k += 32) df_fma(hi, lo, make_float2(gq[k], 0.0f), ys[k]);
    double r = (double)hi + (double)lo;
    for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    r -= (double)gq[n];
    if (lane == 0) ed = fma(r, r, ed);
  }
  return ed;
}

// sum over the CTA of v (the result in thread 0)
template <int NT>
__device__ __forceinline__ double pix_block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < NT / 32; ++w) s += red[w];
  return s;
}

// ln P from its parts, then one step of the search (thread 0 of the sample's last kernel);
// *open counts the samples whose search goes on after this pass
__device__ __forceinline__ void pix_conclude(const SysDev &S, const PixDev &pd, int b, double t,
                                             double half_logdet, int bad, double ES, double ED,
                                             int *open) {
  const double lnP = -ED - exp(t) * ES - half_logdet + 0.5 * S.spx_ns * t + S.spx_const;
  const double phi = (bad || !isfinite(lnP)) ? INFINITY : -lnP;
  brent_step(pd.srch[b], phi, S.spx_iters);
  if (pd.nfac) atomicAdd(pd.nfac, 1ull);
  if (open && pd.srch[b].phase != 2) atomicAdd(open, 1);
}

// ---------------------------------------------------------------------------------------
// One evidence evaluation per sample at its pending ln lambda, one CTA per sample, in one
// launch (glad_set_pix_path mode 1; final_pass: at the best point, with s_MP written to
// s_out[b * s_stride ..]).
__global__ void __launch_bounds__(PIX_THREADS, 2) k_pix_eval(const SysDev *__restrict__ sysv,
                                                          const int *__restrict__ sys_id, WsDev ws,
                                                          PixDev pd, int final_pass, double *s_out,
                                                          int s_stride, int *open) {
  const int b = blockIdx.x;
  const SysDev &S = sysv[sys_id[b]];
  double t;
  if (!pix_active(S, ws, pd, b, final_pass, t)) return;
  const int n = S.spx_ns, lda = n + 1, tid = threadIdx.x;
  float2 *A = pix_A(pd, b);
  float2 *rd = pd.rd + (size_t)b * pd.max_ns, *s = pd.s + (size_t)b * pd.max_ns;
  pix_assemble(S, pd, b, exp(t), tid, PIX_THREADS);
  __shared__ float2 Ds[32][33], Rs[32], sb[32];
  __shared__ float2 Pi[64][33], Pj[64][33];  // (hi, lo) pairs of the panel rows
  __shared__ double red[PIX_THREADS / 32];
  __shared__ int bad;
  if (tid == 0) bad = 0;
  float2 pm = make_float2(1.0f, 0.0f);  // product of the pivots, pm * 2^pe (thread 0)
  int pe = 0;
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += 32) {
    const int kb = min(32, n - k0), r0 = k0 + kb;
    pix_diag<PIX_THREADS>(A, lda, k0, kb, Ds, Rs, &bad);
    if (tid < 32) pix_pivot_product(Ds, kb, pm, pe);
    if (tid < kb) rd[k0 + tid] = Rs[tid];
    for (int e = tid; e < 32 * 32; e += PIX_THREADS) {
      const int i = e >> 5, j = e & 31;
      if (i < kb && j <= i) A[(size_t)(k0 + i) * lda + k0 + j] = Ds[i][j];
    }
    pix_panel_rows(A, lda, k0, kb, Ds, Rs, r0 + tid, n + 1, PIX_THREADS);
    __syncthreads();
    // trailing update M22 -= L21 L21^T, 64 x 64 tiles
    const int T = (n + 1 - r0 + 63) / 64;
    for (int ti = 0; ti < T; ++ti)
      for (int tj = 0; tj <= ti; ++tj) pix_tile<PIX_THREADS>(A, lda, n, k0, kb, r0, ti, tj, Pi, Pj);
  }
  for (int k0 = ((n - 1) / 32) * 32; k0 >= 0; k0 -= 32)
    pix_bsolve_block<PIX_THREADS>(A, lda, n, rd, s, k0, min(32, n - k0), tid, PIX_THREADS, Pi, Pj[0],
                                  sb);
  if (final_pass) {
    if (s_out)
      for (int i = tid; i < n; i += PIX_THREADS) s_out[(size_t)b * s_stride + i] = df_val(s[i]);
    return;
  }
  const double es = pix_es_part(S, s, tid, PIX_THREADS);
  const double ed = pix_ed_rows(S, pd, b, s, tid >> 5, S.n_mask, PIX_THREADS / 32);
  const double ES = pix_block_sum<PIX_THREADS>(es, red);
  const double ED = pix_block_sum<PIX_THREADS>(ed, red);
  if (tid == 0) pix_conclude(S, pd, b, t, pix_half_logdet(pm, pe), bad, 0.5 * ES, 0.5 * ED, open);
}

// ---------------------------------------------------------------------------------------
// The same evaluation as a sequence of launches (the default form, faster than one CTA per
// sample at every batch size measured): the kernel boundaries order the steps, and each step
// spreads over many CTAs per sample (grid y = sample).
//   k_pixm_begin    M assembled; the sample's pivot product and flag reset
//   per 32-column panel step k0:
//     k_pixm_panel    every CTA factors the diagonal block (read from M, which nothing writes
//                     in this launch) and solves its share of the panel rows (row N_s among
//                     them); CTA 0 keeps the factored block in dgf, the reciprocals in rd, and
//                     folds the pivots into the sample's product
//     k_pixm_trail    the 64 x 64 tiles of tile column 0 (next diagonal block and panel), one
//                     per CTA; CTA 0 also moves dgf into M's diagonal block (which nothing
//                     else touches in this launch)
//     k_pixm_rest     the other tiles, several per CTA, on a second, low-priority stream
//                     beside tile column 0 and the next panel (the lookahead)
//   per 32-row block of the backward solve, from the bottom:
//     k_pixm_bsolve   every CTA solves the block (its y entries are not written in this
//                     launch), CTA 0 writes s_MP there, each CTA updates its share of y above
//   k_pixm_es       E_S (or, in the final pass, s_MP to the caller)
//   k_pixm_ed       E_D over chunks of PIXM_ED_ROWS masked rows, one partial sum per chunk
//   k_pixm_fin      the partials summed in order, ln P, one search step

__global__ void __launch_bounds__(PIX_THREADS) k_pixm_begin(const SysDev *__restrict__ sysv,
                                                          const int *__restrict__ sys_id, WsDev ws,
                                                          PixDev pd, int final_pass) {
  const int b = blockIdx.y;
  const SysDev &S = sysv[sys_id[b]];
  double t;
  if (!pix_active(S, ws, pd, b, final_pass, t)) return;
  pix_assemble(S, pd, b, exp(t), (size_t)blockIdx.x * PIX_THREADS + threadIdx.x,
               (size_t)gridDim.x * PIX_THREADS);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    pd.pm[b] = make_float2(1.0f, 0.0f);
    pd.pe[b] = 0;
    pd.bad[b] = 0;
  }
}

__global__ void __launch_bounds__(PIXM_PANEL_THREADS) k_pixm_panel(const SysDev *__restrict__ sysv,
                                                                 const int *__restrict__ sys_id,
                                                                 WsDev ws, PixDev pd, int final_pass,
                                                                 int k0) {
  constexpr int NT = PIXM_PANEL_THREADS;
  const int b = blockIdx.y;
  const SysDev &S = sysv[sys_id[b]];
  double t;
  if (!pix_active(S, ws, pd, b, final_pass, t)) return;
  const int n = S.spx_ns;
  if (k0 >= n) return;
  const int kb = min(32, n - k0), r0 = k0 + kb, lda = n + 1, tid = threadIdx.x;
  if (blockIdx.x > 0 && r0 + (int)blockIdx.x * NT > n) return;
  float2 *A = pix_A(pd, b);
  __shared__ float2 Ds[32][33], Rs[32];
  __shared__ float2 X[32][NT];
  __shared__ int bad;
  if (tid == 0) bad = 0;
  __syncthreads();
  pix_diag<NT>(A, lda, k0, kb, Ds, Rs, &bad);
  if (blockIdx.x == 0) {
    float2 *dst = pd.dgf + (size_t)b * 32 * 32;
    for (int e = tid; e < 32 * 32; e += NT) dst[e] = Ds[e >> 5][e & 31];
    if (tid < kb) pd.rd[(size_t)b * pd.max_ns + k0 + tid] = Rs[tid];
    if (tid < 32) {
      float2 pm = pd.pm[b];
      int pe = pd.pe[b];
      pix_pivot_product(Ds, kb, pm, pe);
      if (tid == 0) {
        pd.pm[b] = pm;
        pd.pe[b] = pe;
        if (bad) pd.bad[b] = 1;
      }
    }
  }
  pix_panel_rows_smem<NT>(A, lda, k0, kb, Ds, Rs, X, r0 + blockIdx.x * NT + tid, n + 1, gridDim.x * NT);
}

// The tiles of tile column 0 (the next diagonal block and panel among them), one per CTA; CTA 0
// also moves the factored diagonal block from dgf into M.
__global__ void __launch_bounds__(PIX_THREADS, 3) k_pixm_trail(const SysDev *__restrict__ sysv,
                                                             const int *__restrict__ sys_id, WsDev ws,
                                                             PixDev pd, int final_pass, int k0) {
  const int b = blockIdx.y;
  const SysDev &S = sysv[sys_id[b]];
  double t;
  if (!pix_active(S, ws, pd, b, final_pass, t)) return;
  const int n = S.spx_ns;
  if (k0 >= n) return;
  const int kb = min(32, n - k0), r0 = k0 + kb, lda = n + 1;
  float2 *A = pix_A(pd, b);
  if (blockIdx.x == 0) {
    const float2 *src = pd.dgf + (size_t)b * 32 * 32;
    for (int e = threadIdx.x; e < 32 * 32; e += PIX_THREADS) {
      const int i = e >> 5, j = e & 31;
      if (i < kb && j <= i) A[(size_t)(k0 + i) * lda + k0 + j] = src[e];
    }
  }
  const int T = (n + 1 - r0 + 63) / 64;
  if ((int)blockIdx.x >= T) return;
  __shared__ float2 Pi[64][33], Pj[64][33];
  pix_tile<PIX_THREADS>(A, lda, n, k0, kb, r0, blockIdx.x, 0, Pi, Pj);
}

// The other tiles (tj >= 1), which the next panel step does not read: CTA x takes tiles x,
// x + gridDim.x, ... of its sample, the next tile's panel rows copied into the second shared
// buffer (cp.async) while the current one is computed.  Dynamic shared memory: two stages of
// Pi, Pj (PIXM_REST_SMEM bytes).
__global__ void __launch_bounds__(PIX_THREADS, 3) k_pixm_rest(const SysDev *__restrict__ sysv,
                                                            const int *__restrict__ sys_id, WsDev ws,
                                                            PixDev pd, int final_pass, int k0) {
  const int b = blockIdx.y;
  const SysDev &S = sysv[sys_id[b]];
  double t;
  if (!pix_active(S, ws, pd, b, final_pass, t)) return;
  const int n = S.spx_ns;
  if (k0 >= n) return;
  const int kb = min(32, n - k0), r0 = k0 + kb, lda = n + 1;
  const int T = (n + 1 - r0 + 63) / 64, ntile = T * (T - 1) / 2;
  int idx = blockIdx.x;
  if (idx >= ntile) return;
  float2 *A = pix_A(pd, b);
  extern __shared__ float2 pbuf[];
  auto P = [&](int stage, int which) {
    return reinterpret_cast<float2(*)[33]>(pbuf + (size_t)(2 * stage + which) * 64 * 33);
  };
  int ti, tj;
  pix_rest_tile(idx, ti, tj);
  pix_tile_fetch<PIX_THREADS>(A, lda, n, k0, kb, r0, ti, tj, P(0, 0), P(0, 1));
  for (int stage = 0; idx < ntile; idx += gridDim.x, stage ^= 1) {
    const int next = idx + gridDim.x;
    int ni = 0, nj = 0;
    if (next < ntile) {
      pix_rest_tile(next, ni, nj);
      pix_tile_fetch<PIX_THREADS>(A, lda, n, k0, kb, r0, ni, nj, P(stage ^ 1, 0), P(stage ^ 1, 1));
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    pix_tile_compute<PIX_THREADS>(A, lda, n, r0, ti, tj, P(stage, 0), P(stage, 1));
    __syncthreads();  // this stage is refilled two tiles on
    ti = ni;
    tj = nj;
  }
}

__global__ void __launch_bounds__(PIX_THREADS) k_pixm_bsolve(const SysDev *__restrict__ sysv,
                                                           const int *__restrict__ sys_id, WsDev ws,
                                                           PixDev pd, int final_pass, int k0) {
  const int b = blockIdx.y;
  const SysDev &S = sysv[sys_id[b]];
  double t;
  if (!pix_active(S, ws, pd, b, final_pass, t)) return;
  const int n = S.spx_ns;
  if (k0 >= n) return;
  if (blockIdx.x > 0 && (int)blockIdx.x * PIX_THREADS >= k0) return;
  __shared__ float2 Lb[32][33], rb[32], sb[32];
  pix_bsolve_block<PIX_THREADS>(pix_A(pd, b), n + 1, n, pd.rd + (size_t)b * pd.max_ns,
                                blockIdx.x == 0 ? pd.s + (size_t)b * pd.max_ns : nullptr, k0,
                                min(32, n - k0), blockIdx.x * PIX_THREADS + threadIdx.x,
                                gridDim.x * PIX_THREADS, Lb, rb, sb);
}

__global__ void __launch_bounds__(PIX_THREADS) k_pixm_es(const SysDev *__restrict__ sysv,
                                                       const int *__restrict__ sys_id, WsDev ws,
                                                       PixDev pd, int final_pass, double *s_out,
                                                       int s_stride) {
  const int b = blockIdx.x;
  const SysDev &S = sysv[sys_id[b]];
  double t;
  if (!pix_active(S, ws, pd, b, final_pass, t)) return;
  const float2 *s = pd.s + (size_t)b * pd.max_ns;
  if (final_pass) {
    if (s_out)
      for (int i = threadIdx.x; i < S.spx_ns; i += PIX_THREADS) s_out[(size_t)b * s_stride + i] = df_val(s[i]);
    return;
  }
  __shared__ double red[PIX_THREADS / 32];
  const double ES = pix_block_sum<PIX_THREADS>(pix_es_part(S, s, threadIdx.x, PIX_THREADS), red);
  if (threadIdx.x == 0) pd.es[b] = ES;
}

__global__ void __launch_bounds__(PIX_THREADS) k_pixm_ed(const SysDev *__restrict__ sysv,
                                                       const int *__restrict__ sys_id, WsDev ws,
                                                       PixDev pd) {
  const int b = blockIdx.y;
  const SysDev &S = sysv[sys_id[b]];
  double t;
  if (!pix_active(S, ws, pd, b, 0, t)) return;
  const int q0 = blockIdx.x * PIXM_ED_ROWS;
  if (q0 >= S.n_mask) return;
  __shared__ double red[PIX_THREADS / 32];
  const double ed = pix_ed_rows(S, pd, b, pd.s + (size_t)b * pd.max_ns, q0 + (threadIdx.x >> 5),
                                min(S.n_mask, q0 + PIXM_ED_ROWS), PIX_THREADS / 32);
  const double ED = pix_block_sum<PIX_THREADS>(ed, red);
  if (threadIdx.x == 0) pd.edp[(size_t)b * pd.ed_chunks + blockIdx.x] = ED;
}

__global__ void k_pixm_fin(const SysDev *__restrict__ sysv, const int *__restrict__ sys_id,
                           WsDev ws, PixDev pd, int B, int *open) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const SysDev &S = sysv[sys_id[b]];
  double t;
  if (!pix_active(S, ws, pd, b, 0, t)) return;
  const int nch = (S.n_mask + PIXM_ED_ROWS - 1) / PIXM_ED_ROWS;
  double ED = 0.0;
  for (int c = 0; c < nch; ++c) ED += pd.edp[(size_t)b * pd.ed_chunks + c];
  pix_conclude(S, pd, b, t, pix_half_logdet(pd.pm[b], pd.pe[b]), pd.bad[b], 0.5 * pd.es[b], 0.5 * ED,
               open);
}

// the image term of logL: terms[0] = -2 ln P at the best lambda
__global__ void k_pix_finish(const SysDev *__restrict__ sysv, const int *__restrict__ sys_id,
                             WsDev ws, PixDev pd, int B, double *lam_out, double *lnP_out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (!S.src_pix) return;
  const PixSearch &s = pd.srch[b];
  ws.terms[4 * (size_t)b] = 2.0 * s.fx;
  if (lam_out) lam_out[b] = exp(s.x);
  if (lnP_out) lnP_out[b] = -s.fx;
}

}  // namespace

cudaError_t pixsrc_ws_ensure(glad_ctx *c, int B) {
  if (!c->n_pix) return cudaSuccess;
  if (!c->pws) c->pws = new PixWs();
  PixWs &w = *c->pws;
  if (!w.aux) {
    int dev = 0, nsm = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    w.slots = 3 * nsm;
    if (cudaFuncSetAttribute(k_pixm_rest, cudaFuncAttributeMaxDynamicSharedMemorySize, PIXM_REST_SMEM) !=
        cudaSuccess)
      return cudaErrorInvalidValue;
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (cudaStreamCreateWithPriority(&w.hi, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&w.aux, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&w.ev_p, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&w.ev_r, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&w.ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&w.ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&w.ev_grp[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&w.ev_grp[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaMalloc(&w.d_open, sizeof(int) * (SPX_MAX_ITERS + 1)) != cudaSuccess ||
        cudaHostAlloc(&w.h_open, sizeof(int) * (SPX_MAX_ITERS + 1), cudaHostAllocDefault) != cudaSuccess)
      return cudaErrorMemoryAllocation;
  }
  if (w.B >= B) return cudaSuccess;
  B = std::max(B, w.B);
  cudaDeviceSynchronize();
  for (void *p : w.allocs) cudaFree(p);
  w.allocs.clear();
  w.B = 0;
  const int ldg = ((c->max_ns + 1) + 3) / 4 * 4;
  const size_t b = B;
  auto take = [&](void **p, size_t bytes) {
    if (cudaMalloc(p, bytes) != cudaSuccess) {
      *p = nullptr;
      return false;
    }
    w.allocs.push_back(*p);
    return true;
  };
  PixDev &d = w.d;
  d.ldg = ldg;
  d.max_ns = c->max_ns;
  d.max_nd = c->max_nd;
  d.ed_chunks = (c->max_nd + PIXM_ED_ROWS - 1) / PIXM_ED_ROWS;
  const bool ok = take((void **)&d.g, sizeof(float) * b * c->max_nd * ldg) &&
                  take((void **)&d.F, sizeof(double) * b * ldg * ldg) &&
                  take((void **)&d.A, sizeof(float2) * b * (c->max_ns + 1) * (c->max_ns + 1)) &&
                  take((void **)&d.s, sizeof(float2) * b * c->max_ns) &&
                  take((void **)&d.rd, sizeof(float2) * b * c->max_ns) &&
                  take((void **)&d.srch, sizeof(PixSearch) * b) &&
                  take((void **)&d.nfac, sizeof(unsigned long long)) &&
                  take((void **)&d.pm, sizeof(float2) * b) &&
                  take((void **)&d.pe, sizeof(int) * b) &&
                  take((void **)&d.bad, sizeof(int) * b) &&
                  take((void **)&d.es, sizeof(double) * b) &&
                  take((void **)&d.edp, sizeof(double) * b * d.ed_chunks) &&
                  take((void **)&d.dgf, sizeof(float2) * b * 32 * 32);
  if (!ok) {
    for (void *p : w.allocs) cudaFree(p);
    w.allocs.clear();
    return cudaErrorMemoryAllocation;
  }
  cudaMemset(d.nfac, 0, sizeof(unsigned long long));
  w.B = B;
  return cudaSuccess;
}

void pixsrc_ws_free(glad_ctx *c) {
  if (!c->pws) return;
  for (void *p : c->pws->allocs) cudaFree(p);
  for (cudaEvent_t e : {c->pws->ev_p, c->pws->ev_r, c->pws->ev_in, c->pws->ev_out, c->pws->ev_grp[0],
                        c->pws->ev_grp[1]})
    if (e) cudaEventDestroy(e);
  if (c->pws->d_open) cudaFree(c->pws->d_open);
  if (c->pws->h_open) cudaFreeHost(c->pws->h_open);
  if (c->pws->hi) cudaStreamDestroy(c->pws->hi);
  if (c->pws->aux) cudaStreamDestroy(c->pws->aux);
  delete c->pws;
  c->pws = nullptr;
}

// the multi-launch form unless the context fixes the one-CTA-per-sample kernel: measured at
// 16 to 1,184 samples of the 30 x 30 grid (RXJ1131 scale), it is the faster one throughout,
// by 3.6x at 16 samples and 7 % at 1,184
bool pixsrc_multi_launch(glad_ctx *c, int B) {
  (void)B;
  return c->tune.pix_path != 1;
}

unsigned long long pixsrc_launches(glad_ctx *c) {
  if (!c->pws) return 0;
  const unsigned long long n = c->pws->launches;
  c->pws->launches = 0;
  return n;
}

unsigned long long pixsrc_factorizations(glad_ctx *c) {
  if (!c->pws || !c->pws->d.nfac) return 0;
  unsigned long long n = 0;
  cudaMemcpy(&n, c->pws->d.nfac, sizeof(n), cudaMemcpyDeviceToHost);
  cudaMemset(c->pws->d.nfac, 0, sizeof(n));
  return n;
}

cudaError_t launch_pixsrc(glad_ctx *c, const int *sys_id, int B, cudaStream_t st,
                          double *lam_out, double *lnP_out, double *s_out) {
  PixWs &w = *c->pws;
  const PixDev &pd = w.d;
  int max_iter = 0, max_tri = 0;
  for (auto &sd : c->h_sysdev)
    if (sd.src_pix) {
      max_iter = std::max(max_iter, sd.spx_iters);
      const int nt = (sd.spx_ns + 1 + 63) / 64;
      max_tri = std::max(max_tri, nt * (nt + 1) / 2);
    }
  const size_t fsm = sizeof(float) * PIX_F_WARPS * pd.ldg;
  cudaError_t e = cudaSuccess;
  if (fsm > 48 * 1024)
    e = cudaFuncSetAttribute(k_pix_f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm);
  if (e != cudaSuccess) return e;
  auto op = [&]() -> cudaError_t {
    k_pix_f<<<dim3((c->max_nd + PIX_F_WARPS - 1) / PIX_F_WARPS, B), PIX_F_WARPS * 32, fsm, st>>>(
        c->d_sys, sys_id, c->ws.d, pd, c->max_pix);
    ++w.launches;
    k_pix_gram<<<dim3(max_tri, B), PIX_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d, pd);
    ++w.launches;
    k_pix_dcol<<<dim3((c->max_ns + PIX_THREADS) / PIX_THREADS, B), PIX_THREADS, 0, st>>>(
        c->d_sys, sys_id, c->ws.d, pd);
    ++w.launches;
    return cudaGetLastError();
  };
  // one evaluation per sample: one CTA per sample, or the multi-launch form
  const bool multi = pixsrc_multi_launch(c, B);
  // the multi-launch form runs on the context's high-priority stream q, forked from st
  const cudaStream_t q = multi ? w.hi : st;
  auto eval = [&](int final_pass, double *so, int *open) {
    if (!multi) {
      k_pix_eval<<<B, PIX_THREADS, 0, q>>>(c->d_sys, sys_id, c->ws.d, pd, final_pass, so,
                                           GLAD_MAX_SRCPIX, open);
      ++w.launches;
      return;
    }
    // the grids from the largest system (smaller ones leave the extra CTAs idle)
    const int ns = pd.max_ns;
    const int nbeg = std::max(1, (int)(((size_t)(ns + 1) * ns + PIX_THREADS * 16 - 1) / (PIX_THREADS * 16)));
    k_pixm_begin<<<dim3(nbeg, B), PIX_THREADS, 0, q>>>(c->d_sys, sys_id, c->ws.d, pd, final_pass);
    ++w.launches;
    // Lookahead: the tiles of tile column 0 of step k (which hold step k + 1's diagonal block
    // and panel) run on q, then panel k + 1, while the other tiles of step k run on the
    // low-priority stream beside them.  Tile column 0 of step k + 1 waits for those: its
    // columns, 32 to the right of step k's, overlap step k's tile column 1.  (Each wait
    // follows a record of the same pass: the sequence captures into a graph.)
    bool side_work = false;
    for (int k0 = 0; k0 < ns; k0 += 32) {
      const int rows = std::max(1, ns + 1 - k0 - 32);  // panel rows, row N_s among them
      const int T = (rows + 63) / 64;
      const int np = (rows + PIXM_PANEL_THREADS - 1) / PIXM_PANEL_THREADS;
      k_pixm_panel<<<dim3(np, B), PIXM_PANEL_THREADS, 0, q>>>(c->d_sys, sys_id, c->ws.d, pd,
                                                              final_pass, k0);
      ++w.launches;
      if (T > 1) cudaEventRecord(w.ev_p, q);
      if (side_work) cudaStreamWaitEvent(q, w.ev_r, 0);
      k_pixm_trail<<<dim3(T, B), PIX_THREADS, 0, q>>>(c->d_sys, sys_id, c->ws.d, pd, final_pass, k0);
      ++w.launches;
      side_work = T > 1;
      if (side_work) {
        // tiles per CTA: enough CTAs for one wave of three per SM, at most PIXM_REST_TPC tiles
        // each for up to 32 samples and one for larger batches (late in the search only a few
        // samples are still open, and their tiles then need many CTAs each; measured at 64
        // samples: 488 logL/s with one, 469 with two)
        const long rest = (long)T * (T - 1) / 2;
        const long cap = B <= 32 ? PIXM_REST_TPC : 1;
        const int tpc = (int)std::min<long>(cap, std::max<long>(1, (rest * B + w.slots - 1) / w.slots));
        cudaStreamWaitEvent(w.aux, w.ev_p, 0);
        k_pixm_rest<<<dim3((int)((rest + tpc - 1) / tpc), B), PIX_THREADS, PIXM_REST_SMEM, w.aux>>>(
            c->d_sys, sys_id, c->ws.d, pd, final_pass, k0);
        ++w.launches;
        cudaEventRecord(w.ev_r, w.aux);
      }
    }
    if (side_work) cudaStreamWaitEvent(q, w.ev_r, 0);
    for (int k0 = ((ns - 1) / 32) * 32; k0 >= 0; k0 -= 32) {
      k_pixm_bsolve<<<dim3(std::max(1, (k0 + PIX_THREADS - 1) / PIX_THREADS), B), PIX_THREADS, 0, q>>>(
          c->d_sys, sys_id, c->ws.d, pd, final_pass, k0);
      ++w.launches;
    }
    k_pixm_es<<<B, PIX_THREADS, 0, q>>>(c->d_sys, sys_id, c->ws.d, pd, final_pass, so, GLAD_MAX_SRCPIX);
    ++w.launches;
    if (!final_pass) {
      k_pixm_ed<<<dim3(pd.ed_chunks, B), PIX_THREADS, 0, q>>>(c->d_sys, sys_id, c->ws.d, pd);
      ++w.launches;
      k_pixm_fin<<<(B + 127) / 128, 128, 0, q>>>(c->d_sys, sys_id, c->ws.d, pd, B, open);
      ++w.launches;
    }
  };
  auto ev = [&]() -> cudaError_t {
    if (multi) {
      cudaEventRecord(w.ev_in, st);
      cudaStreamWaitEvent(q, w.ev_in, 0);
    }
    k_pix_init<<<(B + 127) / 128, 128, 0, q>>>(c->d_sys, sys_id, c->ws.d, pd, B);
    ++w.launches;
    // The first pass evaluates the starting point, each later one a trial point.  Under graph
    // capture all max_iter passes are recorded (converged samples return at once).  Otherwise
    // the passes go out in groups of PIX_GROUP, each group's last count of open searches is
    // copied to the host, and after enqueueing group g + 1 the host waits for group g: when no
    // search is open the call ends there, so at most one group of idle passes runs.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(st, &cs);
    if (cs != cudaStreamCaptureStatusNone) {
      for (int it = 0; it < max_iter; ++it) eval(0, nullptr, nullptr);
    } else {
      cudaError_t e2 = cudaMemsetAsync(w.d_open, 0, sizeof(int) * max_iter, q);
      if (e2 != cudaSuccess) return e2;
      int it = 0, g = 0;
      auto group = [&](int gi) -> cudaError_t {
        for (int k = 0; k < PIX_GROUP && it < max_iter; ++k, ++it) eval(0, nullptr, w.d_open + it);
        cudaMemcpyAsync(w.h_open + gi % 2, w.d_open + it - 1, sizeof(int), cudaMemcpyDeviceToHost, q);
        return cudaEventRecord(w.ev_grp[gi % 2], q);
      };
      if ((e2 = group(0)) != cudaSuccess) return e2;
      while (it < max_iter) {
        if ((e2 = group(g + 1)) != cudaSuccess) return e2;
        if ((e2 = cudaEventSynchronize(w.ev_grp[g % 2])) != cudaSuccess) return e2;
        if (w.h_open[g % 2] == 0) break;
        ++g;
      }
    }
    k_pix_finish<<<(B + 127) / 128, 128, 0, q>>>(c->d_sys, sys_id, c->ws.d, pd, B, lam_out, lnP_out);
    ++w.launches;
    if (s_out) eval(1, s_out, nullptr);
    if (multi) {
      cudaEventRecord(w.ev_out, q);
      cudaStreamWaitEvent(st, w.ev_out, 0);
    }
    return cudaGetLastError();
  };
  e = GLAD_PROF(c, st, KID_PIX_OP, op());
  if (e != cudaSuccess) return e;
  return GLAD_PROF(c, st, KID_PIX_EV, ev());
}
