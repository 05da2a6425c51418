// Pixelated source reconstruction (Sect. 3.1.1, Eqs. dpre, s_MP, evi_ext; Table 1).
//  k_image (k_lens.cu) leaves, for every image pixel of a pixelated-source system, the
//    bilinear grid entries of its ss^2 rays (the lensing operator L), and the PSF kernels the
//    arcs d_esr = data - B (lens light).
//  k_pix_f: one warp per masked pixel q builds row q of the response f = B L (the PSF taps
//    around q gather their pixels' ray entries into a shared row of N_s) and stores
//    g_q = [f_q, d_q] / sigma_q in FP32.
//  k_pix_gram: [F D; D^T d^T C_D^-1 d] = g^T g, lower triangle, 64 x 64 tiles: FP32 products
//    summed in FP32 over 256 rows and in FP64 across them; k_pix_dcol then redoes the data
//    row (D and d^T C_D^-1 d) with FP64 sums.
//  k_pix_eval: one CTA per sample (two resident per SM): A = F + lambda C, blocked Cholesky (32-wide panels,
//    64 x 64 trailing tiles), s_MP by the two triangular solves, and the log-evidence
//      ln P = -E_D - lambda E_S - sum ln L_ii + (N_s/2) ln lambda + const,
//    E_D = |f s_MP - d|^2 / 2 (units of sigma) from the residuals of the masked pixels,
//    E_S = |H s_MP|^2 / 2 (both in FP64), then one step of Brent's minimisation of -ln P over
//    ln lambda; its last pass writes s_MP for the caller.  E_D + lambda E_S is stationary at
//    s_MP, so an error in s_MP moves it only at second order; written as the difference
//    d^T C_D^-1 d - D^T s_MP it would lose ~1e-8 of two sums that reach N_d (S/N)^2.
// The factorisation keeps ~FP64 accuracy because the evidence needs ln det(F + lambda C) to
// ~1e-2 absolute over N_s ~ 1e3 pivots of a matrix whose conditioning grows as lambda falls:
// the matrix, the diagonal blocks, the panels and the solves are FP64, and the trailing update
// (nearly all of the N_s^3/3 flops) runs in double-float on the FP32 pipes, since this GPU's
// FP64 rate is 1/73 of its FP32 rate with or without tensor cores.
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
  double *A;            // [B * max_ns * max_ns] F + lambda C and its factor (row stride N_s),
                        // held as double-float (hi, lo) pairs of floats
  double *y;            // [B * max_ns]
  PixSearch *srch;      // [B]
  unsigned long long *nfac;  // [1] factorisations run
  int ldg, max_ns, max_nd;
};

struct PixWs {
  int B = 0;
  PixDev d{};
  std::vector<void *> allocs;
};

namespace {

constexpr double GOLD = 0.3819660112501051;  // (3 - sqrt 5) / 2
constexpr double TTOL = 1e-3;                // tolerance in ln lambda (ln P moves by ~P"/2 TTOL^2)

#define PIX_F_WARPS 8
#define PIX_THREADS 256

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
__global__ void __launch_bounds__(PIX_THREADS) k_pix_gram(const SysDev *__restrict__ sysv,
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
  float acc[4][4];
  double acc64[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      acc[u][v] = 0.0f;
      acc64[u][v] = 0.0;
    }
  const int lr = tid >> 4, lc = (tid & 15) * 4;  // loader: row lr, columns lc .. lc + 3
  for (int q0 = 0, ch = 0; q0 < nd; q0 += 16, ++ch) {
    const int qq = q0 + lr;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int ca = ti * 64 + lc + k, cb = tj * 64 + lc + k;
      As[lr][lc + k] = (qq < nd && ca < n1) ? g[(size_t)qq * pd.ldg + ca] : 0.0f;
      Bs[lr][lc + k] = (qq < nd && cb < n1) ? g[(size_t)qq * pd.ldg + cb] : 0.0f;
    }
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
          acc64[u][v] += (double)acc[u][v];
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
      if (i < n1 && j <= i) F[(size_t)i * pd.ldg + j] = acc64[u][v] + (double)acc[u][v];
    }
}

// the data row of the Gram matrix again in FP64: D_j = sum_q g_qj g_qn and d^T C_D^-1 d
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
  double acc = 0.0;
  for (int q = 0; q < S.n_mask; ++q) {
    const float *gq = g + (size_t)q * pd.ldg;
    acc = fma((double)gq[j], (double)gq[n], acc);
  }
  pd.F[(size_t)b * pd.ldg * pd.ldg + (size_t)n * pd.ldg + j] = acc;
}

__global__ void k_pix_init(const SysDev *__restrict__ sysv, const int *__restrict__ sys_id,
                           WsDev ws, PixDev pd, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (!S.src_pix) return;
  brent_start(pd.srch[b], S.spx_tlo, S.spx_thi);
}

// One evidence evaluation per sample at its pending ln lambda (final_pass: at the best one,
// with s_MP written to s_out[b * s_stride ..]).
__global__ void __launch_bounds__(PIX_THREADS, 2) k_pix_eval(const SysDev *__restrict__ sysv,
                                                          const int *__restrict__ sys_id, WsDev ws,
                                                          PixDev pd, int final_pass, double *s_out,
                                                          int s_stride) {
  const int b = blockIdx.x;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (!S.src_pix) return;
  PixSearch *sp = pd.srch + b;
  const int phase = sp->phase;
  if (!final_pass && phase == 2) return;
  const double t = (final_pass || phase == 0) ? sp->x : sp->u;
  const double lam = exp(t);
  const int n = S.spx_ns, ldg = pd.ldg;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const double *F = pd.F + (size_t)b * ldg * ldg;
  // the matrix and its factor as double-float (hi, lo) pairs (8 bytes, as a double)
  float2 *A = reinterpret_cast<float2 *>(pd.A + (size_t)b * pd.max_ns * pd.max_ns);
  double *y = pd.y + (size_t)b * pd.max_ns;
  // A = F + lambda C (lower triangle), y = D (row N_s of the Gram matrix)
  for (size_t e = tid; e < (size_t)n * n; e += PIX_THREADS) {
    const int i = (int)(e / n), j = (int)(e - (size_t)i * n);
    if (j <= i) A[e] = df_split(F[(size_t)i * ldg + j] + lam * S.spx_C[e]);
  }
  for (int i = tid; i < n; i += PIX_THREADS) y[i] = F[(size_t)n * ldg + i];
  __shared__ double Dg[32][33];
  __shared__ float2 Pi[64][33], Pj[64][33];  // (hi, lo) pairs of the panel rows
  __shared__ double red[PIX_THREADS / 32];
  __shared__ int bad;
  if (tid == 0) bad = 0;
  double half_logdet = 0.0;  // sum ln L_ii (thread 0)
  __syncthreads();
  for (int k0 = 0; k0 < n; k0 += 32) {
    const int kb = min(32, n - k0);
    // diagonal block, factored by warp 0
    for (int e = tid; e < 32 * 32; e += PIX_THREADS) {
      const int i = e >> 5, j = e & 31;
      Dg[i][j] = (i < kb && j <= i) ? df_val(A[(size_t)(k0 + i) * n + k0 + j]) : (i == j ? 1.0 : 0.0);
    }
    __syncthreads();
    if (warp == 0) {
      for (int j = 0; j < kb; ++j) {
        if (lane == j) {
          double d = Dg[j][j];
          if (!(d > 0.0)) {
            bad = 1;
            d = 1.0;
          }
          Dg[j][j] = sqrt(d);
        }
        __syncwarp();
        if (lane > j && lane < kb) Dg[lane][j] /= Dg[j][j];
        __syncwarp();
        if (lane > j && lane < kb) {
          const double lij = Dg[lane][j];
          for (int cc = j + 1; cc <= lane; ++cc) Dg[lane][cc] -= lij * Dg[cc][j];
        }
        __syncwarp();
      }
    }
    __syncthreads();
    if (tid == 0)
      for (int j = 0; j < kb; ++j) half_logdet += log(Dg[j][j]);
    // panel below the block: x L11^T = a, row by row; the sums in double-float against the
    // block's (hi, lo) copy (kept in Pi's space until the trailing update), the divisions in
    // FP64
    float2(*Dgs)[33] = Pi;
    for (int e = tid; e < 32 * 32; e += PIX_THREADS) {
      const int i = e >> 5, j = e & 31;
      Dgs[i][j] = df_split(Dg[i][j]);
      if (i < kb && j <= i) A[(size_t)(k0 + i) * n + k0 + j] = Dgs[i][j];
    }
    __syncthreads();
    const int r0 = k0 + kb;
    for (int i = r0 + tid; i < n; i += PIX_THREADS) {
      float2 xs[32];
      float2 *ai = A + (size_t)i * n + k0;
#pragma unroll
      for (int m = 0; m < 32; ++m) {
        xs[m] = make_float2(0.0f, 0.0f);
        if (m < kb) {
          float hi = 0.0f, lo = 0.0f;
#pragma unroll
          for (int qd = 0; qd < m; ++qd) df_fma(hi, lo, xs[qd], Dgs[m][qd]);
          xs[m] = df_split((df_val(ai[m]) - ((double)hi + (double)lo)) / Dg[m][m]);
        }
      }
#pragma unroll
      for (int m = 0; m < 32; ++m)
        if (m < kb) ai[m] = xs[m];
    }
    __syncthreads();
    // trailing update A22 -= L21 L21^T, lower triangle, 64 x 64 tiles
    const int T = (n - r0 + 63) / 64;
    const int ty = tid >> 4, tx = tid & 15;
    for (int ti = 0; ti < T; ++ti)
      for (int tj = 0; tj <= ti; ++tj) {
        for (int e = tid; e < 64 * 32; e += PIX_THREADS) {
          const int r = e >> 5, m = e & 31;
          const int gi = r0 + ti * 64 + r, gj = r0 + tj * 64 + r;
          const float2 z = make_float2(0.0f, 0.0f);
          Pi[r][m] = (gi < n && m < kb) ? A[(size_t)gi * n + k0 + m] : z;
          Pj[r][m] = (gj < n && m < kb) ? A[(size_t)gj * n + k0 + m] : z;
        }
        __syncthreads();
        float ah[4][4], al[4][4];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) ah[u][v] = al[u][v] = 0.0f;
#pragma unroll 4
        for (int m = 0; m < 32; ++m) {
          float2 av[4], bv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            av[u] = Pi[ty * 4 + u][m];
            bv[u] = Pj[tx * 4 + u][m];
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
            const int gi = r0 + ti * 64 + ty * 4 + u, gj = r0 + tj * 64 + tx * 4 + v;
            if (gi < n && gj <= gi) A[(size_t)gi * n + gj] = df_sub(A[(size_t)gi * n + gj], ah[u][v], al[u][v]);
          }
        __syncthreads();
      }
  }
  // y = L^-1 D, 32 rows at a time: warp 0 solves the block, the CTA updates the rows below
  for (int k0 = 0; k0 < n; k0 += 32) {
    const int kb = min(32, n - k0);
    if (warp == 0) {
      double yv = lane < kb ? y[k0 + lane] : 0.0;
      for (int j = 0; j < kb; ++j) {
        const double yj = __shfl_sync(0xffffffffu, yv, j) / df_val(A[(size_t)(k0 + j) * n + k0 + j]);
        if (lane == j) yv = yj;
        if (lane > j && lane < kb) yv -= df_val(A[(size_t)(k0 + lane) * n + k0 + j]) * yj;
      }
      if (lane < kb) y[k0 + lane] = yv;
    }
    __syncthreads();
    for (int i = k0 + kb + tid; i < n; i += PIX_THREADS) {
      const float2 *ai = A + (size_t)i * n + k0;
      double sacc = 0.0;
      for (int m = 0; m < kb; ++m) sacc = fma(df_val(ai[m]), y[k0 + m], sacc);
      y[i] -= sacc;
    }
    __syncthreads();
  }
  // s_MP: L^T s = y from the bottom, 32 rows at a time
  for (int k0 = ((n - 1) / 32) * 32; k0 >= 0; k0 -= 32) {
    const int kb = min(32, n - k0);
    if (warp == 0) {
      double sv = lane < kb ? y[k0 + lane] : 0.0;
      for (int j = kb - 1; j >= 0; --j) {
        const double sj = __shfl_sync(0xffffffffu, sv, j) / df_val(A[(size_t)(k0 + j) * n + k0 + j]);
        if (lane == j) sv = sj;
        if (lane < j) sv -= df_val(A[(size_t)(k0 + j) * n + k0 + lane]) * sj;
      }
      if (lane < kb) y[k0 + lane] = sv;
    }
    __syncthreads();
    for (int i = tid; i < k0; i += PIX_THREADS) {
      double sacc = 0.0;
      for (int m = 0; m < kb; ++m) sacc = fma(df_val(A[(size_t)(k0 + m) * n + i]), y[k0 + m], sacc);
      y[i] -= sacc;
    }
    __syncthreads();
  }
  if (final_pass) {
    if (s_out)
      for (int i = tid; i < n; i += PIX_THREADS) s_out[(size_t)b * s_stride + i] = y[i];
    return;
  }
  // E_S = |H s|^2 / 2 (C = H^T H: second differences along x and y, zero outside the grid)
  double es = 0.0;
  for (int p = tid; p < n; p += PIX_THREADS) {
    const int i = p / S.spx_nx, j = p - i * S.spx_nx;
    const double c2 = -2.0 * y[p];
    const double hx = c2 + (j > 0 ? y[p - 1] : 0.0) + (j + 1 < S.spx_nx ? y[p + 1] : 0.0);
    const double hy = c2 + (i > 0 ? y[p - S.spx_nx] : 0.0) + (i + 1 < S.spx_ny ? y[p + S.spx_nx] : 0.0);
    es = fma(hx, hx, fma(hy, hy, es));
  }
  // E_D = |f s - d|^2 / 2 in units of sigma, from the residuals themselves: the difference
  // d^T C_D^-1 d - D^T s_MP of two sums ~ N_d (S/N)^2 would cancel to ~1e-8 of them
  // (the rows' dot products in double-float against s_MP split in place into (hi, lo))
  __syncthreads();
  float2 *ys = reinterpret_cast<float2 *>(y);
  for (int i = tid; i < n; i += PIX_THREADS) {
    const double v = y[i];
    ys[i] = df_split(v);
  }
  __syncthreads();
  double ed = 0.0;
  const float *g = pd.g + (size_t)b * pd.max_nd * ldg;
  for (int q = warp; q < S.n_mask; q += PIX_THREADS / 32) {
    const float *gq = g + (size_t)q * ldg;
    float hi = 0.0f, lo = 0.0f;
    for (int k = lane; k < n; k += 32) df_fma(hi, lo, make_float2(gq[k], 0.0f), ys[k]);
    double r = (double)hi + (double)lo;
    for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    r -= (double)gq[n];
    if (lane == 0) ed = fma(r, r, ed);
  }
  for (int off = 16; off > 0; off >>= 1) {
    es += __shfl_xor_sync(0xffffffffu, es, off);
    ed += __shfl_xor_sync(0xffffffffu, ed, off);
  }
  __shared__ double red2[PIX_THREADS / 32];
  if (lane == 0) {
    red[warp] = es;
    red2[warp] = ed;
  }
  __syncthreads();
  if (tid == 0) {
    double ES = 0.0, ED = 0.0;
    for (int w = 0; w < PIX_THREADS / 32; ++w) {
      ES += red[w];
      ED += red2[w];
    }
    ES *= 0.5;
    ED *= 0.5;
    const double lnP = -ED - lam * ES - half_logdet + 0.5 * n * t + S.spx_const;
    const double phi = (bad || !isfinite(lnP)) ? INFINITY : -lnP;
    brent_step(*sp, phi, S.spx_iters);
    if (pd.nfac) atomicAdd(pd.nfac, 1ull);
  }
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
  const bool ok = take((void **)&d.g, sizeof(float) * b * c->max_nd * ldg) &&
                  take((void **)&d.F, sizeof(double) * b * ldg * ldg) &&
                  take((void **)&d.A, sizeof(double) * b * c->max_ns * c->max_ns) &&
                  take((void **)&d.y, sizeof(double) * b * c->max_ns) &&
                  take((void **)&d.srch, sizeof(PixSearch) * b) &&
                  take((void **)&d.nfac, sizeof(unsigned long long));
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
  delete c->pws;
  c->pws = nullptr;
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
  const PixDev &pd = c->pws->d;
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
    k_pix_gram<<<dim3(max_tri, B), PIX_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d, pd);
    k_pix_dcol<<<dim3((c->max_ns + PIX_THREADS) / PIX_THREADS, B), PIX_THREADS, 0, st>>>(
        c->d_sys, sys_id, c->ws.d, pd);
    return cudaGetLastError();
  };
  auto ev = [&]() -> cudaError_t {
    k_pix_init<<<(B + 127) / 128, 128, 0, st>>>(c->d_sys, sys_id, c->ws.d, pd, B);
    // the first pass evaluates the starting point, each later one a trial point
    for (int it = 0; it < max_iter; ++it)
      k_pix_eval<<<B, PIX_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d, pd, 0, nullptr, 0);
    k_pix_finish<<<(B + 127) / 128, 128, 0, st>>>(c->d_sys, sys_id, c->ws.d, pd, B, lam_out, lnP_out);
    if (s_out)
      k_pix_eval<<<B, PIX_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d, pd, 1, s_out, GLAD_MAX_SRCPIX);
    return cudaGetLastError();
  };
  e = GLAD_PROF(c, st, KID_PIX_OP, op());
  if (e != cudaSuccess) return e;
  return GLAD_PROF(c, st, KID_PIX_EV, ev());
}
