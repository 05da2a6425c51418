// Lensing half of the likelihood (FP32 bulk, FP64 chi^2):
//  k_image: one thread per image pixel; each of its ss x ss sub-pixels is ray-shot
//    through EPL + shear + SIS, scaled by lambda_int and joined by the internal mass sheet
//    for systems that have one (Sect. 3.3) (lens equation beta = theta - alpha, Sect. 3.1.1),
//    the Sersic source is evaluated at beta and the lens-light Sersics at theta,
//    and the average is stored.
//  k_conv: PSF blurring (discrete convolution, zero outside the image) of a 32x8
//    output tile staged with its halo in shared memory, and the masked pixel chi^2
//    (Eq. chi2 of lens_light) reduced in FP64 per sample.
#include <algorithm>

#include "glad_internal.cuh"

namespace {

// system geometry in the ray shooting's float type: pixel scale, source axis ratio and angle
struct SrcGeom {
  float pix, q, c, s;
};
struct SrcGeom64 {
  double pix, q, c, s;
};
__device__ __forceinline__ SrcGeom geom_of(const SysDev &S, float) {
  return {S.pix, S.src_q, S.src_cphi, S.src_sphi};
}
__device__ __forceinline__ SrcGeom64 geom_of(const SysDev &S, double) {
  return {S.pix64, S.src_q64, S.src_cphi64, S.src_sphi64};
}

// float / double versions of the few functions the ray shooting uses
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ const LensPT<float> *lp_of(const WsDev &w, float) { return w.lp; }
__device__ __forceinline__ const LensPT<double> *lp_of(const WsDev &w, double) { return w.lp64; }
__device__ __forceinline__ float *img_of(const WsDev &w, float) { return w.img; }
__device__ __forceinline__ double *img_of(const WsDev &w, double) { return w.img64; }

template <class T>
__device__ __forceinline__ T sersic_f(T R2_scaled, T Ie, T ninv, T bn) {
  // Ie * exp(-bn * (R^(1/n) - 1)) with R2_scaled = (R/Re)^2
  const T w = exp2(T(0.5) * ninv * log2(R2_scaled));
  return Ie * exp(-bn * (w - T(1)));
}

// Composite galaxy (Sect. 3.3) at frame position (xp, yp): adds to the frame deflection.
// Softened isothermal ellipsoid pair of each Chameleon, b = 2 q A (A = Upsilon L_scale I0/(1+q)):
//   alpha = b/e (arctan(e x/(psi + s)), arctanh(e y/(psi + q^2 s))), psi = sqrt(q^2 (s^2 + x^2) + y^2),
// its round limit 2 A (x, y)/(sqrt(R^2 + s^2) + s) for e < 1e-3; halo CSE i (amplitude amp, core s):
//   alpha = 2 q amp (x (psi + q^2 s), y (psi + s)) / (s psi D), D = (psi + s)^2 + (1 - q^2) x^2
// (the y denominator q^2 D written without the cancelling form).
template <class T>
__device__ __forceinline__ void composite_frame(const LensPT<T> &L, int n_lcomp, T xp, T yp, T &ax,
                                                T &ay) {
  for (int c = 0; c < n_lcomp && c < 4; ++c) {
    const T q = L.ch_q[c], e = L.ch_e[c], A = L.ch_A[c];
    T sx = T(0.0), sy = T(0.0);
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const T s = t == 0 ? L.ch_sc[c] : L.ch_st[c];
      const T sg = t == 0 ? T(1.0) : -T(1.0);
      if (e > 1e-3f) {
        const T ps = sqrt(q * q * (s * s + xp * xp) + yp * yp);
        const T b = T(2.0) * q * A / e;
        sx += sg * b * atan(e * xp / (ps + s));
        sy += sg * b * atanh(e * yp / (ps + q * q * s));
      } else {
        const T fac = T(2.0) * A / (sqrt(xp * xp + yp * yp + s * s) + s);
        sx += sg * fac * xp;
        sy += sg * fac * yp;
      }
    }
    ax += sx;
    ay += sy;
  }
  const T q = L.h_q, q2 = q * q;
  const T base = q2 * xp * xp + yp * yp, ex2 = L.h_e2 * xp * xp;
  T hx = T(0.0), hy = T(0.0);
  for (int i = 0; i < GLAD_N_CSE; ++i) {
    const T s = L.cse_sc[i], amp = L.cse_amp[i];
    const T ps = sqrt(base + q2 * s * s);
    const T D = (ps + s) * (ps + s) + ex2;
    const T w = amp / (s * ps * D);
    hx += w * (ps + q2 * s);
    hy += w * (ps + s);
  }
  ax += T(2.0) * q * xp * hx;
  ay += T(2.0) * q * yp * hy;
}

// Round Gaussian black hole of mass M: alpha = M (1 - e^-t)/(pi R^2) (dx, dy), t = R^2/(2 sigma^2)
template <class T>
__device__ __forceinline__ T bh_gauss_factor(T M, T s2x2, T dx, T dy) {
  const T t = (dx * dx + dy * dy) / s2x2;
  const T h1 = t < 1e-3f ? T(1.0) - T(0.5) * t : -expm1(-t) / t;
  return M * h1 / (T(3.14159265358979) * s2x2);
}

template <class T>
__global__ void __launch_bounds__(LENS_THREADS) k_image(const SysDev *__restrict__ sysv,
                                                        const int *__restrict__ sys_id, WsDev ws,
                                                        int max_pix) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  const int p = blockIdx.x * LENS_THREADS + threadIdx.x;
  __shared__ LensPT<T> L;
  {
    const int *src = reinterpret_cast<const int *>(&lp_of(ws, T(0))[b]);
    int *dst = reinterpret_cast<int *>(&L);
    for (int i = threadIdx.x; i < (int)(sizeof(LensPT<T>) / 4); i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  if (p >= S.npix) return;
  const int i = p / S.nx, j = p - i * S.nx;
  const int ss = S.ss;
  const auto G = geom_of(S, T(0));
  const T pix = G.pix;
  const T x0 = (j - T(0.5) * (S.nx - 1)) * pix;
  const T y0 = (i - T(0.5) * (S.ny - 1)) * pix;
  const T q = L.q, omt = T(1.0) - L.t;
  T acc = T(0.0);
  for (int my = 0; my < ss; ++my) {
    const T y = y0 + ((my + T(0.5)) / ss - T(0.5)) * pix;
    for (int mx = 0; mx < ss; ++mx) {
      const T x = x0 + ((mx + T(0.5)) / ss - T(0.5)) * pix;
      const T dx = x - L.xc, dy = y - L.yc;
      const T xp = L.cphi * dx + L.sphi * dy, yp = -L.sphi * dx + L.cphi * dy;
      T apx = T(0.0), apy = T(0.0);
      if (L.mclass == 1) {
        composite_frame(L, S.n_lcomp, xp, yp, apx, apy);
      } else {
        // EPL (Tessore & Metcalf series)
        // at the exact centre alpha is taken as 0 (its direction is undefined there)
        const T R = sqrt(q * q * xp * xp + yp * yp);
        const T iR = R > T(0.0) ? T(1.0) / R : T(0.0);
        const T wr = q * xp * iR, wi = yp * iR;
        const T w2r = wr * wr - wi * wi, w2i = T(2.0) * wr * wi;
        T omr = wr, omi = wi, Sr = wr, Si = wi;
        for (int n = 0; n < L.nterms; ++n) {
          const T rr = L.rho[n];
          const T nr = rr * (w2r * omr - w2i * omi);
          const T ni = rr * (w2r * omi + w2i * omr);
          omr = nr;
          omi = ni;
          Sr += omr;
          Si += omi;
        }
        const T amp = R > T(0.0) ? L.pref * exp2(omt * log2(R)) : T(0.0);
        apx = amp * Sr;
        apy = amp * Si;
      }
      T ax = L.cphi * apx - L.sphi * apy;
      T ay = L.sphi * apx + L.cphi * apy;
      if (L.mclass == 1 && L.bh_M > T(0.0)) {
        const T g = bh_gauss_factor(L.bh_M, L.bh_2s2, dx, dy);
        ax += g * dx;
        ay += g * dy;
      }
      ax += L.g1 * dx + L.g2 * dy;
      ay += L.g2 * dx - L.g1 * dy;
      for (int k = 0; k < S.n_sis; ++k) {
        const T te = (T)S.sis[3 * k];
        const T sx = x - (T)S.sis[3 * k + 1], sy = y - (T)S.sis[3 * k + 2];
        const T r2 = sx * sx + sy * sy;
        const T ir = r2 > T(0.0) ? rsq(r2) : T(0.0);
        ax += te * sx * ir;
        ay += te * sy * ir;
      }
      if (L.sheet) {
        // internal mass sheet: lambda x galaxy + (1 - lambda) u(R^2) (x - x_c, y - y_c)
        T u = T(1.0);
        if (L.sheet == 1) {
          const T R2 = dx * dx + dy * dy;
          const T Qc = sqrt(R2 + L.sh_rc2), Qt = sqrt(R2 + L.sh_rt2);
          u = T(2.0) * L.sh_rc * L.sh_rt * (T(1.0) + (L.sh_rc + L.sh_rt) / (Qc + Qt)) /
              ((L.sh_rc + Qc) * (L.sh_rt + Qt));
        }
        const T om = (T(1.0) - L.lam) * u;
        ax = L.lam * ax + om * dx;
        ay = L.lam * ay + om * dy;
      }
      T v = T(0.0);
      if (S.src_pix) {
        // pixelated source: the ray's bilinear entries into the grid (weight / ss^2; zero
        // outside the span of the pixel centres) for the response f = B L
        T u = (x - ax - (T)S.spx_x0) * (T)S.spx_idx - T(0.5);
        T w = (y - ay - (T)S.spx_y0) * (T)S.spx_idy - T(0.5);
        u = fmin(fmax(u, T(-2.0)), (T)(S.spx_nx + 2));
        w = fmin(fmax(w, T(-2.0)), (T)(S.spx_ny + 2));
        const T fu = floor(u), fw = floor(w);
        const int j0 = (int)fu, i0 = (int)fw;
        const bool in = j0 >= 0 && j0 + 1 < S.spx_nx && i0 >= 0 && i0 + 1 < S.spx_ny;
        const T tu = u - fu, tv = w - fw, sc = in ? T(1.0) / (T)(ss * ss) : T(0.0);
        const int e0 = in ? i0 * S.spx_nx + j0 : 0;
        const size_t o = (size_t)b * ws.max_lpix + ((size_t)p * ss * ss + my * ss + mx) * 4;
        ws.pix_Li[o] = e0;
        ws.pix_Li[o + 1] = e0 + 1;
        ws.pix_Li[o + 2] = e0 + S.spx_nx;
        ws.pix_Li[o + 3] = e0 + S.spx_nx + 1;
        ws.pix_Lw[o] = (float)(sc * (T(1.0) - tu) * (T(1.0) - tv));
        ws.pix_Lw[o + 1] = (float)(sc * tu * (T(1.0) - tv));
        ws.pix_Lw[o + 2] = (float)(sc * (T(1.0) - tu) * tv);
        ws.pix_Lw[o + 3] = (float)(sc * tu * tv);
      } else {
        // source at beta
        const T bx = x - ax - L.src_x, by = y - ay - L.src_y;
        const T xs = G.c * bx + G.s * by, ys = -G.s * bx + G.c * by;
        const T Rs2 = (xs * xs + ys * ys / (G.q * G.q)) * (L.src_Rei * L.src_Rei);
        v = sersic_f(Rs2, L.src_Ie, L.src_ninv, L.src_bn);
      }
      // lens light (same centre and PA as the mass): Sersic, or Chameleon in the composite class
      if (L.mclass == 1) {
        for (int c = 0; c < S.n_lcomp && c < 4; ++c) {
          const T m2 = xp * xp + yp * yp / (L.ch_q[c] * L.ch_q[c]);
          v += L.li_A[c] * (rsq(m2 + L.ch_sc[c] * L.ch_sc[c]) - rsq(m2 + L.ch_st[c] * L.ch_st[c]));
        }
      } else {
        for (int c = 0; c < S.n_lcomp; ++c) {
          const T R2 = (xp * xp + yp * yp * L.ll_qi2[c]) * (L.ll_Rei[c] * L.ll_Rei[c]);
          v += sersic_f(R2, L.ll_Ie[c], L.ll_ninv[c], L.ll_bn[c]);
        }
      }
      acc += v;
    }
  }
  img_of(ws, T(0))[(size_t)b * max_pix + p] = acc / (T)(ss * ss);
}

template <class T>
__global__ void __launch_bounds__(CONV_TX *CONV_TY) k_conv(const SysDev *__restrict__ sysv,
                                                           const int *__restrict__ sys_id, WsDev ws,
                                                           int max_pix, float *image_out,
                                                           float *resid_out) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (S.psf_km != 0 && sizeof(T) == 4) return;  // blurred by k_conv_r (FP32)
  const int ntx = (S.nx + CONV_TX - 1) / CONV_TX;
  const int nty = (S.ny + CONV_TY - 1) / CONV_TY;
  if ((int)blockIdx.x >= ntx * nty) return;
  const int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
  const int K = S.psf_k, h = (K - 1) / 2;
  const int W = CONV_TX + 2 * h, H = CONV_TY + 2 * h;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *tile = reinterpret_cast<T *>(smraw);  // [H*W]
  T *psf = tile + H * W;                   // [K*K]
  const int tid = threadIdx.y * CONV_TX + threadIdx.x;
  const int i0 = ty * CONV_TY - h, j0 = tx * CONV_TX - h;
  const T *img = img_of(ws, T(0)) + (size_t)b * max_pix;
  for (int e = tid; e < H * W; e += CONV_TX * CONV_TY) {
    const int li = e / W, lj = e - li * W;
    const int gi = i0 + li, gj = j0 + lj;
    tile[e] = (gi >= 0 && gi < S.ny && gj >= 0 && gj < S.nx) ? img[gi * S.nx + gj] : T(0);
  }
  for (int e = tid; e < K * K; e += CONV_TX * CONV_TY) psf[e] = (T)S.psf[e];
  __syncthreads();
  const int oi = ty * CONV_TY + threadIdx.y, oj = tx * CONV_TX + threadIdx.x;
  double chi = 0.0;
  if (oi < S.ny && oj < S.nx) {
    // m[i,j] = sum_{a,c} P[a,c] img[i-(a-h), j-(c-h)]; tile row of image row r is r - i0
    double m = 0.0;
    for (int a = 0; a < K; ++a) {
      const T *trow = tile + (threadIdx.y + 2 * h - a) * W + threadIdx.x + 2 * h;
      const T *prow = psf + a * K;
      T rs = T(0);
      for (int c = 0; c < K; ++c) rs = fma(prow[c], trow[-c], rs);
      m += (double)rs;
    }
    const int o = oi * S.nx + oj;
    if (image_out) {
      image_out[o] = (float)m;
    } else if (S.src_pix) {
      // the arcs left by the lens light, fitted by the pixelated source (k_pixsrc.cu)
      ws.pix_dres[(size_t)b * max_pix + o] = (float)((double)S.data[o] - m);
    } else {
      const double r = ((double)S.data[o] - m) * S.wgt[o];
      chi = r * r;
      // d logL / d m = mask (d - m) / sigma^2, for the adjoint
      if (resid_out) resid_out[(size_t)b * max_pix + o] = (float)(r * S.wgt[o]);
    }
  }
  if (image_out) return;
  // block reduction of chi^2 in FP64
  for (int off = 16; off > 0; off >>= 1) chi += __shfl_down_sync(0xffffffffu, chi, off);
  __shared__ double red[CONV_TX * CONV_TY / 32];
  if ((tid & 31) == 0) red[tid >> 5] = chi;
  __syncthreads();
  if (tid < 32) {
    double v = tid < CONV_TX * CONV_TY / 32 ? red[tid] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (tid == 0 && v != 0.0) atomicAdd(&ws.terms[4 * (size_t)b], v);
  }
}

// Register-blocked PSF blurring for PSF sides up to KM (the PSF centred in KM x KM zeros:
// the extra taps add exact zeros).  A CTA of 32 x 8 threads owns 32 columns x 8*CONV_R rows
// of output; each thread one column and CONV_R consecutive rows.  For each PSF column c the
// thread loads the CONV_R + KM - 1 tile values its outputs need (a vertical window, lanes on
// consecutive columns: conflict-free) and the column of taps (float4 broadcasts), then does
// CONV_R x KM FMAs from registers.  Per-column FP32 partial sums are added with Kahan
// compensation; chi^2 as in k_conv.
template <int KM>
__global__ void __launch_bounds__(CONV_TX *CONV_TY) k_conv_r(const SysDev *__restrict__ sysv,
                                                             const int *__restrict__ sys_id,
                                                             WsDev ws, int max_pix,
                                                             float *image_out, float *resid_out) {
  constexpr int R = CONV_R, TR = CONV_TY * R, W = CONV_TX + KM - 1, H = TR + KM - 1;
  constexpr int PT = CONV_PT(KM);
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (S.psf_km != KM) return;
  const int ntx = (S.nx + CONV_TX - 1) / CONV_TX;
  const int nty = (S.ny + TR - 1) / TR;
  if ((int)blockIdx.x >= ntx * nty) return;
  const int tx = blockIdx.x % ntx, ty = blockIdx.x / ntx;
  constexpr int h = (KM - 1) / 2;
  __shared__ float tile[H * W];
  __shared__ __align__(16) float pt[KM * PT];
  const int lane = threadIdx.x, warp = threadIdx.y;
  const int tid = warp * CONV_TX + lane;
  const int i0 = ty * TR - h, j0 = tx * CONV_TX - h;
  const float *img = ws.img + (size_t)b * max_pix;
  for (int e = tid; e < H * W; e += CONV_TX * CONV_TY) {
    const int li = e / W, lj = e - li * W;
    const int gi = i0 + li, gj = j0 + lj;
    tile[e] = (gi >= 0 && gi < S.ny && gj >= 0 && gj < S.nx) ? img[gi * S.nx + gj] : 0.0f;
  }
  for (int e = tid; e < KM * PT; e += CONV_TX * CONV_TY) pt[e] = S.psf_t[e];
  __syncthreads();
  // output (i0 + h + warp*R + r, j0 + h + lane) = sum_{a,c} P[a][c] tile[warp*R + r + KM-1-a][lane + KM-1-c]
  float sum[R], cmp[R];
#pragma unroll
  for (int r = 0; r < R; ++r) sum[r] = cmp[r] = 0.0f;
  for (int c = 0; c < KM; ++c) {
    float w[R + KM - 1];
    const float *col = tile + warp * R * W + lane + KM - 1 - c;
#pragma unroll
    for (int q = 0; q < R + KM - 1; ++q) w[q] = col[q * W];
    float p[PT];
    const float4 *pc = reinterpret_cast<const float4 *>(pt + c * PT);
#pragma unroll
    for (int a4 = 0; a4 < PT / 4; ++a4) {
      const float4 v = pc[a4];
      p[4 * a4] = v.x;
      p[4 * a4 + 1] = v.y;
      p[4 * a4 + 2] = v.z;
      p[4 * a4 + 3] = v.w;
    }
#pragma unroll
    for (int r = 0; r < R; ++r) {
      float part = 0.0f;
#pragma unroll
      for (int a = 0; a < KM; ++a) part = fmaf(p[a], w[r + KM - 1 - a], part);
      // Kahan: sum - cmp carries the column partials
      const float y = part - cmp[r];
      const float t = sum[r] + y;
      cmp[r] = (t - sum[r]) - y;
      sum[r] = t;
    }
  }
  double chi = 0.0;
  const int oj = tx * CONV_TX + lane;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int oi = ty * TR + warp * R + r;
    if (oi >= S.ny || oj >= S.nx) continue;
    const double m = (double)sum[r] - (double)cmp[r];
    const int o = oi * S.nx + oj;
    if (image_out) {
      image_out[o] = (float)m;
    } else if (S.src_pix) {
      ws.pix_dres[(size_t)b * max_pix + o] = (float)((double)S.data[o] - m);
    } else {
      const double rr = ((double)S.data[o] - m) * S.wgt[o];
      chi += rr * rr;
      if (resid_out) resid_out[(size_t)b * max_pix + o] = (float)(rr * S.wgt[o]);
    }
  }
  if (image_out) return;
  for (int off = 16; off > 0; off >>= 1) chi += __shfl_down_sync(0xffffffffu, chi, off);
  __shared__ double red[CONV_TX * CONV_TY / 32];
  if (lane == 0) red[warp] = chi;
  __syncthreads();
  if (tid < 32) {
    double v = tid < CONV_TX * CONV_TY / 32 ? red[tid] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
    if (tid == 0 && v != 0.0) atomicAdd(&ws.terms[4 * (size_t)b], v);
  }
}

}  // namespace

cudaError_t launch_lens(glad_ctx *c, const int *sys_id, int B, float *image_out, cudaStream_t st,
                        float *resid_out) {
  dim3 g1(c->max_img_tiles, B);
  const dim3 blk(CONV_TX, CONV_TY);
  if (c->ws.d.prec > 0 && !resid_out) {
    // FP64 lensing modes: ray shooting, light and PSF blurring in FP64 (general convolution)
    k_image<double><<<g1, LENS_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d, c->max_pix);
    int tiles = 0, kmax = 1;
    for (auto &sd : c->h_sysdev) {
      tiles = std::max(tiles, ((sd.nx + CONV_TX - 1) / CONV_TX) * ((sd.ny + CONV_TY - 1) / CONV_TY));
      kmax = std::max(kmax, sd.psf_k);
    }
    const int h = (kmax - 1) / 2;
    const size_t smem = sizeof(double) * ((CONV_TX + 2 * h) * (CONV_TY + 2 * h) + kmax * kmax);
    k_conv<double><<<dim3(tiles, B), blk, smem, st>>>(c->d_sys, sys_id, c->ws.d, c->max_pix, image_out,
                                                      nullptr);
    return cudaGetLastError();
  }
  k_image<float><<<g1, LENS_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d, c->max_pix);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // one blocked launch per padded PSF side present (samples of other systems exit at
  // once); systems with a PSF side above 31 go through the general kernel
  int tiles_r[3] = {0, 0, 0}, max_conv_tiles = 0, max_k = 0;
  for (auto &sd : c->h_sysdev) {
    const int t = ((sd.nx + CONV_TX - 1) / CONV_TX) * ((sd.ny + CONV_TY * CONV_R - 1) / (CONV_TY * CONV_R));
    if (sd.psf_km == 11) tiles_r[0] = std::max(tiles_r[0], t);
    if (sd.psf_km == 21) tiles_r[1] = std::max(tiles_r[1], t);
    if (sd.psf_km == 31) tiles_r[2] = std::max(tiles_r[2], t);
    if (sd.psf_km == 0) {
      max_conv_tiles = std::max(max_conv_tiles, ((sd.nx + CONV_TX - 1) / CONV_TX) *
                                                    ((sd.ny + CONV_TY - 1) / CONV_TY));
      max_k = std::max(max_k, sd.psf_k);
    }
  }
  if (tiles_r[0])
    k_conv_r<11><<<dim3(tiles_r[0], B), blk, 0, st>>>(c->d_sys, sys_id, c->ws.d, c->max_pix,
                                                      image_out, resid_out);
  if (tiles_r[1])
    k_conv_r<21><<<dim3(tiles_r[1], B), blk, 0, st>>>(c->d_sys, sys_id, c->ws.d, c->max_pix,
                                                      image_out, resid_out);
  if (tiles_r[2])
    k_conv_r<31><<<dim3(tiles_r[2], B), blk, 0, st>>>(c->d_sys, sys_id, c->ws.d, c->max_pix,
                                                      image_out, resid_out);
  if (max_conv_tiles) {
    const int h = (max_k - 1) / 2;
    const size_t smem = sizeof(float) * ((CONV_TX + 2 * h) * (CONV_TY + 2 * h) + max_k * max_k);
    k_conv<float><<<dim3(max_conv_tiles, B), blk, smem, st>>>(c->d_sys, sys_id, c->ws.d, c->max_pix,
                                                       image_out, resid_out);
  }
  return cudaGetLastError();
}

void set_conv_smem_limit() {
  const int h = (GLAD_MAX_PSF - 1) / 2;
  const int smem = sizeof(float) * ((CONV_TX + 2 * h) * (CONV_TY + 2 * h) + GLAD_MAX_PSF * GLAD_MAX_PSF);
  cudaFuncSetAttribute(k_conv<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  cudaFuncSetAttribute(k_conv<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * smem);
}
