// Dynamics half of the likelihood.
//  k_jam: Sigma v_los^2 at every sub-sample of the sky grid by the (tracer k, mass j,
//    Gauss-Legendre node g) pair sum of the cylindrically aligned JAM solution,
//      Sigma v^2(x', y') = sum_e (Q0_e + Q1_e x'^2) 2^(ax_e x'^2 + ay_e y'^2),
//    with the table streamed through shared memory in chunks and FP32 partial
//    sums flushed to FP64 per chunk; the tracer surface brightness (Eq. sb_mge_2D)
//    at the same points; then both maps go straight through the binning-after-PSF
//    operator W (bin sums of the PSF_kin-blurred maps, Eq. binned) into per-bin
//    FP64 accumulators, so the maps are never stored.
//  k_kin_finalize: v_rms,l = sqrt(num_l/den_l) (Eq. Vrms) and chi^2_dyn (Eq. chi2_dyn).
//  k_combine: logL = -(chi2_pix + chi2_dyn + chi2_tmd + chi2_img)/2 (Eq. chi_general).
#include <algorithm>

#include "glad_internal.cuh"
#include "jam_common.cuh"

namespace {

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int PTS, int UNR>
__device__ __forceinline__ void jam_tile(const SysDev &S, const WsDev &ws, JamSmem &sm, int b,
                                         int tile, int max_light, int max_ent, int max_bins) {
  constexpr int NP = PTS / 2;
  constexpr int TH = (JAM_THREADS / JAM_TW) * PTS;
  const int tid = threadIdx.x;
  const DynP dp = ws.dp[b];
  const int ntx = (S.nsx + JAM_TW - 1) / JAM_TW;
  const int c0 = (tile % ntx) * JAM_TW, r0 = (tile / ntx) * TH;
  const int c1 = min(c0 + JAM_TW, S.nsx) - 1, r1 = min(r0 + TH, S.nsy) - 1;
  for (int l = tid; l < S.n_bins; l += JAM_THREADS) {
    sm.bnum[l] = 0.0f;
    sm.bden[l] = 0.0f;
  }
  for (int k = tid; k < S.n_light; k += JAM_THREADS) {
    sm.sI0[k] = ws.I0f[(size_t)b * max_light + k];
    sm.scx[k] = S.sb_cx[k];
    sm.scy[k] = S.sb_cy[k];
  }
  const float cphi = (float)dp.cphi, sphi = (float)dp.sphi;
  const float xc = (float)dp.xc, yc = (float)dp.yc;
  const float hx = 0.5f * (S.nsx - 1), hy = 0.5f * (S.nsy - 1);
  float Xmin, Ymin;
  jam_tile_bounds(S, dp, c0, c1, r0, r1, Xmin, Ymin);
  const float Xmax = jam_tile_xmax(S, dp, c0, c1, r0, r1);
  const float4 *gt = ws.tab + (size_t)b * max_ent;
  const int n_ent = S.n_ent;
  const int n_chunks = (n_ent + JAM_CHUNK - 1) / JAM_CHUNK;
  const int lane = tid & 31, warp = tid >> 5;
  // Reference value of the tile's sums: the full sum at its four corners (their minimum).
  // Terms whose magnitude stays below 2^-(JAM_REL_MARGIN + log2 n_ent) of it over the whole
  // tile are left out; after the sum, the left-out magnitudes (a bound on their total) must
  // stay below 2^-JAM_REL_CHECK of the smallest |sum| in the tile, else the tile is summed
  // again with only the exact skipping.
  float lref = 0.0f, lrel = -INFINITY;
  if (ws.neg_mode != 0) {
    float cX[4], cY[4], cv[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float x = ((q & 1 ? c1 : c0) - hx) * S.dsub - xc;
      const float y = ((q & 2 ? r1 : r0) - hy) * S.dsub - yc;
      const float xp = cphi * x + sphi * y, yp = -sphi * x + cphi * y;
      cX[q] = xp * xp;
      cY[q] = yp * yp;
      cv[q] = 0.0f;
    }
    for (int e = tid; e < n_ent; e += JAM_THREADS) {
      const float4 c = gt[e];
#pragma unroll
      for (int q = 0; q < 4; ++q)
        cv[q] = fmaf(fmaf(c.w, cX[q], c.z), ex2(fmaf(c.y, cY[q], c.x * cX[q])), cv[q]);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      for (int off = 16; off > 0; off >>= 1) cv[q] += __shfl_xor_sync(0xffffffffu, cv[q], off);
      if (lane == 0) sm.red[q][warp] = cv[q];
    }
    __syncthreads();
    if (tid == 0) {
      float ref = 3.4e38f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float t = 0.0f;
        for (int w = 0; w < JAM_THREADS / 32; ++w) t += sm.red[q][w];
        ref = fminf(ref, t);
      }
      sm.flag = (ref > 0.0f && ref < 3.4e38f) ? __float_as_int(__log2f(ref)) : 0x7fffffff;
    }
    __syncthreads();
    const int f = sm.flag;
    lref = f == 0x7fffffff ? 0.0f : __int_as_float(f);
    // threshold relative to the reference; -inf (no usable reference): exact skipping only
    lrel = f == 0x7fffffff ? -INFINITY : -(JAM_REL_MARGIN + __log2f((float)max(n_ent, 1)));
  }
  if (tid == 0) {
    sm.tb[0] = Xmin;
    sm.tb[1] = Ymin;
    sm.tb[2] = Xmax;
    sm.tb[3] = lref;
    sm.tb[4] = lrel;
  }
  __syncthreads();
  // evaluations this tile executes (thread 0 keeps the count)
  const unsigned long long npts = (unsigned long long)(c1 - c0 + 1) * (unsigned long long)(r1 - r0 + 1);
  unsigned long long n_eval = 0;
  // this thread's points: column col, rows row0 .. row0 + PTS - 1 (clamped into the tile)
  const int col = c0 + (tid % JAM_TW);
  const int row0 = r0 + (tid / JAM_TW) * PTS;
  float2 X[NP], Y[NP], acc[NP];
  double accd[PTS];
#pragma unroll
  for (int i = 0; i < PTS; ++i) {
    const int J = min(col, c1), I = min(row0 + i, r1);
    const float x = (J - hx) * S.dsub - xc;
    const float y = (I - hy) * S.dsub - yc;
    const float xp = cphi * x + sphi * y, yp = -sphi * x + cphi * y;
    if (i & 1) {
      X[i >> 1].y = xp * xp;
      Y[i >> 1].y = yp * yp;
    } else {
      X[i >> 1].x = xp * xp;
      Y[i >> 1].x = yp * yp;
    }
  }
  for (;;) {
#pragma unroll
    for (int i = 0; i < PTS; ++i) accd[i] = 0.0;
#pragma unroll
    for (int p = 0; p < NP; ++p) acc[p] = make_float2(0.f, 0.f);
    float drel = 0.0f;
    JamStager stg;
    stg.count_rel(gt, n_ent, 0, sm.tb, sm.wcount[0], drel);
    __syncthreads();
    stg.write(sm.tab[0], sm.wcount[0], &sm.n_kept[0]);
    __syncthreads();
    for (int ch = 0; ch < n_chunks; ++ch) {
      const int cur = ch & 1;
      const bool more = ch + 1 < n_chunks;
      if (more)
        stg.count_rel(gt, n_ent, (ch + 1) * JAM_CHUNK, sm.tb, sm.wcount[cur ^ 1], drel);
      const float4 *t = sm.tab[cur];
      const int nk = sm.n_kept[cur];
      n_eval += (unsigned long long)nk * npts;
#pragma unroll UNR
      for (int e = 0; e < nk; ++e) {
        const float4 c = t[e];
        const float2 cx = make_float2(c.x, c.x), cy = make_float2(c.y, c.y);
        const float2 cz = make_float2(c.z, c.z), cw = make_float2(c.w, c.w);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const float2 arg = __ffma2_rn(cy, Y[p], __fmul2_rn(cx, X[p]));
          const float2 E = make_float2(ex2(arg.x), ex2(arg.y));
          acc[p] = __ffma2_rn(__ffma2_rn(cw, X[p], cz), E, acc[p]);
        }
      }
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        accd[2 * p] += (double)acc[p].x;
        accd[2 * p + 1] += (double)acc[p].y;
        acc[p] = make_float2(0.f, 0.f);
      }
      __syncthreads();
      if (more) stg.write(sm.tab[cur ^ 1], sm.wcount[cur ^ 1], &sm.n_kept[cur ^ 1]);
      __syncthreads();
    }
    if (lrel == -INFINITY) break;
    // a-posteriori check: left-out magnitudes against the smallest |sum| of the tile
    float vmin = 3.4e38f;
#pragma unroll
    for (int i = 0; i < PTS; ++i)
      if (col <= c1 && row0 + i <= r1) vmin = fminf(vmin, fabsf((float)accd[i]));
    for (int off = 16; off > 0; off >>= 1) {
      vmin = fminf(vmin, __shfl_xor_sync(0xffffffffu, vmin, off));
      drel += __shfl_xor_sync(0xffffffffu, drel, off);
    }
    if (lane == 0) {
      sm.red[0][warp] = vmin;
      sm.red[1][warp] = drel;
    }
    __syncthreads();
    if (tid == 0) {
      float vm = 3.4e38f, dr = 0.0f;
      for (int w = 0; w < JAM_THREADS / 32; ++w) {
        vm = fminf(vm, sm.red[0][w]);
        dr += sm.red[1][w];
      }
      // dropped total <= dr * 2^lref; accept when that is <= 2^-JAM_REL_CHECK * vm
      sm.flag = (ws.neg_mode == 1 && __log2f(dr) + lref <= __log2f(vm) - JAM_REL_CHECK) ? 1 : 0;
    }
    __syncthreads();
    const bool ok = sm.flag != 0;
    __syncthreads();
    if (ok) break;
    lrel = -INFINITY;  // sum the tile again with the exact skipping only
    if (tid == 0) sm.tb[4] = -INFINITY;
    __syncthreads();
  }
  if (tid == 0 && ws.evals) atomicAdd(ws.evals, n_eval);
  // tracer surface brightness and the binning-after-PSF scatter
#pragma unroll
  for (int i = 0; i < PTS; ++i) {
    if (col > c1 || row0 + i > r1) continue;
    const int s = (row0 + i) * S.nsx + col;
    const float Xi = (i & 1) ? X[i >> 1].y : X[i >> 1].x;
    const float Yi = (i & 1) ? Y[i >> 1].y : Y[i >> 1].x;
    float sb = 0.0f;
    for (int k = 0; k < S.n_light; ++k)
      sb = fmaf(sm.sI0[k], ex2(-fmaf(sm.scy[k], Yi, sm.scx[k] * Xi)), sb);
    const float v = (float)accd[i];
    for (int e = S.w_off[s]; e < S.w_off[s + 1]; ++e) {
      const int l = S.w_bin[e];
      const float w = S.w_val[e];
      atomicAdd(&sm.bnum[l], w * v);
      atomicAdd(&sm.bden[l], w * sb);
    }
  }
  __syncthreads();
  double *acc_g = ws.binacc + (size_t)b * max_bins * 2;
  for (int l = tid; l < S.n_bins; l += JAM_THREADS) {
    if (sm.bnum[l] != 0.0f) atomicAdd(&acc_g[2 * l], (double)sm.bnum[l]);
    if (sm.bden[l] != 0.0f) atomicAdd(&acc_g[2 * l + 1], (double)sm.bden[l]);
  }
  __syncthreads();  // the shared arrays are reused by the next tile of a persistent CTA
}

// one CTA per (tile, sample) of the largest system; tiles beyond a sample's system exit
template <int PTS, int MINB, int UNR>
__global__ void __launch_bounds__(JAM_THREADS, MINB) k_jam(const SysDev *__restrict__ sysv,
                                                           const int *__restrict__ sys_id, WsDev ws,
                                                           int max_light, int max_ent, int max_bins) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (S.jam_align != 0 || (int)blockIdx.x >= jam_tiles(S.nsx, S.nsy, PTS)) return;
  __shared__ JamSmem sm;
  jam_tile<PTS, UNR>(S, ws, sm, b, blockIdx.x, max_light, max_ent, max_bins);
}

// Work list for the persistent form: wl_off[b] = first item of sample b, wl_off[B] = total,
// items of a sample = its tiles (none for invalid samples).  One CTA; resets the counter.
__global__ void k_worklist(const SysDev *__restrict__ sysv, const int *__restrict__ sys_id,
                           WsDev ws, int B, int pts) {
  __shared__ int part[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < B; base += blockDim.x) {
    const int b = base + threadIdx.x;
    int n = 0;
    if (b < B && ws.status[b] == GLAD_SAMPLE_OK) {
      const SysDev &S = sysv[sys_id[b]];
      n = S.jam_align == 0 ? jam_tiles(S.nsx, S.nsy, pts) : 0;
    }
    part[threadIdx.x] = n;
    __syncthreads();
    // inclusive scan (Hillis-Steele) over the block
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
      const int v = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
      __syncthreads();
      part[threadIdx.x] += v;
      __syncthreads();
    }
    if (b < B) ws.wl_off[b] = carry + part[threadIdx.x] - n;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry += part[threadIdx.x];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ws.wl_off[B] = carry;
    *ws.wl_counter = 0;
  }
}

// Persistent form: a fixed grid of SM-count x occupancy CTAs takes (sample, tile) items
// from a global counter until the list is exhausted, so uneven batches leave no idle slots.
template <int PTS, int MINB, int UNR>
__global__ void __launch_bounds__(JAM_THREADS, MINB) k_jam_persist(
    const SysDev *__restrict__ sysv, const int *__restrict__ sys_id, WsDev ws, int B,
    int max_light, int max_ent, int max_bins) {
  __shared__ JamSmem sm;
  __shared__ int item_s, b_s;
  const int total = ws.wl_off[B];
  for (;;) {
    if (threadIdx.x == 0) {
      const int it = atomicAdd(ws.wl_counter, 1);
      int bb = -1;
      if (it < total) {
        // last sample whose first item is <= it
        int lo = 0, hi = B - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (ws.wl_off[mid] <= it) lo = mid;
          else hi = mid - 1;
        }
        bb = lo;
      }
      item_s = it;
      b_s = bb;
    }
    __syncthreads();
    const int it = item_s, b = b_s;
    __syncthreads();
    if (b < 0) return;
    const SysDev &S = sysv[sys_id[b]];
    jam_tile<PTS, UNR>(S, ws, sm, b, it - ws.wl_off[b], max_light, max_ent, max_bins);
  }
}

// The pair sum in FP64 (precision mode 2, glad_set_precision): one thread per sky sub-sample,
// every table entry (no skipping), the FP64 table staged through shared memory in chunks, exp()
// in FP64; then the tracer surface brightness and the binning-after-PSF scatter in FP64.
__global__ void __launch_bounds__(256) k_jam64(const SysDev *__restrict__ sysv,
                                               const int *__restrict__ sys_id, WsDev ws,
                                               int max_light, int max_ent, int max_bins) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (S.jam_align != 0) return;
  const int s = blockIdx.x * 256 + threadIdx.x;
  if ((int)blockIdx.x * 256 >= S.n_sub) return;
  const DynP dp = ws.dp[b];
  const int I = s / S.nsx, J = s - I * S.nsx;
  const double x = (J - 0.5 * (S.nsx - 1)) * S.dsub64 - dp.xc;
  const double y = (I - 0.5 * (S.nsy - 1)) * S.dsub64 - dp.yc;
  const double xp = dp.cphi * x + dp.sphi * y, yp = -dp.sphi * x + dp.cphi * y;
  const double X = xp * xp, Y = yp * yp;
  __shared__ double4_16a ch[256];
  const double4_16a *tab = ws.tab64 + (size_t)b * max_ent;
  double v = 0.0;
  for (int e0 = 0; e0 < S.n_ent; e0 += 256) {
    __syncthreads();
    if (e0 + threadIdx.x < S.n_ent) ch[threadIdx.x] = tab[e0 + threadIdx.x];
    __syncthreads();
    const int ne = min(256, S.n_ent - e0);
    for (int k = 0; k < ne; ++k) {
      const double4_16a t = ch[k];
      v += (t.z + t.w * X) * exp(t.x * X + t.y * Y);
    }
  }
  if (s >= S.n_sub) return;
  double sb = 0.0;
  for (int k = 0; k < S.n_light; ++k) {
    const double sg = S.sig_light[k], q = S.qp_light[k];
    sb += ws.I0d[(size_t)b * max_light + k] * exp(-(X + Y / (q * q)) / (2.0 * sg * sg));
  }
  double *acc_g = ws.binacc + (size_t)b * max_bins * 2;
  for (int e = S.w_off[s]; e < S.w_off[s + 1]; ++e) {
    const int l = S.w_bin[e];
    const double w = S.w_val[e];
    atomicAdd(&acc_g[2 * l], w * v);
    atomicAdd(&acc_g[2 * l + 1], w * sb);
  }
}

__global__ void k_kin_finalize(const SysDev *__restrict__ sysv, const int *__restrict__ sys_id,
                               WsDev ws, int max_bins, float *vrms_out) {
  const int b = blockIdx.x;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  const double *acc = ws.binacc + (size_t)b * max_bins * 2;
  double chi = 0.0;
  for (int l = threadIdx.x; l < S.n_bins; l += blockDim.x) {
    const double v = sqrt(acc[2 * l] / acc[2 * l + 1]);
    if (vrms_out) vrms_out[l] = (float)v;
    const double r = ((double)S.v_obs[l] - v) / (double)S.v_sig[l];
    chi += r * r;
  }
  for (int off = 16; off > 0; off >>= 1) chi += __shfl_down_sync(0xffffffffu, chi, off);
  __shared__ double red[32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = chi;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) t += red[w];
    ws.terms[4 * (size_t)b + 1] = t;
  }
}

__global__ void k_combine(WsDev ws, int B, double *logL, int *status, double *terms) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  int st = ws.status[b];
  const double t0 = ws.terms[4 * b], t1 = ws.terms[4 * b + 1], t2 = ws.terms[4 * b + 2],
               t3 = ws.terms[4 * b + 3];
  double L = -INFINITY;
  if (st == GLAD_SAMPLE_OK) {
    const double s = t0 + t1 + t2 + t3;
    if (isfinite(s)) L = -0.5 * s;
    else st = GLAD_SAMPLE_NONFINITE;
  }
  logL[b] = L;
  status[b] = st;
  if (terms) {
    terms[4 * b] = st == GLAD_SAMPLE_OK ? t0 : NAN;
    terms[4 * b + 1] = st == GLAD_SAMPLE_OK ? t1 : NAN;
    terms[4 * b + 2] = st == GLAD_SAMPLE_OK ? t2 : NAN;
    terms[4 * b + 3] = st == GLAD_SAMPLE_OK ? t3 : NAN;
  }
}

}  // namespace

// candidate launch shapes of the JAM pair sum: (points per thread, minimum CTAs per SM
// requested from the register allocator, unroll of the table-entry loop); the tuner times
// these and the persistent forms
#define GLAD_JAM_SHAPES(X) X(4, 5, 2) X(4, 5, 4) X(4, 6, 4) X(8, 3, 2) X(8, 4, 2) X(8, 4, 4) X(16, 2, 1)

bool jam_shape_supported(int pts, int minb, int unr) {
#define GLAD_JAM_MATCH(P, M, U) if (pts == P && minb == M && unr == U) return true;
  GLAD_JAM_SHAPES(GLAD_JAM_MATCH)
#undef GLAD_JAM_MATCH
  return false;
}

int jam_shape_list(int (*out)[3], int cap) {
  int n = 0;
#define GLAD_JAM_LIST(P, M, U) \
  if (n < cap) {               \
    out[n][0] = P;             \
    out[n][1] = M;             \
    out[n][2] = U;             \
  }                            \
  ++n;
  GLAD_JAM_SHAPES(GLAD_JAM_LIST)
#undef GLAD_JAM_LIST
  return n;
}

cudaError_t launch_jam(glad_ctx *c, const int *sys_id, int B, cudaStream_t st) {
  const int pts = c->tune.jam_pts;
  const int minb = c->tune.jam_minb;
  const int unr = c->tune.jam_unroll;
  if (!jam_shape_supported(pts, minb, unr)) return cudaErrorInvalidConfiguration;
  if (c->tune.jam_persistent && c->ws.d.wl_off) {
    k_worklist<<<1, 1024, 0, st>>>(c->d_sys, sys_id, c->ws.d, B, pts);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
#define GLAD_JAM_PERSIST(P, M, U)                                                                \
  if (pts == P && minb == M && unr == U) {                                                       \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_jam_persist<P, M, U>, JAM_THREADS, 0); \
    k_jam_persist<P, M, U><<<nsm * (occ > 0 ? occ : 1), JAM_THREADS, 0, st>>>(                   \
        c->d_sys, sys_id, c->ws.d, B, c->max_light, c->max_ent, c->max_bins);                    \
  }
    GLAD_JAM_SHAPES(GLAD_JAM_PERSIST)
#undef GLAD_JAM_PERSIST
    return cudaGetLastError();
  }
  int tiles = 0;
  for (auto &sd : c->h_sysdev) tiles = std::max(tiles, jam_tiles(sd.nsx, sd.nsy, pts));
  dim3 grid(tiles, B);
#define GLAD_JAM_LAUNCH(P, M, U)                                                                \
  if (pts == P && minb == M && unr == U)                                                        \
    k_jam<P, M, U><<<grid, JAM_THREADS, 0, st>>>(c->d_sys, sys_id, c->ws.d, c->max_light,       \
                                                 c->max_ent, c->max_bins);
  GLAD_JAM_SHAPES(GLAD_JAM_LAUNCH)
#undef GLAD_JAM_LAUNCH
  return cudaGetLastError();
}

cudaError_t launch_jam64(glad_ctx *c, const int *sys_id, int B, cudaStream_t st) {
  int blocks = 0;
  for (auto &sd : c->h_sysdev) blocks = std::max(blocks, (sd.n_sub + 255) / 256);
  k_jam64<<<dim3(blocks, B), 256, 0, st>>>(c->d_sys, sys_id, c->ws.d, c->max_light, c->max_ent,
                                            c->max_bins);
  return cudaGetLastError();
}

cudaError_t launch_kin_finalize(glad_ctx *c, const int *sys_id, int B, float *vrms_out,
                                cudaStream_t st) {
  k_kin_finalize<<<B, 256, 0, st>>>(c->d_sys, sys_id, c->ws.d, c->max_bins, vrms_out);
  return cudaGetLastError();
}

cudaError_t launch_combine(glad_ctx *c, int B, double *logL, int *status, double *terms,
                           cudaStream_t st) {
  k_combine<<<(B + 127) / 128, 128, 0, st>>>(c->ws.d, B, logL, status, terms);
  return cudaGetLastError();
}
