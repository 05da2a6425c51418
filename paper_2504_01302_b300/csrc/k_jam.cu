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
#include <type_traits>

#include "glad_internal.cuh"
#include "jam_common.cuh"

namespace {

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Recurrence form of the pair sum (the project's own; no counterpart in the paper).  Along a
// thread's rows the exponent is quadratic in the row offset i from a chain's first point:
//   a(i) = ax x'(i)^2 + ay y'(i)^2 = a(0) + i B + i^2 C,  B = 2 (ax x'(0) ux + ay y'(0) uy),
//   C = ax ux^2 + ay uy^2,  (ux, uy) = the row step in the galaxy frame,
// so 2^a(i) = P(i) k(i) with P(i) = 2^a(0) (2^B)^i and k(i) = 2^(C i^2).  P takes one multiply
// per point, k(i) folds into the entry's two prefactor terms while the chunk is staged, and
// each chain of JAM_REC_LEN points costs two ex2 instead of JAM_REC_LEN.  It is used for the
// entries with |C| <= JAM_REC_MAXC; there, a term that reaches 2^-JAM_REC_LOST of its prefactor
// at some point of a chain cannot sit on a chain whose first value 2^a(0) underflows (the
// chain's exponent rises by at most 9|C| + 6 sqrt(JAM_REC_LOST |C|) <= 126 - JAM_REC_LOST from
// its first point), so only terms below that fraction can be lost; their bound joins the
// left-out total of the negligible-term check.  The other entries are summed directly.
#define JAM_REC_LEN 4
#define JAM_REC_MAXC 1.0f
#define JAM_REC_LOST 67.0f

// k-scaled prefactors of the recurrence entries, after JamSmem in dynamic shared memory
struct JamRec {
  union {
    float2 kq[2][JAM_CHUNK][3];            // point-paired form: (Q0 k(i), Q1 k(i)), i = 1, 2, 3
    float4 kq4[2][JAM_CHUNK / 2 + 1][3];   // entry-paired form: two entries per float4
  };
};

// Staging for the recurrence form: like JamStager::count_rel / write, with the kept entries
// split into the directly summed ones (first) and the recurrence ones (after them, each with
// its k-scaled prefactors).
struct JamStagerRec {
  float4 v0, v1;
  bool k0, k1, w0, w1;  // kept; kept and summed by the recurrence
  __device__ __forceinline__ void count(const float4 *gt, int n_ent, int base, const volatile float *tb,
                                        float ux2, float uy2, int (*wc)[2][JAM_THREADS / 32],
                                        float &drel) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float Xmin = tb[0], Ymin = tb[1], Xmax = tb[2], lref = tb[3], lrel = tb[4];
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const int e0 = base + tid, e1 = base + tid + JAM_THREADS;
    v0 = e0 < n_ent ? gt[e0] : z;
    v1 = e1 < n_ent ? gt[e1] : z;
    const float b0 = fmaf(v0.y, Ymin, v0.x * Xmin), b1 = fmaf(v1.y, Ymin, v1.x * Xmin);
    const float l0 = __log2f(fabsf(v0.z) + fabsf(v0.w) * Xmax) - lref;
    const float l1 = __log2f(fabsf(v1.z) + fabsf(v1.w) * Xmax) - lref;
    const float m0 = b0 + l0, m1 = b1 + l1;
    const bool x0 = e0 < n_ent && b0 >= JAM_SKIP_LOG2, x1 = e1 < n_ent && b1 >= JAM_SKIP_LOG2;
    k0 = x0 && m0 >= lrel;
    k1 = x1 && m1 >= lrel;
    if (x0 && !k0) drel += jam_ex2(m0);
    if (x1 && !k1) drel += jam_ex2(m1);
    w0 = k0 && fabsf(fmaf(v0.y, uy2, v0.x * ux2)) <= JAM_REC_MAXC;
    w1 = k1 && fabsf(fmaf(v1.y, uy2, v1.x * ux2)) <= JAM_REC_MAXC;
    // what the recurrence may lose: below 2^-JAM_REC_LOST of the prefactor bound
    if (w0) drel += jam_ex2(fminf(b0, -JAM_REC_LOST) + l0);
    if (w1) drel += jam_ex2(fminf(b1, -JAM_REC_LOST) + l1);
    const unsigned d0 = __ballot_sync(0xffffffffu, k0 && !w0), r0 = __ballot_sync(0xffffffffu, w0);
    const unsigned d1 = __ballot_sync(0xffffffffu, k1 && !w1), r1 = __ballot_sync(0xffffffffu, w1);
    if (lane == 0) {
      wc[0][0][warp] = __popc(d0);
      wc[0][1][warp] = __popc(r0);
      wc[1][0][warp] = __popc(d1);
      wc[1][1][warp] = __popc(r1);
    }
  }
  __device__ __forceinline__ static void kq_of(const float4 &v, float ux2, float uy2, float2 *kq) {
    const float C = fmaf(v.y, uy2, v.x * ux2);
    const float k1 = jam_ex2(C), k2 = jam_ex2(4.0f * C), k3 = jam_ex2(9.0f * C);
    kq[0] = make_float2(v.z * k1, v.w * k1);
    kq[1] = make_float2(v.z * k2, v.w * k2);
    kq[2] = make_float2(v.z * k3, v.w * k3);
  }
  __device__ __forceinline__ void write(float4 *tab, float2 (*kq)[3], int (*wc)[2][JAM_THREADS / 32],
                                        int *n_kept, int *n_direct, float ux2, float uy2) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned d0 = __ballot_sync(0xffffffffu, k0 && !w0), r0 = __ballot_sync(0xffffffffu, w0);
    const unsigned d1 = __ballot_sync(0xffffffffu, k1 && !w1), r1 = __ballot_sync(0xffffffffu, w1);
    int od0 = 0, td0 = 0, od1 = 0, td1 = 0, or0 = 0, tr0 = 0, or1 = 0, tr1 = 0;
#pragma unroll
    for (int w = 0; w < JAM_THREADS / 32; ++w) {
      const int a0 = wc[0][0][w], a1 = wc[1][0][w], c0 = wc[0][1][w], c1 = wc[1][1][w];
      od0 += w < warp ? a0 : 0;
      od1 += w < warp ? a1 : 0;
      or0 += w < warp ? c0 : 0;
      or1 += w < warp ? c1 : 0;
      td0 += a0;
      td1 += a1;
      tr0 += c0;
      tr1 += c1;
    }
    const int nd = td0 + td1;
    if (k0 && !w0) tab[od0 + __popc(d0 & lt)] = v0;
    if (k1 && !w1) tab[td0 + od1 + __popc(d1 & lt)] = v1;
    if (w0) {
      const int p = or0 + __popc(r0 & lt);
      tab[nd + p] = v0;
      kq_of(v0, ux2, uy2, kq[p]);
    }
    if (w1) {
      const int p = tr0 + or1 + __popc(r1 & lt);
      tab[nd + p] = v1;
      kq_of(v1, ux2, uy2, kq[p]);
    }
    if (tid == 0) {
      *n_kept = nd + tr0 + tr1;
      *n_direct = nd;
    }
  }
};

// Staging for the entry-paired forms: the kept entries, compacted in order, are stored two to
// a pair of float4 -- (ax, ax', ay, ay') and (Q0, Q0', Q1, Q1') of entries 2m and 2m + 1 --
// so that one packed f32x2 operation evaluates two entries at one point with no duplicated
// operands.  With REC the kept entries are split as in JamStagerRec: directly summed pairs
// first, then the recurrence pairs, each with (Q0 k(i), Q0' k'(i), Q1 k(i), Q1' k'(i)) for
// i = 1, 2, 3; an odd list is padded with a zero entry (no term).
template <bool REC>
struct JamStagerPair {
  float4 v0, v1;
  bool k0, k1, w0, w1;  // kept; kept and summed by the recurrence
  __device__ __forceinline__ void count(const float4 *gt, int n_ent, int base, const volatile float *tb,
                                        float ux2, float uy2, int (*wc)[2][JAM_THREADS / 32],
                                        float &drel) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float Xmin = tb[0], Ymin = tb[1], Xmax = tb[2], lref = tb[3], lrel = tb[4];
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const int e0 = base + tid, e1 = base + tid + JAM_THREADS;
    v0 = e0 < n_ent ? gt[e0] : z;
    v1 = e1 < n_ent ? gt[e1] : z;
    const float b0 = fmaf(v0.y, Ymin, v0.x * Xmin), b1 = fmaf(v1.y, Ymin, v1.x * Xmin);
    const float l0 = __log2f(fabsf(v0.z) + fabsf(v0.w) * Xmax) - lref;
    const float l1 = __log2f(fabsf(v1.z) + fabsf(v1.w) * Xmax) - lref;
    const float m0 = b0 + l0, m1 = b1 + l1;
    const bool x0 = e0 < n_ent && b0 >= JAM_SKIP_LOG2, x1 = e1 < n_ent && b1 >= JAM_SKIP_LOG2;
    k0 = x0 && m0 >= lrel;
    k1 = x1 && m1 >= lrel;
    if (x0 && !k0) drel += jam_ex2(m0);
    if (x1 && !k1) drel += jam_ex2(m1);
    w0 = REC && k0 && fabsf(fmaf(v0.y, uy2, v0.x * ux2)) <= JAM_REC_MAXC;
    w1 = REC && k1 && fabsf(fmaf(v1.y, uy2, v1.x * ux2)) <= JAM_REC_MAXC;
    if (w0) drel += jam_ex2(fminf(b0, -JAM_REC_LOST) + l0);
    if (w1) drel += jam_ex2(fminf(b1, -JAM_REC_LOST) + l1);
    const unsigned d0 = __ballot_sync(0xffffffffu, k0 && !w0), r0 = __ballot_sync(0xffffffffu, w0);
    const unsigned d1 = __ballot_sync(0xffffffffu, k1 && !w1), r1 = __ballot_sync(0xffffffffu, w1);
    if (lane == 0) {
      wc[0][0][warp] = __popc(d0);
      wc[0][1][warp] = __popc(r0);
      wc[1][0][warp] = __popc(d1);
      wc[1][1][warp] = __popc(r1);
    }
  }
  // entry v at place j of its list, pairs from `pair0` on
  __device__ __forceinline__ static void put(float4 *tab, int pair0, int j, const float4 &v) {
    float *A = reinterpret_cast<float *>(&tab[2 * (pair0 + (j >> 1))]);
    const int s = j & 1;
    A[s] = v.x;
    A[2 + s] = v.y;
    A[4 + s] = v.z;
    A[6 + s] = v.w;
  }
  __device__ __forceinline__ static void put_kq(float4 (*kq)[3], int j, const float4 &v, float ux2,
                                                float uy2) {
    const float C = fmaf(v.y, uy2, v.x * ux2);
    const float k[3] = {jam_ex2(C), jam_ex2(4.0f * C), jam_ex2(9.0f * C)};
    const int s = j & 1;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float *K = reinterpret_cast<float *>(&kq[j >> 1][i]);
      K[s] = v.z * k[i];
      K[2 + s] = v.w * k[i];
    }
  }
  // tab: 2 float4 per pair; n_kept = kept entries, n_direct = directly summed entries
  __device__ __forceinline__ void write(float4 *tab, float4 (*kq)[3], int (*wc)[2][JAM_THREADS / 32],
                                        int *n_kept, int *n_direct, float ux2, float uy2) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned d0 = __ballot_sync(0xffffffffu, k0 && !w0), r0 = __ballot_sync(0xffffffffu, w0);
    const unsigned d1 = __ballot_sync(0xffffffffu, k1 && !w1), r1 = __ballot_sync(0xffffffffu, w1);
    int od0 = 0, td0 = 0, od1 = 0, td1 = 0, or0 = 0, tr0 = 0, or1 = 0, tr1 = 0;
#pragma unroll
    for (int w = 0; w < JAM_THREADS / 32; ++w) {
      const int a0 = wc[0][0][w], a1 = wc[1][0][w], c0 = wc[0][1][w], c1 = wc[1][1][w];
      od0 += w < warp ? a0 : 0;
      od1 += w < warp ? a1 : 0;
      or0 += w < warp ? c0 : 0;
      or1 += w < warp ? c1 : 0;
      td0 += a0;
      td1 += a1;
      tr0 += c0;
      tr1 += c1;
    }
    const int nd = td0 + td1, nr = tr0 + tr1, pd = (nd + 1) >> 1;
    if (k0 && !w0) put(tab, 0, od0 + __popc(d0 & lt), v0);
    if (k1 && !w1) put(tab, 0, td0 + od1 + __popc(d1 & lt), v1);
    if (w0) {
      const int j = or0 + __popc(r0 & lt);
      put(tab, pd, j, v0);
      put_kq(kq, j, v0, ux2, uy2);
    }
    if (w1) {
      const int j = tr0 + or1 + __popc(r1 & lt);
      put(tab, pd, j, v1);
      put_kq(kq, j, v1, ux2, uy2);
    }
    if (tid == 0) {
      const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
      if (nd & 1) put(tab, 0, nd, z);
      if (REC && (nr & 1)) {
        put(tab, pd, nr, z);
        put_kq(kq, nr, z, ux2, uy2);
      }
      *n_kept = nd + nr;
      *n_direct = nd;
    }
  }
};

// Forms of the pair sum (the launch shape's last number): 0 direct, two points per packed
// f32x2 operation; 1 recurrence, two points per packed operation (PTS a multiple of 8);
// 2 direct, two table entries per packed operation; 3 recurrence, two entries per packed
// operation (PTS a multiple of 4).
template <int PTS, int UNR, int FORM>
__device__ __forceinline__ void jam_tile(const SysDev &S, const WsDev &ws, JamSmem &sm, JamRec *sr,
                                         int b, int tile, int max_light, int max_ent, int max_bins) {
  constexpr bool REC = FORM == 1 || FORM == 3, PAIR = FORM >= 2;
  constexpr int NP = PTS / 2;
  constexpr int NSEG = (PAIR ? PTS : NP) / JAM_REC_LEN;
  static_assert(!REC || (PAIR ? PTS : NP) % JAM_REC_LEN == 0, "recurrence chains of 4 rows");
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
  // the row step in the galaxy frame (x' and y' per sky row)
  const float ux = sphi * S.dsub, uy = cphi * S.dsub;
  const float ux2 = ux * ux, uy2 = uy * uy;
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
  // this thread's points: column col, rows row0 .. row0 + PTS - 1 (rows past the tile are
  // evaluated and discarded)
  const int col = c0 + (tid % JAM_TW);
  const int row0 = r0 + (tid / JAM_TW) * PTS;
  const float xs = (min(col, c1) - hx) * S.dsub - xc;
  // forms 0, 1: two points per packed register, X[p] = (x'^2 at row p, at row NP + p);
  // forms 2, 3: one point per register pair, X[i] = (x'^2, x'^2) at row i
  constexpr int NX = PAIR ? PTS : NP;
  float2 X[NX], Y[NX], acc[NX];
  double accd[PTS];
#pragma unroll
  for (int i = 0; i < PTS; ++i) {
    const float y = (row0 + i - hy) * S.dsub - yc;
    const float xp = cphi * xs + sphi * y, yp = -sphi * xs + cphi * y;
    if (PAIR) {
      X[i] = make_float2(xp * xp, xp * xp);
      Y[i] = make_float2(yp * yp, yp * yp);
    } else if (i < NP) {
      X[i].x = xp * xp;
      Y[i].x = yp * yp;
    } else {
      X[i - NP].y = xp * xp;
      Y[i - NP].y = yp * yp;
    }
  }
  // recurrence chains: segment s starts at point CH * s of the chain layout; XB, YB hold
  // 2 x'(start) ux and 2 y'(start) uy, so that B = ax XB + ay YB
  float2 XB[REC ? NSEG : 1], YB[REC ? NSEG : 1];
  if constexpr (REC) {
#pragma unroll
    for (int s = 0; s < NSEG; ++s) {
      const float ya = (row0 + JAM_REC_LEN * s - hy) * S.dsub - yc;
      const float yb = PAIR ? ya : (row0 + NP + JAM_REC_LEN * s - hy) * S.dsub - yc;
      XB[s] = make_float2(2.0f * (cphi * xs + sphi * ya) * ux, 2.0f * (cphi * xs + sphi * yb) * ux);
      YB[s] = make_float2(2.0f * (-sphi * xs + cphi * ya) * uy, 2.0f * (-sphi * xs + cphi * yb) * uy);
    }
  }
  for (;;) {
#pragma unroll
    for (int i = 0; i < PTS; ++i) accd[i] = 0.0;
#pragma unroll
    for (int p = 0; p < NX; ++p) acc[p] = make_float2(0.f, 0.f);
    float drel = 0.0f;
    typename std::conditional<
        FORM == 0, JamStager,
        typename std::conditional<FORM == 1, JamStagerRec, JamStagerPair<REC>>::type>::type stg;
    auto count = [&](int base, int buf) {
      if constexpr (FORM == 0)
        stg.count_rel(gt, n_ent, base, sm.tb, sm.wcount[buf], drel);
      else
        stg.count(gt, n_ent, base, sm.tb, ux2, uy2, sm.wc[buf], drel);
    };
    auto write = [&](int buf) {
      if constexpr (FORM == 0)
        stg.write(sm.tab[buf], sm.wcount[buf], &sm.n_kept[buf]);
      else if constexpr (FORM == 1)
        stg.write(sm.tab[buf], sr->kq[buf], sm.wc[buf], &sm.n_kept[buf], &sm.n_direct[buf], ux2, uy2);
      else
        stg.write(sm.tab[buf], REC ? sr->kq4[buf] : nullptr, sm.wc[buf], &sm.n_kept[buf],
                  &sm.n_direct[buf], ux2, uy2);
    };
    count(0, 0);
    __syncthreads();
    write(0);
    __syncthreads();
    for (int ch = 0; ch < n_chunks; ++ch) {
      const int cur = ch & 1;
      const bool more = ch + 1 < n_chunks;
      if (more) count((ch + 1) * JAM_CHUNK, cur ^ 1);
      const float4 *t = sm.tab[cur];
      const int nk = sm.n_kept[cur];
      const int nd = FORM == 0 ? nk : sm.n_direct[cur];
      n_eval += (unsigned long long)nk * npts;
      if constexpr (!PAIR) {
        // direct, two points per packed operation
#pragma unroll UNR
        for (int e = 0; e < nd; ++e) {
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
      } else {
        // direct, two entries per packed operation
        const int npd = (nd + 1) >> 1;
#pragma unroll UNR
        for (int m = 0; m < npd; ++m) {
          const float4 a = t[2 * m], q = t[2 * m + 1];
          const float2 cx = make_float2(a.x, a.y), cy = make_float2(a.z, a.w);
          const float2 cz = make_float2(q.x, q.y), cw = make_float2(q.z, q.w);
#pragma unroll
          for (int i = 0; i < PTS; ++i) {
            const float2 arg = __ffma2_rn(cy, Y[i], __fmul2_rn(cx, X[i]));
            const float2 E = make_float2(ex2(arg.x), ex2(arg.y));
            acc[i] = __ffma2_rn(__ffma2_rn(cw, X[i], cz), E, acc[i]);
          }
        }
      }
      if constexpr (FORM == 1) {
        const float2 (*kq)[3] = sr->kq[cur];
#pragma unroll UNR
        for (int e = nd; e < nk; ++e) {
          const float4 c = t[e];
          const float2 q1 = kq[e - nd][0], q2 = kq[e - nd][1], q3 = kq[e - nd][2];
          const float2 cx = make_float2(c.x, c.x), cy = make_float2(c.y, c.y);
          const float2 cz = make_float2(c.z, c.z), cw = make_float2(c.w, c.w);
          const float2 z1 = make_float2(q1.x, q1.x), w1 = make_float2(q1.y, q1.y);
          const float2 z2 = make_float2(q2.x, q2.x), w2 = make_float2(q2.y, q2.y);
          const float2 z3 = make_float2(q3.x, q3.x), w3 = make_float2(q3.y, q3.y);
#pragma unroll
          for (int s = 0; s < NSEG; ++s) {
            const int p = JAM_REC_LEN * s;
            const float2 a = __ffma2_rn(cy, Y[p], __fmul2_rn(cx, X[p]));
            const float2 B = __ffma2_rn(cy, YB[s], __fmul2_rn(cx, XB[s]));
            // a chain whose first value underflows stays at zero: the ratio is kept finite
            float2 P = make_float2(ex2(a.x), ex2(a.y));
            const float2 R = make_float2(ex2(fminf(B.x, 100.0f)), ex2(fminf(B.y, 100.0f)));
            acc[p] = __ffma2_rn(__ffma2_rn(cw, X[p], cz), P, acc[p]);
            P = __fmul2_rn(P, R);
            acc[p + 1] = __ffma2_rn(__ffma2_rn(w1, X[p + 1], z1), P, acc[p + 1]);
            P = __fmul2_rn(P, R);
            acc[p + 2] = __ffma2_rn(__ffma2_rn(w2, X[p + 2], z2), P, acc[p + 2]);
            P = __fmul2_rn(P, R);
            acc[p + 3] = __ffma2_rn(__ffma2_rn(w3, X[p + 3], z3), P, acc[p + 3]);
          }
        }
      }
      if constexpr (FORM == 3) {
        const float4 (*kq)[3] = sr->kq4[cur];
        const int pd = (nd + 1) >> 1, npr = (nk - nd + 1) >> 1;
#pragma unroll UNR
        for (int m = 0; m < npr; ++m) {
          const float4 a = t[2 * (pd + m)], q = t[2 * (pd + m) + 1];
          const float4 q1 = kq[m][0], q2 = kq[m][1], q3 = kq[m][2];
          const float2 cx = make_float2(a.x, a.y), cy = make_float2(a.z, a.w);
          const float2 cz = make_float2(q.x, q.y), cw = make_float2(q.z, q.w);
          const float2 z1 = make_float2(q1.x, q1.y), w1 = make_float2(q1.z, q1.w);
          const float2 z2 = make_float2(q2.x, q2.y), w2 = make_float2(q2.z, q2.w);
          const float2 z3 = make_float2(q3.x, q3.y), w3 = make_float2(q3.z, q3.w);
#pragma unroll
          for (int s = 0; s < NSEG; ++s) {
            const int p = JAM_REC_LEN * s;
            const float2 av = __ffma2_rn(cy, Y[p], __fmul2_rn(cx, X[p]));
            const float2 B = __ffma2_rn(cy, YB[s], __fmul2_rn(cx, XB[s]));
            float2 P = make_float2(ex2(av.x), ex2(av.y));
            const float2 R = make_float2(ex2(fminf(B.x, 100.0f)), ex2(fminf(B.y, 100.0f)));
            acc[p] = __ffma2_rn(__ffma2_rn(cw, X[p], cz), P, acc[p]);
            P = __fmul2_rn(P, R);
            acc[p + 1] = __ffma2_rn(__ffma2_rn(w1, X[p + 1], z1), P, acc[p + 1]);
            P = __fmul2_rn(P, R);
            acc[p + 2] = __ffma2_rn(__ffma2_rn(w2, X[p + 2], z2), P, acc[p + 2]);
            P = __fmul2_rn(P, R);
            acc[p + 3] = __ffma2_rn(__ffma2_rn(w3, X[p + 3], z3), P, acc[p + 3]);
          }
        }
      }
#pragma unroll
      for (int p = 0; p < NX; ++p) {
        if (PAIR) {
          accd[p] += (double)acc[p].x + (double)acc[p].y;
        } else {
          accd[p] += (double)acc[p].x;
          accd[NP + p] += (double)acc[p].y;
        }
        acc[p] = make_float2(0.f, 0.f);
      }
      __syncthreads();
      if (more) write(cur ^ 1);
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
    const float Xi = PAIR ? X[i].x : (i < NP ? X[i].x : X[i - NP].y);
    const float Yi = PAIR ? Y[i].x : (i < NP ? Y[i].x : Y[i - NP].y);
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

// dynamic shared memory of the pair-sum kernels: JamSmem, and JamRec after it in the
// recurrence forms (1, 3)
constexpr size_t jam_smem_bytes(int form) {
  return (form == 1 || form == 3) ? sizeof(JamSmem) + sizeof(JamRec) : sizeof(JamSmem);
}

// one CTA per (tile, sample) of the largest system; tiles beyond a sample's system exit
template <int PTS, int MINB, int UNR, int FORM>
__global__ void __launch_bounds__(JAM_THREADS, MINB) k_jam(const SysDev *__restrict__ sysv,
                                                           const int *__restrict__ sys_id, WsDev ws,
                                                           int max_light, int max_ent, int max_bins) {
  const int b = blockIdx.y;
  if (ws.status[b] != GLAD_SAMPLE_OK) return;
  const SysDev &S = sysv[sys_id[b]];
  if (S.jam_align != 0 || (int)blockIdx.x >= jam_tiles(S.nsx, S.nsy, PTS)) return;
  extern __shared__ __align__(16) unsigned char jam_dyn[];
  JamRec *sr = (FORM == 1 || FORM == 3) ? reinterpret_cast<JamRec *>(jam_dyn + sizeof(JamSmem)) : nullptr;
  jam_tile<PTS, UNR, FORM>(S, ws, *reinterpret_cast<JamSmem *>(jam_dyn), sr, b, blockIdx.x,
                          max_light, max_ent, max_bins);
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
template <int PTS, int MINB, int UNR, int FORM>
__global__ void __launch_bounds__(JAM_THREADS, MINB) k_jam_persist(
    const SysDev *__restrict__ sysv, const int *__restrict__ sys_id, WsDev ws, int B,
    int max_light, int max_ent, int max_bins) {
  extern __shared__ __align__(16) unsigned char jam_dyn[];
  JamSmem &sm = *reinterpret_cast<JamSmem *>(jam_dyn);
  JamRec *sr = (FORM == 1 || FORM == 3) ? reinterpret_cast<JamRec *>(jam_dyn + sizeof(JamSmem)) : nullptr;
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
    jam_tile<PTS, UNR, FORM>(S, ws, sm, sr, b, it - ws.wl_off[b], max_light, max_ent, max_bins);
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
// requested from the register allocator, unroll of the table-entry loop, form of the sum:
// 0 direct / 1 recurrence with two points per packed operation, 2 direct / 3 recurrence with
// two table entries per packed operation); the tuner times these and the persistent forms
#define GLAD_JAM_SHAPES(X)                                                                        \
  X(2, 6, 4, 0) X(2, 8, 4, 0) X(4, 5, 2, 0) X(4, 5, 4, 0) X(4, 6, 4, 0) X(8, 3, 2, 0) X(8, 4, 2, 0)  \
  X(8, 4, 4, 0) X(16, 2, 1, 0)                                                                     \
  X(8, 3, 2, 1) X(8, 4, 1, 1) X(8, 4, 2, 1) X(16, 2, 1, 1)                                         \
  X(4, 4, 2, 2) X(4, 5, 2, 2) X(4, 5, 1, 2) X(8, 3, 1, 2)                                          \
  X(4, 4, 2, 3) X(4, 4, 1, 3) X(4, 5, 1, 3) X(8, 3, 1, 3)

bool jam_shape_supported(int pts, int minb, int unr, int rec) {
#define GLAD_JAM_MATCH(P, M, U, R) if (pts == P && minb == M && unr == U && rec == R) return true;
  GLAD_JAM_SHAPES(GLAD_JAM_MATCH)
#undef GLAD_JAM_MATCH
  return false;
}

int jam_shape_list(int (*out)[4], int cap) {
  int n = 0;
#define GLAD_JAM_LIST(P, M, U, R) \
  if (n < cap) {                  \
    out[n][0] = P;                \
    out[n][1] = M;                \
    out[n][2] = U;                \
    out[n][3] = R;                \
  }                               \
  ++n;
  GLAD_JAM_SHAPES(GLAD_JAM_LIST)
#undef GLAD_JAM_LIST
  return n;
}

// the recurrence forms' dynamic shared memory exceeds the default 48 KB: raise the limit
template <class K>
static cudaError_t jam_smem_limit(K kern, int form) {
  if (jam_smem_bytes(form) <= 48 * 1024) return cudaSuccess;
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)jam_smem_bytes(form));
}

cudaError_t launch_jam(glad_ctx *c, const int *sys_id, int B, cudaStream_t st) {
  const int pts = c->tune.jam_pts;
  const int minb = c->tune.jam_minb;
  const int unr = c->tune.jam_unroll;
  const int rec = c->tune.jam_form;
  if (!jam_shape_supported(pts, minb, unr, rec)) return cudaErrorInvalidConfiguration;
  cudaError_t e = cudaSuccess;
  if (c->tune.jam_persistent && c->ws.d.wl_off) {
    k_worklist<<<1, 1024, 0, st>>>(c->d_sys, sys_id, c->ws.d, B, pts);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    int dev = 0, nsm = 0, occ = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
#define GLAD_JAM_PERSIST(P, M, U, R)                                                              \
  if (pts == P && minb == M && unr == U && rec == R) {                                            \
    e = jam_smem_limit(k_jam_persist<P, M, U, R>, R);                                             \
    if (e != cudaSuccess) return e;                                                               \
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_jam_persist<P, M, U, R>, JAM_THREADS,  \
                                                  jam_smem_bytes(R));                             \
    k_jam_persist<P, M, U, R><<<nsm * (occ > 0 ? occ : 1), JAM_THREADS, jam_smem_bytes(R), st>>>( \
        c->d_sys, sys_id, c->ws.d, B, c->max_light, c->max_ent, c->max_bins);                     \
  }
    GLAD_JAM_SHAPES(GLAD_JAM_PERSIST)
#undef GLAD_JAM_PERSIST
    return cudaGetLastError();
  }
  int tiles = 0;
  for (auto &sd : c->h_sysdev) tiles = std::max(tiles, jam_tiles(sd.nsx, sd.nsy, pts));
  dim3 grid(tiles, B);
#define GLAD_JAM_LAUNCH(P, M, U, R)                                                             \
  if (pts == P && minb == M && unr == U && rec == R) {                                          \
    e = jam_smem_limit(k_jam<P, M, U, R>, R);                                                   \
    if (e != cudaSuccess) return e;                                                             \
    k_jam<P, M, U, R><<<grid, JAM_THREADS, jam_smem_bytes(R), st>>>(                            \
        c->d_sys, sys_id, c->ws.d, c->max_light, c->max_ent, c->max_bins);                      \
  }
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
