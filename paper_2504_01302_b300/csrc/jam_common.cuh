// Sky tiling and table staging shared by the JAM pair-sum kernels (forward and the
// gradient's derivative pass).
#pragma once
#include "glad_internal.cuh"

__device__ __forceinline__ float jam_ex2(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Sky tiles are JAM_TW columns x (8 * PTS) rows of sub-samples; each warp covers JAM_TW
// columns and PTS consecutive rows, each thread one column.  For a tile, a lower bound of
// x'^2 and y'^2 over its points (from its corners: x', y' are linear in the pixel indices)
// bounds every exponent ax x'^2 + ay y'^2 (ax, ay < 0) from above; table entries whose bound
// is below -130 give 2^arg < 2^-130, which ex2.approx.ftz flushes to exactly 0, so they are
// dropped while staging the chunk.  The kept entries keep their order and the chunk
// boundaries of the FP32 partial sums are unchanged: every point's sum is bit-identical to
// the one without skipping.
#define JAM_TW 32
#define JAM_SKIP_LOG2 (-130.0f)
// Negligible terms (forward pair sum): a term is left out when its largest magnitude over
// the tile is below 2^-(JAM_REL_MARGIN + log2 n_ent) of the tile's reference sum, and the
// bound on everything left out must come to at most 2^-JAM_REL_CHECK of the smallest |sum|
// in the tile (2^-26: below the FP32 rounding of each sum), else the tile is summed again
// without it.
#define JAM_REL_MARGIN 22.0f
// the derivative pass keeps more (its left-out bounds also cover the derivatives, whose
// factor ln2 |ax| is largest for the narrow Gaussians that this rule leaves out)
#define JAM_REL_MARGIN_GRAD 30.0f
#define JAM_REL_CHECK 26.0f

struct JamSmem {
  float4 tab[2][JAM_CHUNK + 4];        // (+4: the entry-paired forms pad two odd lists)
  int wcount[2][2][JAM_THREADS / 32];  // [buffer][half of the chunk][warp]
  int wc[2][2][2][JAM_THREADS / 32];   // [buffer][half][direct, recurrence][warp] (k_jam forms 1-3)
  int n_kept[2];
  int n_direct[2];
  float red[4][JAM_THREADS / 32];      // block reductions of the negligible-term test
  int flag;
  float tb[5];                         // tile constants: Xmin, Ymin, Xmax, lref, lrel
  float bnum[GLAD_MAX_BINS], bden[GLAD_MAX_BINS];
  float sI0[GLAD_MAX_LIGHT], scx[GLAD_MAX_LIGHT], scy[GLAD_MAX_LIGHT];
};

__host__ __device__ inline int jam_tiles(int nsx, int nsy, int pts) {
  return ((nsx + JAM_TW - 1) / JAM_TW) * ((nsy + (JAM_THREADS / JAM_TW) * pts - 1) /
                                         ((JAM_THREADS / JAM_TW) * pts));
}


// Lower bounds of x'^2 and y'^2 over the tile [c0, c1] x [r0, r1] of sub-sample indices
// (x', y' are linear in the indices, so the extremes sit at the corners), slightly lowered
// against rounding.
__device__ __forceinline__ void jam_tile_bounds(const SysDev &S, const DynP &dp, int c0, int c1,
                                                int r0, int r1, float &Xmin, float &Ymin) {
  const float cphi = (float)dp.cphi, sphi = (float)dp.sphi;
  const float xc = (float)dp.xc, yc = (float)dp.yc;
  const float hx = 0.5f * (S.nsx - 1), hy = 0.5f * (S.nsy - 1);
  float xmn = 1e30f, xmx = -1e30f, ymn = 1e30f, ymx = -1e30f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float x = ((q & 1 ? c1 : c0) - hx) * S.dsub - xc;
    const float y = ((q & 2 ? r1 : r0) - hy) * S.dsub - yc;
    const float xp = cphi * x + sphi * y, yp = -sphi * x + cphi * y;
    xmn = fminf(xmn, xp);
    xmx = fmaxf(xmx, xp);
    ymn = fminf(ymn, yp);
    ymx = fmaxf(ymx, yp);
  }
  Xmin = (xmn <= 0.0f && xmx >= 0.0f) ? 0.0f : 0.999f * fminf(xmn * xmn, xmx * xmx);
  Ymin = (ymn <= 0.0f && ymx >= 0.0f) ? 0.0f : 0.999f * fminf(ymn * ymn, ymx * ymx);
}

// Upper bound of x'^2 over the same tile (the extremes of x' sit at the corners).
__device__ __forceinline__ float jam_tile_xmax(const SysDev &S, const DynP &dp, int c0, int c1,
                                               int r0, int r1) {
  const float cphi = (float)dp.cphi, sphi = (float)dp.sphi;
  const float xc = (float)dp.xc, yc = (float)dp.yc;
  const float hx = 0.5f * (S.nsx - 1), hy = 0.5f * (S.nsy - 1);
  float m = 0.0f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float x = ((q & 1 ? c1 : c0) - hx) * S.dsub - xc;
    const float y = ((q & 2 ? r1 : r0) - hy) * S.dsub - yc;
    const float xp = cphi * x + sphi * y;
    m = fmaxf(m, xp * xp);
  }
  return 1.001f * m;
}

// Order-preserving compaction of one JAM_CHUNK of table entries into shared memory, keeping
// the entries whose exponent bound over the tile is >= JAM_SKIP_LOG2.  count() loads two
// entries per thread and publishes per-warp counts; after a barrier write() stores the kept
// entries at their prefix positions and the number kept.
struct JamStager {
  float4 v0, v1;
  bool k0, k1;
  __device__ __forceinline__ void count(const float4 *gt, int n_ent, int base, float Xmin, float Ymin,
                                        int (*wcount)[JAM_THREADS / 32]) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const int e0 = base + tid, e1 = base + tid + JAM_THREADS;
    v0 = e0 < n_ent ? gt[e0] : z;
    v1 = e1 < n_ent ? gt[e1] : z;
    k0 = e0 < n_ent && fmaf(v0.y, Ymin, v0.x * Xmin) >= JAM_SKIP_LOG2;
    k1 = e1 < n_ent && fmaf(v1.y, Ymin, v1.x * Xmin) >= JAM_SKIP_LOG2;
    const unsigned m0 = __ballot_sync(0xffffffffu, k0), m1 = __ballot_sync(0xffffffffu, k1);
    if (lane == 0) {
      wcount[0][warp] = __popc(m0);
      wcount[1][warp] = __popc(m1);
    }
  }
  // count() with the negligible-term criterion as well: an entry is also dropped when
  // 2^(bound) (|Q0| + |Q1| Xmax), the largest magnitude its term reaches over the tile,
  // is below 2^lrel (lrel relative to a reference value of the tile's sums); the dropped
  // magnitudes, relative to that reference, are added to drel.
  // (tb: Xmin, Ymin, Xmax, lref, lrel of the tile, in shared memory)
  __device__ __forceinline__ void count_rel(const float4 *gt, int n_ent, int base,
                                            const volatile float *tb,
                                            int (*wcount)[JAM_THREADS / 32], float &drel) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float Xmin = tb[0], Ymin = tb[1], Xmax = tb[2], lref = tb[3], lrel = tb[4];
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const int e0 = base + tid, e1 = base + tid + JAM_THREADS;
    v0 = e0 < n_ent ? gt[e0] : z;
    v1 = e1 < n_ent ? gt[e1] : z;
    const float b0 = fmaf(v0.y, Ymin, v0.x * Xmin), b1 = fmaf(v1.y, Ymin, v1.x * Xmin);
    // log2 of the term's largest magnitude relative to the reference
    const float m0 = b0 + __log2f(fabsf(v0.z) + fabsf(v0.w) * Xmax) - lref;
    const float m1 = b1 + __log2f(fabsf(v1.z) + fabsf(v1.w) * Xmax) - lref;
    const bool x0 = e0 < n_ent && b0 >= JAM_SKIP_LOG2, x1 = e1 < n_ent && b1 >= JAM_SKIP_LOG2;
    k0 = x0 && m0 >= lrel;
    k1 = x1 && m1 >= lrel;
    if (x0 && !k0) drel += jam_ex2(m0);
    if (x1 && !k1) drel += jam_ex2(m1);
    const unsigned c0 = __ballot_sync(0xffffffffu, k0), c1 = __ballot_sync(0xffffffffu, k1);
    if (lane == 0) {
      wcount[0][warp] = __popc(c0);
      wcount[1][warp] = __popc(c1);
    }
  }
  // count_rel() for the derivative pass: the left-out bounds of the term, of its X
  // derivative (|Q1| 2^bound + ln2 |ax| M) and of its Y derivative (ln2 |ay| M), M the term
  // bound, each relative to the reference, go to dv, dx, dy.
  __device__ __forceinline__ void count_rel_grad(const float4 *gt, int n_ent, int base,
                                                 const volatile float *tb,
                                                 int (*wcount)[JAM_THREADS / 32], float &dv,
                                                 float &dx, float &dy) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const float Xmin = tb[0], Ymin = tb[1], Xmax = tb[2], lref = tb[3], lrel = tb[4];
    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
    const int e0 = base + tid, e1 = base + tid + JAM_THREADS;
    v0 = e0 < n_ent ? gt[e0] : z;
    v1 = e1 < n_ent ? gt[e1] : z;
    const float b0 = fmaf(v0.y, Ymin, v0.x * Xmin), b1 = fmaf(v1.y, Ymin, v1.x * Xmin);
    const float m0 = b0 + __log2f(fabsf(v0.z) + fabsf(v0.w) * Xmax) - lref;
    const float m1 = b1 + __log2f(fabsf(v1.z) + fabsf(v1.w) * Xmax) - lref;
    const bool x0 = e0 < n_ent && b0 >= JAM_SKIP_LOG2, x1 = e1 < n_ent && b1 >= JAM_SKIP_LOG2;
    k0 = x0 && m0 >= lrel;
    k1 = x1 && m1 >= lrel;
    constexpr float L2 = 0.6931471805599453f;
    if (x0 && !k0) {
      const float M = jam_ex2(m0);
      dv += M;
      dx += jam_ex2(b0 + __log2f(fabsf(v0.w)) - lref) + L2 * fabsf(v0.x) * M;
      dy += L2 * fabsf(v0.y) * M;
    }
    if (x1 && !k1) {
      const float M = jam_ex2(m1);
      dv += M;
      dx += jam_ex2(b1 + __log2f(fabsf(v1.w)) - lref) + L2 * fabsf(v1.x) * M;
      dy += L2 * fabsf(v1.y) * M;
    }
    const unsigned c0 = __ballot_sync(0xffffffffu, k0), c1 = __ballot_sync(0xffffffffu, k1);
    if (lane == 0) {
      wcount[0][warp] = __popc(c0);
      wcount[1][warp] = __popc(c1);
    }
  }
  __device__ __forceinline__ void write(float4 *tab, int (*wcount)[JAM_THREADS / 32], int *n_kept) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const unsigned m0 = __ballot_sync(0xffffffffu, k0), m1 = __ballot_sync(0xffffffffu, k1);
    int off0 = 0, tot0 = 0, off1 = 0, tot1 = 0;
#pragma unroll
    for (int w = 0; w < JAM_THREADS / 32; ++w) {
      const int a0 = wcount[0][w], a1 = wcount[1][w];
      off0 += w < warp ? a0 : 0;
      off1 += w < warp ? a1 : 0;
      tot0 += a0;
      tot1 += a1;
    }
    if (k0) tab[off0 + __popc(m0 & lt)] = v0;
    if (k1) tab[tot0 + off1 + __popc(m1 & lt)] = v1;
    if (tid == 0) *n_kept = tot0 + tot1;
  }
};
