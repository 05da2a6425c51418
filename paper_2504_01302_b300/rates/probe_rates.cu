// Throughput probe for the roofline denominators of the JAM kernel: ex2.approx.ftz.f32
// (MUFU), FFMA and DFMA issued from 8 independent chains per thread over a grid of
// 8 CTAs x 256 threads per SM.  Every loop is bounded; nothing waits on anything.
#include <cstdio>
#include <cuda_runtime.h>

__device__ __forceinline__ float ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void k_ex2(float *out, int iters) {
  float y[8];
  for (int i = 0; i < 8; ++i) y[i] = 0.001f * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) y[i] = ex2(fmaf(y[i], -0.5f, 0.25f));
  }
  float s = 0;
  for (int i = 0; i < 8; ++i) s += y[i];
  if (s == 12345.f) out[0] = s;
}

__global__ void k_ffma(float *out, int iters) {
  float y[8];
  for (int i = 0; i < 8; ++i) y[i] = 0.001f * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) y[i] = fmaf(y[i], 0.999f, 0.001f);
  }
  float s = 0;
  for (int i = 0; i < 8; ++i) s += y[i];
  if (s == 12345.f) out[0] = s;
}

__global__ void k_dfma(double *out, int iters) {
  double y[8];
  for (int i = 0; i < 8; ++i) y[i] = 0.001 * (threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) y[i] = fma(y[i], 0.999, 0.001);
  }
  double s = 0;
  for (int i = 0; i < 8; ++i) s += y[i];
  if (s == 12345.) out[0] = s;
}

// The JAM pair-sum instruction mix without memory: per pair of points FMUL2, FFMA2,
// two MUFU.EX2 and two FFMA2, over 4 independent pairs per thread.
__global__ void k_jam_mix(float *out, int iters) {
  float2 X[4], Y[4], acc[4];
  for (int p = 0; p < 4; ++p) {
    X[p] = make_float2(0.01f * (threadIdx.x + p), 0.02f * p);
    Y[p] = make_float2(0.03f * p, 0.01f * threadIdx.x);
    acc[p] = make_float2(0.f, 0.f);
  }
  float cxv = -0.5f, cyv = -0.25f, czv = 0.5f, cwv = 0.125f;
  for (int it = 0; it < iters; ++it) {
    const float2 cx = make_float2(cxv, cxv), cy = make_float2(cyv, cyv);
    const float2 cz = make_float2(czv, czv), cw = make_float2(cwv, cwv);
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const float2 arg = __ffma2_rn(cy, Y[p], __fmul2_rn(cx, X[p]));
      const float2 E = make_float2(ex2(arg.x), ex2(arg.y));
      acc[p] = __ffma2_rn(__ffma2_rn(cw, X[p], cz), E, acc[p]);
    }
    cxv += 1e-7f;
    cyv -= 1e-7f;
  }
  float s = 0;
  for (int p = 0; p < 4; ++p) s += acc[p].x + acc[p].y;
  if (s == 12345.f) out[0] = s;
}

int main() {
  int nsm = 0, clk_khz = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, 0);
  cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, 0);
  float *o;
  double *od;
  cudaMalloc(&o, 4);
  cudaMalloc(&od, 8);
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  const int blocks = nsm * 8, thr = 256;
  for (int rep = 0; rep < 3; ++rep) {
    const int it = 20000;
    float ms;
    cudaEventRecord(a);
    k_ex2<<<blocks, thr>>>(o, it);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    const double ex2s = (double)blocks * thr * it * 8 / (ms * 1e-3);
    cudaEventRecord(a);
    k_ffma<<<blocks, thr>>>(o, it * 4);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    const double ffs = (double)blocks * thr * it * 4 * 8 / (ms * 1e-3);
    cudaEventRecord(a);
    k_dfma<<<blocks, thr>>>(od, it / 8);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    const double dfs = (double)blocks * thr * (it / 8) * 8 / (ms * 1e-3);
    // ratios to FFMA, whose issue rate is 128 lanes/clk/SM, cancel the unknown clock
    printf("rep=%d sm=%d ex2/s=%.4e ffma/s=%.4e dfma/s=%.4e ex2_per_ffma=%.4f dfma_per_ffma=%.5f "
           "ex2_per_clk_sm(at 128 ffma/clk)=%.2f dfma_per_clk_sm=%.2f\n",
           rep, nsm, ex2s, ffs, dfs, ex2s / ffs, dfs / ffs, 128.0 * ex2s / ffs, 128.0 * dfs / ffs);
  }
  for (int rep = 0; rep < 2; ++rep) {
    const int it = 4000;
    float ms, ms_f;
    cudaEventRecord(a);
    k_jam_mix<<<blocks, thr>>>(o, it);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms, a, b);
    cudaEventRecord(a);
    k_ffma<<<blocks, thr>>>(o, it * 4);
    cudaEventRecord(b);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(&ms_f, a, b);
    const double evals = (double)blocks * thr * it * 8 / (ms * 1e-3);
    const double ffs = (double)blocks * thr * it * 4 * 8 / (ms_f * 1e-3);
    printf("jam_mix rep=%d evals/s=%.4e evals_per_clk_sm(at 128 ffma/clk)=%.2f\n", rep, evals,
           128.0 * evals / ffs);
  }
  printf("status=%s\n", cudaGetErrorString(cudaDeviceSynchronize()));
  return 0;
}
