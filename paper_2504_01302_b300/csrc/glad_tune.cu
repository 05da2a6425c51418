// Autotuner for the launch shapes of the JAM kernels: sky points per thread of the
// pair-sum kernel with a register cap for a minimum number of resident CTAs per SM
// (the candidate list in k_jam.cu), grid or persistent form, and table entries per
// thread of its adjoint (2, 4).  Each
// candidate is timed with CUDA events on the caller's batch; the fastest is kept in the
// context and, when GLAD_TUNE_CACHE names a file, stored there keyed by the batch shape
// and the device name so later processes skip the timing.
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>

#include "glad_internal.cuh"

glad_status glad_set_error(glad_status s, const char *msg);
cudaError_t grad_ws_ensure(glad_ctx *c, int B);
cudaError_t launch_jam_fg(glad_ctx *c, const int *sys_id, int B, cudaStream_t st);
float *grad_resid_buffer(glad_ctx *c);
cudaError_t time_jam_adj(glad_ctx *c, const int *sys_id, int B, cudaStream_t st);

namespace {

// launch shape of the JAM pair sum as one integer: 1000000 * form of the sum +
// 100000 * persistent + 1000 * points per thread + 10 * min CTAs per SM + unroll
int jam_code(const glad_ctx *c) {
  return c->tune.jam_form * 1000000 + c->tune.jam_persistent * 100000 + c->tune.jam_pts * 1000 +
         c->tune.jam_minb * 10 + c->tune.jam_unroll;
}

// decodes a jam_code into the context's tuning; false (nothing changed) for codes this build
// does not have
bool set_jam_code(glad_ctx *c, int code) {
  if (code < 0) return false;
  const int form = code / 1000000, pers = (code / 100000) % 10, pts = (code % 100000) / 1000;
  const int minb = (code % 1000) / 10, unr = code % 10;
  if (form > 3 || pers > 1 || !jam_shape_supported(pts, minb, unr, form)) return false;
  c->tune.jam_form = form;
  c->tune.jam_persistent = pers;
  c->tune.jam_pts = pts;
  c->tune.jam_minb = minb;
  c->tune.jam_unroll = unr;
  return true;
}

std::string tune_key(glad_ctx *c, int B) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaGetDeviceProperties(&prop, dev);
  std::string k = std::string(prop.name) + "|B=" + std::to_string(B);
  for (auto &s : c->h_sysdev)
    k += "|" + std::to_string(s.n_sub) + "x" + std::to_string(s.n_ent);
  for (auto &ch : k)
    if (ch == ' ') ch = '_';
  return k;
}

bool cache_lookup(const std::string &key, int *pts, int *ept) {
  const char *path = getenv("GLAD_TUNE_CACHE");
  if (!path) return false;
  FILE *f = fopen(path, "r");
  if (!f) return false;
  char k[4096];
  int a, b;
  bool found = false;
  while (fscanf(f, "%4095s %d %d", k, &a, &b) == 3)
    if (key == k) {
      *pts = a;
      *ept = b;
      found = true;
    }
  fclose(f);
  return found;
}

void cache_store(const std::string &key, int pts, int ept) {
  const char *path = getenv("GLAD_TUNE_CACHE");
  if (!path) return;
  FILE *f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s %d %d\n", key.c_str(), pts, ept);
  fclose(f);
}

template <class F>
float time_ms(cudaStream_t st, F &&launch, int reps) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  launch();  // warm-up
  cudaEventRecord(a, st);
  for (int r = 0; r < reps; ++r) launch();
  cudaEventRecord(b, st);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

}  // namespace

extern "C" glad_status glad_autotune(glad_ctx *c, const int *sys_id, const double *theta, int B,
                                     int with_grad, void *stream) {
  if (!c || !sys_id || !theta || B < 1) return glad_set_error(GLAD_EINVAL, "glad_autotune: bad arguments");
  cudaStream_t st = (cudaStream_t)stream;
  const std::string key = tune_key(c, B);
  int pts = 8, ept = 4;
  int code = 0;
  // a cached choice counts only while this build still has that launch shape
  if (cache_lookup(key, &code, &ept) && (ept == 2 || ept == 4) && set_jam_code(c, code)) {
    c->tune.adj_ept = ept;
    return GLAD_OK;
  }
  // a forward pass (gradient flavour when asked) leaves tables and point data in place
  double *logL = nullptr, *grad = nullptr;
  int *status = nullptr;
  glad_status s;
  // use the library's own entry points for the warm state
  extern glad_status glad_loglike(glad_ctx *, const int *, const double *, int, double *, int *,
                                  double *, void *);
  extern glad_status glad_loglike_grad(glad_ctx *, const int *, const double *, int, double *,
                                       double *, int *, double *, void *);
  if (cudaMalloc(&logL, sizeof(double) * B) != cudaSuccess ||
      cudaMalloc(&status, sizeof(int) * B) != cudaSuccess ||
      cudaMalloc(&grad, sizeof(double) * B * GLAD_NTHETA) != cudaSuccess) {
    cudaFree(logL);
    cudaFree(status);
    cudaFree(grad);
    return glad_set_error(GLAD_ENOMEM, "glad_autotune: scratch allocation failed");
  }
  s = with_grad ? glad_loglike_grad(c, sys_id, theta, B, logL, grad, status, nullptr, stream)
                : glad_loglike(c, sys_id, theta, B, logL, status, nullptr, stream);
  if (s == GLAD_OK) {
    // (points per thread, minimum CTAs per SM asked of the register allocator)
    int cand[32][4];
    const int ncand = jam_shape_list(cand, 32);
    float best = 1e30f;
    int minb = 4, unr = 2, form = 0;
    c->tune.jam_persistent = 0;
    for (int ic = 0; ic < ncand && ic < 32; ++ic) {
      const int *cd = cand[ic];
      c->tune.jam_pts = cd[0];
      c->tune.jam_minb = cd[1];
      c->tune.jam_unroll = cd[2];
      c->tune.jam_form = cd[3];
      const float ms = time_ms(st, [&]() { launch_jam(c, sys_id, B, st); }, 2);
      if (ms < best) {
        best = ms;
        pts = cd[0];
        minb = cd[1];
        unr = cd[2];
        form = cd[3];
      }
    }
    c->tune.jam_pts = pts;
    c->tune.jam_minb = minb;
    c->tune.jam_unroll = unr;
    c->tune.jam_form = form;
    // the same shape as one persistent launch over the (sample, tile) work list
    c->tune.jam_persistent = 1;
    const float ms_p = time_ms(st, [&]() { launch_jam(c, sys_id, B, st); }, 2);
    c->tune.jam_persistent = ms_p < best ? 1 : 0;
    if (with_grad) {
      const int cand_ept[2] = {2, 4};
      best = 1e30f;
      for (int e : cand_ept) {
        c->tune.adj_ept = e;
        const float ms = time_ms(st, [&]() { time_jam_adj(c, sys_id, B, st); }, 2);
        if (ms < best) {
          best = ms;
          ept = e;
        }
      }
      c->tune.adj_ept = ept;
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = glad_set_error(GLAD_ECUDA, cudaGetErrorString(e));
    else
      cache_store(key, jam_code(c), c->tune.adj_ept);
  }
  cudaFree(logL);
  cudaFree(status);
  cudaFree(grad);
  return s;
}

extern "C" int glad_tuning(glad_ctx *c, int *jam_pts, int *adj_ept) {
  if (!c) return -1;
  if (jam_pts) *jam_pts = jam_code(c);
  if (adj_ept) *adj_ept = c->tune.adj_ept;
  return 0;
}

extern "C" glad_status glad_set_tuning(glad_ctx *c, int jam_code, int adj_ept) {
  if (!c) return glad_set_error(GLAD_EINVAL, "glad_set_tuning: null context");
  if ((adj_ept != 2 && adj_ept != 4) || !set_jam_code(c, jam_code))
    return glad_set_error(GLAD_EINVAL, "glad_set_tuning: unsupported launch shape");
  c->tune.adj_ept = adj_ept;
  return GLAD_OK;
}
