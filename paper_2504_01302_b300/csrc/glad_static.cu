// glad_loglike_static: the batched log-likelihood for callers that must not allocate
// device memory while they run -- code that runs inside a CUDA-graph capture owned by
// someone else, a real-time sampler loop with a fixed memory budget, or a host process
// that shares the device under an allocator it does not control.  The per-sample
// scratch (coefficient tables, unblurred images, bin sums, chi^2 terms) lives in one
// file-scope device array instead of the context's cudaMalloc'd workspace; the kernels
// are the ones glad_loglike launches.
#include <mutex>
#include <string>

#include "glad_internal.cuh"

glad_status glad_set_error(glad_status s, const char *msg);

namespace {

// 64 MiB, held by every device that loads the library until the process exits.
constexpr size_t kStaticScratchBytes = size_t(64) << 20;
__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// Device address of g_static_scratch on the current device (the host-side symbol is
// only a stand-in).  Looked up once per device, on the first call made on it.
cudaError_t scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

// Lay the per-sample arrays of a batch of B out in the scratch; returns the bytes used.
size_t carve(const glad_ctx *c, int B, unsigned char *base, WsDev *w) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> void * {
    void *p = base ? base + off : nullptr;
    off += align256(bytes);
    return p;
  };
  const size_t b = (size_t)B;
  w->lp = (LensP *)take(b * sizeof(LensP));
  w->dp = (DynP *)take(b * sizeof(DynP));
  w->nu0 = (double *)take(b * c->max_light * sizeof(double));
  w->c0 = (double *)take(b * c->max_light * sizeof(double));
  w->Cj = (double *)take(b * c->max_mass_tot * sizeof(double));
  w->e2 = (double *)take(b * c->max_mass_tot * sizeof(double));
  w->I0f = (float *)take(b * c->max_light * sizeof(float));
  w->tab = (float4 *)take(b * c->max_ent * sizeof(float4));
  w->img = (float *)take(b * c->max_pix * sizeof(float));
  w->binacc = (double *)take(b * c->max_bins * 2 * sizeof(double));
  w->terms = (double *)take(b * 4 * sizeof(double));
  w->status = (int *)take(b * sizeof(int));
  // work list of the persistent JAM form (k_worklist writes every entry and the counter)
  w->wl_off = (int *)take((b + 1) * sizeof(int));
  w->wl_counter = (int *)take(sizeof(int));
  w->sph_mt = (float4 *)take(b * c->max_smg * sizeof(float4));
  w->sph_mrz = (float *)take(b * c->max_smg * sizeof(float));
  w->sph_tr = (float4 *)take(b * c->max_light * sizeof(float4));
  w->sgrid = (float2 *)take(b * c->max_sgrid * sizeof(float2));
  return off;
}

}  // namespace

extern "C" glad_status glad_loglike_static(glad_ctx *c, const int *sys_id, const double *theta,
                                           int B, double *logL, int *sample_status, double *terms,
                                           void *stream) {
  glad_set_error(GLAD_OK, "");  // a successful call leaves glad_last_error() empty
  if (!c || !sys_id || !theta || !logL || !sample_status || B < 1)
    return glad_set_error(GLAD_EINVAL, "glad_loglike_static: bad arguments");
  if (c->n_pix)
    return glad_set_error(GLAD_EUNSUPPORTED, "glad_loglike_static: pixelated-source systems need "
                                             "the allocating entry points");
  WsDev w{};
  const size_t need = carve(c, B, nullptr, &w);
  if (need > kStaticScratchBytes) {
    const size_t per = carve(c, 1, nullptr, &w);
    std::string m = "glad_loglike_static: a batch of " + std::to_string(B) + " needs " +
                    std::to_string(need) + " bytes of scratch; the static array holds " +
                    std::to_string(kStaticScratchBytes) + " (about " +
                    std::to_string(kStaticScratchBytes / per) + " samples of these systems)";
    return glad_set_error(GLAD_EUNSUPPORTED, m.c_str());
  }
  void *base = nullptr;
  cudaError_t e = scratch_address(&base);
  if (e != cudaSuccess) {
    std::string m = std::string("glad_loglike_static: cudaGetSymbolAddress failed: ") +
                    cudaGetErrorString(e);
    return glad_set_error(GLAD_ECUDA, m.c_str());
  }
  carve(c, B, (unsigned char *)base, &w);
  // same JAM summation and launch shape as glad_loglike; evaluations are not counted
  // (w.evals stays null), so glad_jam_evaluations keeps the figure of the last counted call
  w.neg_mode = c->tune.neg_mode;
  cudaStream_t st = (cudaStream_t)stream;
  // the launchers read the context's workspace view: point it at the scratch for the
  // duration of the launches (kernel arguments are copied at launch) and restore it
  const WsDev saved = c->ws.d;
  c->ws.d = w;
  // accumulators that the kernels add into start at zero on every call
  e = cudaMemsetAsync(w.terms, 0, sizeof(double) * 4 * (size_t)B, st);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(w.binacc, 0, sizeof(double) * 2 * c->max_bins * (size_t)B, st);
  if (e == cudaSuccess) e = launch_prep(c, sys_id, theta, B, st);
  if (e == cudaSuccess) e = launch_dyn_tables(c, sys_id, B, st);
  if (e == cudaSuccess) e = launch_lens(c, sys_id, B, nullptr, st);
  if (e == cudaSuccess) e = launch_dyn_sums(c, sys_id, B, st);
  if (e == cudaSuccess) e = launch_kin_finalize(c, sys_id, B, nullptr, st);
  if (e == cudaSuccess) e = launch_combine(c, B, logL, sample_status, terms, st);
  c->ws.d = saved;
  if (e != cudaSuccess) {
    std::string m = std::string("glad_loglike_static: launch failed: ") + cudaGetErrorString(e);
    return glad_set_error(GLAD_ECUDA, m.c_str());
  }
  return GLAD_OK;
}
