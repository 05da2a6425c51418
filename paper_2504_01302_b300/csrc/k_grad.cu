// Gradient of the joint log-likelihood (adjoint kernels).
#include "glad_internal.cuh"

cudaError_t launch_grad(glad_ctx *c, const int *sys_id, const double *theta, int B, double *grad,
                        cudaStream_t st) {
  (void)c; (void)sys_id; (void)theta; (void)B; (void)grad; (void)st;
  return cudaErrorNotSupported;
}
cudaError_t grad_ws_ensure(glad_ctx *c, int B) { (void)c; (void)B; return cudaSuccess; }
void grad_ws_free(glad_ctx *c) { (void)c; }
