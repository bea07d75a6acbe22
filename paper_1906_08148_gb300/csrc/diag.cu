// diag.cu -- a check of the device-timeout path (no counterpart in the paper).
//
// Every device-side wait of the library is bounded: when it runs out the
// kernel sets the context's error word and returns, and the host maps the
// word to SPAMM_E_TIMEOUT.  This entry point exercises exactly that path
// without faulting anything: one thread waits, with a short bound, on an
// mbarrier phase that nothing completes.
#include "internal.cuh"
#include "ptx.cuh"

namespace spamm {

__global__ void timeout_probe_kernel(uint64_t wait_ns, int* __restrict__ err) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  mbar_init(&bar, 1);
  fence_mbar_init();
  // phase 0 needs one arrival; none comes, so the bounded wait gives up
  if (!mbar_wait_bounded(&bar, 0u, 1ll << 40, wait_ns)) atomicOr(err, DEV_ERR_TIMEOUT);
}

}  // namespace spamm

using namespace spamm;

extern "C" SPAMM_API spamm_status spamm_check_timeout_path(spamm_ctx ctx, int64_t wait_ns) {
  if (!ctx || wait_ns <= 0 || wait_ns > 2000000000ll) return SPAMM_E_INVALID_ARG;
  try {
    CK(cudaSetDevice(ctx->device));
    timeout_probe_kernel<<<1, 32, 0, ctx->stream>>>((uint64_t)wait_ns, ctx->d_err);
    CK_LAUNCH("timeout_probe_kernel");
    sync_and_check(ctx);  // maps the error word (and clears it)
    return SPAMM_OK;
  } catch (const Error& e) {
    ctx->last_error = e.msg;
    return e.status;
  }
}
