// noalloc.cu -- leaf squared norms and their total without any device
// allocation: the reduction scratch is a fixed file-scope device array.
#include <mutex>

#include "internal.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int64_t kLeavesPerPartial = 64;  // a block's share: grids of ~nleaves / 64 blocks fill the SMs evenly
constexpr int64_t kMaxPartials = SPAMM_NOALLOC_MAX_LEAVES / kLeavesPerPartial;

// One FP64 partial sum per 64 leaves, shared by every call on a device.
static __device__ __align__(256) double g_noalloc_partials[kMaxPartials];

// Device address of g_noalloc_partials per device ordinal, looked up once.
constexpr int kMaxDevices = 64;
double* g_partials_addr[kMaxDevices] = {};
std::mutex g_setup_mutex;

// Warp per leaf; lane l reads the 16-byte pairs l, l+32, ... and squares are
// accumulated with FMAs in that fixed order, then combined by a butterfly.
__global__ void noalloc_sqnorm_kernel(const double* __restrict__ payload, int64_t nleaves, int bs,
                                      double* __restrict__ sq_out, double* __restrict__ partials) {
  __shared__ double warp_sum[kThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t e = (int64_t)bs * bs;
  const int pairs = (int)(e / 2);
  // block b owns leaves [b * 64, (b + 1) * 64); each warp takes every 8th of them
  const int64_t first = (int64_t)blockIdx.x * kLeavesPerPartial;
  double block_part = 0.0;
  for (int64_t i = warp; i < kLeavesPerPartial; i += kThreads / 32) {
    const int64_t q = first + i;
    if (q >= nleaves) break;
    const double2* src = reinterpret_cast<const double2*>(payload + q * e);
    double s = 0.0;
    for (int p = lane; p < pairs; p += 32) {
      const double2 v = __ldg(src + p);
      s = __fma_rn(v.x, v.x, s);
      s = __fma_rn(v.y, v.y, s);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) sq_out[q] = s;
    block_part += s;
  }
  if (lane == 0) warp_sum[warp] = block_part;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) t += warp_sum[w];
    partials[blockIdx.x] = t;
  }
}

// One warp adds the partials: lane l those at l, l + 32, ... in index order,
// then a butterfly (a fixed order, so the total is reproducible).
__global__ void noalloc_total_kernel(const double* __restrict__ partials, int64_t nparts, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  double t = 0.0;
  for (int64_t i = lane; i < nparts; i += 32) t += partials[i];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
  if (lane == 0) *out = t;
}

// Set-up, once per device, with that device current: the kernel needs the
// array's device address, which host code can only learn from the runtime.
spamm_status partials_address(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return SPAMM_E_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_partials_addr[device]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_partials) != cudaSuccess || !p) {
      cudaGetLastError();
      return SPAMM_E_CUDA;
    }
    g_partials_addr[device] = static_cast<double*>(p);
  }
  *out = g_partials_addr[device];
  return SPAMM_OK;
}

}  // namespace

extern "C" spamm_status spamm_leaf_sqnorms_noalloc(const double* payload, int64_t nleaves, int bs, double* sq_out,
                                                   double* total_out, void* cuda_stream) {
  if (bs != 32 && bs != 64 && bs != 128 && bs != 256) return SPAMM_E_INVALID_ARG;
  if (nleaves < 0 || !total_out || (nleaves > 0 && (!payload || !sq_out))) return SPAMM_E_INVALID_ARG;
  if (nleaves > SPAMM_NOALLOC_MAX_LEAVES) return SPAMM_E_CAPACITY;
  // the kernel reads the payload in 16-byte pairs and writes 8-byte results:
  // a misaligned pointer is refused here, before anything reaches the GPU
  if (nleaves > 0 && (reinterpret_cast<uintptr_t>(payload) % 16 != 0 || reinterpret_cast<uintptr_t>(sq_out) % 8 != 0))
    return SPAMM_E_INVALID_ARG;
  if (reinterpret_cast<uintptr_t>(total_out) % 8 != 0) return SPAMM_E_INVALID_ARG;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) {
    cudaGetLastError();
    return SPAMM_E_CUDA;
  }
  double* partials = nullptr;
  const spamm_status st = partials_address(device, &partials);
  if (st != SPAMM_OK) return st;
  cudaStream_t stream = static_cast<cudaStream_t>(cuda_stream);
  const int64_t nparts = (nleaves + kLeavesPerPartial - 1) / kLeavesPerPartial;
  if (nparts > 0) {
    noalloc_sqnorm_kernel<<<(unsigned)nparts, kThreads, 0, stream>>>(payload, nleaves, bs, sq_out, partials);
    ++spamm::g_kernel_launches;
  }
  noalloc_total_kernel<<<1, 32, 0, stream>>>(partials, nparts, total_out);
  ++spamm::g_kernel_launches;
  return cudaGetLastError() == cudaSuccess ? SPAMM_OK : SPAMM_E_CUDA;
}
