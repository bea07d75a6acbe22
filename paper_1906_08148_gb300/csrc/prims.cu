// prims.cu -- errors, device memory, prefix sums and radix sort.
#include <cstdio>
#include <cstring>

#include "internal.cuh"

namespace spamm {

thread_local unsigned long long g_kernel_launches = 0;  // per host thread: a context is used by one thread

void fail(spamm_status st, const std::string& msg) { throw Error{st, msg}; }

void check_cuda(cudaError_t e, const char* what, const char* file, int line) {
  if (e == cudaSuccess) return;
  char buf[512];
  snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    fail(SPAMM_E_OOM, buf);
  }
  fail(SPAMM_E_CUDA, buf);
}

Buf::~Buf() {
  if (!p) return;
  if (ctx->ufree)
    ctx->ufree(p, ctx->user);
  else
    cudaFreeAsync(p, ctx->stream);
}

BufP alloc_bytes(spamm_ctx ctx, size_t bytes) {
  auto b = std::make_shared<Buf>();
  b->ctx = ctx;
  b->bytes = bytes;
  if (bytes == 0) return b;
  size_t rounded = (bytes + 255) & ~(size_t)255;
  if (ctx->ualloc) {
    b->p = ctx->ualloc(rounded, ctx->user);
    if (!b->p) fail(SPAMM_E_OOM, "allocator returned NULL for " + std::to_string(rounded) + " bytes");
  } else {
    cudaError_t e = cudaMallocAsync(&b->p, rounded, ctx->stream);
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (e == cudaErrorMemoryAllocation && cudaStreamIsCapturing(ctx->stream, &cap) == cudaSuccess &&
        cap == cudaStreamCaptureStatusNone) {
      // the pool keeps freed blocks; hand them back to the device and try once more
      cudaGetLastError();
      cudaMemPool_t pool;
      if (cudaStreamSynchronize(ctx->stream) == cudaSuccess &&
          cudaDeviceGetDefaultMemPool(&pool, ctx->device) == cudaSuccess &&
          cudaMemPoolTrimTo(pool, 0) == cudaSuccess)
        e = cudaMallocAsync(&b->p, rounded, ctx->stream);
    }
    if (e != cudaSuccess) {
      b->p = nullptr;
      cudaGetLastError();
      fail(e == cudaErrorMemoryAllocation ? SPAMM_E_OOM : SPAMM_E_CUDA,
           "device allocation of " + std::to_string(rounded) + " bytes failed: " + cudaGetErrorString(e));
    }
  }
  return b;
}

template <class T>
T read_scalar(spamm_ctx ctx, const T* d) {
  CK(cudaMemcpyAsync(ctx->h_pinned, d, sizeof(T), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  T v;
  memcpy(&v, ctx->h_pinned, sizeof(T));
  return v;
}
template uint64_t read_scalar<uint64_t>(spamm_ctx, const uint64_t*);
template int64_t read_scalar<int64_t>(spamm_ctx, const int64_t*);
template double read_scalar<double>(spamm_ctx, const double*);
template int read_scalar<int>(spamm_ctx, const int*);

void clear_device_error(spamm_ctx ctx) { CK(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream)); }

void sync_and_check(spamm_ctx ctx) {
  CK(cudaStreamSynchronize(ctx->stream));
  CK(cudaGetLastError());
  int err = read_scalar<int>(ctx, ctx->d_err);
  if (!err) return;
  clear_device_error(ctx);
  if (err & DEV_ERR_TIMEOUT) fail(SPAMM_E_TIMEOUT, "a bounded device-side wait ran out");
  if (err & DEV_ERR_NONFINITE) fail(SPAMM_E_NONFINITE, "input contains Inf or NaN");
  if (err & DEV_ERR_DUPLICATE) fail(SPAMM_E_INVALID_ARG, "repeated leaf coordinate");
  fail(SPAMM_E_INVALID_ARG, "index out of range");
}

// ------------------------------------------------------------ prefix sums
constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

// Exclusive scan across the 256 threads of a block; *total = block sum.
// T = uint64_t (exact) or double (fixed tiling, so the rounding is the same
// on every run).
template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* total) {
  __shared__ T warp_tot[kScanThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T x = v;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, off);
    if (lane >= off) x += y;
  }
  if (lane == 31) warp_tot[warp] = x;
  __syncthreads();
  T before = 0, all = 0;
#pragma unroll
  for (int w = 0; w < kScanThreads / 32; ++w) {
    T t = warp_tot[w];
    if (w < warp) before += t;
    all += t;
  }
  __syncthreads();
  *total = all;
  const T prev = __shfl_up_sync(0xffffffffu, x, 1);  // the previous lane's inclusive sum
  return lane == 0 ? before : before + prev;
}

template <class T>
__global__ void scan_reduce_kernel(const T* __restrict__ in, int64_t n, T* __restrict__ bsum) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  T s = 0;
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    int64_t q = base + i;
    if (q < n) s += in[q];
  }
  T total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

template <class T>
__global__ void scan_blocksums_kernel(T* bsum, int64_t nblocks, T* d_total) {
  T carry = 0;
  for (int64_t base = 0; base < nblocks; base += kScanThreads) {
    int64_t q = base + threadIdx.x;
    T v = q < nblocks ? bsum[q] : 0;
    T total;
    T ex = block_exclusive_scan(v, &total);
    if (q < nblocks) bsum[q] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0 && d_total) *d_total = carry;
}

// inclusive = false: out[q] = sum of in[0 .. q-1]; true: sum of in[0 .. q]
template <class T>
__global__ void scan_down_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t n, const T* __restrict__ bsum,
                                 bool inclusive) {
  __shared__ T tile[kScanTile];
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    int64_t q = base + i;
    tile[i] = q < n ? in[q] : 0;
  }
  __syncthreads();
  T loc[kScanItems];
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    loc[i] = s;
    s += tile[threadIdx.x * kScanItems + i];
  }
  T total;
  T ex = block_exclusive_scan(s, &total) + bsum[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const T mine = tile[threadIdx.x * kScanItems + i];
    tile[threadIdx.x * kScanItems + i] = inclusive ? (ex + loc[i]) + mine : ex + loc[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    int64_t q = base + i;
    if (q < n) out[q] = tile[i];
  }
}

// n <= kScanTile: the whole scan in one block, one launch.
template <class T>
__global__ void scan_one_tile_kernel(const T* __restrict__ in, T* __restrict__ out, int64_t n, T* d_total,
                                     bool inclusive) {
  __shared__ T tile[kScanTile];
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) tile[i] = i < n ? in[i] : 0;
  __syncthreads();
  T loc[kScanItems];
  T s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    loc[i] = s;
    s += tile[threadIdx.x * kScanItems + i];
  }
  T total;
  const T ex = block_exclusive_scan(s, &total);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const T mine = tile[threadIdx.x * kScanItems + i];
    tile[threadIdx.x * kScanItems + i] = inclusive ? (ex + loc[i]) + mine : ex + loc[i];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads)
    if (i < n) out[i] = tile[i];
  if (threadIdx.x == 0 && d_total) *d_total = total;
}

template <class T>
static void scan_any(spamm_ctx ctx, const T* in, T* out, int64_t n, T* d_total, bool inclusive) {
  if (n <= 0) {
    if (d_total) CK(cudaMemsetAsync(d_total, 0, sizeof(T), ctx->stream));
    return;
  }
  if (n <= kScanTile) {
    scan_one_tile_kernel<T><<<1, kScanThreads, 0, ctx->stream>>>(in, out, n, d_total, inclusive);
    CK_LAUNCH("scan_one_tile_kernel");
    return;
  }
  const int64_t nblocks = (n + kScanTile - 1) / kScanTile;
  BufP bs = alloc_n<T>(ctx, nblocks);
  scan_reduce_kernel<T><<<(unsigned)nblocks, kScanThreads, 0, ctx->stream>>>(in, n, P<T>(bs));
  CK_LAUNCH("scan_reduce_kernel");
  scan_blocksums_kernel<T><<<1, kScanThreads, 0, ctx->stream>>>(P<T>(bs), nblocks, d_total);
  CK_LAUNCH("scan_blocksums_kernel");
  scan_down_kernel<T><<<(unsigned)nblocks, kScanThreads, 0, ctx->stream>>>(in, out, n, P<T>(bs), inclusive);
  CK_LAUNCH("scan_down_kernel");
}

void scan_exclusive_u64(spamm_ctx ctx, const uint64_t* in, uint64_t* out, int64_t n, uint64_t* d_total) {
  scan_any<uint64_t>(ctx, in, out, n, d_total, false);
}

void scan_inclusive_f64(spamm_ctx ctx, const double* in, double* out, int64_t n) {
  scan_any<double>(ctx, in, out, n, nullptr, true);
}

// ------------------------------------------------------------- radix sort
constexpr int kRadixBits = 4;
constexpr int kRadixBins = 1 << kRadixBits;

__global__ void radix_hist_kernel(const uint64_t* __restrict__ keys, int64_t n, int shift,
                                  uint64_t* __restrict__ hist, int64_t nblocks) {
  __shared__ unsigned cnt[kRadixBins];
  if (threadIdx.x < kRadixBins) cnt[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += kScanThreads) {
    int64_t q = base + i;
    if (q < n) atomicAdd(&cnt[(keys[q] >> shift) & (kRadixBins - 1)], 1u);
  }
  __syncthreads();
  if (threadIdx.x < kRadixBins) hist[(int64_t)threadIdx.x * nblocks + blockIdx.x] = cnt[threadIdx.x];
}

__global__ void radix_scatter_kernel(const uint64_t* __restrict__ kin, const int64_t* __restrict__ vin,
                                     uint64_t* __restrict__ kout, int64_t* __restrict__ vout, int64_t n, int shift,
                                     const uint64_t* __restrict__ offs, int64_t nblocks) {
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  unsigned c[kRadixBins];
#pragma unroll
  for (int d = 0; d < kRadixBins; ++d) c[d] = 0;
  for (int i = 0; i < kScanItems; ++i) {
    int64_t q = base + i;
    if (q < n) c[(kin[q] >> shift) & (kRadixBins - 1)]++;
  }
  uint64_t pre[kRadixBins];
#pragma unroll
  for (int d = 0; d < kRadixBins; ++d) {
    uint64_t tot;
    pre[d] = block_exclusive_scan<uint64_t>(c[d], &tot) + offs[(int64_t)d * nblocks + blockIdx.x];
  }
  for (int i = 0; i < kScanItems; ++i) {
    int64_t q = base + i;
    if (q >= n) break;
    uint64_t k = kin[q];
    int d = (int)((k >> shift) & (kRadixBins - 1));
    uint64_t pos = 0;
#pragma unroll
    for (int e = 0; e < kRadixBins; ++e)
      if (e == d) pos = pre[e]++;
    kout[pos] = k;
    vout[pos] = vin[q];
  }
}

void radix_sort_pairs(spamm_ctx ctx, uint64_t* keys, int64_t* vals, int64_t n, int bits) {
  if (n <= 1 || bits <= 0) return;
  const int64_t nblocks = (n + kScanTile - 1) / kScanTile;
  BufP k2 = alloc_n<uint64_t>(ctx, n), v2 = alloc_n<int64_t>(ctx, n);
  BufP hist = alloc_n<uint64_t>(ctx, nblocks * kRadixBins);
  uint64_t *ka = keys, *kb = P<uint64_t>(k2);
  int64_t *va = vals, *vb = P<int64_t>(v2);
  for (int shift = 0; shift < bits; shift += kRadixBits) {
    radix_hist_kernel<<<(unsigned)nblocks, kScanThreads, 0, ctx->stream>>>(ka, n, shift, P<uint64_t>(hist), nblocks);
    CK_LAUNCH("radix_hist_kernel");
    scan_exclusive_u64(ctx, P<uint64_t>(hist), P<uint64_t>(hist), nblocks * kRadixBins, nullptr);
    radix_scatter_kernel<<<(unsigned)nblocks, kScanThreads, 0, ctx->stream>>>(ka, va, kb, vb, n, shift,
                                                                            P<uint64_t>(hist), nblocks);
    CK_LAUNCH("radix_scatter_kernel");
    std::swap(ka, kb);
    std::swap(va, vb);
  }
  if (ka != keys) {
    CK(cudaMemcpyAsync(keys, ka, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(vals, va, n * sizeof(int64_t), cudaMemcpyDeviceToDevice, ctx->stream));
  }
}

}  // namespace spamm
