// gemm_fp64.cu -- kernel (c), FP64 form, with the C-leaf norms of kernel (d)
// fused into its epilogue.
//
// C_ij = sum over the kept k (ascending) of A_ik B_kj, one output leaf per
// work item (Algorithm 1, "C = AB" at the lowest level, run batched over the
// task list as Section 4.4 describes).  Persistent CTAs claim output leaves
// from an atomic counter; every output leaf is owned by one CTA, so there are
// no atomics on C and the k order is fixed (results do not depend on the
// schedule).  Operand leaves are contiguous bs*bs FP64 blocks and are staged
// in shared memory by 1-D TMA bulk copies, double-buffered on mbarriers; the
// product is register-tiled DFMA (FP64 has no tcgen05 kind; DFMA measures
// faster than the FP64 mma.sync path on this part).
#include "internal.cuh"
#include "ptx.cuh"

namespace spamm {

constexpr int kGemmThreads = 256;

template <int BS>
__global__ void __launch_bounds__(kGemmThreads) gemm_fp64_kernel(
    int64_t G, const int64_t* __restrict__ gstart, const int32_t* __restrict__ ta, const int32_t* __restrict__ tb,
    const int64_t* __restrict__ slotA, const int64_t* __restrict__ slotB, const double* __restrict__ poolA,
    const double* __restrict__ poolB, double* __restrict__ cpool, double* __restrict__ csq,
    unsigned long long* __restrict__ work, int* __restrict__ err) {
  constexpr int LEAF = BS * BS;
  constexpr uint32_t LEAF_BYTES = LEAF * sizeof(double);
  constexpr int TM = BS / 16;  // per-thread tile TM x TM: rows tr + 16 i, cols tc + 16 j
  extern __shared__ __align__(128) unsigned char smem_raw[];
  double* sA[2] = {reinterpret_cast<double*>(smem_raw), reinterpret_cast<double*>(smem_raw) + 2 * LEAF};
  double* sB[2] = {reinterpret_cast<double*>(smem_raw) + LEAF, reinterpret_cast<double*>(smem_raw) + 3 * LEAF};
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int64_t s_g;
  __shared__ int s_abort;
  __shared__ double s_red[kGemmThreads / 32];

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int tr = tid >> 4, tc = tid & 15;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    s_abort = 0;
  }
  __syncthreads();
  uint32_t phase[2] = {0u, 0u};
  uint32_t inflight = 0;  // bit s: stage s has a copy that nobody waited for

  auto issue = [&](int64_t q, int s) {
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(&bar[s], 2 * LEAF_BYTES);
    bulk_g2s(sA[s], poolA + slotA[ta[q]] * LEAF, LEAF_BYTES, &bar[s]);
    bulk_g2s(sB[s], poolB + slotB[tb[q]] * LEAF, LEAF_BYTES, &bar[s]);
  };

  for (;;) {
    if (tid == 0) s_g = (int64_t)atomicAdd(work, 1ull);
    __syncthreads();
    const int64_t g = s_g;
    if (g >= G || s_abort) break;
    const int64_t q0 = gstart[g], q1 = gstart[g + 1];
    double acc[TM][TM];
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) acc[i][j] = 0.0;
    if (tid == 0 && q0 < q1) issue(q0, 0);
    inflight |= 1u;
    for (int64_t q = q0; q < q1; ++q) {
      const int s = (int)((q - q0) & 1);
      if (q + 1 < q1) {
        if (tid == 0) issue(q + 1, s ^ 1);
        inflight |= 1u << (s ^ 1);
      }
      if (!mbar_wait_bounded(&bar[s], phase[s])) {
        atomicOr(err, DEV_ERR_TIMEOUT);
        s_abort = 1;
      } else {
        phase[s] ^= 1u;
        inflight &= ~(1u << s);
      }
      __syncthreads();
      if (s_abort) break;
      const double* As = sA[s];
      const double* Bs = sB[s];
#pragma unroll 4
      for (int kk = 0; kk < BS; ++kk) {
        double a[TM], b[TM];
#pragma unroll
        for (int i = 0; i < TM; ++i) a[i] = As[(tr + 16 * i) * BS + kk];
#pragma unroll
        for (int j = 0; j < TM; ++j) b[j] = Bs[kk * BS + tc + 16 * j];
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TM; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
      }
      __syncthreads();
    }
    if (q0 >= q1) inflight &= ~1u;
    if (s_abort) break;
    // epilogue: write C leaf g and its squared Frobenius norm (kernel (d))
    double* C = cpool + g * LEAF;
    double s2 = 0.0;
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) {
        C[(tr + 16 * i) * BS + tc + 16 * j] = acc[i][j];
        s2 = __fma_rn(acc[i][j], acc[i][j], s2);
      }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
    if (lane == 0) s_red[warp] = s2;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int w = 0; w < kGemmThreads / 32; ++w) t += s_red[w];
      csq[g] = t;
    }
  }
  // leave no bulk copy in flight into this CTA's shared memory
  if (tid == 0) {
    for (int s = 0; s < 2; ++s)
      if (inflight & (1u << s)) mbar_wait_bounded(&bar[s], phase[s]);
  }
  __syncthreads();
}

template <int BS>
static void launch_fp64(spamm_mat A, spamm_mat B, const TaskList& T, double* cpool, double* csq) {
  spamm_ctx ctx = A->ctx;
  const size_t smem = 4 * (size_t)BS * BS * sizeof(double);
  CK(cudaFuncSetAttribute(gemm_fp64_kernel<BS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, gemm_fp64_kernel<BS>, kGemmThreads, smem));
  if (per_sm < 1) per_sm = 1;
  int64_t grid = (int64_t)ctx->num_sms * per_sm;
  if (grid > T.ngroups) grid = T.ngroups;
  unsigned long long* work = ctx->d_scratch + 8;
  CK(cudaMemsetAsync(work, 0, sizeof(unsigned long long), ctx->stream));
  gemm_fp64_kernel<BS><<<(unsigned)grid, kGemmThreads, smem, ctx->stream>>>(
      T.ngroups, P<int64_t>(T.gstart), P<int32_t>(T.ta), P<int32_t>(T.tb), P<int64_t>(A->slot), P<int64_t>(B->slot),
      P<double>(A->pool), P<double>(B->pool), cpool, csq, work, ctx->d_err);
  CK_LAUNCH("gemm_fp64_kernel");
}

void gemm_fp64(spamm_mat A, spamm_mat B, const TaskList& T, double* cpool, double* csq) {
  if (T.ngroups == 0) return;
  switch (A->bs) {
    case 32: launch_fp64<32>(A, B, T, cpool, csq); break;
    case 64: launch_fp64<64>(A, B, T, cpool, csq); break;
    default: fail(SPAMM_E_UNSUPPORTED, "FP64 leaf products are built for bs = 32 and 64");
  }
}

}  // namespace spamm
