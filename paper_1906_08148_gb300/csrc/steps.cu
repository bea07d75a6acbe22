// steps.cu -- the plan-time step list of the tensor-core leaf GEMM: for every
// quad of output leaves (2I + h, 2J + c), the four kept-product runs merged by
// k, one 32-byte record per k step (the leaves to load, each child's scale),
// so the GEMM reads its steps sequentially.
#include "internal.cuh"

namespace spamm {

// ------------------------------------------------------------- quad steps
// The four kept-product runs of a quad (child c = 2h + cj, tasks of one C leaf
// in ascending k) merged by k.
struct QuadMerge {
  int64_t p[4], e[4];
  __device__ QuadMerge(const int32_t* g, const int64_t* gstart) {
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      p[c] = g[c] >= 0 ? gstart[g[c]] : 0;
      e[c] = g[c] >= 0 ? gstart[g[c] + 1] : 0;
    }
  }
  __device__ bool more() const { return p[0] < e[0] || p[1] < e[1] || p[2] < e[2] || p[3] < e[3]; }
  // advance past the next k; bit c of the result: child c has a kept product there, task q[c]
  __device__ unsigned next(const int32_t* ta, const uint32_t* codeA, int64_t* q) {
    uint32_t k[4];
    uint32_t kmin = 0xFFFFFFFFu;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      k[c] = p[c] < e[c] ? code_col(codeA[ta[p[c]]]) : 0xFFFFFFFFu;
      kmin = k[c] < kmin ? k[c] : kmin;
    }
    unsigned has = 0;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      q[c] = p[c];
      if (k[c] == kmin) {
        has |= 1u << c;
        ++p[c];
      }
    }
    return has;
  }
};

// One thread per quad.  Count pass (out == null): count[Q] = its steps.
// Write pass: its steps at out[qstart[Q] ...].
__global__ void quad_steps_kernel(int64_t nquads, const int32_t* __restrict__ quads, const int64_t* __restrict__ gstart,
                                  const int32_t* __restrict__ ta, const int32_t* __restrict__ tb,
                                  const uint32_t* __restrict__ codeA, const int32_t* __restrict__ expA,
                                  const int32_t* __restrict__ expB, const int32_t* __restrict__ bmap,
                                  uint64_t* __restrict__ count, const uint64_t* __restrict__ qstart,
                                  QuadStep* __restrict__ out) {
  for (int64_t Q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; Q < nquads; Q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t g[4] = {quads[4 * Q], quads[4 * Q + 1], quads[4 * Q + 2], quads[4 * Q + 3]};
    QuadMerge m(g, gstart);
    QuadStep* o = out ? out + qstart[Q] : nullptr;
    int64_t s = 0;
    while (m.more()) {
      int64_t q[4];
      const unsigned has = m.next(ta, codeA, q);
      if (o) {
        QuadStep st;
        // children 0/1 share the A leaf of row half 0, 2/3 that of half 1; 0/2 and 1/3 share B leaves
        st.a[0] = (has & 1u) ? ta[q[0]] : ((has & 2u) ? ta[q[1]] : -1);
        st.a[1] = (has & 4u) ? ta[q[2]] : ((has & 8u) ? ta[q[3]] : -1);
        st.b[0] = (has & 1u) ? tb[q[0]] : ((has & 4u) ? tb[q[2]] : -1);
        st.b[1] = (has & 2u) ? tb[q[1]] : ((has & 8u) ? tb[q[3]] : -1);
        if (bmap) {
          if (st.b[0] >= 0) st.b[0] = bmap[st.b[0]];
          if (st.b[1] >= 0) st.b[1] = bmap[st.b[1]];
        }
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          float sc = 0.f;
          if (has & (1u << c)) {
            sc = 1.f;
            if (expA) {
              // 2^-(eA + eB) as a product of two normal powers of two (|e| <= 120)
              const int ea = expA[ta[q[c]]], eb = expB[bmap ? bmap[tb[q[c]]] : tb[q[c]]];
              sc = __int_as_float((127 - ea) << 23) * __int_as_float((127 - eb) << 23);
            }
          }
          st.scale[c] = sc;
        }
        o[s] = st;
      }
      ++s;
    }
    if (count) count[Q] = (uint64_t)s;
  }
}

// Leaf (k, j) of M -> index of leaf (j, k): binary search over M's
// Morton-sorted leaf codes; misses are counted in *missing.
__global__ void transpose_map_kernel(int64_t n, const uint32_t* __restrict__ code, int32_t* __restrict__ map,
                                     unsigned long long* missing) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t want = morton2(code_col(code[q]), code_row(code[q]));
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (code[mid] < want)
        lo = mid + 1;
      else
        hi = mid;
    }
    const bool hit = code[lo] == want;
    map[q] = hit ? (int32_t)lo : -1;
    if (!hit) atomicAdd(missing, 1ull);
  }
}

int64_t transpose_map(spamm_mat M, BufP* map, spamm_ctx on) {
  spamm_ctx ctx = on ? on : M->ctx;
  const int64_t n = M->nleaves;
  *map = alloc_n<int32_t>(ctx, n);
  if (n == 0) return 0;
  unsigned long long* missing = ctx->d_scratch + 10;
  CK(cudaMemsetAsync(missing, 0, sizeof(unsigned long long), ctx->stream));
  const int64_t want = (n + 255) / 256, cap = (int64_t)ctx->num_sms * 16;
  transpose_map_kernel<<<(unsigned)(want < cap ? want : cap), 256, 0, ctx->stream>>>(
      n, P<uint32_t>(M->lv[M->L].code), P<int32_t>(*map), missing);
  CK_LAUNCH("transpose_map_kernel");
  return (int64_t)read_scalar(ctx, reinterpret_cast<const uint64_t*>(missing));
}

// ------------------------------------------------------ 128 x 128 leaves
// A 128-leaf product is one unit of the tensor-core kernel: its four 64 x 64
// quadrants (2h + c) are the unit's children, and kept product q of output
// leaf g runs as steps 2q and 2q + 1, the two K halves kh, on operand tiles
// 4 leaf + 2 h + kh (A) and 4 leaf + 2 c + kh (B) of the tile-split terms.
// So the steps of leaf g start at 2 gstart[g], in the leaf's k order.
__global__ void leaf128_steps_kernel(int64_t ntasks, const int32_t* __restrict__ ta, const int32_t* __restrict__ tb,
                                     const int32_t* __restrict__ expA, const int32_t* __restrict__ expB,
                                     const int32_t* __restrict__ bmap, QuadStep* __restrict__ out) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ntasks; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t la = ta[q], lb = bmap ? bmap[tb[q]] : tb[q];
#pragma unroll
    for (int kh = 0; kh < 2; ++kh) {
      QuadStep st;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        st.a[h] = 4 * la + 2 * h + kh;
        st.b[h] = 4 * lb + 2 * h + kh;
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int ea = expA[st.a[c >> 1]], eb = expB[st.b[c & 1]];
        st.scale[c] = __int_as_float((127 - ea) << 23) * __int_as_float((127 - eb) << 23);
      }
      out[2 * q + kh] = st;
    }
  }
}

__global__ void twice_kernel(int64_t n, const int64_t* __restrict__ in, uint64_t* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = 2 * (uint64_t)in[i];
}

int64_t build_leaf128_steps(spamm_ctx ctx, const TaskList& T, const int32_t* expA, const int32_t* expB,
                            const int32_t* bmap, BufP* qstart, BufP* qsteps) {
  const int64_t ng = T.ngroups;
  *qstart = alloc_n<uint64_t>(ctx, ng + 1);
  *qsteps = alloc_n<QuadStep>(ctx, 2 * T.ntasks);
  const int64_t cap = (int64_t)ctx->num_sms * 16;
  const int64_t g1 = (ng + 1 + 255) / 256;
  twice_kernel<<<(unsigned)(g1 < cap ? g1 : cap), 256, 0, ctx->stream>>>(ng + 1, P<int64_t>(T.gstart),
                                                                          P<uint64_t>(*qstart));
  CK_LAUNCH("twice_kernel");
  if (T.ntasks > 0) {
    const int64_t g2 = (T.ntasks + 255) / 256;
    leaf128_steps_kernel<<<(unsigned)(g2 < cap ? g2 : cap), 256, 0, ctx->stream>>>(
        T.ntasks, P<int32_t>(T.ta), P<int32_t>(T.tb), expA, expB, bmap, P<QuadStep>(*qsteps));
    CK_LAUNCH("leaf128_steps_kernel");
  }
  return 2 * T.ntasks;
}

int64_t build_quad_steps(spamm_ctx ctx, const TaskList& T, const uint32_t* codeA, const int32_t* expA,
                         const int32_t* expB, const int32_t* bmap, BufP* qstart, BufP* qsteps) {
  const int64_t nq = T.ngroups > 0 ? T.nquads : 0;
  *qstart = alloc_n<uint64_t>(ctx, nq + 1);
  *qsteps = nullptr;
  if (nq == 0) {
    CK(cudaMemsetAsync(P<uint64_t>(*qstart), 0, sizeof(uint64_t), ctx->stream));
    return 0;
  }
  BufP cnt = alloc_n<uint64_t>(ctx, nq);
  const int64_t want = (nq + 255) / 256, cap = (int64_t)ctx->num_sms * 16;
  const unsigned grid = (unsigned)(want < cap ? want : cap);
  quad_steps_kernel<<<grid, 256, 0, ctx->stream>>>(nq, P<int32_t>(T.quads), P<int64_t>(T.gstart), P<int32_t>(T.ta),
                                                   P<int32_t>(T.tb), codeA, expA, expB, bmap, P<uint64_t>(cnt),
                                                   nullptr, nullptr);
  CK_LAUNCH("quad_steps_kernel(count)");
  scan_exclusive_u64(ctx, P<uint64_t>(cnt), P<uint64_t>(*qstart), nq, P<uint64_t>(*qstart) + nq);
  const int64_t total = (int64_t)read_scalar(ctx, P<uint64_t>(*qstart) + nq);
  *qsteps = alloc_n<QuadStep>(ctx, total);
  quad_steps_kernel<<<grid, 256, 0, ctx->stream>>>(nq, P<int32_t>(T.quads), P<int64_t>(T.gstart), P<int32_t>(T.ta),
                                                   P<int32_t>(T.tb), codeA, expA, expB, bmap, nullptr,
                                                   P<uint64_t>(*qstart), P<QuadStep>(*qsteps));
  CK_LAUNCH("quad_steps_kernel(write)");
  return total;
}

}  // namespace spamm
