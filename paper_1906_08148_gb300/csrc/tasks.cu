// tasks.cu -- kernel (b): the SpAMM task-list builder.
//
// Algorithm 1 descends both quadtrees together: a pair (A_IK, B_KJ) that was
// entered on level t spawns the eight child pairs (A_ik, B_kj), i in {2I,
// 2I+1}, k in {2K, 2K+1}, j in {2J, 2J+1}; a child pair is entered iff both
// children are non-null and ||A_ik|| ||B_kj|| >= tau (Truncmul: no test).  The
// test is carried down to leaf pairs (Section 4.4) and the whole output
// structure is known before any leaf product runs, as the batched "in
// advance" multiplication of Section 4.4 does.
//
// Representation on level t: "groups" are the output nodes (I, J) that have
// at least one entered pair, in Morton order, each owning a contiguous run of
// pairs (a = node index in A, b = node index in B) ordered by K ascending.
// One level step:
//   count  (thread per pair) evaluate the 8 children of every pair and store
//          an 8-bit kept mask per pair; then (warp per group) per child output
//          node c = 2ci + cj the number of kept pairs, packed as
//          (count | nonempty << 36).
//   scan   exclusive prefix over the 4 * groups packed values: output offset
//          of every child group and its index among the non-empty ones.
//   write  (warp per group): every lane takes one pair, per child group two
//          warp ballots (k-child 0 and 1) place the kept pairs; within a
//          child group pairs stay in parent order with k = 2K, 2K+1, so the
//          children are again sorted by k.  Lane 0 writes the child groups.
// Because a parent's squared norm is a floating-point sum of non-negative
// children, the test is monotone down the tree and the pruned descent keeps
// exactly the leaf pairs that pass the leaf-level test.
#include "internal.cuh"
#include "screen.cuh"

namespace spamm {

constexpr int kWarpsPerBlock = 8;
constexpr uint64_t kCountMask = (1ull << 36) - 1;

__device__ __forceinline__ int comp4(const int4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

__device__ __forceinline__ double comp4d(const double4& v, int i) {
  return i == 0 ? v.x : (i == 1 ? v.y : (i == 2 ? v.z : v.w));
}

// Per node of a level, one 16-byte record: the index of its first child on
// the next level (the children of a node are consecutive there: every level
// is in Morton order) and the four children's 24-bit norm keys (screen.cuh;
// kNullKey where a child is null), so the descent reads one 16-byte load per
// node of a pair.  The norms themselves (-1 where null) go to a second array
// that only the pairs the screen leaves undecided read.  One launch covers
// both operands' levels (A's nodes first); a node whose children are not
// consecutive sets the range error (a broken quadtree).
struct __align__(16) NodeRec {
  uint32_t base;
  uint32_t w[3];  // keys k0..k3, 24 bits each, k0 in the low bits of w[0]
};

__device__ __forceinline__ uint32_t rec_key(const NodeRec& r, int c) {
  switch (c) {
    case 0: return r.w[0] & 0xFFFFFFu;
    case 1: return (r.w[0] >> 24) | ((r.w[1] & 0xFFFFu) << 8);
    case 2: return (r.w[1] >> 16) | ((r.w[2] & 0xFFu) << 16);
    default: return r.w[2] >> 8;
  }
}

// Next-level indices of the four children (-1 where null).
__device__ __forceinline__ int4 rec_children(const NodeRec& r) {
  unsigned pres = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) pres |= (unsigned)(rec_key(r, i) != kNullKey) << i;
  const int b = (int)r.base;
  return make_int4(pres & 1u ? b : -1, pres & 2u ? b + __popc(pres & 1u) : -1, pres & 4u ? b + __popc(pres & 3u) : -1,
                   pres & 8u ? b + __popc(pres & 7u) : -1);
}

__global__ void node_rec_kernel(int64_t nA, const int4* __restrict__ childA, const double* __restrict__ sqA,
                                NodeRec* __restrict__ recA, double4* __restrict__ normA, int64_t nB,
                                const int4* __restrict__ childB, const double* __restrict__ sqB,
                                NodeRec* __restrict__ recB, double4* __restrict__ normB, int* err) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nA + nB; q += (int64_t)gridDim.x * blockDim.x) {
    const bool a = q < nA;
    const int64_t r = a ? q : q - nA;
    const int4 c = (a ? childA : childB)[r];
    const double* sq = a ? sqA : sqB;
    const double4 v = make_double4(c.x >= 0 ? sqrt(sq[c.x]) : -1.0, c.y >= 0 ? sqrt(sq[c.y]) : -1.0,
                                   c.z >= 0 ? sqrt(sq[c.z]) : -1.0, c.w >= 0 ? sqrt(sq[c.w]) : -1.0);
    const int ch[4] = {c.x, c.y, c.z, c.w};
    uint32_t k[4];
    int base = -1, rank = 0;
    bool ok = true;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (ch[i] < 0) {
        k[i] = kNullKey;
        continue;
      }
      if (base < 0) base = ch[i];
      ok &= ch[i] == base + rank;
      ++rank;
      k[i] = pack_norm(comp4d(v, i));
    }
    if (!ok) atomicOr(err, DEV_ERR_RANGE);
    NodeRec rec;
    rec.base = (uint32_t)(base < 0 ? 0 : base);
    rec.w[0] = k[0] | (k[1] << 24);
    rec.w[1] = (k[1] >> 8) | (k[2] << 16);
    rec.w[2] = (k[2] >> 16) | (k[3] << 8);
    (a ? recA : recB)[r] = rec;
    (a ? normA : normB)[r] = v;
  }
}

// The FP64 decision p >= tau (and the borderline count at the leaf level).
__device__ __forceinline__ bool exact_keep(double na, double nb, double tau, bool leaf, long long* border) {
  const double prod = __dmul_rn(na, nb);
  const long long pb = __double_as_longlong(prod), tb = __double_as_longlong(tau);
  const long long dist = pb > tb ? pb - tb : tb - pb;
  if (leaf && dist <= (1ll << 14) && fabs(prod - tau) <= 1e-12 * tau) ++*border;
  return pb >= tb;  // prod >= tau for prod, tau >= 0
}

// mask bit (2*c + ck) for child group c = 2*ci + cj and child k-index ck;
// na / nb: the children's norms of the pair's A and B nodes.  The product is
// the FP64 round-to-nearest product of the two norms; the comparisons use its
// bits (non-negative doubles order like their bit patterns), because this part
// issues FP64 instructions at two per clock per SM.  The borderline test
// |prod - tau| <= 1e-12 tau is evaluated in FP64 only for products within
// 2^14 units in the last place of tau (1e-12 relative is about 4500 of them).
__device__ __forceinline__ unsigned child_mask(const NodeRec& ra, const NodeRec& rb, const double4* na,
                                               const double4* nb, const TauScreen& sc, double tau, int test,
                                               bool leaf, long long* cand, long long* border) {
  uint32_t ka[4], kb[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    ka[i] = rec_key(ra, i);
    kb[i] = rec_key(rb, i);
  }
  unsigned m = 0;
#pragma unroll
  for (int ci = 0; ci < 2; ++ci)
#pragma unroll
    for (int cj = 0; cj < 2; ++cj)
#pragma unroll
      for (int ck = 0; ck < 2; ++ck) {
        const int ia = 2 * ci + ck, ib = 2 * ck + cj;
        if (ka[ia] == kNullKey || kb[ib] == kNullKey) continue;
        ++*cand;
        bool keep = true;
        if (test) {
          const int d = screen_decide(ka[ia], kb[ib], sc);
          keep = d >= 0 ? d == 1 : exact_keep(comp4d(*na, ia), comp4d(*nb, ib), tau, leaf, border);
        }
        if (keep) m |= 1u << (2 * (2 * ci + cj) + ck);
      }
  return m;
}

// count, part 1: the norm test of every entered pair, one thread per pair
// (the pairs of a level, flat: no group loop, so every thread has one chain
// of gathers in flight and the level's pairs all run at once); the 8-bit
// child mask of each pair, and the level's candidate and borderline counts.
__global__ void __launch_bounds__(256)
    task_mask_kernel(const int64_t* __restrict__ dQ, const int32_t* __restrict__ ta,
                     const int32_t* __restrict__ tb, const NodeRec* __restrict__ recA,
                     const NodeRec* __restrict__ recB, const double4* __restrict__ normA,
                     const double4* __restrict__ normB, TauScreen sc, double tau, int test, int leaf,
                     uint8_t* __restrict__ mask, unsigned long long* stats) {
  const int64_t Q = *dQ;
  long long cand = 0, border = 0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < Q; q += (int64_t)gridDim.x * blockDim.x) {
    const int32_t ia = ta[q], ib = tb[q];
    mask[q] = (uint8_t)child_mask(recA[ia], recB[ib], normA + ia, normB + ib, sc, tau, test, leaf, &cand, &border);
  }
  // warp sums, then one atomic per block (atomics on one address from every
  // warp of the grid would queue at a single L2 slice)
  __shared__ long long s_cnt[8][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    cand += __shfl_xor_sync(0xffffffffu, cand, off);
    border += __shfl_xor_sync(0xffffffffu, border, off);
  }
  if (lane == 0) {
    s_cnt[warp][0] = cand;
    s_cnt[warp][1] = border;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    long long c = 0, b = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      c += s_cnt[w][0];
      b += s_cnt[w][1];
    }
    if (c) atomicAdd(stats + 0, (unsigned long long)c);
    if (b) atomicAdd(stats + 1, (unsigned long long)b);
  }
}

// count, part 2 (warp per group): per child group c = 2 ci + cj the number of
// kept pairs, from the masks; packed as (count | nonempty << 36).  Groups past
// this level's count (up to the capacity the scan runs over) get zeros.
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    task_group_count_kernel(int64_t Gcap, const int64_t* __restrict__ dG, const int64_t* __restrict__ gstart,
                            const uint8_t* __restrict__ mask, uint64_t* __restrict__ packed) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t G = *dG;
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < Gcap; g += nw) {
    if (g >= G) {
      if (lane < 4) packed[4 * g + lane] = 0;
      continue;
    }
    const int64_t q0 = gstart[g], q1 = gstart[g + 1];
    unsigned cnt[4] = {0, 0, 0, 0};
    for (int64_t q = q0 + lane; q < q1; q += 32) {
      const unsigned m = mask[q];
#pragma unroll
      for (int c = 0; c < 4; ++c) cnt[c] += __popc((m >> (2 * c)) & 3u);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) cnt[c] += __shfl_xor_sync(0xffffffffu, cnt[c], off);
    }
    if (lane == 0) {
#pragma unroll
      for (int c = 0; c < 4; ++c) packed[4 * g + c] = (uint64_t)cnt[c] | ((uint64_t)(cnt[c] > 0) << 36);
    }
  }
}

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    task_write_kernel(const int64_t* __restrict__ dG, const int64_t* __restrict__ gstart,
                      const uint32_t* __restrict__ gcode,
                      const int32_t* __restrict__ ta, const int32_t* __restrict__ tb, const NodeRec* __restrict__ recA,
                      const NodeRec* __restrict__ recB, const uint8_t* __restrict__ mask,
                      const uint64_t* __restrict__ packed, const uint64_t* __restrict__ off,
                      int32_t* __restrict__ ta2, int32_t* __restrict__ tb2, uint32_t* __restrict__ gcode2,
                      int64_t* __restrict__ gstart2, int32_t* __restrict__ quad) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t G = *dG;
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {
    const int64_t q0 = gstart[g], q1 = gstart[g + 1];
    int64_t base[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) base[c] = (int64_t)(off[4 * g + c] & kCountMask);
    if (lane < 4) {
      const uint64_t o = off[4 * g + lane];
      const bool present = (packed[4 * g + lane] & kCountMask) != 0;
      if (present) {
        const int64_t gid = (int64_t)(o >> 36);
        gcode2[gid] = 4u * gcode[g] + (uint32_t)lane;
        gstart2[gid] = (int64_t)(o & kCountMask);
      }
      if (quad) quad[4 * g + lane] = present ? (int32_t)(o >> 36) : -1;
    }
    for (int64_t qb = q0; qb < q1; qb += 32) {
      const int64_t q = qb + lane;
      const bool active = q < q1;
      const unsigned m = active ? mask[q] : 0u;
      int4 ca = make_int4(-1, -1, -1, -1), cb = ca;
      if (m) {
        ca = rec_children(recA[ta[q]]);
        cb = rec_children(recB[tb[q]]);
      }
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const unsigned bits = (m >> (2 * c)) & 3u;
        // warp ballots compact the kept children: a lane's entries follow
        // every kept child of the lanes before it (k-child 0, then 1)
        const unsigned b0 = __ballot_sync(0xffffffffu, bits & 1u), b1 = __ballot_sync(0xffffffffu, bits & 2u);
        const unsigned lt = (1u << lane) - 1u;
        const int tot = __popc(b0) + __popc(b1);
        int64_t pos = base[c] + __popc(b0 & lt) + __popc(b1 & lt);
        const int ci = c >> 1, cj = c & 1;
        if (bits & 1u) {
          ta2[pos] = comp4(ca, 2 * ci + 0);
          tb2[pos] = comp4(cb, 0 + cj);
          ++pos;
        }
        if (bits & 2u) {
          ta2[pos] = comp4(ca, 2 * ci + 1);
          tb2[pos] = comp4(cb, 2 + cj);
        }
        base[c] += tot;
      }
    }
  }
}

__global__ void root_test_kernel(const double* sqA, const double* sqB, double tau, int test, int64_t* gstart,
                                 unsigned long long* stats) {
  if (threadIdx.x != 0) return;
  const double prod = __dmul_rn(sqrt(sqA[0]), sqrt(sqB[0]));
  const bool keep = !test || prod >= tau;
  gstart[1] = keep ? 1 : 0;
  stats[0] = 1;
  stats[1] = (test && fabs(prod - tau) <= 1e-12 * tau) ? 1 : 0;
}

static unsigned warps_grid(spamm_ctx ctx, int64_t items) {
  int64_t g = (items + kWarpsPerBlock - 1) / kWarpsPerBlock;
  int64_t cap = (int64_t)ctx->num_sms * 16;
  if (g > cap) g = cap;
  return (unsigned)(g < 1 ? 1 : g);
}

// Sizes of the next level from the scan total, on the device: its pair and
// group counts, the closing entry of its group offsets, and this level's
// statistics (lv[4 t ..]: candidates, borderline pairs, pairs, groups).
__global__ void level_finish_kernel(const uint64_t* __restrict__ tot, unsigned long long* __restrict__ stats,
                                    int64_t* __restrict__ dQ2, int64_t* __restrict__ dG2, int64_t* __restrict__ gstart2,
                                    int64_t* __restrict__ lv) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int64_t Q2 = (int64_t)(*tot & kCountMask), G2 = (int64_t)(*tot >> 36);
  *dQ2 = Q2;
  *dG2 = G2;
  gstart2[G2] = Q2;
  lv[0] = (int64_t)stats[0];
  lv[1] = (int64_t)stats[1];
  stats[0] = stats[1] = 0;  // for the next level's count
  lv[2] = Q2;
  lv[3] = G2;
}

// Upper bounds on the next level's sizes below which the host does not wait
// for the exact counts (buffers are allocated at the bound instead).  The
// leaf level always waits: its arrays are the plan's task list, kept for the
// leaf products.  (Waiting less often measured slower: the kernels of a level
// allocated at the bound run over the bound, 4 G groups, and the scan too.)
constexpr int64_t kPairsNoSync = 1ll << 22;
constexpr int64_t kGroupsNoSync = 1ll << 20;

TaskList build_tasks(spamm_mat A, spamm_mat B, double tau, int test_norms, spamm_ctx on) {
  spamm_ctx ctx = on ? on : A->ctx;
  TaskList T;
  if (A->nleaves == 0 || B->nleaves == 0) {
    T.gstart = alloc_n<int64_t>(ctx, 1);
    CK(cudaMemsetAsync(P<int64_t>(T.gstart), 0, sizeof(int64_t), ctx->stream));
    return T;
  }
  // level 0: the root pair is entered
  int64_t G = 1, Q = 1;  // capacities; exact when `exact`
  bool exact = true;
  BufP gcode = alloc_n<uint32_t>(ctx, 1), gstart = alloc_n<int64_t>(ctx, 2);
  BufP ta = alloc_n<int32_t>(ctx, 1), tb = alloc_n<int32_t>(ctx, 1);
  // device sizes: [2 t] pairs, [2 t + 1] groups of level t; per-level statistics after them
  const int nlev = A->L + 1;
  BufP sizes = alloc_n<int64_t>(ctx, 2 * nlev + 4 * nlev);
  int64_t* dsz = P<int64_t>(sizes);
  int64_t* dlv = dsz + 2 * nlev;
  {
    const int64_t h_gstart[2] = {0, 1};
    const int64_t h_sz[2] = {1, 1};
    CK(cudaMemsetAsync(dsz, 0, (2 * nlev + 4 * nlev) * sizeof(int64_t), ctx->stream));
    CK(cudaMemsetAsync(P<uint32_t>(gcode), 0, sizeof(uint32_t), ctx->stream));
    CK(cudaMemsetAsync(P<int32_t>(ta), 0, sizeof(int32_t), ctx->stream));
    CK(cudaMemsetAsync(P<int32_t>(tb), 0, sizeof(int32_t), ctx->stream));
    CK(cudaMemcpyAsync(P<int64_t>(gstart), h_gstart, sizeof(h_gstart), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(dsz, h_sz, sizeof(h_sz), cudaMemcpyHostToDevice, ctx->stream));
  }
  unsigned long long* stats = ctx->d_scratch;  // [0] candidates, [1] borderline
  uint64_t* hp = static_cast<uint64_t*>(ctx->h_pinned);
  if (A->L == 0) {
    // a single leaf: the root pair is the only leaf pair and takes the leaf test
    root_test_kernel<<<1, 32, 0, ctx->stream>>>(P<double>(A->lv[0].sq), P<double>(B->lv[0].sq), tau, test_norms,
                                                P<int64_t>(gstart), stats);
    CK_LAUNCH("root_test_kernel");
    CK(cudaMemcpyAsync(hp, P<int64_t>(gstart) + 1, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(hp + 1, stats, 2 * sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    Q = (int64_t)hp[0];
    G = Q;
    T.n_borderline = (int64_t)hp[2];
    if (G > 0) {
      // one output leaf: a quad holding only child 0
      const int32_t q4[4] = {0, -1, -1, -1};
      T.nquads = 1;
      T.quads = alloc_n<int32_t>(ctx, 4);
      CK(cudaMemcpyAsync(P<int32_t>(T.quads), q4, sizeof(q4), cudaMemcpyHostToDevice, ctx->stream));
    }
  }
  const TauScreen screen = make_screen(tau);
  int last = 0;  // level whose sizes describe the current arrays
  CK(cudaMemsetAsync(stats, 0, 2 * sizeof(unsigned long long), ctx->stream));  // level_finish re-zeroes them
  for (int t = 0; t < A->L; ++t) {
    const bool leaf = (t + 1 == A->L);
    const int64_t* dG = dsz + 2 * t + 1;
    BufP mask = alloc_n<uint8_t>(ctx, Q);
    BufP packed = alloc_n<uint64_t>(ctx, 4 * G), off = alloc_n<uint64_t>(ctx, 4 * G), tot = alloc_n<uint64_t>(ctx, 1);
    const int64_t nA = A->lv[t].count, nB = B->lv[t].count;
    BufP normA = alloc_n<double4>(ctx, nA), normB = alloc_n<double4>(ctx, nB);
    BufP recA = alloc_n<NodeRec>(ctx, nA), recB = alloc_n<NodeRec>(ctx, nB);
    {
      const int64_t g = (nA + nB + 255) / 256, cap = (int64_t)ctx->num_sms * 16;
      node_rec_kernel<<<(unsigned)(g < cap ? g : cap), 256, 0, ctx->stream>>>(
          nA, P<int4>(A->lv[t].child), P<double>(A->lv[t + 1].sq), P<NodeRec>(recA), P<double4>(normA), nB,
          P<int4>(B->lv[t].child), P<double>(B->lv[t + 1].sq), P<NodeRec>(recB), P<double4>(normB), ctx->d_err);
      CK_LAUNCH("node_rec_kernel");
    }
    {
      const int64_t g = (Q + 255) / 256, cap = (int64_t)ctx->num_sms * 16;
      task_mask_kernel<<<(unsigned)(g < cap ? (g > 0 ? g : 1) : cap), 256, 0, ctx->stream>>>(
          dsz + 2 * t, P<int32_t>(ta), P<int32_t>(tb), P<NodeRec>(recA), P<NodeRec>(recB), P<double4>(normA),
          P<double4>(normB), screen, tau, test_norms, leaf, P<uint8_t>(mask), stats);
      CK_LAUNCH("task_mask_kernel");
    }
    task_group_count_kernel<<<warps_grid(ctx, G), kWarpsPerBlock * 32, 0, ctx->stream>>>(
        G, dG, P<int64_t>(gstart), P<uint8_t>(mask), P<uint64_t>(packed));
    CK_LAUNCH("task_group_count_kernel");
    scan_exclusive_u64(ctx, P<uint64_t>(packed), P<uint64_t>(off), 4 * G, P<uint64_t>(tot));
    // capacities of the next level: exact after a wait, else the bounds 8 Q and 4 G
    int64_t Q2 = 8 * Q, G2 = 4 * G;
    const bool wait = Q2 > kPairsNoSync || G2 > kGroupsNoSync || leaf;
    BufP gstart2;
    if (wait) {
      CK(cudaMemcpyAsync(hp, P<uint64_t>(tot), sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
      CK(cudaStreamSynchronize(ctx->stream));
      Q2 = (int64_t)(hp[0] & kCountMask);
      G2 = (int64_t)(hp[0] >> 36);
    }
    gstart2 = alloc_n<int64_t>(ctx, G2 + 1);
    level_finish_kernel<<<1, 32, 0, ctx->stream>>>(P<uint64_t>(tot), stats, dsz + 2 * (t + 1), dsz + 2 * (t + 1) + 1,
                                                   P<int64_t>(gstart2), dlv + 4 * (t + 1));
    CK_LAUNCH("level_finish_kernel");
    BufP gcode2 = alloc_n<uint32_t>(ctx, G2);
    if (leaf) T.quads = alloc_n<int32_t>(ctx, 4 * G);  // the four children of each parent of the C leaves
    BufP ta2 = alloc_n<int32_t>(ctx, Q2), tb2 = alloc_n<int32_t>(ctx, Q2);
    if (G2 > 0) {
      task_write_kernel<<<warps_grid(ctx, G), kWarpsPerBlock * 32, 0, ctx->stream>>>(
          dG, P<int64_t>(gstart), P<uint32_t>(gcode), P<int32_t>(ta), P<int32_t>(tb), P<NodeRec>(recA),
          P<NodeRec>(recB), P<uint8_t>(mask), P<uint64_t>(packed), P<uint64_t>(off), P<int32_t>(ta2),
          P<int32_t>(tb2), P<uint32_t>(gcode2), P<int64_t>(gstart2), leaf ? P<int32_t>(T.quads) : nullptr);
      CK_LAUNCH("task_write_kernel");
    }
    G = G2;
    Q = Q2;
    exact = wait;
    gcode = gcode2;
    gstart = gstart2;
    ta = ta2;
    tb = tb2;
    last = t + 1;
    if (exact && G == 0) break;
  }
  // exact sizes of every level and per-level statistics, one read-back (the
  // two arrays are adjacent)
  std::vector<int64_t> h(6 * nlev);
  CK(cudaMemcpyAsync(h.data(), dsz, 6 * nlev * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  const int64_t* hl = h.data() + 2 * nlev;
  if (A->L > 0) {
    Q = h[2 * last];
    G = h[2 * last + 1];
    for (int t = 1; t <= last; ++t) {
      T.n_candidates[t] = hl[4 * t + 0];
      T.n_kept_level[t] = hl[4 * t + 2];
    }
    if (last == A->L) {
      T.n_borderline = hl[4 * A->L + 1];
      T.nquads = h[2 * (A->L - 1) + 1];  // the groups one level up are the parents of the C leaves
    }
  }
  T.ngroups = G;
  T.ntasks = Q;
  T.gcode = gcode;
  T.gstart = gstart;
  T.ta = ta;
  T.tb = tb;
  return T;
}

// (i, k, j) of every task, for the parity hook.
__global__ void tasks_to_ikj_kernel(int64_t G, const int64_t* __restrict__ gstart, const uint32_t* __restrict__ gcode,
                                    const int32_t* __restrict__ ta, const uint32_t* __restrict__ codeA,
                                    int32_t* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; g < G; g += nw) {
    const int32_t i = (int32_t)code_row(gcode[g]), j = (int32_t)code_col(gcode[g]);
    for (int64_t q = gstart[g] + lane; q < gstart[g + 1]; q += 32) {
      out[3 * q + 0] = i;
      out[3 * q + 1] = (int32_t)code_col(codeA[ta[q]]);
      out[3 * q + 2] = j;
    }
  }
}

void tasks_to_ikj(spamm_mat A, const TaskList& T, int32_t* d_out) {
  spamm_ctx ctx = A->ctx;
  if (T.ngroups == 0) return;
  tasks_to_ikj_kernel<<<warps_grid(ctx, T.ngroups), kWarpsPerBlock * 32, 0, ctx->stream>>>(
      T.ngroups, P<int64_t>(T.gstart), P<uint32_t>(T.gcode), P<int32_t>(T.ta), P<uint32_t>(A->lv[A->L].code), d_out);
  CK_LAUNCH("tasks_to_ikj_kernel");
}

}  // namespace spamm
