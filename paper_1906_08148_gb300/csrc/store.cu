// store.cu -- the device quadtree store: leaf norms (kernel a), parent norms,
// input truncation, builders from dense / blocks / COO / generator, exports
// and the error walk.
//
// Layout in HBM: a matrix is a payload pool of bs*bs row-major FP64 leaves
// plus, for every quadtree level t = 0..L, the nodes of that level sorted by
// the Morton code of their (row, col) position, their squared Frobenius norms
// and (t < L) an int4 of child node indices (-1 = null child).  Leaf m's
// payload is at pool + slot[m]*bs*bs, so truncated views share the pool.
#include <cstdio>

#include "../../synth/decaygen.h"
#include "internal.cuh"

namespace spamm {

constexpr int kThreads = 256;

void fill_iota_u32(spamm_ctx ctx, uint32_t* p, int64_t n);
void fill_iota_i64(spamm_ctx ctx, int64_t* p, int64_t n);
void and_u8(spamm_ctx ctx, uint8_t* a, const uint8_t* b, int64_t n);

static unsigned grid_for(spamm_ctx ctx, int64_t items, int per_block, int max_per_sm = 32) {
  int64_t g = (items + per_block - 1) / per_block;
  int64_t cap = (int64_t)ctx->num_sms * max_per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// ------------------------------------------------------------------------
// Kernel (a): squared Frobenius norm of each leaf (Section 2, Section 4.2:
// every matrix stores its squared norm).  One warp per leaf; lane l reads
// the 16-byte pairs l, l+32, ... (coalesced 512-byte rows), squares are
// accumulated with explicit FMAs in that fixed order and the 32 partial sums
// are combined by a butterfly, so every build path gives identical bits.
// The FMA is the only FP64 instruction per element: this part issues two FP64
// operations per clock per SM, so the non-zero and finiteness checks work on
// the bit patterns in the integer pipe (any bit besides the sign set: non-zero;
// exponent field all ones: Inf or NaN).
template <class Get>
__device__ __forceinline__ void warp_leaf_sumsq(Get get, int bs, int lane, double* s_out, bool* nz_out, bool* bad_out) {
  const int pairs = bs * bs / 2;
  double s = 0.0;
  uint32_t bits = 0, emax = 0;
  for (int i = lane; i < pairs; i += 32) {
    double2 v = get(i);
    s = __fma_rn(v.x, v.x, s);
    s = __fma_rn(v.y, v.y, s);
    const uint32_t hx = (uint32_t)__double2hiint(v.x), hy = (uint32_t)__double2hiint(v.y);
    bits |= (uint32_t)__double2loint(v.x) | (uint32_t)__double2loint(v.y) | ((hx | hy) & 0x7fffffffu);
    emax = max(emax, max(hx & 0x7ff00000u, hy & 0x7ff00000u));
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  *s_out = s;
  *nz_out = __any_sync(0xffffffffu, bits != 0);
  *bad_out = __any_sync(0xffffffffu, emax == 0x7ff00000u);
}

// Block b takes leaves [64 b, 64 b + 64), each of its 8 warps every 8th of
// them (a grid of about nleaves / 64 blocks spreads evenly over the SMs;
// larger grids stride by whole blocks).
constexpr int64_t kNormLeavesPerBlock = 64;
__global__ void leaf_sqnorm_kernel(const double* __restrict__ pool, const int64_t* __restrict__ slot, int64_t m,
                                   int bs, double* __restrict__ sq, uint8_t* __restrict__ nonzero, int check_finite,
                                   int* err) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwb = blockDim.x >> 5;
  const int64_t e = (int64_t)bs * bs;
  for (int64_t q0 = (int64_t)blockIdx.x * kNormLeavesPerBlock; q0 < m; q0 += (int64_t)gridDim.x * kNormLeavesPerBlock)
  for (int64_t q = q0 + warp; q < q0 + kNormLeavesPerBlock && q < m; q += nwb) {
    const double2* src = reinterpret_cast<const double2*>(pool + (slot ? slot[q] : q) * e);
    double s;
    bool nz, bad;
    warp_leaf_sumsq([&](int i) { return __ldg(src + i); }, bs, lane, &s, &nz, &bad);
    if (lane == 0) {
      sq[q] = s;
      if (nonzero) nonzero[q] = nz;
      if (bad && check_finite) atomicOr(err, DEV_ERR_NONFINITE);
    }
  }
}

void leaf_sqnorms(spamm_ctx ctx, const double* pool, const int64_t* slot, int64_t nleaves, int bs, double* sq,
                  uint8_t* nonzero, int check_finite) {
  if (nleaves <= 0) return;
  const int64_t nblk = (nleaves + kNormLeavesPerBlock - 1) / kNormLeavesPerBlock;
  leaf_sqnorm_kernel<<<(unsigned)(nblk < (1ll << 30) ? nblk : (1ll << 30)), kThreads, 0, ctx->stream>>>(
      pool, slot, nleaves, bs, sq, nonzero, check_finite, ctx->d_err);
  CK_LAUNCH("leaf_sqnorm_kernel");
}

// ------------------------------------------------------------ compaction
__global__ void keep_to_u64_kernel(const uint8_t* __restrict__ keep, int64_t n, uint64_t* __restrict__ out) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    out[q] = keep[q] ? 1u : 0u;
}

__global__ void compact_leaves_kernel(int64_t n, const uint8_t* __restrict__ keep, const uint64_t* __restrict__ pos,
                                      const uint32_t* __restrict__ code, const double* __restrict__ sq,
                                      const int64_t* __restrict__ slot, uint32_t* __restrict__ ocode,
                                      double* __restrict__ osq, int64_t* __restrict__ oslot) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    if (!keep[q]) continue;
    int64_t p = (int64_t)pos[q];
    ocode[p] = code[q];
    osq[p] = sq[q];
    oslot[p] = slot ? slot[q] : q;
  }
}

spamm_mat new_mat(spamm_ctx ctx, int64_t n, int bs) {
  spamm_mat m = new spamm_mat_s();
  m->ctx = ctx;
  m->n = n;
  m->bs = bs;
  m->L = levels_for(n, bs);
  m->lv.resize(m->L + 1);
  return m;
}

void set_leaves_compacted(spamm_mat m, int64_t ncand, const uint32_t* code, const double* sq, const int64_t* slot,
                          const uint8_t* keep) {
  spamm_ctx ctx = m->ctx;
  Level& leaf = m->lv[m->L];
  if (ncand <= 0) {
    m->nleaves = 0;
    leaf.count = 0;
    build_tree(m);
    return;
  }
  BufP flags = alloc_n<uint64_t>(ctx, ncand), pos = alloc_n<uint64_t>(ctx, ncand), tot = alloc_n<uint64_t>(ctx, 1);
  keep_to_u64_kernel<<<grid_for(ctx, ncand, kThreads), kThreads, 0, ctx->stream>>>(keep, ncand, P<uint64_t>(flags));
  CK_LAUNCH("keep_to_u64_kernel");
  scan_exclusive_u64(ctx, P<uint64_t>(flags), P<uint64_t>(pos), ncand, P<uint64_t>(tot));
  int64_t cnt = (int64_t)read_scalar<uint64_t>(ctx, P<uint64_t>(tot));
  leaf.count = cnt;
  m->nleaves = cnt;
  leaf.code = alloc_n<uint32_t>(ctx, cnt);
  leaf.sq = alloc_n<double>(ctx, cnt);
  m->slot = alloc_n<int64_t>(ctx, cnt);
  if (cnt > 0) {
    compact_leaves_kernel<<<grid_for(ctx, ncand, kThreads), kThreads, 0, ctx->stream>>>(
        ncand, keep, P<uint64_t>(pos), code, sq, slot, P<uint32_t>(leaf.code), P<double>(leaf.sq),
        P<int64_t>(m->slot));
    CK_LAUNCH("compact_leaves_kernel");
  }
  build_tree(m);
}

// ----------------------------------------------------- parents (Section 2)
// ||A^t||_F^2 = sum of the four children's squared norms, added in the fixed
// order (0,0), (0,1), (1,0), (1,1); children are found from the sorted codes
// of the level below (parent code = child code >> 2).
// The level below holds *dn nodes (the arrays have room for ncap); flags past
// *dn are 0 so that a scan over the capacity gives the parent count.
__global__ void parent_flags_kernel(const uint32_t* __restrict__ code, int64_t ncap, const uint64_t* __restrict__ dn,
                                    uint64_t* __restrict__ flags) {
  const int64_t n = (int64_t)*dn;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ncap; q += (int64_t)gridDim.x * blockDim.x)
    flags[q] = q < n && (q == 0 || (code[q] >> 2) != (code[q - 1] >> 2)) ? 1u : 0u;
}

__global__ void parent_link_kernel(const uint32_t* __restrict__ code, const uint64_t* __restrict__ dn,
                                   const uint64_t* __restrict__ flags, const uint64_t* __restrict__ excl,
                                   uint32_t* __restrict__ pcode, int4* __restrict__ pchild) {
  const int64_t n = (int64_t)*dn;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t p = (int64_t)(excl[q] + flags[q]) - 1;
    uint32_t c = code[q];
    if (flags[q]) pcode[p] = c >> 2;
    reinterpret_cast<int*>(pchild + p)[c & 3u] = (int)q;
  }
}

__global__ void parent_sum_kernel(int64_t np, const int4* __restrict__ child, const double* __restrict__ csq,
                                  double* __restrict__ psq) {
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < np; p += (int64_t)gridDim.x * blockDim.x) {
    int4 ch = child[p];
    double s = 0.0;
    if (ch.x >= 0) s += csq[ch.x];
    if (ch.y >= 0) s += csq[ch.y];
    if (ch.z >= 0) s += csq[ch.z];
    if (ch.w >= 0) s += csq[ch.w];
    psq[p] = s;
  }
}

// Node counts stay on the device while the levels are built (each level's
// arrays sized by an upper bound: no more parents than children, and no more
// than the level's grid); one read-back at the end gives the exact counts.
void build_skeleton(spamm_mat m) {
  spamm_ctx ctx = m->ctx;
  const int L = m->L;
  if (L == 0) return;
  BufP dcnt = alloc_n<uint64_t>(ctx, L + 1);
  uint64_t* d = P<uint64_t>(dcnt);
  const uint64_t nleaf = (uint64_t)m->lv[L].count;
  CK(cudaMemcpyAsync(d + L, &nleaf, sizeof(uint64_t), cudaMemcpyHostToDevice, ctx->stream));
  std::vector<BufP> keep;  // scan buffers live until the counts are read
  int64_t ncap = m->lv[L].count;
  int top = L;  // lowest level index built
  for (int t = L; t >= 1 && ncap > 0; --t) {
    Level& ch = m->lv[t];
    Level& pa = m->lv[t - 1];
    const int64_t grid_nodes = (int64_t)1 << (2 * (t - 1));
    const int64_t pcap = ncap < grid_nodes ? ncap : grid_nodes;
    BufP flags = alloc_n<uint64_t>(ctx, ncap), excl = alloc_n<uint64_t>(ctx, ncap);
    parent_flags_kernel<<<grid_for(ctx, ncap, kThreads), kThreads, 0, ctx->stream>>>(P<uint32_t>(ch.code), ncap,
                                                                                    d + t, P<uint64_t>(flags));
    CK_LAUNCH("parent_flags_kernel");
    scan_exclusive_u64(ctx, P<uint64_t>(flags), P<uint64_t>(excl), ncap, d + t - 1);
    pa.code = alloc_n<uint32_t>(ctx, pcap);
    pa.sq.reset();
    pa.child = alloc_n<int4>(ctx, pcap);
    CK(cudaMemsetAsync(P<int4>(pa.child), 0xFF, pcap * sizeof(int4), ctx->stream));
    parent_link_kernel<<<grid_for(ctx, ncap, kThreads), kThreads, 0, ctx->stream>>>(
        P<uint32_t>(ch.code), d + t, P<uint64_t>(flags), P<uint64_t>(excl), P<uint32_t>(pa.code), P<int4>(pa.child));
    CK_LAUNCH("parent_link_kernel");
    keep.push_back(flags);
    keep.push_back(excl);
    ncap = pcap;
    top = t - 1;
  }
  std::vector<uint64_t> h(L + 1, 0);
  CK(cudaMemcpyAsync(h.data(), d, (L + 1) * sizeof(uint64_t), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  for (int t = 0; t < L; ++t) {
    Level& pa = m->lv[t];
    pa.count = t >= top ? (int64_t)h[t] : 0;
    if (pa.count == 0) {
      pa.code.reset();
      pa.sq.reset();
      pa.child.reset();
    }
  }
}

void alloc_level_norms(spamm_mat m) {
  for (int t = 0; t < m->L; ++t)
    if (m->lv[t].count > 0) m->lv[t].sq = alloc_n<double>(m->ctx, m->lv[t].count);
}

void propagate_norms(spamm_mat m) {
  spamm_ctx ctx = m->ctx;
  for (int t = m->L; t >= 1; --t) {
    const Level& ch = m->lv[t];
    const Level& pa = m->lv[t - 1];
    if (pa.count == 0) continue;
    parent_sum_kernel<<<grid_for(ctx, pa.count, kThreads), kThreads, 0, ctx->stream>>>(
        pa.count, P<int4>(pa.child), P<double>(ch.sq), P<double>(pa.sq));
    CK_LAUNCH("parent_sum_kernel");
  }
}

// Parent norms of several matrices, one launch per height above the leaves:
// segment q of height h is one matrix's level L - h.
struct NormSeg {
  const int4* child;
  const double* csq;
  double* psq;
};
__global__ void parent_sum_batch_kernel(const NormSeg* __restrict__ seg, const int64_t* __restrict__ begin, int nseg,
                                        int64_t total) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < total; u += (int64_t)gridDim.x * blockDim.x) {
    int lo = 0, hi = nseg - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (begin[mid] <= u)
        lo = mid;
      else
        hi = mid - 1;
    }
    const NormSeg sg = seg[lo];
    const int64_t p = u - begin[lo];
    const int4 ch = sg.child[p];
    double s = 0.0;
    if (ch.x >= 0) s += sg.csq[ch.x];
    if (ch.y >= 0) s += sg.csq[ch.y];
    if (ch.z >= 0) s += sg.csq[ch.z];
    if (ch.w >= 0) s += sg.csq[ch.w];
    sg.psq[p] = s;
  }
}

BufP norm_batch_tables(spamm_ctx ctx, const std::vector<spamm_mat>& ms, std::vector<NormBatchLevel>* levels) {
  int H = 0;
  for (spamm_mat m : ms) H = m->L > H ? m->L : H;
  std::vector<NormSeg> segs;
  std::vector<int64_t> begins;
  levels->clear();
  for (int h = 1; h <= H; ++h) {
    NormBatchLevel lv;
    lv.first = (int)segs.size();
    int64_t tot = 0;
    for (spamm_mat m : ms) {
      if (m->L < h) continue;
      const Level& pa = m->lv[m->L - h];
      if (pa.count == 0) continue;
      segs.push_back({P<int4>(pa.child), P<double>(m->lv[m->L - h + 1].sq), P<double>(pa.sq)});
      begins.push_back(tot);
      tot += pa.count;
    }
    lv.nseg = (int)segs.size() - lv.first;
    lv.total = tot;
    levels->push_back(lv);
  }
  // pageable sources: each copy has read them by the time it returns
  const size_t sb = segs.size() * sizeof(NormSeg), bb = begins.size() * sizeof(int64_t);
  BufP tab = alloc_bytes(ctx, sb + bb + 16);
  if (!segs.empty()) {
    CK(cudaMemcpyAsync(tab->p, segs.data(), sb, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(static_cast<uint8_t*>(tab->p) + sb, begins.data(), bb, cudaMemcpyHostToDevice, ctx->stream));
  }
  for (NormBatchLevel& lv : *levels) {
    lv.seg = static_cast<const void*>(static_cast<const NormSeg*>(tab->p) + lv.first);
    lv.begin = reinterpret_cast<const int64_t*>(static_cast<const uint8_t*>(tab->p) + sb) + lv.first;
  }
  return tab;
}

void propagate_norms_batch(spamm_ctx ctx, const std::vector<NormBatchLevel>& levels) {
  for (const NormBatchLevel& lv : levels) {
    if (lv.total == 0) continue;
    parent_sum_batch_kernel<<<grid_for(ctx, lv.total, kThreads), kThreads, 0, ctx->stream>>>(
        static_cast<const NormSeg*>(lv.seg), lv.begin, lv.nseg, lv.total);
    CK_LAUNCH("parent_sum_batch_kernel");
  }
}

void build_tree(spamm_mat m) {
  build_skeleton(m);
  alloc_level_norms(m);
  propagate_norms(m);
}

// ----------------------------------------------------------- truncation
// Block rule: drop leaf iff sqrt(s) < tau (the pool is shared, no copy).
__global__ void block_keep_kernel(const double* __restrict__ sq, int64_t n, double tau, uint8_t* __restrict__ keep) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    keep[q] = !(sqrt(sq[q]) < tau);
}

spamm_mat truncate_block(spamm_mat in, double tau, spamm_ctx on) {
  spamm_ctx ctx = on ? on : in->ctx;
  spamm_mat out = new_mat(ctx, in->n, in->bs);
  out->symmetric = in->symmetric;
  out->pool = in->pool;
  const int64_t n = in->nleaves;
  BufP keep = alloc_n<uint8_t>(ctx, n);
  if (n > 0) {
    block_keep_kernel<<<grid_for(ctx, n, kThreads), kThreads, 0, ctx->stream>>>(P<double>(in->lv[in->L].sq), n, tau,
                                                                               P<uint8_t>(keep));
    CK_LAUNCH("block_keep_kernel");
  }
  set_leaves_compacted(out, n, P<uint32_t>(in->lv[in->L].code), P<double>(in->lv[in->L].sq), P<int64_t>(in->slot),
                       P<uint8_t>(keep));
  return out;
}

// Error-controlled rule: drop the smallest leaves (ascending squared norm,
// ties in Morton order) as long as the sum of their squared norms, added in
// that order, stays <= tau^2, so ||A - A~||_F <= tau.  The squared norms are
// non-negative doubles, so their bit patterns sort like their values.
__global__ void sq_sort_keys_kernel(const double* __restrict__ sq, int64_t n, uint64_t* __restrict__ keys,
                                    int64_t* __restrict__ idx) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    keys[q] = (uint64_t)__double_as_longlong(sq[q]);
    idx[q] = q;
  }
}

__global__ void sorted_sq_kernel(const uint64_t* __restrict__ keys, int64_t n, double* __restrict__ v) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    v[q] = __longlong_as_double((long long)keys[q]);
}

__global__ void within_budget_kernel(const double* __restrict__ csum, int64_t n, double budget,
                                     uint64_t* __restrict__ flag) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    flag[q] = csum[q] <= budget ? 1u : 0u;
}

// The first *ndrop leaves of the sorted order are dropped (a prefix, even if
// rounding made the running sums non-monotone by an ulp).
__global__ void drop_prefix_kernel(const int64_t* __restrict__ idx, int64_t n, const uint64_t* __restrict__ ndrop,
                                   uint8_t* __restrict__ keep) {
  const int64_t k = (int64_t)*ndrop;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    keep[idx[q]] = q >= k;
}

spamm_mat truncate_error_controlled(spamm_mat in, double tau, spamm_ctx on) {
  spamm_ctx ctx = on ? on : in->ctx;
  spamm_mat out = new_mat(ctx, in->n, in->bs);
  out->symmetric = in->symmetric;
  out->pool = in->pool;
  const int64_t n = in->nleaves;
  BufP keep = alloc_n<uint8_t>(ctx, n);
  if (n > 0) {
    BufP keys = alloc_n<uint64_t>(ctx, n), idx = alloc_n<int64_t>(ctx, n), v = alloc_n<double>(ctx, n);
    BufP csum = alloc_n<double>(ctx, n), flag = alloc_n<uint64_t>(ctx, n), pos = alloc_n<uint64_t>(ctx, n);
    BufP ndrop = alloc_n<uint64_t>(ctx, 1);
    const unsigned g = grid_for(ctx, n, kThreads);
    sq_sort_keys_kernel<<<g, kThreads, 0, ctx->stream>>>(P<double>(in->lv[in->L].sq), n, P<uint64_t>(keys),
                                                          P<int64_t>(idx));
    CK_LAUNCH("sq_sort_keys_kernel");
    radix_sort_pairs(ctx, P<uint64_t>(keys), P<int64_t>(idx), n, 64);  // stable: ties keep Morton order
    sorted_sq_kernel<<<g, kThreads, 0, ctx->stream>>>(P<uint64_t>(keys), n, P<double>(v));
    CK_LAUNCH("sorted_sq_kernel");
    scan_inclusive_f64(ctx, P<double>(v), P<double>(csum), n);
    within_budget_kernel<<<g, kThreads, 0, ctx->stream>>>(P<double>(csum), n, tau * tau, P<uint64_t>(flag));
    CK_LAUNCH("within_budget_kernel");
    scan_exclusive_u64(ctx, P<uint64_t>(flag), P<uint64_t>(pos), n, P<uint64_t>(ndrop));
    drop_prefix_kernel<<<g, kThreads, 0, ctx->stream>>>(P<int64_t>(idx), n, P<uint64_t>(ndrop), P<uint8_t>(keep));
    CK_LAUNCH("drop_prefix_kernel");
  }
  set_leaves_compacted(out, n, P<uint32_t>(in->lv[in->L].code), P<double>(in->lv[in->L].sq), P<int64_t>(in->slot),
                       P<uint8_t>(keep));
  return out;
}

// Element rule (Theorem 1): a -> 0 iff |a| < tau, into a fresh pool.
__global__ void element_trunc_copy_kernel(const double* __restrict__ src, const int64_t* __restrict__ slot, int64_t n,
                                          int bs, double tau, double* __restrict__ dst) {
  const int64_t e = (int64_t)bs * bs;
  for (int64_t q = blockIdx.x; q < n; q += gridDim.x) {
    const double* s = src + slot[q] * e;
    double* d = dst + q * e;
    for (int64_t i = threadIdx.x; i < e; i += blockDim.x) {
      double v = s[i];
      d[i] = fabs(v) < tau ? 0.0 : v;
    }
  }
}

spamm_mat truncate_element(spamm_mat in, double tau) {
  spamm_ctx ctx = in->ctx;
  const int64_t n = in->nleaves, e = (int64_t)in->bs * in->bs;
  spamm_mat out = new_mat(ctx, in->n, in->bs);
  out->symmetric = in->symmetric;
  out->pool = alloc_n<double>(ctx, n * e);
  BufP sq = alloc_n<double>(ctx, n), nz = alloc_n<uint8_t>(ctx, n);
  if (n > 0) {
    element_trunc_copy_kernel<<<grid_for(ctx, n, 1), kThreads, 0, ctx->stream>>>(
        P<double>(in->pool), P<int64_t>(in->slot), n, in->bs, tau, P<double>(out->pool));
    CK_LAUNCH("element_trunc_copy_kernel");
    leaf_sqnorms(ctx, P<double>(out->pool), nullptr, n, in->bs, P<double>(sq), P<uint8_t>(nz), 0);
  }
  set_leaves_compacted(out, n, P<uint32_t>(in->lv[in->L].code), P<double>(sq), nullptr, P<uint8_t>(nz));
  return out;
}

// --------------------------------------------------------------- builders
__global__ void block_codes_kernel(const int32_t* __restrict__ bi, const int32_t* __restrict__ bj, int64_t n,
                                   int64_t nb, uint64_t* __restrict__ keys, int64_t* __restrict__ vals, int* err) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    int32_t r = bi[q], c = bj[q];
    if (r < 0 || c < 0 || r >= nb || c >= nb) {
      atomicOr(err, DEV_ERR_RANGE);
      r = 0;
      c = 0;
    }
    keys[q] = morton2((uint32_t)r, (uint32_t)c);
    vals[q] = q;
  }
}

__global__ void gather_sorted_kernel(int64_t n, const uint64_t* __restrict__ keys, const int64_t* __restrict__ vals,
                                     const double* __restrict__ sq_by_input, const uint8_t* __restrict__ nz_by_input,
                                     double tau, int block_rule, uint32_t* __restrict__ code, double* __restrict__ sq,
                                     int64_t* __restrict__ slot, uint8_t* __restrict__ keep, int* err) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t v = vals[q];
    code[q] = (uint32_t)keys[q];
    sq[q] = sq_by_input[v];
    slot[q] = v;
    bool k = nz_by_input[v] != 0;
    if (block_rule && tau > 0.0 && sqrt(sq_by_input[v]) < tau) k = false;
    keep[q] = k;
    if (q > 0 && keys[q] == keys[q - 1]) atomicOr(err, DEV_ERR_DUPLICATE);
  }
}

__global__ void zero_below_kernel(double* __restrict__ a, int64_t n, double tau) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    if (fabs(a[q]) < tau) a[q] = 0.0;
}

// Leaves given as a pool of `nblocks` payloads already on the device in input order.
static spamm_mat finish_from_pool(spamm_ctx ctx, int64_t n, int bs, BufP pool, int64_t nblocks, const int32_t* d_bi,
                                  const int32_t* d_bj, double tau, spamm_trunc_rule rule) {
  spamm_mat m = new_mat(ctx, n, bs);
  m->pool = pool;
  const int64_t e = (int64_t)bs * bs;
  if (rule == SPAMM_TRUNC_ELEMENT && tau > 0.0 && nblocks > 0) {
    zero_below_kernel<<<grid_for(ctx, nblocks * e, kThreads), kThreads, 0, ctx->stream>>>(P<double>(pool),
                                                                                         nblocks * e, tau);
    CK_LAUNCH("zero_below_kernel");
  }
  BufP sq = alloc_n<double>(ctx, nblocks), nz = alloc_n<uint8_t>(ctx, nblocks);
  BufP keys = alloc_n<uint64_t>(ctx, nblocks), vals = alloc_n<int64_t>(ctx, nblocks);
  BufP code = alloc_n<uint32_t>(ctx, nblocks), ssq = alloc_n<double>(ctx, nblocks);
  BufP slot = alloc_n<int64_t>(ctx, nblocks), keep = alloc_n<uint8_t>(ctx, nblocks);
  if (nblocks > 0) {
    leaf_sqnorms(ctx, P<double>(pool), nullptr, nblocks, bs, P<double>(sq), P<uint8_t>(nz), 1);
    const int64_t nb = (n + bs - 1) / bs;
    block_codes_kernel<<<grid_for(ctx, nblocks, kThreads), kThreads, 0, ctx->stream>>>(
        d_bi, d_bj, nblocks, nb, P<uint64_t>(keys), P<int64_t>(vals), ctx->d_err);
    CK_LAUNCH("block_codes_kernel");
    radix_sort_pairs(ctx, P<uint64_t>(keys), P<int64_t>(vals), nblocks, 2 * m->L);
    gather_sorted_kernel<<<grid_for(ctx, nblocks, kThreads), kThreads, 0, ctx->stream>>>(
        nblocks, P<uint64_t>(keys), P<int64_t>(vals), P<double>(sq), P<uint8_t>(nz), tau,
        rule == SPAMM_TRUNC_BLOCK_FROB, P<uint32_t>(code), P<double>(ssq), P<int64_t>(slot), P<uint8_t>(keep),
        ctx->d_err);
    CK_LAUNCH("gather_sorted_kernel");
    sync_and_check(ctx);
  }
  set_leaves_compacted(m, nblocks, P<uint32_t>(code), P<double>(ssq), P<int64_t>(slot), P<uint8_t>(keep));
  return m;
}

spamm_mat build_from_blocks(spamm_ctx ctx, int64_t n, int bs, int64_t nblocks, const int32_t* bi, const int32_t* bj,
                            const double* payload, int on_device, double tau, spamm_trunc_rule rule) {
  const int64_t e = (int64_t)bs * bs;
  BufP pool = alloc_n<double>(ctx, nblocks * e);
  BufP dbi = alloc_n<int32_t>(ctx, nblocks), dbj = alloc_n<int32_t>(ctx, nblocks);
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  if (nblocks > 0) {
    CK(cudaMemcpyAsync(P<double>(pool), payload, nblocks * e * sizeof(double), kind, ctx->stream));
    CK(cudaMemcpyAsync(P<int32_t>(dbi), bi, nblocks * sizeof(int32_t), kind, ctx->stream));
    CK(cudaMemcpyAsync(P<int32_t>(dbj), bj, nblocks * sizeof(int32_t), kind, ctx->stream));
  }
  return finish_from_pool(ctx, n, bs, pool, nblocks, P<int32_t>(dbi), P<int32_t>(dbj), tau, rule);
}

// Candidate leaves in Morton order over the 2^L x 2^L grid, those inside
// the ceil(n/bs) x ceil(n/bs) block range only.  Warp per candidate.
template <class Elem>
__global__ void candidate_stats_kernel(Elem elem, int64_t ncand, int bs, int64_t nb, double tau, int rule,
                                       double* __restrict__ sq, uint8_t* __restrict__ keep, int* err) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < ncand; q += nw) {
    const uint32_t r = code_row((uint32_t)q), c = code_col((uint32_t)q);
    if (r >= nb || c >= nb || elem.skip(r, c, tau, rule)) {
      if (lane == 0) {
        keep[q] = 0;
        sq[q] = 0.0;
      }
      continue;
    }
    double s;
    bool nz, bad;
    warp_leaf_sumsq(
        [&](int i) {
          int e0 = 2 * i;
          double x = elem(r, c, e0 / bs, e0 % bs), y = elem(r, c, e0 / bs, e0 % bs + 1);
          if (rule == SPAMM_TRUNC_ELEMENT) {
            if (fabs(x) < tau) x = 0.0;
            if (fabs(y) < tau) y = 0.0;
          }
          return make_double2(x, y);
        },
        bs, lane, &s, &nz, &bad);
    if (lane == 0) {
      bool k = nz;
      if (rule == SPAMM_TRUNC_BLOCK_FROB && tau > 0.0 && sqrt(s) < tau) k = false;
      keep[q] = k;
      sq[q] = s;
      if (bad) atomicOr(err, DEV_ERR_NONFINITE);
    }
  }
}

template <class Elem>
__global__ void candidate_fill_kernel(Elem elem, int64_t nleaves, const uint32_t* __restrict__ code, int bs,
                                      double tau, int rule, double* __restrict__ pool) {
  const int64_t e = (int64_t)bs * bs;
  for (int64_t q = blockIdx.x; q < nleaves; q += gridDim.x) {
    const uint32_t r = code_row(code[q]), c = code_col(code[q]);
    for (int64_t i = threadIdx.x; i < e; i += blockDim.x) {
      double x = elem(r, c, (int)(i / bs), (int)(i % bs));
      if (rule == SPAMM_TRUNC_ELEMENT && fabs(x) < tau) x = 0.0;
      pool[q * e + i] = x;
    }
  }
}

struct DenseElem {
  const double* a;
  int64_t lda, n;
  int bs;
  __device__ double operator()(uint32_t r, uint32_t c, int i, int j) const {
    int64_t gi = (int64_t)r * bs + i, gj = (int64_t)c * bs + j;
    return (gi < n && gj < n) ? a[gi * lda + gj] : 0.0;
  }
  __device__ bool skip(uint32_t, uint32_t, double, int) const { return false; }
};

struct GenElem {
  synth_params p;
  int bs;
  __device__ double operator()(uint32_t r, uint32_t c, int i, int j) const {
    return synth_element(&p, (int64_t)r * bs + i, (int64_t)c * bs + j);
  }
  // A leaf whose bound says every element is below the cutoff is null; under
  // the block rule a leaf whose norm bound bs * max|a| is below tau is dropped.
  __device__ bool skip(uint32_t r, uint32_t c, double tau, int rule) const {
    double b = synth_leaf_bound(&p, bs, r, c);
    if (b < p.cutoff) return true;
    if (rule == SPAMM_TRUNC_ELEMENT && b < tau) return true;
    if (rule == SPAMM_TRUNC_BLOCK_FROB && tau > 0.0 && b * bs < tau) return true;
    return false;
  }
};

template <class Elem>
static spamm_mat build_from_elements(spamm_ctx ctx, int64_t n, int bs, Elem elem, double tau, spamm_trunc_rule rule) {
  spamm_mat m = new_mat(ctx, n, bs);
  const int64_t nb = (n + bs - 1) / bs;
  const int64_t ncand = (int64_t)1 << (2 * m->L);
  BufP sq = alloc_n<double>(ctx, ncand), keep = alloc_n<uint8_t>(ctx, ncand), code = alloc_n<uint32_t>(ctx, ncand);
  candidate_stats_kernel<<<grid_for(ctx, ncand, kThreads / 32), kThreads, 0, ctx->stream>>>(
      elem, ncand, bs, nb, tau, (int)rule, P<double>(sq), P<uint8_t>(keep), ctx->d_err);
  CK_LAUNCH("candidate_stats_kernel");
  sync_and_check(ctx);
  // the candidates' codes are their indices 0 .. 4^L - 1
  uint32_t* c32 = P<uint32_t>(code);
  fill_iota_u32(ctx, c32, ncand);
  set_leaves_compacted(m, ncand, c32, P<double>(sq), nullptr, P<uint8_t>(keep));
  // payload for the kept leaves, slot = leaf index
  const int64_t e = (int64_t)bs * bs;
  m->pool = alloc_n<double>(ctx, m->nleaves * e);
  if (m->nleaves > 0) {
    candidate_fill_kernel<<<grid_for(ctx, m->nleaves, 1, 64), kThreads, 0, ctx->stream>>>(
        elem, m->nleaves, P<uint32_t>(m->lv[m->L].code), bs, tau, (int)rule, P<double>(m->pool));
    CK_LAUNCH("candidate_fill_kernel");
    fill_iota_i64(ctx, P<int64_t>(m->slot), m->nleaves);
  }
  return m;
}

__global__ void iota_u32_kernel(uint32_t* p, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    p[q] = (uint32_t)q;
}
__global__ void iota_i64_kernel(int64_t* p, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    p[q] = q;
}
void fill_iota_u32(spamm_ctx ctx, uint32_t* p, int64_t n) {
  if (n <= 0) return;
  iota_u32_kernel<<<grid_for(ctx, n, kThreads), kThreads, 0, ctx->stream>>>(p, n);
  CK_LAUNCH("iota_u32_kernel");
}
void fill_iota_i64(spamm_ctx ctx, int64_t* p, int64_t n) {
  if (n <= 0) return;
  iota_i64_kernel<<<grid_for(ctx, n, kThreads), kThreads, 0, ctx->stream>>>(p, n);
  CK_LAUNCH("iota_i64_kernel");
}

spamm_mat build_from_dense(spamm_ctx ctx, int64_t n, const double* a, int64_t lda, int on_device, int bs, double tau,
                           spamm_trunc_rule rule) {
  BufP tmp;
  const double* da = a;
  int64_t dlda = lda;
  if (!on_device) {
    tmp = alloc_n<double>(ctx, n * n);
    CK(cudaMemcpy2DAsync(P<double>(tmp), n * sizeof(double), a, lda * sizeof(double), n * sizeof(double), n,
                         cudaMemcpyHostToDevice, ctx->stream));
    da = P<double>(tmp);
    dlda = n;
  }
  DenseElem el{da, dlda, n, bs};
  spamm_mat m = build_from_elements(ctx, n, bs, el, tau, rule);
  sync_and_check(ctx);  // the temporary copy must outlive the fill
  return m;
}

spamm_mat build_generated(spamm_ctx ctx, const spamm_gen_params* gp, int bs, double tau, spamm_trunc_rule rule) {
  GenElem el;
  el.p.n = gp->n;
  el.p.kind = gp->kind;
  el.p.law = gp->law;
  el.p.alpha = gp->alpha;
  el.p.c = gp->c;
  el.p.cutoff = gp->cutoff;
  el.p.seed = gp->seed;
  el.bs = bs;
  spamm_mat m = build_from_elements(ctx, gp->n, bs, el, tau, rule);
  m->symmetric = 1;  // u_ij and the decay law are symmetric in (i, j)
  return m;
}

// COO: sort (leaf code, in-leaf offset) keys stably, sum runs of equal keys
// in input order, scatter into zeroed leaves.
__global__ void coo_keys_kernel(const int64_t* __restrict__ row, const int64_t* __restrict__ col,
                                const double* __restrict__ val, int64_t nnz, int64_t n, int bs, int lbs,
                                uint64_t* __restrict__ keys, int64_t* __restrict__ vals, int* err) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = row[q], c = col[q];
    if (r < 0 || c < 0 || r >= n || c >= n) {
      atomicOr(err, DEV_ERR_RANGE);
      r = 0;
      c = 0;
    }
    if (!isfinite(val[q])) atomicOr(err, DEV_ERR_NONFINITE);
    uint64_t leaf = morton2((uint32_t)(r / bs), (uint32_t)(c / bs));
    uint64_t off = (uint64_t)((r % bs) * bs + (c % bs));
    keys[q] = (leaf << (2 * lbs)) | off;
    vals[q] = q;
  }
}

__global__ void coo_leaf_flags_kernel(const uint64_t* __restrict__ keys, int64_t nnz, int lbs,
                                      uint64_t* __restrict__ flags) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x)
    flags[q] = (q == 0 || (keys[q] >> (2 * lbs)) != (keys[q - 1] >> (2 * lbs))) ? 1u : 0u;
}

__global__ void coo_scatter_kernel(const uint64_t* __restrict__ keys, const int64_t* __restrict__ vals,
                                   const double* __restrict__ val, int64_t nnz, int lbs,
                                   const uint64_t* __restrict__ flags, const uint64_t* __restrict__ excl,
                                   double* __restrict__ pool, uint32_t* __restrict__ code) {
  const int64_t e = (int64_t)1 << (2 * lbs);
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += (int64_t)gridDim.x * blockDim.x) {
    if (q > 0 && keys[q] == keys[q - 1]) continue;  // not the head of its run
    int64_t leaf = (int64_t)(excl[q] + flags[q]) - 1;
    if (flags[q]) code[leaf] = (uint32_t)(keys[q] >> (2 * lbs));
    double s = 0.0;
    for (int64_t p = q; p < nnz && keys[p] == keys[q]; ++p) s += val[vals[p]];
    pool[leaf * e + (int64_t)(keys[q] & (uint64_t)(e - 1))] = s;
  }
}

spamm_mat build_from_coo(spamm_ctx ctx, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col,
                         const double* val, int on_device, int bs, double tau, spamm_trunc_rule rule) {
  spamm_mat m = new_mat(ctx, n, bs);
  int lbs = 0;
  while ((1 << lbs) < bs) ++lbs;
  const int64_t e = (int64_t)bs * bs;
  BufP drow, dcol, dval;
  const int64_t *r = row, *c = col;
  const double* v = val;
  if (!on_device && nnz > 0) {
    drow = alloc_n<int64_t>(ctx, nnz);
    dcol = alloc_n<int64_t>(ctx, nnz);
    dval = alloc_n<double>(ctx, nnz);
    CK(cudaMemcpyAsync(P<int64_t>(drow), row, nnz * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(P<int64_t>(dcol), col, nnz * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(P<double>(dval), val, nnz * 8, cudaMemcpyHostToDevice, ctx->stream));
    r = P<int64_t>(drow);
    c = P<int64_t>(dcol);
    v = P<double>(dval);
  }
  if (nnz == 0) {
    set_leaves_compacted(m, 0, nullptr, nullptr, nullptr, nullptr);
    return m;
  }
  BufP keys = alloc_n<uint64_t>(ctx, nnz), vals = alloc_n<int64_t>(ctx, nnz);
  coo_keys_kernel<<<grid_for(ctx, nnz, kThreads), kThreads, 0, ctx->stream>>>(
      r, c, v, nnz, n, bs, lbs, P<uint64_t>(keys), P<int64_t>(vals), ctx->d_err);
  CK_LAUNCH("coo_keys_kernel");
  sync_and_check(ctx);
  radix_sort_pairs(ctx, P<uint64_t>(keys), P<int64_t>(vals), nnz, 2 * m->L + 2 * lbs);
  BufP flags = alloc_n<uint64_t>(ctx, nnz), excl = alloc_n<uint64_t>(ctx, nnz), tot = alloc_n<uint64_t>(ctx, 1);
  coo_leaf_flags_kernel<<<grid_for(ctx, nnz, kThreads), kThreads, 0, ctx->stream>>>(P<uint64_t>(keys), nnz, lbs,
                                                                                   P<uint64_t>(flags));
  CK_LAUNCH("coo_leaf_flags_kernel");
  scan_exclusive_u64(ctx, P<uint64_t>(flags), P<uint64_t>(excl), nnz, P<uint64_t>(tot));
  const int64_t nl = (int64_t)read_scalar<uint64_t>(ctx, P<uint64_t>(tot));
  BufP pool = alloc_n<double>(ctx, nl * e), code = alloc_n<uint32_t>(ctx, nl);
  CK(cudaMemsetAsync(P<double>(pool), 0, nl * e * sizeof(double), ctx->stream));
  coo_scatter_kernel<<<grid_for(ctx, nnz, kThreads), kThreads, 0, ctx->stream>>>(
      P<uint64_t>(keys), P<int64_t>(vals), v, nnz, lbs, P<uint64_t>(flags), P<uint64_t>(excl), P<double>(pool),
      P<uint32_t>(code));
  CK_LAUNCH("coo_scatter_kernel");
  if (rule == SPAMM_TRUNC_ELEMENT && tau > 0.0) {
    zero_below_kernel<<<grid_for(ctx, nl * e, kThreads), kThreads, 0, ctx->stream>>>(P<double>(pool), nl * e, tau);
    CK_LAUNCH("zero_below_kernel");
  }
  BufP sq = alloc_n<double>(ctx, nl), nz = alloc_n<uint8_t>(ctx, nl);
  leaf_sqnorms(ctx, P<double>(pool), nullptr, nl, bs, P<double>(sq), P<uint8_t>(nz), 0);
  if (rule == SPAMM_TRUNC_BLOCK_FROB && tau > 0.0) {
    BufP keep2 = alloc_n<uint8_t>(ctx, nl);
    block_keep_kernel<<<grid_for(ctx, nl, kThreads), kThreads, 0, ctx->stream>>>(P<double>(sq), nl, tau,
                                                                                P<uint8_t>(keep2));
    CK_LAUNCH("block_keep_kernel");
    and_u8(ctx, P<uint8_t>(nz), P<uint8_t>(keep2), nl);
  }
  m->pool = pool;
  set_leaves_compacted(m, nl, P<uint32_t>(code), P<double>(sq), nullptr, P<uint8_t>(nz));
  return m;
}

__global__ void and_u8_kernel(uint8_t* a, const uint8_t* b, int64_t n) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x)
    a[q] = a[q] && b[q];
}
void and_u8(spamm_ctx ctx, uint8_t* a, const uint8_t* b, int64_t n) {
  if (n <= 0) return;
  and_u8_kernel<<<grid_for(ctx, n, kThreads), kThreads, 0, ctx->stream>>>(a, b, n);
  CK_LAUNCH("and_u8_kernel");
}

// ---------------------------------------------------------------- exports
__global__ void to_dense_kernel(const double* __restrict__ pool, const int64_t* __restrict__ slot,
                                const uint32_t* __restrict__ code, int64_t nleaves, int bs, int64_t n,
                                double* __restrict__ out, int64_t ld) {
  const int64_t e = (int64_t)bs * bs;
  for (int64_t q = blockIdx.x; q < nleaves; q += gridDim.x) {
    const int64_t r0 = (int64_t)code_row(code[q]) * bs, c0 = (int64_t)code_col(code[q]) * bs;
    const double* src = pool + slot[q] * e;
    for (int64_t i = threadIdx.x; i < e; i += blockDim.x) {
      int64_t r = r0 + i / bs, c = c0 + i % bs;
      if (r < n && c < n) out[r * ld + c] = src[i];
    }
  }
}

void export_dense(spamm_mat m, double* out, int64_t ld, int on_device) {
  spamm_ctx ctx = m->ctx;
  BufP tmp;
  double* dst = out;
  int64_t dld = ld;
  if (!on_device) {
    tmp = alloc_n<double>(ctx, m->n * m->n);
    dst = P<double>(tmp);
    dld = m->n;
  }
  CK(cudaMemset2DAsync(dst, dld * sizeof(double), 0, m->n * sizeof(double), m->n, ctx->stream));
  if (m->nleaves > 0) {
    to_dense_kernel<<<grid_for(ctx, m->nleaves, 1, 64), kThreads, 0, ctx->stream>>>(
        P<double>(m->pool), P<int64_t>(m->slot), P<uint32_t>(m->lv[m->L].code), m->nleaves, m->bs, m->n, dst, dld);
    CK_LAUNCH("to_dense_kernel");
  }
  if (!on_device)
    CK(cudaMemcpy2DAsync(out, ld * sizeof(double), dst, dld * sizeof(double), m->n * sizeof(double), m->n,
                         cudaMemcpyDeviceToHost, ctx->stream));
  sync_and_check(ctx);
}

__global__ void to_blocks_kernel(const double* __restrict__ pool, const int64_t* __restrict__ slot,
                                 const uint32_t* __restrict__ code, int64_t nleaves, int bs, int32_t* bi, int32_t* bj,
                                 double* __restrict__ payload) {
  const int64_t e = (int64_t)bs * bs;
  for (int64_t q = blockIdx.x; q < nleaves; q += gridDim.x) {
    if (threadIdx.x == 0) {
      if (bi) bi[q] = (int32_t)code_row(code[q]);
      if (bj) bj[q] = (int32_t)code_col(code[q]);
    }
    if (payload) {
      const double2* src = reinterpret_cast<const double2*>(pool + slot[q] * e);
      double2* dst = reinterpret_cast<double2*>(payload + q * e);
      for (int64_t i = threadIdx.x; i < e / 2; i += blockDim.x) dst[i] = src[i];
    }
  }
}

void export_blocks(spamm_mat m, int32_t* bi, int32_t* bj, double* payload, double* sq, int on_device) {
  spamm_ctx ctx = m->ctx;
  const int64_t nl = m->nleaves, e = (int64_t)m->bs * m->bs;
  if (nl == 0) return;
  BufP tbi, tbj, tpay;
  int32_t *dbi = bi, *dbj = bj;
  double* dpay = payload;
  if (!on_device) {
    if (bi) dbi = P<int32_t>(tbi = alloc_n<int32_t>(ctx, nl));
    if (bj) dbj = P<int32_t>(tbj = alloc_n<int32_t>(ctx, nl));
    if (payload) dpay = P<double>(tpay = alloc_n<double>(ctx, nl * e));
  }
  to_blocks_kernel<<<grid_for(ctx, nl, 1, 64), kThreads, 0, ctx->stream>>>(
      P<double>(m->pool), P<int64_t>(m->slot), P<uint32_t>(m->lv[m->L].code), nl, m->bs, dbi, dbj, dpay);
  CK_LAUNCH("to_blocks_kernel");
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (!on_device) {
    if (bi) CK(cudaMemcpyAsync(bi, dbi, nl * sizeof(int32_t), kind, ctx->stream));
    if (bj) CK(cudaMemcpyAsync(bj, dbj, nl * sizeof(int32_t), kind, ctx->stream));
    if (payload) CK(cudaMemcpyAsync(payload, dpay, nl * e * sizeof(double), kind, ctx->stream));
  }
  if (sq) CK(cudaMemcpyAsync(sq, P<double>(m->lv[m->L].sq), nl * sizeof(double), kind, ctx->stream));
  sync_and_check(ctx);
}

__global__ void gather_leaves_kernel(const double* __restrict__ pool, const int64_t* __restrict__ slot,
                                     const uint32_t* __restrict__ code, int64_t nleaves, int bs, int64_t nq,
                                     const int32_t* __restrict__ bi, const int32_t* __restrict__ bj,
                                     double* __restrict__ out, int32_t* __restrict__ found);

void gather_leaves(spamm_mat m, int64_t nq, const int32_t* bi, const int32_t* bj, double* out, int32_t* found,
                   int on_device) {
  spamm_ctx ctx = m->ctx;
  if (nq <= 0) return;
  const int64_t e = (int64_t)m->bs * m->bs;
  BufP tbi, tbj, tout, tfound;
  const int32_t *dbi = bi, *dbj = bj;
  double* dout = out;
  int32_t* dfound = found;
  if (!on_device) {
    tbi = alloc_n<int32_t>(ctx, nq);
    tbj = alloc_n<int32_t>(ctx, nq);
    tout = alloc_n<double>(ctx, nq * e);
    tfound = alloc_n<int32_t>(ctx, nq);
    CK(cudaMemcpyAsync(P<int32_t>(tbi), bi, nq * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(P<int32_t>(tbj), bj, nq * sizeof(int32_t), cudaMemcpyHostToDevice, ctx->stream));
    dbi = P<int32_t>(tbi);
    dbj = P<int32_t>(tbj);
    dout = P<double>(tout);
    dfound = P<int32_t>(tfound);
  }
  gather_leaves_kernel<<<grid_for(ctx, nq, 1, 64), kThreads, 0, ctx->stream>>>(
      P<double>(m->pool), P<int64_t>(m->slot), P<uint32_t>(m->lv[m->L].code), m->nleaves, m->bs, nq, dbi, dbj, dout,
      dfound);
  CK_LAUNCH("gather_leaves_kernel");
  if (!on_device) {
    CK(cudaMemcpyAsync(out, dout, nq * e * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    if (found) CK(cudaMemcpyAsync(found, dfound, nq * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  }
  sync_and_check(ctx);
}

// ------------------------------------------------------- error ||X - Y||_F
__device__ __forceinline__ int64_t find_code(const uint32_t* __restrict__ codes, int64_t n, uint32_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    int64_t mid = (lo + hi) >> 1;
    if (codes[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return (lo < n && codes[lo] == key) ? lo : -1;
}

__global__ void error_x_kernel(const double* __restrict__ xpool, const int64_t* __restrict__ xslot,
                               const uint32_t* __restrict__ xcode, const double* __restrict__ xsq, int64_t nx,
                               const double* __restrict__ ypool, const int64_t* __restrict__ yslot,
                               const uint32_t* __restrict__ ycode, int64_t ny, int bs, double* __restrict__ part) {
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t e = (int64_t)bs * bs;
  for (int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; q < nx; q += nw) {
    int64_t p = find_code(ycode, ny, xcode[q]);
    if (p < 0) {
      if (lane == 0) part[q] = xsq[q];
      continue;
    }
    const double2* xs = reinterpret_cast<const double2*>(xpool + xslot[q] * e);
    const double2* ys = reinterpret_cast<const double2*>(ypool + yslot[p] * e);
    double s;
    bool nz, bad;
    warp_leaf_sumsq(
        [&](int i) {
          double2 a = __ldg(xs + i), b = __ldg(ys + i);
          return make_double2(a.x - b.x, a.y - b.y);
        },
        bs, lane, &s, &nz, &bad);
    if (lane == 0) part[q] = s;
  }
}

__global__ void error_y_kernel(const uint32_t* __restrict__ xcode, int64_t nx, const uint32_t* __restrict__ ycode,
                               const double* __restrict__ ysq, int64_t ny, double* __restrict__ part) {
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < ny; q += (int64_t)gridDim.x * blockDim.x)
    part[q] = find_code(xcode, nx, ycode[q]) < 0 ? ysq[q] : 0.0;
}

// Deterministic sum: fixed 4096-element tiles reduced by a fixed tree, then
// the tile sums in order by one block.
__global__ void sum_tiles_kernel(const double* __restrict__ in, int64_t n, double* __restrict__ out) {
  __shared__ double sh[kThreads];
  const int64_t base = (int64_t)blockIdx.x * 4096;
  double s = 0.0;
  for (int i = 0; i < 16; ++i) {
    int64_t q = base + threadIdx.x + (int64_t)i * kThreads;
    if (q < n) s += in[q];
  }
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[blockIdx.x] = sh[0];
}

double device_sum(spamm_ctx ctx, const double* in, int64_t n) {
  if (n <= 0) return 0.0;
  BufP a = alloc_n<double>(ctx, (n + 4095) / 4096 + 1);
  const double* src = in;
  BufP cur;
  while (true) {
    int64_t nb = (n + 4095) / 4096;
    BufP out = alloc_n<double>(ctx, nb);
    sum_tiles_kernel<<<(unsigned)nb, kThreads, 0, ctx->stream>>>(src, n, P<double>(out));
    CK_LAUNCH("sum_tiles_kernel");
    cur = out;
    src = P<double>(cur);
    n = nb;
    if (nb == 1) break;
  }
  return read_scalar<double>(ctx, src);
}

__global__ void gather_leaves_kernel(const double* __restrict__ pool, const int64_t* __restrict__ slot,
                                     const uint32_t* __restrict__ code, int64_t nleaves, int bs, int64_t nq,
                                     const int32_t* __restrict__ bi, const int32_t* __restrict__ bj,
                                     double* __restrict__ out, int32_t* __restrict__ found) {
  const int64_t e = (int64_t)bs * bs;
  const int64_t side = (int64_t)1 << 16;
  for (int64_t q = blockIdx.x; q < nq; q += gridDim.x) {
    const int32_t r = bi[q], c = bj[q];
    int64_t p = -1;
    if (r >= 0 && c >= 0 && r < side && c < side) p = find_code(code, nleaves, morton2((uint32_t)r, (uint32_t)c));
    if (threadIdx.x == 0 && found) found[q] = p >= 0;
    for (int64_t i = threadIdx.x; i < e; i += blockDim.x) out[q * e + i] = p >= 0 ? pool[slot[p] * e + i] : 0.0;
  }
}

double error_fro(spamm_mat X, spamm_mat Y) {
  spamm_ctx ctx = X->ctx;
  const int64_t nx = X->nleaves, ny = Y->nleaves;
  BufP px = alloc_n<double>(ctx, nx), py = alloc_n<double>(ctx, ny);
  double total = 0.0;
  if (nx > 0) {
    error_x_kernel<<<grid_for(ctx, nx, kThreads / 32), kThreads, 0, ctx->stream>>>(
        P<double>(X->pool), P<int64_t>(X->slot), P<uint32_t>(X->lv[X->L].code), P<double>(X->lv[X->L].sq), nx,
        P<double>(Y->pool), P<int64_t>(Y->slot), P<uint32_t>(Y->lv[Y->L].code), ny, X->bs, P<double>(px));
    CK_LAUNCH("error_x_kernel");
    total += device_sum(ctx, P<double>(px), nx);
  }
  if (ny > 0) {
    error_y_kernel<<<grid_for(ctx, ny, kThreads), kThreads, 0, ctx->stream>>>(
        P<uint32_t>(X->lv[X->L].code), nx, P<uint32_t>(Y->lv[Y->L].code), P<double>(Y->lv[Y->L].sq), ny,
        P<double>(py));
    CK_LAUNCH("error_y_kernel");
    total += device_sum(ctx, P<double>(py), ny);
  }
  sync_and_check(ctx);
  return sqrt(total);
}

}  // namespace spamm
