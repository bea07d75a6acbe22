// internal.cuh -- shared internals of libspamm (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <memory>
#include <string>
#include <vector>

#include "spamm.h"

namespace spamm {

struct Error {
  spamm_status status;
  std::string msg;
};

[[noreturn]] void fail(spamm_status st, const std::string& msg);
void check_cuda(cudaError_t e, const char* what, const char* file, int line);
#define CK(x) ::spamm::check_cuda((x), #x, __FILE__, __LINE__)
// Every kernel launch is followed by CK_LAUNCH, which also counts it.
extern thread_local unsigned long long g_kernel_launches;
#define CK_LAUNCH(what) \
  (++::spamm::g_kernel_launches, ::spamm::check_cuda(cudaGetLastError(), what, __FILE__, __LINE__))

// Device buffer owned through the context allocator.
struct Buf {
  spamm_ctx ctx = nullptr;
  void* p = nullptr;
  size_t bytes = 0;
  ~Buf();
};
using BufP = std::shared_ptr<Buf>;
BufP alloc_bytes(spamm_ctx ctx, size_t bytes);
template <class T>
BufP alloc_n(spamm_ctx ctx, int64_t count) {
  return alloc_bytes(ctx, (size_t)(count > 0 ? count : 0) * sizeof(T));
}
template <class T>
T* P(const BufP& b) {
  return b ? static_cast<T*>(b->p) : nullptr;
}

// One quadtree level: nodes sorted by Morton code of (row, col) at that level.
struct Level {
  int64_t count = 0;
  BufP code;   // uint32 Morton code
  BufP sq;     // double squared Frobenius norm
  BufP child;  // int4: node index of child (2*ci + cj) on the next level, -1 if null (levels < L)
};

// Bits of the device error word.
enum : int { DEV_ERR_TIMEOUT = 1, DEV_ERR_RANGE = 2, DEV_ERR_NONFINITE = 4, DEV_ERR_DUPLICATE = 8 };

// Bounded waits: iterations of a try_wait loop before a device wait gives up.
constexpr long long kWaitLimit = 1ll << 26;

// Morton codes of (row, col) with the row bit above the column bit, so the
// four children of code m are 4m + 2*ci + cj.
__host__ __device__ __forceinline__ uint32_t part1by1(uint32_t x) {
  x &= 0x0000FFFFu;
  x = (x | (x << 8)) & 0x00FF00FFu;
  x = (x | (x << 4)) & 0x0F0F0F0Fu;
  x = (x | (x << 2)) & 0x33333333u;
  x = (x | (x << 1)) & 0x55555555u;
  return x;
}
__host__ __device__ __forceinline__ uint32_t compact1by1(uint32_t x) {
  x &= 0x55555555u;
  x = (x | (x >> 1)) & 0x33333333u;
  x = (x | (x >> 2)) & 0x0F0F0F0Fu;
  x = (x | (x >> 4)) & 0x00FF00FFu;
  x = (x | (x >> 8)) & 0x0000FFFFu;
  return x;
}
__host__ __device__ __forceinline__ uint32_t morton2(uint32_t r, uint32_t c) { return (part1by1(r) << 1) | part1by1(c); }
__host__ __device__ __forceinline__ uint32_t code_row(uint32_t m) { return compact1by1(m >> 1); }
__host__ __device__ __forceinline__ uint32_t code_col(uint32_t m) { return compact1by1(m); }

inline int levels_for(int64_t n, int bs) {
  int64_t nb = (n + bs - 1) / bs;
  int L = 0;
  while (((int64_t)1 << L) < nb) ++L;
  return L;
}

// ---- primitives (prims.cu) ----
// Exclusive prefix sum of n uint64 values; total written to d_total (device) if not null.
void scan_exclusive_u64(spamm_ctx ctx, const uint64_t* in, uint64_t* out, int64_t n, uint64_t* d_total);
// Inclusive prefix sum of n doubles (fixed tiling: the same rounding on every run).
void scan_inclusive_f64(spamm_ctx ctx, const double* in, double* out, int64_t n);
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits of the key.
void radix_sort_pairs(spamm_ctx ctx, uint64_t* keys, int64_t* vals, int64_t n, int bits);
// Copy a device scalar to the host (synchronises the context stream).
template <class T>
T read_scalar(spamm_ctx ctx, const T* d);
void sync_and_check(spamm_ctx ctx);  // synchronise, map the device error word to a status
void clear_device_error(spamm_ctx ctx);

}  // namespace spamm

struct spamm_ctx_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  void* (*ualloc)(size_t, void*) = nullptr;
  void (*ufree)(void*, void*) = nullptr;
  void* user = nullptr;
  std::string last_error;
  int* d_err = nullptr;                      // device error word
  unsigned long long* d_scratch = nullptr;   // 64 counters (statistics, work queues)
  void* h_pinned = nullptr;                  // 4 KB pinned staging for scalar read-backs
  int num_sms = 0;
  int gemm_sm_limit = 0;                     // 0: leaf GEMM may use every SM
  int exec_graph = 0;                        // run the execute phase as a captured CUDA graph
  int claim_order = 0;                       // spamm_claim_order of the plans created on this context
  cudaStream_t capture_stream = nullptr;     // created on first graph capture
  cudaGraphExec_t graph_exec = nullptr;      // the last execute graph, updated in place for the next batch
  int64_t graph_instantiations = 0, graph_updates = 0;
  int live_handles = 0;
};

struct spamm_mat_s {
  spamm_ctx ctx = nullptr;
  int64_t n = 0;
  int bs = 0;
  int L = 0;
  int64_t nleaves = 0;
  spamm::BufP pool;  // double payload, bs*bs per slot
  spamm::BufP slot;  // int64 per leaf: payload slot of leaf m (leaves in Morton order)
  int symmetric = 0;  // the matrix equals its transpose (set by the generator or the caller)
  std::vector<spamm::Level> lv;  // levels 0..L
};

namespace spamm {
// ---- quadtree store (store.cu) ----
spamm_mat new_mat(spamm_ctx ctx, int64_t n, int bs);
void build_tree(spamm_mat m);  // levels L-1..0 from m->lv[L]
// build_tree in parts: the structure (codes, child links; synchronises per
// level for the counts), then norm buffers, then the norms (no host sync, so
// it can be captured in a CUDA graph).  The addition order is build_tree's.
void build_skeleton(spamm_mat m);
void alloc_level_norms(spamm_mat m);
void propagate_norms(spamm_mat m);
// propagate_norms of several matrices at once: one launch per height above the
// leaves.  norm_batch_tables uploads the per-height segment tables (norm
// buffers must already exist); propagate_norms_batch launches (no host sync).
struct NormBatchLevel {
  const void* seg = nullptr;       // device segment table of this height
  const int64_t* begin = nullptr;  // device: first parent of each segment
  int first = 0, nseg = 0;
  int64_t total = 0;
};
BufP norm_batch_tables(spamm_ctx ctx, const std::vector<spamm_mat>& ms, std::vector<NormBatchLevel>* levels);
void propagate_norms_batch(spamm_ctx ctx, const std::vector<NormBatchLevel>& levels);
// Leaf set from candidate leaves: keep[q] selects rows of (code, sq, slot) already sorted by code.
void set_leaves_compacted(spamm_mat m, int64_t ncand, const uint32_t* code, const double* sq, const int64_t* slot,
                          const uint8_t* keep);
spamm_mat truncate_block(spamm_mat in, double tau, spamm_ctx on = nullptr);  // work on `on` (default: in's context)
spamm_mat truncate_element(spamm_mat in, double tau);
spamm_mat truncate_error_controlled(spamm_mat in, double tau, spamm_ctx on = nullptr);
void leaf_sqnorms(spamm_ctx ctx, const double* pool, const int64_t* slot, int64_t nleaves, int bs, double* sq,
                  uint8_t* nonzero, int check_finite);
double error_fro(spamm_mat X, spamm_mat Y);
double device_sum(spamm_ctx ctx, const double* in, int64_t n);  // deterministic reduction, synchronises

// ---- purification-chain operations (algebra.cu) ----
spamm_mat add_scaled(double alpha, spamm_mat X, double beta, spamm_mat Y, spamm_ctx ctx);
spamm_mat identity_mat(spamm_ctx ctx, int64_t n, int bs);
double trace_of(spamm_mat X);

// ---- task-list builder (tasks.cu) ----
struct TaskList {
  int64_t ngroups = 0;  // C leaves
  int64_t ntasks = 0;   // kept leaf products
  BufP gcode;           // uint32 Morton code of each C leaf, ascending
  BufP gstart;          // int64 [ngroups + 1] first task of each C leaf
  BufP ta, tb;          // int32 leaf index in A / B of each task (k ascending within a C leaf)
  int64_t nquads = 0;   // output nodes one level above the leaves
  BufP quads;           // int32 [4 * nquads]: C leaf (group) index of child 2*ci + cj, -1 if absent
  int64_t n_candidates[SPAMM_MAX_LEVELS] = {};
  int64_t n_kept_level[SPAMM_MAX_LEVELS] = {};
  int64_t n_borderline = 0;
};
TaskList build_tasks(spamm_mat A, spamm_mat B, double tau, int test_norms, spamm_ctx on = nullptr);

// ---- batched leaf products (gemm_fp64.cu, gemm_tc.cu) ----
// One k step of a quad of output leaves (2I + h, 2J + c) in the tensor-core
// kernel: the four kept-product runs of the quad merged by k.
struct __align__(16) QuadStep {
  int32_t a[2];    // A leaf (2I + h, k), -1 where no kept product of row half h uses k
  int32_t b[2];    // B leaf (k, 2J + c), -1 where no kept product of column c uses k
  float scale[4];  // child 2h + c: its operand scale factor if the product (2I+h, k, 2J+c) is kept, else 0
};
static_assert(sizeof(QuadStep) == 32, "QuadStep is two 16-byte words");

// Device view of one planned multiplication.  A batch is an array of these;
// its work units (output leaves, or quads of output leaves for the
// tensor-core kernel) are numbered consecutively across plans: plan r owns
// units [ubegin[r], ubegin[r+1]).  Output leaf g of plan r is the sum over its
// tasks of A[ta] B[tb], written to cpool + g*bs*bs with its squared norm in csq[g].
struct PlanDev {
  const int64_t* gstart;
  const int32_t* ta;
  const int32_t* tb;
  const int32_t* quads;
  const double* poolA;
  const int64_t* slotA;
  const double* poolB;
  const int64_t* slotB;
  const uint8_t* termsA;  // tensor forms: operand terms per leaf
  const uint8_t* termsB;
  const int64_t* qstart;    // tensor forms: steps of quad Q are qsteps[qstart[Q] .. qstart[Q+1])
  const QuadStep* qsteps;
  double* cpool;
  double* csq;
  const int64_t* uorder;  // unit (FP64: output leaf; tensor forms: quad or 128-leaf) at each claiming position, or null for identity
  double* csq_part;       // FP64 form, leaves split into sub-tile units: partial squared norms [leaf][sub-tile]
  int32_t tc_bs;          // tensor forms: 64 (units are quads of output leaves) or 128 (units are output leaves)
  int64_t ufirst;         // tensor forms without uorder: unit number of this view's unit 0 (sliced execution)
};
struct BatchDev {
  const PlanDev* plans;
  const int64_t* ubegin;  // nplans + 1 entries
  int nplans;
  int64_t nunits;
};
// Plan owning unit u (the last r with ubegin[r] <= u).
__device__ __forceinline__ int plan_of(const int64_t* __restrict__ ubegin, int nplans, int64_t u) {
  int lo = 0, hi = nplans - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (ubegin[mid] <= u)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}
void gemm_fp64_batch(spamm_ctx ctx, int bs, const BatchDev& b);
// Work units per output leaf of the FP64 kernel (sub-tiles of 64 x 64 for larger leaves).
int fp64_units_per_leaf(int bs);
// Output leaves ordered by their number of kept products, largest first
// (stable), for the FP64 kernel's unit claiming; an empty buffer when the
// leaves are small enough that the claiming tail does not matter.
// Units 0..n-1 sorted by their work start[u+1] - start[u], largest first,
// ties in index order (stable); empty for n <= 1.
BufP unit_order_longest(spamm_ctx ctx, const int64_t* start, int64_t n);
// The tensor-core forms' persistent quad kernel (gemm_tc.cu).
void gemm_tc_batch(spamm_ctx ctx, spamm_prec prec, const BatchDev& b);
// Kernel (d) of the tensor-core forms: the GEMM's two-float output slots to
// FP64 in place, and each leaf's squared norm (kernel (a)'s order).
void tc_finish(spamm_ctx ctx, spamm_prec prec, double* pool, int64_t nleaves, int bs, double* sq);
// 64 x 64 operand tiles per leaf of the tensor forms (bs 64: 1, bs 128: 4).
inline int tc_tiles_per_leaf(int bs) { return (bs / 64) * (bs / 64); }
// Operand terms of a leaf set for a tensor form (role 0: used as A, 1: as B),
// and each tile's power-of-two scale exponent.
void prep_terms(spamm_mat M, spamm_prec prec, int role, BufP* terms, BufP* expo, spamm_ctx on = nullptr);
// Step list of every quad of T for the tensor-core kernel; returns the step count.
// codeA: Morton codes of A's leaves (the k of a task is the column of its A
// leaf); expA/expB: the leaves' scale exponents (null: no scaling).
// bmap (may be null): for B's leaf q, the index of the leaf whose terms serve
// as its B operand (a symmetric matrix times itself uses A's terms of the
// transposed leaf); the step list then refers to that index.
int64_t build_quad_steps(spamm_ctx ctx, const TaskList& T, const uint32_t* codeA, const int32_t* expA,
                         const int32_t* expB, const int32_t* bmap, BufP* qstart, BufP* qsteps);
// The same for 128 x 128 leaves: one unit per output leaf, two K-half steps
// per kept product (T.gstart doubled), on the tile-split operand terms.
int64_t build_leaf128_steps(spamm_ctx ctx, const TaskList& T, const int32_t* expA, const int32_t* expB,
                            const int32_t* bmap, BufP* qstart, BufP* qsteps);
// For every leaf (k, j) of M, the index of leaf (j, k) in M (-1 if absent);
// returns the number of absent ones (synchronises).
int64_t transpose_map(spamm_mat M, BufP* map, spamm_ctx on = nullptr);
// Tensor-core flops one quad step executes (every term product over the full 128 x 128 tile).
double quad_step_flops(spamm_prec prec);
}  // namespace spamm
