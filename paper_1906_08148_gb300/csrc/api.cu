// api.cu -- the extern "C" entry points of libspamm (declared in spamm.h).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "internal.cuh"

namespace spamm {
spamm_mat build_from_blocks(spamm_ctx, int64_t, int, int64_t, const int32_t*, const int32_t*, const double*, int,
                            double, spamm_trunc_rule);
spamm_mat build_from_dense(spamm_ctx, int64_t, const double*, int64_t, int, int, double, spamm_trunc_rule);
spamm_mat build_generated(spamm_ctx, const spamm_gen_params*, int, double, spamm_trunc_rule);
spamm_mat build_from_coo(spamm_ctx, int64_t, int64_t, const int64_t*, const int64_t*, const double*, int, int, double,
                         spamm_trunc_rule);
void export_dense(spamm_mat, double*, int64_t, int);
void export_blocks(spamm_mat, int32_t*, int32_t*, double*, double*, int);
void tasks_to_ikj(spamm_mat A, const TaskList& T, int32_t* d_out);
void fill_iota_i64(spamm_ctx ctx, int64_t* p, int64_t n);
void gather_leaves(spamm_mat m, int64_t nq, const int32_t* bi, const int32_t* bj, double* out, int32_t* found,
                   int on_device);
}  // namespace spamm

using namespace spamm;

namespace {

spamm_status set_error(spamm_ctx ctx, spamm_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

template <class F>
spamm_status guarded(spamm_ctx ctx, F&& f) {
  if (ctx) {
    ctx->last_error.clear();
    cudaSetDevice(ctx->device);
  }
  try {
    f();
    return SPAMM_OK;
  } catch (const Error& e) {
    return set_error(ctx, e.status, e.msg);
  } catch (const std::bad_alloc&) {
    return set_error(ctx, SPAMM_E_OOM, "host allocation failed");
  } catch (...) {
    return set_error(ctx, SPAMM_E_CUDA, "unexpected exception");
  }
}

void need(bool ok, const char* what) {
  if (!ok) fail(SPAMM_E_INVALID_ARG, what);
}

void check_bs(int bs) { need(bs == 32 || bs == 64 || bs == 128 || bs == 256, "bs must be 32, 64, 128 or 256"); }
void check_tau(double tau) { need(std::isfinite(tau) && tau >= 0.0, "tau must be finite and >= 0"); }
void check_rule(spamm_trunc_rule r) {
  need(r == SPAMM_TRUNC_BLOCK_FROB || r == SPAMM_TRUNC_ELEMENT || r == SPAMM_TRUNC_ERROR_CONTROL,
       "unknown truncation rule");
}
void check_n(int64_t n, int bs) {
  need(n > 0, "n must be > 0");
  need(levels_for(n, bs) <= 16, "n / bs exceeds 65536 leaves per dimension");
}

// The builders truncate per leaf while building (block and element rules); the
// error-controlled rule needs every leaf's norm first, so it runs afterwards.
double build_tau(double tau, spamm_trunc_rule r) { return r == SPAMM_TRUNC_ERROR_CONTROL ? 0.0 : tau; }
spamm_trunc_rule build_rule(spamm_trunc_rule r) { return r == SPAMM_TRUNC_ERROR_CONTROL ? SPAMM_TRUNC_BLOCK_FROB : r; }
spamm_mat after_build(spamm_mat m, double tau, spamm_trunc_rule r) {
  if (r != SPAMM_TRUNC_ERROR_CONTROL || tau <= 0.0) return m;
  std::unique_ptr<spamm_mat_s> full(m);
  return truncate_error_controlled(m, tau);
}

spamm_mat registered(spamm_mat m) {
  m->ctx->live_handles++;
  return m;
}

// Device time between two events on the context stream (events are synchronised).
double elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, a, b));
  return (double)ms;
}

struct Events {
  cudaEvent_t e[5] = {};
  Events() {
    for (auto& x : e) CK(cudaEventCreate(&x));
  }
  ~Events() {
    for (auto& x : e)
      if (x) cudaEventDestroy(x);
  }
};

}  // namespace

extern "C" {

spamm_status spamm_create(int device, void* cuda_stream, spamm_ctx* out) {
  if (!out) return SPAMM_E_INVALID_ARG;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return SPAMM_E_INVALID_ARG;
  }
  spamm_ctx ctx = new spamm_ctx_s();
  spamm_status st = guarded(nullptr, [&] {
    ctx->device = device;
    CK(cudaSetDevice(device));
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    CK(cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device));
    CK(cudaMalloc(&ctx->d_err, sizeof(int)));
    CK(cudaMemset(ctx->d_err, 0, sizeof(int)));
    CK(cudaMalloc(&ctx->d_scratch, 64 * sizeof(unsigned long long)));
    CK(cudaMemset(ctx->d_scratch, 0, 64 * sizeof(unsigned long long)));
    CK(cudaMallocHost(&ctx->h_pinned, 4096));
    // keep freed stream-ordered memory in the pool instead of returning it
    cudaMemPool_t pool;
    CK(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t thr = UINT64_MAX;
    CK(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  });
  if (st != SPAMM_OK) {
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->d_scratch) cudaFree(ctx->d_scratch);
    if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
    delete ctx;
    return st;
  }
  *out = ctx;
  return SPAMM_OK;
}

spamm_status spamm_destroy(spamm_ctx ctx) {
  if (!ctx) return SPAMM_E_INVALID_ARG;
  if (ctx->live_handles > 0) return set_error(ctx, SPAMM_E_BUSY, "release all handles before destroying the context");
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(ctx->d_err);
  cudaFree(ctx->d_scratch);
  cudaFreeHost(ctx->h_pinned);
  if (ctx->graph_exec) cudaGraphExecDestroy(ctx->graph_exec);
  if (ctx->capture_stream) cudaStreamDestroy(ctx->capture_stream);
  delete ctx;
  return SPAMM_OK;
}

spamm_status spamm_set_stream(spamm_ctx ctx, void* cuda_stream) {
  if (!ctx) return SPAMM_E_INVALID_ARG;
  return guarded(ctx, [&] {
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
  });
}

spamm_status spamm_set_allocator(spamm_ctx ctx, void* (*alloc)(size_t, void*), void (*free_fn)(void*, void*),
                                 void* user) {
  if (!ctx) return SPAMM_E_INVALID_ARG;
  return guarded(ctx, [&] {
    need((alloc == nullptr) == (free_fn == nullptr), "alloc and free must both be set or both be NULL");
    if (ctx->live_handles > 0) fail(SPAMM_E_BUSY, "the allocator can only change while no handle is alive");
    ctx->ualloc = alloc;
    ctx->ufree = free_fn;
    ctx->user = user;
  });
}

spamm_status spamm_sync(spamm_ctx ctx) {
  if (!ctx) return SPAMM_E_INVALID_ARG;
  return guarded(ctx, [&] { sync_and_check(ctx); });
}

spamm_status spamm_trim(spamm_ctx ctx) {
  if (!ctx) return SPAMM_E_INVALID_ARG;
  return guarded(ctx, [&] {
    sync_and_check(ctx);
    if (ctx->ualloc) return;
    cudaMemPool_t pool;
    CK(cudaDeviceGetDefaultMemPool(&pool, ctx->device));
    CK(cudaMemPoolTrimTo(pool, 0));
  });
}

const char* spamm_last_error(spamm_ctx ctx) { return ctx ? ctx->last_error.c_str() : "invalid context"; }

spamm_status spamm_from_dense(spamm_ctx ctx, int64_t n, const double* a, int64_t lda, int on_device, int bs,
                              double tau, spamm_trunc_rule rule, spamm_mat* out) {
  if (!ctx || !out) return SPAMM_E_INVALID_ARG;
  *out = nullptr;
  return guarded(ctx, [&] {
    check_bs(bs);
    check_n(n, bs);
    check_tau(tau);
    check_rule(rule);
    need(a != nullptr && lda >= n, "a must be non-NULL with lda >= n");
    spamm_mat m = after_build(build_from_dense(ctx, n, a, lda, on_device, bs, build_tau(tau, rule), build_rule(rule)),
                              tau, rule);
    *out = registered(m);
  });
}

spamm_status spamm_from_blocks(spamm_ctx ctx, int64_t n, int bs, int64_t nblocks, const int32_t* bi,
                               const int32_t* bj, const double* payload, int on_device, double tau,
                               spamm_trunc_rule rule, spamm_mat* out) {
  if (!ctx || !out) return SPAMM_E_INVALID_ARG;
  *out = nullptr;
  return guarded(ctx, [&] {
    check_bs(bs);
    check_n(n, bs);
    check_tau(tau);
    check_rule(rule);
    need(nblocks >= 0, "nblocks must be >= 0");
    need(nblocks == 0 || (bi && bj && payload), "bi, bj and payload must be non-NULL");
    spamm_mat m = after_build(
        build_from_blocks(ctx, n, bs, nblocks, bi, bj, payload, on_device, build_tau(tau, rule), build_rule(rule)), tau,
        rule);
    *out = registered(m);
  });
}

spamm_status spamm_from_coo(spamm_ctx ctx, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col,
                            const double* val, int on_device, int bs, double tau, spamm_trunc_rule rule,
                            spamm_mat* out) {
  if (!ctx || !out) return SPAMM_E_INVALID_ARG;
  *out = nullptr;
  return guarded(ctx, [&] {
    check_bs(bs);
    check_n(n, bs);
    check_tau(tau);
    check_rule(rule);
    need(nnz >= 0, "nnz must be >= 0");
    need(nnz == 0 || (row && col && val), "row, col and val must be non-NULL");
    spamm_mat m = after_build(
        build_from_coo(ctx, n, nnz, row, col, val, on_device, bs, build_tau(tau, rule), build_rule(rule)), tau, rule);
    *out = registered(m);
  });
}

spamm_status spamm_generate(spamm_ctx ctx, const spamm_gen_params* params, int bs, double tau, spamm_trunc_rule rule,
                            spamm_mat* out) {
  if (!ctx || !out || !params) return SPAMM_E_INVALID_ARG;
  *out = nullptr;
  return guarded(ctx, [&] {
    check_bs(bs);
    check_n(params->n, bs);
    check_tau(tau);
    check_rule(rule);
    need(params->kind == 0 || params->kind == 1, "kind must be 0 (1-D) or 1 (3-D lattice)");
    need(std::isfinite(params->alpha) && params->alpha >= 0.0, "alpha must be finite and >= 0");
    need(std::isfinite(params->c) && std::isfinite(params->cutoff) && params->cutoff >= 0.0, "bad c or cutoff");
    spamm_mat m = after_build(build_generated(ctx, params, bs, build_tau(tau, rule), build_rule(rule)), tau, rule);
    *out = registered(m);
  });
}

spamm_status spamm_truncate(spamm_ctx ctx, spamm_mat in, double tau, spamm_trunc_rule rule, spamm_mat* out) {
  if (!ctx || !in || !out) return SPAMM_E_INVALID_ARG;
  *out = nullptr;
  return guarded(ctx, [&] {
    check_tau(tau);
    check_rule(rule);
    spamm_mat m = rule == SPAMM_TRUNC_BLOCK_FROB ? truncate_block(in, tau)
                  : rule == SPAMM_TRUNC_ELEMENT  ? truncate_element(in, tau)
                                                 : truncate_error_controlled(in, tau);
    sync_and_check(ctx);
    *out = registered(m);
  });
}

spamm_status spamm_release(spamm_mat m) {
  if (!m) return SPAMM_E_INVALID_ARG;
  spamm_ctx ctx = m->ctx;
  cudaSetDevice(ctx->device);
  delete m;
  ctx->live_handles--;
  return SPAMM_OK;
}

static void run_truncation(spamm_mat A, spamm_mat B, double tau, spamm_mode mode, spamm_mat* At, spamm_mat* Bt,
                           spamm_ctx on = nullptr) {
  if (mode == SPAMM_MODE_SPAMM) {
    *At = A;
    *Bt = B;
    return;
  }
  *At = truncate_block(A, tau, on);
  *Bt = (B == A) ? *At : truncate_block(B, tau, on);
}

static void check_pair(spamm_mat A, spamm_mat B, double tau, spamm_mode mode) {
  if (A->n != B->n || A->bs != B->bs) fail(SPAMM_E_SHAPE, "A and B differ in n or bs");
  if (A->ctx->device != B->ctx->device) fail(SPAMM_E_INVALID_ARG, "A and B live on different devices");
  check_tau(tau);
  need(mode == SPAMM_MODE_TRUNCATE || mode == SPAMM_MODE_SPAMM || mode == SPAMM_MODE_COMBINED, "unknown mode");
}

}  // extern "C"

// ------------------------------------------------------------ plan / execute
struct spamm_plan_s {
  spamm_ctx ctx = nullptr;
  int64_t n = 0;
  int bs = 0;
  int L = 0;
  spamm_prec prec = SPAMM_PREC_FP64;
  TaskList T;
  BufP poolA, slotA, poolB, slotB, termsA, termsB, expA, expB;
  BufP qstart, qsteps;  // tensor forms: the quad step list
  BufP bmap;            // tensor forms, symmetric X times X: B leaf -> A leaf whose terms serve it
  BufP uorder;          // FP64 form: unit -> output leaf, longest first (empty: identity)
  int64_t nsteps = 0;
  std::vector<Level> cskel;  // output quadtree structure (codes, child links; no norms)
  int64_t na = 0, nb = 0;
  double ms_truncate = 0, ms_tasks = 0, ms_prep = 0;
  int64_t launches = 0;
};

namespace {

size_t held_bytes(const spamm_plan_s& p) {
  size_t b = 0;
  std::vector<const Buf*> seen;
  for (const BufP* x : {&p.T.gcode, &p.T.gstart, &p.T.ta, &p.T.tb, &p.T.quads, &p.qstart, &p.qsteps, &p.slotA,
                        &p.slotB, &p.termsA, &p.termsB, &p.expA, &p.expB, &p.uorder, &p.bmap}) {
    if (!*x) continue;
    bool dup = false;  // shared buffers (symmetric operands) count once
    for (const Buf* q : seen) dup = dup || q == x->get();
    if (dup) continue;
    seen.push_back(x->get());
    b += (*x)->bytes;
  }
  return b;
}

void check_form(spamm_prec prec, int bs) {
  need(prec == SPAMM_PREC_FP64 || prec == SPAMM_PREC_BF16_SPLIT || prec == SPAMM_PREC_FP16_SCALED ||
           prec == SPAMM_PREC_BF16_SPLIT4,
       "unknown precision form");
  if (prec == SPAMM_PREC_FP64 && bs > 256)
    fail(SPAMM_E_UNSUPPORTED, "FP64 leaf products are built for bs = 32, 64, 128 and 256");
  if (prec != SPAMM_PREC_FP64 && bs != 64 && bs != 128)
    fail(SPAMM_E_UNSUPPORTED, "tensor-core precision forms are built for bs = 64 and 128");
}

spamm_plan make_plan(spamm_ctx ctx, spamm_mat A, spamm_mat B, double tau, spamm_mode mode, spamm_prec prec) {
  check_pair(A, B, tau, mode);
  check_form(prec, A->bs);
  Events ev;
  const unsigned long long launches0 = g_kernel_launches;
  std::unique_ptr<spamm_plan_s> p(new spamm_plan_s());
  p->ctx = ctx;
  p->n = A->n;
  p->bs = A->bs;
  p->L = A->L;
  p->prec = prec;
  CK(cudaEventRecord(ev.e[0], ctx->stream));
  spamm_mat At = nullptr, Bt = nullptr;
  run_truncation(A, B, tau, mode, &At, &Bt, ctx);
  std::unique_ptr<spamm_mat_s> ownA(At != A ? At : nullptr), ownB((Bt != B && Bt != At) ? Bt : nullptr);
  CK(cudaEventRecord(ev.e[1], ctx->stream));
  p->T = build_tasks(At, Bt, tau, mode != SPAMM_MODE_TRUNCATE, ctx);
  {
    // the output structure is fixed by the kept set (Section 4.4): build it now
    std::unique_ptr<spamm_mat_s> sk(new_mat(ctx, A->n, A->bs));
    sk->lv[sk->L].count = p->T.ngroups;
    sk->lv[sk->L].code = p->T.gcode;
    build_skeleton(sk.get());
    p->cskel = sk->lv;
  }
  CK(cudaEventRecord(ev.e[2], ctx->stream));
  p->na = At->nleaves;
  p->nb = Bt->nleaves;
  if (prec == SPAMM_PREC_FP64) {
    p->poolA = At->pool;
    p->slotA = At->slot;
    p->poolB = Bt->pool;
    p->slotB = Bt->slot;
    const bool longest = ctx->claim_order == SPAMM_ORDER_LONGEST_FIRST ||
                         (ctx->claim_order == SPAMM_ORDER_AUTO && p->bs >= 128);
    if (longest) p->uorder = unit_order_longest(ctx, P<int64_t>(p->T.gstart), p->T.ngroups);
  } else {
    prep_terms(At, prec, 0, &p->termsA, &p->expA, ctx);
    // X times X with X symmetric: the B operand of leaf (k, j) is the transpose
    // of leaf (j, k), whose A terms are exactly the B terms of (k, j) (rows of
    // (j, k) are columns of (k, j), with the same grid), so one set of terms
    // serves both roles, if every leaf's transpose is present
    if (Bt == At && At->symmetric && transpose_map(At, &p->bmap, ctx) == 0) {
      p->termsB = p->termsA;
      p->expB = p->expA;
    } else {
      p->bmap.reset();
      prep_terms(Bt, prec, 1, &p->termsB, &p->expB, ctx);
    }
    if (p->bs == 128)
      p->nsteps = build_leaf128_steps(ctx, p->T, P<int32_t>(p->expA), P<int32_t>(p->expB), P<int32_t>(p->bmap),
                                      &p->qstart, &p->qsteps);
    else
      p->nsteps = build_quad_steps(ctx, p->T, P<uint32_t>(At->lv[At->L].code), P<int32_t>(p->expA),
                                   P<int32_t>(p->expB), P<int32_t>(p->bmap), &p->qstart, &p->qsteps);
    if (ctx->claim_order == SPAMM_ORDER_LONGEST_FIRST)
      p->uorder = unit_order_longest(ctx, P<int64_t>(p->qstart), p->bs == 128 ? p->T.ngroups : p->T.nquads);
  }
  CK(cudaEventRecord(ev.e[3], ctx->stream));
  sync_and_check(ctx);
  p->ms_truncate = elapsed_ms(ev.e[0], ev.e[1]);
  p->ms_tasks = elapsed_ms(ev.e[1], ev.e[2]);
  p->ms_prep = elapsed_ms(ev.e[2], ev.e[3]);
  p->launches = (int64_t)(g_kernel_launches - launches0);
  ctx->live_handles++;
  return p.release();
}

void fill_stats(const spamm_plan_s& p, spamm_stats* st) {
  memset(st, 0, sizeof(*st));
  for (int t = 0; t < SPAMM_MAX_LEVELS; ++t) {
    st->n_candidates[t] = p.T.n_candidates[t];
    st->n_kept_level[t] = p.T.n_kept_level[t];
  }
  st->n_kept = p.T.ntasks;
  st->n_borderline = p.T.n_borderline;
  st->n_c_leaves = p.T.ngroups;
  st->n_a_leaves = p.na;
  st->n_b_leaves = p.nb;
  st->levels = p.L;
  st->bs = p.bs;
  st->kept_flops = 2.0 * (double)p.bs * p.bs * p.bs * (double)p.T.ntasks;
  st->n_steps = p.prec == SPAMM_PREC_FP64 ? p.T.ntasks : p.nsteps;
  st->executed_flops = p.prec == SPAMM_PREC_FP64 ? st->kept_flops : (double)p.nsteps * quad_step_flops(p.prec);
  st->terms_shared = p.bmap ? 1 : 0;
  st->ms_truncate = p.ms_truncate;
  st->ms_tasks = p.ms_tasks;
  st->ms_prep = p.ms_prep;
}

// The output of one plan (its leaves, slots, norms and quadtree levels, the
// FP64 sub-tile partial norms) and the device view of the plan over all its
// work units: output leaves (or their 64 x 64 sub-tiles) for the FP64 kernel,
// quads of output leaves for the tensor-core kernel.
struct PlanOut {
  std::unique_ptr<spamm_mat_s> C;
  BufP part;
  PlanDev dev{};
  int64_t units = 0;
};

PlanOut make_output(spamm_ctx ctx, const spamm_plan_s& p) {
  PlanOut o;
  const int bs = p.bs;
  const int64_t e = (int64_t)bs * bs;
  o.C.reset(new_mat(ctx, p.n, bs));
  spamm_mat Cm = o.C.get();
  Cm->lv = p.cskel;
  Cm->nleaves = p.T.ngroups;
  Cm->pool = alloc_n<double>(ctx, p.T.ngroups * e);
  Cm->slot = alloc_n<int64_t>(ctx, p.T.ngroups);
  Cm->lv[Cm->L].sq = alloc_n<double>(ctx, p.T.ngroups);
  alloc_level_norms(Cm);
  PlanDev& d = o.dev;
  d.gstart = P<int64_t>(p.T.gstart);
  d.ta = P<int32_t>(p.T.ta);
  d.tb = P<int32_t>(p.T.tb);
  d.quads = P<int32_t>(p.T.quads);
  d.poolA = P<double>(p.poolA);
  d.slotA = P<int64_t>(p.slotA);
  d.poolB = P<double>(p.poolB);
  d.slotB = P<int64_t>(p.slotB);
  d.termsA = P<uint8_t>(p.termsA);
  d.termsB = P<uint8_t>(p.termsB);
  d.qstart = P<int64_t>(p.qstart);
  d.qsteps = P<QuadStep>(p.qsteps);
  d.cpool = P<double>(Cm->pool);
  d.csq = P<double>(Cm->lv[Cm->L].sq);
  d.uorder = P<int64_t>(p.uorder);
  const int64_t per_leaf = p.prec == SPAMM_PREC_FP64 ? fp64_units_per_leaf(bs) : 1;
  if (per_leaf > 1) {
    o.part = alloc_n<double>(ctx, p.T.ngroups * per_leaf);
    d.csq_part = P<double>(o.part);
  }
  d.tc_bs = bs;
  o.units = p.T.ngroups == 0 ? 0
            : p.prec == SPAMM_PREC_FP64 ? p.T.ngroups * per_leaf
            : bs == 128 ? p.T.ngroups
                        : p.T.nquads;
  return o;
}

// The plan's view from work unit `first` on (FP64: a whole number of leaves):
// the kernels number the units of a launch from 0 within each plan, so a
// slice is the same plan with its per-unit arrays advanced.
PlanDev slice_view(const spamm_plan_s& p, const PlanDev& d, int64_t first) {
  PlanDev v = d;
  if (first == 0) return v;
  if (p.prec == SPAMM_PREC_FP64) {
    const int64_t leaf0 = first / fp64_units_per_leaf(p.bs);
    if (v.uorder) {
      v.uorder += leaf0;  // leaves in claiming order; outputs indexed by the leaf itself
    } else {
      v.gstart += leaf0;
      v.cpool += leaf0 * (int64_t)p.bs * p.bs;
      v.csq += leaf0;
      if (v.csq_part) v.csq_part += leaf0 * fp64_units_per_leaf(p.bs);
    }
  } else if (v.uorder) {
    v.uorder += first;  // units in claiming order; steps and outputs indexed by the unit itself
  } else {
    v.ufirst = first;  // steps and outputs indexed by the unit itself (a 128-leaf unit is its output leaf)
  }
  return v;
}

void launch_gemm(spamm_ctx ctx, spamm_prec prec, int bs, const BatchDev& batch) {
  if (prec == SPAMM_PREC_FP64)
    gemm_fp64_batch(ctx, bs, batch);
  else
    gemm_tc_batch(ctx, prec, batch);
}

// One persistent launch over all plans, then every output's parent norms (one
// launch per level for the whole batch).  Buffers are allocated and the plan
// table uploaded first, so the launch sequence has no host synchronisation;
// with ctx->exec_graph it is captured and run as one CUDA graph.
std::vector<spamm_mat> execute_plans(spamm_ctx ctx, const std::vector<spamm_plan>& plans, double* ms_gemm,
                                     double* ms_cnorm, int64_t* launches) {
  const int64_t np = (int64_t)plans.size();
  const spamm_prec prec = plans[0]->prec;
  const int bs = plans[0]->bs;
  for (spamm_plan p : plans)
    if (p->ctx->device != ctx->device || p->prec != prec || p->bs != bs)
      fail(SPAMM_E_INVALID_ARG, "a batch needs one device, one precision form and one leaf size");
  Events ev;
  const unsigned long long launches0 = g_kernel_launches;
  std::vector<PlanOut> pout;
  std::vector<spamm_mat> outp;
  std::vector<PlanDev> host(np);
  std::vector<int64_t> ubegin(np + 1, 0);
  for (int64_t r = 0; r < np; ++r) {
    pout.push_back(make_output(ctx, *plans[r]));
    outp.push_back(pout.back().C.get());
    host[r] = pout.back().dev;
    ubegin[r + 1] = ubegin[r] + pout.back().units;
  }
  BufP dplans = alloc_n<PlanDev>(ctx, np), dub = alloc_n<int64_t>(ctx, np + 1);
  CK(cudaMemcpyAsync(P<PlanDev>(dplans), host.data(), np * sizeof(PlanDev), cudaMemcpyHostToDevice, ctx->stream));
  CK(cudaMemcpyAsync(P<int64_t>(dub), ubegin.data(), (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                     ctx->stream));
  std::vector<NormBatchLevel> nlv;
  BufP ntab = norm_batch_tables(ctx, outp, &nlv);
  BatchDev batch{P<PlanDev>(dplans), P<int64_t>(dub), (int)np, ubegin[np]};

  auto sequence = [&](unsigned evflags) {
    CK(cudaEventRecordWithFlags(ev.e[0], ctx->stream, evflags));
    launch_gemm(ctx, prec, bs, batch);
    CK(cudaEventRecordWithFlags(ev.e[1], ctx->stream, evflags));
    if (prec != SPAMM_PREC_FP64)
      for (int64_t r = 0; r < np; ++r)
        tc_finish(ctx, prec, P<double>(outp[r]->pool), outp[r]->nleaves, bs, P<double>(outp[r]->lv[outp[r]->L].sq));
    for (int64_t r = 0; r < np; ++r) fill_iota_i64(ctx, P<int64_t>(outp[r]->slot), outp[r]->nleaves);
    propagate_norms_batch(ctx, nlv);
    CK(cudaEventRecordWithFlags(ev.e[2], ctx->stream, evflags));
  };
  if (ctx->exec_graph) {
    // capture on the context's capture stream (the legacy stream cannot be captured), run on its stream
    if (!ctx->capture_stream) CK(cudaStreamCreateWithFlags(&ctx->capture_stream, cudaStreamNonBlocking));
    cudaStream_t run = ctx->stream;
    cudaGraph_t g = nullptr;
    cudaGraphExec_t ge = nullptr;
    ctx->stream = ctx->capture_stream;
    CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeRelaxed));
    try {
      sequence(cudaEventRecordExternal);
    } catch (...) {
      cudaStreamEndCapture(ctx->stream, &g);
      if (g) cudaGraphDestroy(g);
      ctx->stream = run;
      throw;
    }
    const cudaError_t ce = cudaStreamEndCapture(ctx->stream, &g);
    ctx->stream = run;
    CK(ce);
    // the instantiated graph of the previous batch is updated in place when
    // the new one has the same topology (new kernel parameters and events);
    // otherwise it is replaced
    bool updated = false;
    if (ctx->graph_exec) {
      cudaGraphExecUpdateResultInfo info;
      updated = cudaGraphExecUpdate(ctx->graph_exec, g, &info) == cudaSuccess;
      if (!updated) {
        cudaGetLastError();
        // not an error: the graph is re-instantiated; the reason is kept for diagnosis
        cudaGraphNodeType nt = cudaGraphNodeTypeEmpty;
        if (info.errorNode) cudaGraphNodeGetType(info.errorNode, &nt);
        ctx->last_error = "execute graph re-instantiated: update result " + std::to_string((int)info.result) +
                          ", node type " + std::to_string((int)nt);
        cudaGraphExecDestroy(ctx->graph_exec);
        ctx->graph_exec = nullptr;
      }
    }
    cudaError_t ie = cudaSuccess;
    if (!updated) ie = cudaGraphInstantiate(&ctx->graph_exec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) ctx->graph_exec = nullptr;
    CK(ie);
    ge = ctx->graph_exec;
    ctx->graph_updates += updated ? 1 : 0;
    ctx->graph_instantiations += updated ? 0 : 1;
    const cudaError_t le = cudaGraphLaunch(ge, ctx->stream);
    CK(le);
    ++g_kernel_launches;  // the graph launch itself; its kernels were counted at capture
    CK(cudaStreamSynchronize(ctx->stream));
  } else {
    sequence(cudaEventRecordDefault);
  }
  sync_and_check(ctx);
  *ms_gemm = elapsed_ms(ev.e[0], ev.e[1]);
  *ms_cnorm = elapsed_ms(ev.e[1], ev.e[2]);
  *launches = (int64_t)(g_kernel_launches - launches0);
  std::vector<spamm_mat> res;
  for (auto& o : pout) res.push_back(o.C.release());
  return res;
}

}  // namespace

extern "C" {

spamm_status spamm_plan_create(spamm_ctx ctx, spamm_mat A, spamm_mat B, double tau, spamm_mode mode, spamm_prec prec,
                               spamm_plan* out) {
  if (!ctx || !A || !B || !out) return SPAMM_E_INVALID_ARG;
  *out = nullptr;
  return guarded(ctx, [&] { *out = make_plan(ctx, A, B, tau, mode, prec); });
}

spamm_status spamm_plan_info(spamm_plan p, int64_t* n_kept, int64_t* n_c_leaves, int64_t* plan_bytes,
                             int64_t* exec_bytes) {
  if (!p) return SPAMM_E_INVALID_ARG;
  if (n_kept) *n_kept = p->T.ntasks;
  if (n_c_leaves) *n_c_leaves = p->T.ngroups;
  if (plan_bytes) *plan_bytes = (int64_t)held_bytes(*p);
  if (exec_bytes) {
    // output payload, slot and squared norm per leaf, the FP64 sub-tile partial
    // norms, the parents' norms (at most a third of the leaves), the batch tables
    const int64_t parts = p->prec == SPAMM_PREC_FP64 && fp64_units_per_leaf(p->bs) > 1 ? fp64_units_per_leaf(p->bs) : 0;
    *exec_bytes = p->T.ngroups * ((int64_t)p->bs * p->bs * 8 + 8 + 8 + 8 * parts) + (p->T.ngroups / 3 + 1) * 8 + 4096;
  }
  return SPAMM_OK;
}

spamm_status spamm_plan_release(spamm_plan p) {
  if (!p) return SPAMM_E_INVALID_ARG;
  spamm_ctx ctx = p->ctx;
  cudaSetDevice(ctx->device);
  delete p;
  ctx->live_handles--;
  return SPAMM_OK;
}

}  // extern "C"

// ------------------------------------------------------------ sliced execution
struct spamm_job_s {
  spamm_ctx ctx = nullptr;
  spamm_plan plan = nullptr;
  PlanOut out;
  int64_t done = 0;            // units run so far (a prefix of the claiming order)
  int nq = 1;                  // units per output leaf (FP64 sub-tiles), slices hold whole leaves
  std::vector<double> wpre;    // work of units [0, u): kept products (FP64) or quad steps
  double ms_gemm = 0.0;        // launches this job took part in
  int64_t launches = 0;
};

namespace {

// Host copy of the work per unit in claiming order, as a prefix sum.
void job_work_prefix(spamm_job j) {
  const spamm_plan_s& p = *j->plan;
  spamm_ctx ctx = j->ctx;
  const int64_t u = j->out.units;
  j->wpre.assign(u + 1, 0.0);
  if (u == 0) return;
  if (p.prec == SPAMM_PREC_FP64) {
    const int64_t ng = p.T.ngroups;
    std::vector<int64_t> gs(ng + 1), ord;
    CK(cudaMemcpyAsync(gs.data(), P<int64_t>(p.T.gstart), (ng + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost,
                       ctx->stream));
    if (p.uorder) {
      ord.resize(ng);
      CK(cudaMemcpyAsync(ord.data(), P<int64_t>(p.uorder), ng * sizeof(int64_t), cudaMemcpyDeviceToHost,
                         ctx->stream));
    }
    sync_and_check(ctx);
    for (int64_t x = 0; x < u; ++x) {
      const int64_t li = x / j->nq, g = ord.empty() ? li : ord[li];
      j->wpre[x + 1] = j->wpre[x] + (double)(gs[g + 1] - gs[g]) / j->nq;
    }
  } else {
    std::vector<int64_t> qs(u + 1), ord;
    CK(cudaMemcpyAsync(qs.data(), P<int64_t>(p.qstart), (u + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost,
                       ctx->stream));
    if (p.uorder) {
      ord.resize(u);
      CK(cudaMemcpyAsync(ord.data(), P<int64_t>(p.uorder), u * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    }
    sync_and_check(ctx);
    for (int64_t x = 0; x < u; ++x) {
      const int64_t q = ord.empty() ? x : ord[x];
      j->wpre[x + 1] = j->wpre[x] + (double)(qs[q + 1] - qs[q]);
    }
  }
}

}  // namespace

extern "C" {

spamm_status spamm_job_begin(spamm_ctx ctx, spamm_plan plan, spamm_job* out) {
  if (!ctx || !plan || !out) return SPAMM_E_INVALID_ARG;
  *out = nullptr;
  return guarded(ctx, [&] {
    if (plan->ctx->device != ctx->device) fail(SPAMM_E_INVALID_ARG, "the plan lives on another device");
    std::unique_ptr<spamm_job_s> j(new spamm_job_s());
    j->ctx = ctx;
    j->plan = plan;
    j->nq = plan->prec == SPAMM_PREC_FP64 ? fp64_units_per_leaf(plan->bs) : 1;
    j->out = make_output(ctx, *plan);
    job_work_prefix(j.get());
    ctx->live_handles++;
    *out = j.release();
  });
}

spamm_status spamm_job_info(spamm_job job, int64_t* units, int64_t* units_done, double* work, double* work_done) {
  if (!job) return SPAMM_E_INVALID_ARG;
  if (units) *units = job->out.units;
  if (units_done) *units_done = job->done;
  if (work) *work = job->wpre.back();
  if (work_done) *work_done = job->wpre[job->done];
  return SPAMM_OK;
}

spamm_status spamm_run(spamm_ctx ctx, int64_t njobs, const spamm_job* jobs, const double* work_budget,
                       int64_t* units_run, double* ms_gemm) {
  if (!ctx || njobs <= 0 || !jobs || !work_budget) return SPAMM_E_INVALID_ARG;
  return guarded(ctx, [&] {
    const spamm_prec prec = jobs[0] ? jobs[0]->plan->prec : SPAMM_PREC_FP64;
    const int bs = jobs[0] ? jobs[0]->plan->bs : 0;
    std::vector<PlanDev> host;
    std::vector<int64_t> ubegin(1, 0), take(njobs, 0);
    for (int64_t r = 0; r < njobs; ++r) {
      spamm_job j = jobs[r];
      need(j != nullptr, "NULL job");
      if (j->plan->prec != prec || j->plan->bs != bs || j->ctx->device != ctx->device)
        fail(SPAMM_E_INVALID_ARG, "one launch needs one device, one precision form and one leaf size");
      const int64_t c = j->done, left = j->out.units - c;
      if (left == 0) continue;
      // the units from c on whose work fits the budget, at least one leaf's worth
      const double lim = j->wpre[c] + (work_budget[r] > 0 ? work_budget[r] : 0.0);
      int64_t n = (int64_t)(std::upper_bound(j->wpre.begin() + c + 1, j->wpre.end(), lim) - j->wpre.begin()) - 1 - c;
      n = std::max<int64_t>(n, 1);
      n = (n + j->nq - 1) / j->nq * j->nq;
      n = std::min(n, left);
      take[r] = n;
      host.push_back(slice_view(*j->plan, j->out.dev, c));
      ubegin.push_back(ubegin.back() + n);
    }
    double ms = 0.0;
    if (!host.empty()) {
      const int64_t np = (int64_t)host.size();
      BufP dplans = alloc_n<PlanDev>(ctx, np), dub = alloc_n<int64_t>(ctx, np + 1);
      CK(cudaMemcpyAsync(P<PlanDev>(dplans), host.data(), np * sizeof(PlanDev), cudaMemcpyHostToDevice,
                         ctx->stream));
      CK(cudaMemcpyAsync(P<int64_t>(dub), ubegin.data(), (np + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                         ctx->stream));
      BatchDev batch{P<PlanDev>(dplans), P<int64_t>(dub), (int)np, ubegin.back()};
      Events ev;
      CK(cudaEventRecord(ev.e[0], ctx->stream));
      launch_gemm(ctx, prec, bs, batch);
      CK(cudaEventRecord(ev.e[1], ctx->stream));
      sync_and_check(ctx);
      ms = elapsed_ms(ev.e[0], ev.e[1]);
    }
    for (int64_t r = 0; r < njobs; ++r) {
      jobs[r]->done += take[r];
      if (take[r] > 0) {
        jobs[r]->ms_gemm += ms;
        jobs[r]->launches++;
      }
      if (units_run) units_run[r] = take[r];
    }
    if (ms_gemm) *ms_gemm = ms;
  });
}

spamm_status spamm_job_finish(spamm_ctx ctx, spamm_job job, spamm_mat* C, spamm_stats* stats) {
  if (!ctx || !job || !C) return SPAMM_E_INVALID_ARG;
  *C = nullptr;
  return guarded(ctx, [&] {
    if (job->done != job->out.units) fail(SPAMM_E_BUSY, "the job has units that have not run");
    if (!job->out.C) fail(SPAMM_E_INVALID_ARG, "the job was already finished");
    spamm_mat Cm = job->out.C.get();
    Events ev;
    CK(cudaEventRecord(ev.e[0], ctx->stream));
    if (job->plan->prec != SPAMM_PREC_FP64)
      tc_finish(ctx, job->plan->prec, P<double>(Cm->pool), Cm->nleaves, job->plan->bs, P<double>(Cm->lv[Cm->L].sq));
    fill_iota_i64(ctx, P<int64_t>(Cm->slot), Cm->nleaves);
    std::vector<NormBatchLevel> nlv;
    BufP ntab = norm_batch_tables(ctx, {Cm}, &nlv);
    propagate_norms_batch(ctx, nlv);
    CK(cudaEventRecord(ev.e[1], ctx->stream));
    sync_and_check(ctx);
    if (stats) {
      fill_stats(*job->plan, stats);
      stats->ms_gemm = job->ms_gemm;
      stats->ms_cnorm = elapsed_ms(ev.e[0], ev.e[1]);
      stats->n_launches = job->launches;
    }
    job->out.part.reset();
    *C = registered(job->out.C.release());
  });
}

spamm_status spamm_job_release(spamm_job job) {
  if (!job) return SPAMM_E_INVALID_ARG;
  spamm_ctx ctx = job->ctx;
  cudaSetDevice(ctx->device);
  delete job;
  ctx->live_handles--;
  return SPAMM_OK;
}

spamm_status spamm_set_gemm_sms(spamm_ctx ctx, int nsms) {
  if (!ctx) return SPAMM_E_INVALID_ARG;
  return guarded(ctx, [&] {
    need(nsms >= 0 && nsms <= ctx->num_sms, "nsms must be in [0, number of SMs]");
    ctx->gemm_sm_limit = nsms;
  });
}

spamm_status spamm_set_claim_order(spamm_ctx ctx, int order) {
  if (!ctx) return SPAMM_E_INVALID_ARG;
  if (order != SPAMM_ORDER_AUTO && order != SPAMM_ORDER_MORTON && order != SPAMM_ORDER_LONGEST_FIRST)
    return SPAMM_E_INVALID_ARG;
  ctx->claim_order = order;
  return SPAMM_OK;
}

spamm_status spamm_set_exec_graph(spamm_ctx ctx, int enable) {
  if (!ctx) return SPAMM_E_INVALID_ARG;
  ctx->exec_graph = enable != 0;
  return SPAMM_OK;
}

spamm_status spamm_exec_graph_info(spamm_ctx ctx, int64_t* instantiations, int64_t* updates) {
  if (!ctx) return SPAMM_E_INVALID_ARG;
  if (instantiations) *instantiations = ctx->graph_instantiations;
  if (updates) *updates = ctx->graph_updates;
  return SPAMM_OK;
}

spamm_status spamm_execute(spamm_ctx ctx, int64_t nplans, const spamm_plan* plans, spamm_mat* C, spamm_stats* stats) {
  if (!ctx || nplans <= 0 || !plans || !C) return SPAMM_E_INVALID_ARG;
  for (int64_t r = 0; r < nplans; ++r) C[r] = nullptr;
  return guarded(ctx, [&] {
    std::vector<spamm_plan> v(plans, plans + nplans);
    for (spamm_plan p : v) need(p != nullptr, "NULL plan");
    double ms_gemm = 0, ms_cnorm = 0;
    int64_t launches = 0;
    std::vector<spamm_mat> out = execute_plans(ctx, v, &ms_gemm, &ms_cnorm, &launches);
    for (int64_t r = 0; r < nplans; ++r) {
      C[r] = registered(out[r]);
      if (stats) {
        fill_stats(*v[r], &stats[r]);
        stats[r].ms_gemm = ms_gemm;
        stats[r].ms_cnorm = ms_cnorm;
        stats[r].n_launches = launches;
      }
    }
  });
}

spamm_status spamm_multiply(spamm_ctx ctx, spamm_mat A, spamm_mat B, double tau, spamm_mode mode, spamm_prec prec,
                            spamm_mat* C, spamm_stats* stats) {
  if (!ctx || !A || !B || !C) return SPAMM_E_INVALID_ARG;
  *C = nullptr;
  return guarded(ctx, [&] {
    std::unique_ptr<spamm_plan_s> p(make_plan(ctx, A, B, tau, mode, prec));
    ctx->live_handles--;  // the plan is internal to this call
    double ms_gemm = 0, ms_cnorm = 0;
    int64_t launches = 0;
    std::vector<spamm_mat> out = execute_plans(ctx, {p.get()}, &ms_gemm, &ms_cnorm, &launches);
    if (stats) {
      fill_stats(*p, stats);
      stats->ms_gemm = ms_gemm;
      stats->ms_cnorm = ms_cnorm;
      stats->n_launches = p->launches + launches;
    }
    *C = registered(out[0]);
  });
}

spamm_status spamm_kept_tasks(spamm_ctx ctx, spamm_mat A, spamm_mat B, double tau, spamm_mode mode, int32_t* ikj_out,
                              int64_t cap, int64_t* count) {
  if (!ctx || !A || !B || !count) return SPAMM_E_INVALID_ARG;
  return guarded(ctx, [&] {
    check_pair(A, B, tau, mode);
    spamm_mat At = nullptr, Bt = nullptr;
    run_truncation(A, B, tau, mode, &At, &Bt);
    std::unique_ptr<spamm_mat_s> ownA(At != A ? At : nullptr), ownB((Bt != B && Bt != At) ? Bt : nullptr);
    TaskList T = build_tasks(At, Bt, tau, mode != SPAMM_MODE_TRUNCATE);
    *count = T.ntasks;
    if (T.ntasks > cap) fail(SPAMM_E_CAPACITY, "ikj_out holds fewer triples than the kept set");
    if (T.ntasks == 0) return;
    need(ikj_out != nullptr, "ikj_out must be non-NULL");
    BufP d = alloc_n<int32_t>(ctx, 3 * T.ntasks);
    tasks_to_ikj(At, T, P<int32_t>(d));
    CK(cudaMemcpyAsync(ikj_out, P<int32_t>(d), 3 * T.ntasks * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    sync_and_check(ctx);
  });
}

spamm_status spamm_add(spamm_ctx ctx, double alpha, spamm_mat X, double beta, spamm_mat Y, spamm_mat* out) {
  if (!ctx || !X || !Y || !out) return SPAMM_E_INVALID_ARG;
  *out = nullptr;
  return guarded(ctx, [&] {
    need(std::isfinite(alpha) && std::isfinite(beta), "alpha and beta must be finite");
    if (X->n != Y->n || X->bs != Y->bs) fail(SPAMM_E_SHAPE, "X and Y differ in n or bs");
    if (X->ctx->device != ctx->device || Y->ctx->device != ctx->device)
      fail(SPAMM_E_INVALID_ARG, "operands live on another device");
    *out = registered(add_scaled(alpha, X, beta, Y, ctx));
  });
}

spamm_status spamm_identity(spamm_ctx ctx, int64_t n, int bs, spamm_mat* out) {
  if (!ctx || !out) return SPAMM_E_INVALID_ARG;
  *out = nullptr;
  return guarded(ctx, [&] {
    check_bs(bs);
    check_n(n, bs);
    *out = registered(identity_mat(ctx, n, bs));
  });
}

spamm_status spamm_trace(spamm_ctx ctx, spamm_mat X, double* out) {
  if (!ctx || !X || !out) return SPAMM_E_INVALID_ARG;
  return guarded(ctx, [&] { *out = trace_of(X); });
}

spamm_status spamm_frob_norm(spamm_ctx ctx, spamm_mat m, double* out) {
  if (!ctx || !m || !out) return SPAMM_E_INVALID_ARG;
  return guarded(ctx, [&] {
    if (m->nleaves == 0) {
      *out = 0.0;
      return;
    }
    *out = std::sqrt(read_scalar<double>(ctx, P<double>(m->lv[0].sq)));
  });
}

spamm_status spamm_error(spamm_ctx ctx, spamm_mat X, spamm_mat Y, double* out) {
  if (!ctx || !X || !Y || !out) return SPAMM_E_INVALID_ARG;
  return guarded(ctx, [&] {
    if (X->n != Y->n || X->bs != Y->bs) fail(SPAMM_E_SHAPE, "X and Y differ in n or bs");
    *out = error_fro(X, Y);
  });
}

spamm_status spamm_set_symmetric(spamm_mat m, int symmetric) {
  if (!m) return SPAMM_E_INVALID_ARG;
  m->symmetric = symmetric != 0;
  return SPAMM_OK;
}

spamm_status spamm_mat_info(spamm_mat m, int64_t* n, int32_t* bs, int32_t* levels, int64_t* nleaves) {
  if (!m) return SPAMM_E_INVALID_ARG;
  if (n) *n = m->n;
  if (bs) *bs = m->bs;
  if (levels) *levels = m->L;
  if (nleaves) *nleaves = m->nleaves;
  return SPAMM_OK;
}

spamm_status spamm_to_dense(spamm_ctx ctx, spamm_mat m, double* out, int64_t ld, int on_device) {
  if (!ctx || !m || !out) return SPAMM_E_INVALID_ARG;
  return guarded(ctx, [&] {
    need(ld >= m->n, "ld must be >= n");
    export_dense(m, out, ld, on_device);
  });
}

spamm_status spamm_to_blocks(spamm_ctx ctx, spamm_mat m, int32_t* bi, int32_t* bj, double* payload, double* sq,
                             int64_t cap, int on_device) {
  if (!ctx || !m) return SPAMM_E_INVALID_ARG;
  return guarded(ctx, [&] {
    if (cap < m->nleaves) fail(SPAMM_E_CAPACITY, "cap is smaller than the number of leaves");
    export_blocks(m, bi, bj, payload, sq, on_device);
  });
}

spamm_status spamm_gather_leaves(spamm_ctx ctx, spamm_mat m, int64_t nq, const int32_t* bi, const int32_t* bj,
                                 double* payload_out, int32_t* found, int on_device) {
  if (!ctx || !m) return SPAMM_E_INVALID_ARG;
  return guarded(ctx, [&] {
    need(nq >= 0, "nq must be >= 0");
    need(nq == 0 || (bi && bj && payload_out), "bi, bj and payload_out must be non-NULL");
    gather_leaves(m, nq, bi, bj, payload_out, found, on_device);
  });
}

spamm_status spamm_level_norms(spamm_ctx ctx, spamm_mat m, int level, uint32_t* codes, double* sq, int64_t cap,
                               int64_t* count) {
  if (!ctx || !m || !count) return SPAMM_E_INVALID_ARG;
  return guarded(ctx, [&] {
    need(level >= 0 && level <= m->L, "level must be in [0, L]");
    const Level& lv = m->lv[level];
    *count = lv.count;
    if (lv.count > cap) fail(SPAMM_E_CAPACITY, "cap is smaller than the node count");
    if (lv.count == 0) return;
    if (codes)
      CK(cudaMemcpyAsync(codes, P<uint32_t>(lv.code), lv.count * sizeof(uint32_t), cudaMemcpyDeviceToHost,
                         ctx->stream));
    if (sq) CK(cudaMemcpyAsync(sq, P<double>(lv.sq), lv.count * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    sync_and_check(ctx);
  });
}

}  // extern "C"
