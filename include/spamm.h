/*
 * spamm.h -- C ABI of libspamm: approximate multiplication C ~ AB of nearly
 * sparse matrices with decay, stored as quadtrees of dense leaf blocks, on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: Artemov, "Approximate multiplication of nearly sparse matrices with
 * decay in a fully recursive distributed task-based parallel framework"
 * (arXiv:1906.08148).  The three methods of Section 5 are provided:
 *   Truncmul  C~ = A~ B~            (Theorem 1: inputs truncated with tau)
 *   SpAMM     C- = SpAMM(A, B, tau) (Algorithm 1 / Theorem 2: a sub-product
 *                                    A_ik B_kj is skipped iff
 *                                    ||A_ik||_F ||B_kj||_F < tau)
 *   Hybrid    C^ = SpAMM(A~, B~, tau), the same tau for both (Theorem 3).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Matrices are n x n, FP64.  A matrix handle (spamm_mat) is a quadtree whose
 *   leaves are dense bs x bs row-major FP64 blocks, bs in {32, 64, 128, 256}; a leaf
 *   is stored iff it has at least one non-zero element and a null sub-matrix is
 *   never stored (Sections 4.2 and 4.4).  Every node carries its squared
 *   Frobenius norm, parents being the sums of their four children (Section 2).
 *   n need not be a multiple of bs: the last leaves are zero-padded and the
 *   padding stays zero.  Leaf grid side 2^L >= ceil(n / bs), L <= 16.
 * - Handles are immutable once returned and are released with
 *   spamm_release().  The library owns all device memory behind a handle; it
 *   allocates through the context's allocator (spamm_set_allocator) or, by
 *   default, stream-ordered cudaMallocAsync on the context stream.  Caller
 *   buffers are only borrowed for the duration of a call.
 * - `on_device` = 1 means a pointer argument is a device pointer on the
 *   context's device; 0 means host memory (pageable or pinned).
 * - All device work runs on the context's CUDA stream.  Calls that return a
 *   host value (norms, errors, counts, statistics, host copies) synchronise
 *   that stream before returning.
 * - Every call returns a spamm_status; nothing aborts or traps.  The message
 *   of the last failure on a context is available from spamm_last_error().
 *   A device-side wait that runs past its bound makes the call return
 *   SPAMM_E_TIMEOUT.
 * - A context is used by one host thread at a time.
 */
#ifndef SPAMM_H
#define SPAMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define SPAMM_API __attribute__((visibility("default")))
#else
#define SPAMM_API
#endif

#define SPAMM_ABI_VERSION 1
#define SPAMM_MAX_LEVELS 17

typedef struct spamm_ctx_s* spamm_ctx;
typedef struct spamm_mat_s* spamm_mat;

typedef enum {
  SPAMM_OK = 0,
  SPAMM_E_INVALID_ARG = 1, /* bad size, tau < 0 or NaN, bs not 32/64/128/256, NULL pointer, index out of range */
  SPAMM_E_SHAPE = 2,       /* operands disagree in n or bs */
  SPAMM_E_NONFINITE = 3,   /* an input element is Inf or NaN */
  SPAMM_E_OOM = 4,         /* device allocation failed */
  SPAMM_E_CUDA = 5,        /* a CUDA call failed */
  SPAMM_E_TIMEOUT = 6,     /* a bounded device-side wait ran out */
  SPAMM_E_BUSY = 7,        /* resource in use */
  SPAMM_E_CAPACITY = 8,    /* caller buffer too small; required size returned where the call says so */
  SPAMM_E_UNSUPPORTED = 9  /* valid request the library does not implement (named in the message) */
} spamm_status;

/* The three methods of Section 5: Truncmul, SpAMM, Hybrid. */
typedef enum { SPAMM_MODE_TRUNCATE = 0, SPAMM_MODE_SPAMM = 1, SPAMM_MODE_COMBINED = 2 } spamm_mode;

/* Input truncation rule.  BLOCK_FROB: a leaf is dropped iff its Frobenius
 * norm is < tau.  ELEMENT: a_ij -> 0 iff |a_ij| < tau (Theorem 1, equation
 * "truncated matrices"), then leaves left without a non-zero are dropped.
 * ERROR_CONTROL: tau is an error budget: the leaves with the smallest squared
 * norms (ties in Morton order) are dropped as long as the sum of their squared
 * norms, added in that order, stays <= tau^2, so ||A - A~||_F <= tau (the
 * error-controlled truncation Section 1 cites, applied to whole leaves). */
typedef enum {
  SPAMM_TRUNC_BLOCK_FROB = 0,
  SPAMM_TRUNC_ELEMENT = 1,
  SPAMM_TRUNC_ERROR_CONTROL = 2
} spamm_trunc_rule;

/* Arithmetic of the leaf products (the paper computes in FP64; the other
 * forms run the leaf products on the tensor cores).  Norms, the tau test and
 * errors are always FP64.
 * FP64: plain double precision.
 * BF16_SPLIT / BF16_SPLIT4: an error-free split taken straight from the FP64
 * elements.  Each leaf is scaled by a power of two (largest |a| in [1, 2));
 * each row of an A leaf and each column of a B leaf is written as 3 (SPLIT)
 * or 4 (SPLIT4) bfloat16 slices on a grid set by the line's largest element:
 * x = sum_s d_s 2^(e - 8 - 9 s) + r, |d_s| <= 256, |r| <= 2^(e - 9 S) with
 * |x| < 2^e on the line.  The slice products with index sum < S are formed
 * on the tensor cores; for each output row and column the products of one
 * index sum are integers on a common grid, so a 64-term sum of them is exact
 * in the FP32 accumulator (sums 0, and 1 for SPLIT4, get accumulators of
 * their own; the smaller rest shares one).  Each leaf product is then added
 * into a two-float (hi + lo) FP32 accumulator with an error-free TwoSum, and
 * the output leaf is hi + lo in FP64.  Relative error about 1e-8 (SPLIT) and
 * 1e-10 (SPLIT4) of |A||B|, from the dropped digits.
 * FP16_SCALED: per-leaf power-of-two scaling, two float16 terms of the
 * element rounded to FP32, FP32 accumulation: about 2e-7 relative, fastest.
 * Range of the tensor-core forms: operand elements below 2^-1022 count as 0,
 * digits whose unit falls below 2^-126 after the leaf scale are dropped, the
 * per-leaf scale exponents are clamped to [-120, 120], so elements must be
 * below about 2^100 in magnitude, and the output leaves are summed in FP32,
 * so output elements must lie within the FP32 range (about 1e-38 .. 3e38,
 * relative precision lost towards the bottom).  A power-of-two rescaling of
 * the inputs within that range rescales the result exactly. */
typedef enum {
  SPAMM_PREC_FP64 = 0,
  SPAMM_PREC_BF16_SPLIT = 1,
  SPAMM_PREC_FP16_SCALED = 2,
  SPAMM_PREC_BF16_SPLIT4 = 3
} spamm_prec;

/* Synthetic matrix with exponential decay (Definition 1 with c, alpha):
 *   a_ij = c u_ij exp(-alpha d(i,j)),  u_ij ~ U[-1,1) symmetric, seeded;
 *   |a_ij| < cutoff -> 0.   kind 0: d = |i - j| (the model problem of
 * Section 5.3); kind 1: d = Euclidean distance between the points of a 3-D
 * unit lattice in Morton order (stand-in for the systems of Section 5.4).
 * law 1: algebraic decay a_ij = c u_ij / (1 + d(i,j))^p, p = alpha rounded
 * down to an integer >= 1 (the other decay class Section 1 mentions). */
typedef struct {
  int64_t n;
  int32_t kind;
  int32_t law; /* 0: exponential, 1: algebraic */
  double alpha;
  double c;
  double cutoff;
  uint64_t seed;
} spamm_gen_params;

/* Statistics of one multiplication.  Level t counts child pairs formed when
 * descending from level t-1 to level t (t = 1..L). */
typedef struct {
  int64_t n_candidates[SPAMM_MAX_LEVELS]; /* pairs with both sub-matrices non-null */
  int64_t n_kept_level[SPAMM_MAX_LEVELS]; /* of those, pairs that passed the norm test */
  int64_t n_kept;        /* leaf products performed (the paper's N_gemm) */
  int64_t n_borderline;  /* leaf candidates with |norm product - tau| <= 1e-12 tau */
  int64_t n_c_leaves;    /* leaves of C */
  int64_t n_a_leaves;    /* leaves of A after input truncation */
  int64_t n_b_leaves;
  int32_t levels;        /* L */
  int32_t bs;
  double kept_flops;     /* 2 bs^3 n_kept (Section 5.3, flop count) */
  double ms_truncate;    /* device time of input truncation */
  double ms_tasks;       /* device time of the task-list build */
  double ms_gemm;        /* device time of the leaf products (incl. C leaf norms) */
  double ms_cnorm;       /* device time of the C quadtree norms */
  int64_t n_launches;    /* CUDA kernels this call launched */
  double ms_prep;        /* device time of the tensor-form operand terms and quad step list (0 for FP64) */
  int64_t n_steps;       /* leaf-GEMM steps: FP64 = n_kept; tensor forms = k steps of output quads */
  double executed_flops; /* flops the leaf-GEMM kernel executes: FP64 = kept_flops; tensor forms =
                            n_steps x every term product over a 128 x 128 x 64 tile */
  int64_t terms_shared;  /* tensor forms: 1 if A and B were one symmetric matrix and one set of
                            operand terms served both roles (see spamm_set_symmetric), else 0 */
} spamm_stats;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` using stream `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  *out receives the
 * handle.  Errors: SPAMM_E_INVALID_ARG (out NULL, bad device), SPAMM_E_CUDA. */
SPAMM_API spamm_status spamm_create(int device, void* cuda_stream, spamm_ctx* out);

/* Destroy a context.  Handles created on it must be released first. */
SPAMM_API spamm_status spamm_destroy(spamm_ctx ctx);

/* Replace the stream all later work of `ctx` runs on. */
SPAMM_API spamm_status spamm_set_stream(spamm_ctx ctx, void* cuda_stream);

/* Install a device allocator: alloc(bytes, user) returns device memory usable
 * on the context stream in stream order (NULL on failure -> SPAMM_E_OOM);
 * free(ptr, user) returns it.  Pass alloc = free = NULL to go back to
 * cudaMallocAsync.  Must be called while no handle of `ctx` is alive. */
SPAMM_API spamm_status spamm_set_allocator(spamm_ctx ctx, void* (*alloc)(size_t bytes, void* user),
                                 void (*free_fn)(void* ptr, void* user), void* user);

/* Block until all work of `ctx` is done; reports a pending device error. */
SPAMM_API spamm_status spamm_sync(spamm_ctx ctx);

/* Wait for the context stream, then return to the driver the device memory
 * that the device's stream-ordered pool keeps cached from freed blocks
 * (cudaMemPoolTrimTo(pool, 0); the library sets that pool to keep freed
 * memory).  Live handles are untouched.  With an allocator installed by
 * spamm_set_allocator the pool is not the library's and nothing is trimmed.
 * Errors: INVALID_ARG (ctx NULL), CUDA. */
SPAMM_API spamm_status spamm_trim(spamm_ctx ctx);

/* Message of the last failing call on `ctx` ("" if none).  Owned by ctx. */
SPAMM_API const char* spamm_last_error(spamm_ctx ctx);

/* -------------------------------------------------------------- building */

/* Build a quadtree matrix from a dense row-major n x n array `a` with leading
 * dimension `lda` >= n.  tau > 0 truncates the input with `rule` while
 * building (tau = 0: only the all-zero leaves are dropped).  Leaf squared
 * norms and parents are computed here (Section 2).
 * Errors: INVALID_ARG (n <= 0, lda < n, bs, tau), NONFINITE, OOM, CUDA. */
SPAMM_API spamm_status spamm_from_dense(spamm_ctx ctx, int64_t n, const double* a, int64_t lda, int on_device, int bs,
                              double tau, spamm_trunc_rule rule, spamm_mat* out);

/* Build from `nblocks` dense leaves: block (bi[q], bj[q]) has its bs*bs
 * row-major payload at payload + q*bs*bs.  Blocks may come in any order;
 * all-zero blocks are dropped; a repeated (bi, bj) is INVALID_ARG, as is a
 * coordinate outside [0, ceil(n/bs)).  Payload entries past n must be 0. */
SPAMM_API spamm_status spamm_from_blocks(spamm_ctx ctx, int64_t n, int bs, int64_t nblocks, const int32_t* bi,
                               const int32_t* bj, const double* payload, int on_device, double tau,
                               spamm_trunc_rule rule, spamm_mat* out);

/* Build from COO triplets (row[q], col[q], val[q]), q < nnz, 0-based.
 * Repeated coordinates are summed in input order.  Explicit zeros are
 * allowed (a leaf holding only zeros is dropped).
 * Errors: INVALID_ARG (index outside [0,n)), NONFINITE, OOM, CUDA. */
SPAMM_API spamm_status spamm_from_coo(spamm_ctx ctx, int64_t n, int64_t nnz, const int64_t* row, const int64_t* col,
                            const double* val, int on_device, int bs, double tau, spamm_trunc_rule rule,
                            spamm_mat* out);

/* Generate a synthetic decay matrix (spamm_gen_params) directly into leaves on
 * the device.  With tau > 0 and the BLOCK_FROB rule, leaves below tau are
 * never stored (identical to truncating the full matrix, the rule being
 * per leaf), so matrices whose untruncated form does not fit can be built. */
SPAMM_API spamm_status spamm_generate(spamm_ctx ctx, const spamm_gen_params* params, int bs, double tau,
                            spamm_trunc_rule rule, spamm_mat* out);

/* Truncated copy of `in` with threshold tau (the vector-space truncation the
 * paper contrasts with SpAMM's product-space truncation, Sections 2 and 3).
 * BLOCK_FROB shares the leaf payload with `in` (no copy).  Also the output
 * truncation of a product (pass a product as `in`). */
SPAMM_API spamm_status spamm_truncate(spamm_ctx ctx, spamm_mat in, double tau, spamm_trunc_rule rule, spamm_mat* out);

/* Release a handle (payload memory shared with views is freed with the last). */
SPAMM_API spamm_status spamm_release(spamm_mat m);

/* ---------------------------------------------------------- multiplication */

/* C ~ A B with method `mode` and threshold tau >= 0 (Algorithm 1; Section 5):
 * TRUNCATE and COMBINED first truncate A and B with the block rule and the
 * same tau.  The quadtrees are descended level by level; a child pair
 * (A_ik, B_kj) is entered iff both are non-null and, except in TRUNCATE mode,
 * fl(sqrt(s_A)) * fl(sqrt(s_B)) >= tau (s = stored squared norm); the norm
 * test is applied down to leaf pairs (Section 4.4).  C's structure is built
 * in advance from the kept set and all leaf products are then run batched
 * (Section 4.4); C_ij = sum over kept k, ascending, of A_ik B_kj.  C carries
 * its leaf and parent squared norms.  `stats` may be NULL.
 * Errors: SHAPE (n or bs differ), INVALID_ARG (tau, mode, prec),
 * UNSUPPORTED (precision form not available for this bs), OOM, CUDA, TIMEOUT. */
SPAMM_API spamm_status spamm_multiply(spamm_ctx ctx, spamm_mat A, spamm_mat B, double tau, spamm_mode mode,
                            spamm_prec prec, spamm_mat* C, spamm_stats* stats);

/* ------------------------------------------------- two-phase, batched form */

typedef struct spamm_plan_s* spamm_plan;

/* First phase of spamm_multiply: input truncation (TRUNCATE, COMBINED), the
 * kept task list from the quadtree descent (the output structure built in
 * advance, Section 4.4) and, for the tensor-core forms, the operand terms.
 * The plan holds its own references to the storage it needs, so A and B may be
 * released afterwards; it is immutable and may be executed many times.
 * Errors as spamm_multiply. */
SPAMM_API spamm_status spamm_plan_create(spamm_ctx ctx, spamm_mat A, spamm_mat B, double tau, spamm_mode mode,
                                         spamm_prec prec, spamm_plan* out);

/* Sizes of a plan, for admission by memory footprint: kept leaf products,
 * output leaves, device bytes the plan holds, device bytes its execution will
 * allocate for the output.  Any output pointer may be NULL. */
SPAMM_API spamm_status spamm_plan_info(spamm_plan p, int64_t* n_kept, int64_t* n_c_leaves, int64_t* plan_bytes,
                                       int64_t* exec_bytes);

/* Second phase, batched: the leaf products of all `nplans` plans (one
 * precision form and one leaf size, made on this context) run in ONE
 * persistent kernel launch (the batched leaf multiplication of Section 4.4,
 * across requests); then every output's leaf norms and quadtree.  C[r]
 * receives the product of plans[r]; each output is bit-identical to executing
 * its plan alone.  Plans may come from other contexts on the same device
 * (e.g. planned on another stream): spamm_plan_create returns only once its
 * work is complete, and a plan must not be released while an execute that
 * uses it is running.  Outputs belong to `ctx`.  `stats`, if not NULL, holds
 * nplans entries (ms_gemm is the shared launch).  Errors: INVALID_ARG (mixed
 * forms/sizes/devices), OOM, CUDA, TIMEOUT. */
SPAMM_API spamm_status spamm_execute(spamm_ctx ctx, int64_t nplans, const spamm_plan* plans, spamm_mat* C,
                                     spamm_stats* stats);

SPAMM_API spamm_status spamm_plan_release(spamm_plan p);

/* ---------------------------------------- sliced execution (continuous batching) */

typedef struct spamm_job_s* spamm_job;

/* The execute phase of a plan, cut into slices that later requests can join:
 * spamm_job_begin allocates the plan's output (spamm_plan_info's exec_bytes)
 * and returns a job whose work units -- output leaves (their 64 x 64
 * sub-tiles for bs 128 and 256) in the FP64 form, quads of output leaves in
 * the tensor forms -- run in later spamm_run calls, in the plan's claiming
 * order.  Each output leaf is computed whole by one unit, with its products
 * in ascending k, so the result does not depend on how the units were cut
 * into launches: it is bit-identical to spamm_execute of the same plan.  The
 * plan must outlive the job.  Errors: INVALID_ARG, OOM, CUDA. */
SPAMM_API spamm_status spamm_job_begin(spamm_ctx ctx, spamm_plan plan, spamm_job* out);

/* Units of the job, how many have run, and the same as work: kept leaf
 * products (FP64) or quad steps (tensor forms).  Any pointer may be NULL. */
SPAMM_API spamm_status spamm_job_info(spamm_job job, int64_t* units, int64_t* units_done, double* work,
                                      double* work_done);

/* ONE persistent leaf-product launch over the next units of `njobs` jobs (one
 * precision form and leaf size, on this device): job r contributes the
 * following units whose work adds up to at most work_budget[r] (at least one
 * unit, one whole leaf in the FP64 form, at most what is left; a finished job
 * contributes nothing).  Returns once the launch has completed; units_run[r]
 * (may be NULL) receives the units job r ran, *ms_gemm (may be NULL) the
 * launch's device time.  A server calls this in a loop, adding new jobs
 * between calls, so requests that arrive while others run share the next
 * launches with them.  Errors: INVALID_ARG (mixed forms, sizes or devices),
 * CUDA, TIMEOUT. */
SPAMM_API spamm_status spamm_run(spamm_ctx ctx, int64_t njobs, const spamm_job* jobs, const double* work_budget,
                                 int64_t* units_run, double* ms_gemm);

/* Once every unit of the job has run: the output's leaf slots and quadtree
 * norms (kernel (d)); *C receives the product.  `stats` (may be NULL) is
 * filled as spamm_execute fills it, ms_gemm summing the launches the job took
 * part in.  Errors: BUSY (units left), INVALID_ARG (already finished), CUDA. */
SPAMM_API spamm_status spamm_job_finish(spamm_ctx ctx, spamm_job job, spamm_mat* C, spamm_stats* stats);

/* Releases a job; an unfinished job's output is freed with it. */
SPAMM_API spamm_status spamm_job_release(spamm_job job);

/* Run the persistent leaf-product launches of `ctx` on at most `nsms` SMs
 * (0 = all), leaving the others to kernels on other streams, e.g. planning
 * the next requests while a batch executes. */
SPAMM_API spamm_status spamm_set_gemm_sms(spamm_ctx ctx, int nsms);

/* Order in which the persistent leaf-product kernels claim their work units
 * (an output leaf, a 64 x 64 sub-tile of one, or a quad of four output leaves),
 * for plans created afterwards on `ctx` -- the tile schedule.  Section 4.4's
 * batched multiply fixes the output structure before any leaf product runs,
 * so the order is free:
 *   SPAMM_ORDER_MORTON: output Morton order; the units in flight on all SMs
 *     share A rows and B columns in L2;
 *   SPAMM_ORDER_LONGEST_FIRST: units with the most kept products (steps)
 *     first, ties in Morton order; shortens the tail of launches that hold
 *     few units per SM;
 *   SPAMM_ORDER_AUTO (default): longest first for FP64 leaves of 128 and 256,
 *     Morton otherwise.
 * Results are identical in every order (each output leaf sums its products
 * in k order on one CTA). */
typedef enum {
  SPAMM_ORDER_AUTO = 0,
  SPAMM_ORDER_MORTON = 1,
  SPAMM_ORDER_LONGEST_FIRST = 2
} spamm_claim_order;
SPAMM_API spamm_status spamm_set_claim_order(spamm_ctx ctx, int order);

/* enable != 0: spamm_execute / spamm_multiply run their execute phase (the
 * persistent leaf-product launch of every plan in the batch, then the output
 * quadtrees' parent norms, one launch per level for the whole batch) as one
 * captured CUDA graph.  Output buffers are allocated and the batch tables
 * uploaded before the capture, so the captured sequence holds kernels and
 * timing events only.  Results are identical either way.  Default 0. */
SPAMM_API spamm_status spamm_set_exec_graph(spamm_ctx ctx, int enable);

/* Graph mode keeps the last instantiated graph in the context and, for the
 * next batch, updates it in place (cudaGraphExecUpdate: new kernel
 * parameters and events) when the captured sequence has the same topology,
 * instantiating a new one only when it does not.  Counts of both since the
 * context was created; either pointer may be NULL. */
SPAMM_API spamm_status spamm_exec_graph_info(spamm_ctx ctx, int64_t* instantiations, int64_t* updates);

/* Parity hook: the kept leaf triples of spamm_multiply(A, B, tau, mode) as
 * (i, k, j) int32 triples (3 per triple, host memory), grouped by C leaf in
 * Morton order of (i, j), k ascending within a group.  *count receives the
 * number of triples; if it exceeds `cap`, nothing is written and
 * SPAMM_E_CAPACITY is returned. */
SPAMM_API spamm_status spamm_kept_tasks(spamm_ctx ctx, spamm_mat A, spamm_mat B, double tau, spamm_mode mode,
                              int32_t* ikj_out, int64_t cap, int64_t* count);

/* ------------------------------------------- operations of a purification chain */

/* *out = alpha X + beta Y (same n and bs), element by element as
 * fl(fl(alpha x) + fl(beta y)) with an absent leaf taken as zero; the leaf set
 * is the union of X's and Y's, without leaves that come out exactly zero
 * (null = zero).  Section 4.4 lists addition and rescaling among the
 * operations of the leaf library; with the identity it gives the shifts and
 * the 2X - X^2 step of density-matrix purification (Section 1).  Errors:
 * INVALID_ARG, SHAPE, NONFINITE (an element overflowed), OOM, CUDA. */
SPAMM_API spamm_status spamm_add(spamm_ctx ctx, double alpha, spamm_mat X, double beta, spamm_mat Y, spamm_mat* out);

/* The n x n identity as a quadtree of bs x bs leaves (diagonal leaves only). */
SPAMM_API spamm_status spamm_identity(spamm_ctx ctx, int64_t n, int bs, spamm_mat* out);

/* Trace of X (the sum of the diagonals of its diagonal leaves, each leaf in
 * row order, the leaf sums by a fixed reduction tree). */
SPAMM_API spamm_status spamm_trace(spamm_ctx ctx, spamm_mat X, double* out);

/* Diagnostic (no counterpart in the paper): launch one kernel whose bounded
 * device-side wait, wait_ns nanoseconds long (1 .. 2e9), runs out because
 * nothing completes the awaited mbarrier phase.  Returns SPAMM_E_TIMEOUT, the
 * status every library kernel reports when one of its waits runs out; the
 * context's error word is cleared and the context stays usable.  Errors:
 * INVALID_ARG, CUDA. */
SPAMM_API spamm_status spamm_check_timeout_path(spamm_ctx ctx, int64_t wait_ns);

/* ------------------------------------------------------------ evaluation */

/* ||M||_F = sqrt of the root's squared norm (Section 2); 0 for an empty M. */
SPAMM_API spamm_status spamm_frob_norm(spamm_ctx ctx, spamm_mat m, double* out);

/* ||X - Y||_F over the union of the two leaf sets (a leaf missing on one side
 * counts as zero), accumulated in FP64 (the error measure of Section 5). */
SPAMM_API spamm_status spamm_error(spamm_ctx ctx, spamm_mat X, spamm_mat Y, double* out);

/* Shape of a handle: any output pointer may be NULL. */
SPAMM_API spamm_status spamm_mat_info(spamm_mat m, int64_t* n, int32_t* bs, int32_t* levels, int64_t* nleaves);

/* Mark m as symmetric (symmetric != 0) or not.  spamm_generate marks its
 * matrices (the decay generators are symmetric in (i, j)); truncation keeps
 * the mark.  When one marked handle is both operands of a tensor-core
 * multiply (X times X, the squarings of a purification chain), the operand
 * terms of X are built once and serve both roles: B's leaf (k, j) uses the
 * terms of leaf (j, k), which are exactly its own B terms for a symmetric X,
 * halving the memory of the terms; if some leaf's transpose is absent from
 * the leaf set (possible after truncation when two norms straddle tau by an
 * ulp), the terms are built separately as for any A and B.  The result is
 * then X X^T, so the mark must only be set on matrices equal to their
 * transpose.  Errors: SPAMM_E_INVALID_ARG (m NULL). */
SPAMM_API spamm_status spamm_set_symmetric(spamm_mat m, int symmetric);

/* Dense copy of M into `out` (row-major, leading dimension ld >= n). */
SPAMM_API spamm_status spamm_to_dense(spamm_ctx ctx, spamm_mat m, double* out, int64_t ld, int on_device);

/* Export the leaves in Morton order of (bi, bj): coordinates, payloads
 * (bs*bs row-major each) and squared norms.  Any of bi/bj/payload/sq may be
 * NULL.  `cap` is the capacity in leaves; fewer than nleaves -> CAPACITY. */
SPAMM_API spamm_status spamm_to_blocks(spamm_ctx ctx, spamm_mat m, int32_t* bi, int32_t* bj, double* payload, double* sq,
                             int64_t cap, int on_device);

/* Copy the leaves at block coordinates (bi[q], bj[q]), q < nq, into
 * payload_out + q*bs*bs (row-major); found[q] = 1 if that leaf is stored, else
 * 0 and its payload is zero-filled.  bi, bj, payload_out and found are all on
 * the host (on_device = 0) or all on the device (1); found may be NULL. */
SPAMM_API spamm_status spamm_gather_leaves(spamm_ctx ctx, spamm_mat m, int64_t nq, const int32_t* bi,
                                           const int32_t* bj, double* payload_out, int32_t* found, int on_device);

/* ------------------------------------------------- allocation-free variant */

/* Largest nleaves spamm_leaf_sqnorms_noalloc accepts. */
#define SPAMM_NOALLOC_MAX_LEAVES (1 << 24)

/* The paper has no counterpart of this call; it serves callers that must not
 * allocate device memory: services that reserve all device memory up front and
 * may not allocate on their request path (an allocation can fail there, and
 * cudaMalloc/cudaFree can synchronise the device), and plug-ins that run inside
 * a host framework which owns the device memory.  No context is needed.
 *
 * Squared Frobenius norm of each of `nleaves` dense bs x bs row-major FP64
 * leaves stored back to back at device address `payload` (leaf q at
 * payload + q*bs*bs) into sq_out[q], and their sum into *total_out.  payload,
 * sq_out and total_out are caller-allocated device memory of the current CUDA
 * device; the work is enqueued on `cuda_stream` (NULL = legacy default stream)
 * and the call returns without waiting for it.  Per-leaf results equal, bit for
 * bit, the leaf norms the library stores for the same payload.
 *
 * It calls no cudaMalloc, cudaFree or allocating library routine.  Its scratch
 * (one FP64 partial sum per 64 leaves, 2 MB) is a fixed device array in this
 * library, which every GPU that loads the library holds until the process
 * exits.  The first call on a device looks up that array's device address with
 * the device current (a one-time set-up); make that first call before any
 * stream capture.  All calls on a device share the array, so calls whose work
 * overlaps on the GPU race: order them on one stream or synchronise between
 * them.  Each call writes every scratch entry it reads before reading it.
 * Errors: SPAMM_E_CAPACITY if nleaves > SPAMM_NOALLOC_MAX_LEAVES,
 * SPAMM_E_INVALID_ARG (bs not 32/64/128/256, nleaves < 0, NULL pointer,
 * payload not 16-byte aligned, sq_out or total_out not 8-byte aligned; these
 * are checked on the host before anything is enqueued), SPAMM_E_CUDA (set-up
 * or launch failed). */
SPAMM_API spamm_status spamm_leaf_sqnorms_noalloc(const double* payload, int64_t nleaves, int bs, double* sq_out,
                                                  double* total_out, void* cuda_stream);

/* Nodes of quadtree level `level` (0 = root, L = leaves): Morton codes of
 * (row, col) at that level and squared norms, host memory.  *count receives
 * the node count; more than `cap` -> CAPACITY, nothing written. */
SPAMM_API spamm_status spamm_level_norms(spamm_ctx ctx, spamm_mat m, int level, uint32_t* codes, double* sq, int64_t cap,
                               int64_t* count);

#ifdef __cplusplus
}
#endif
#endif /* SPAMM_H */
