/*
 * spamm_oracle.c -- plain, slow, FP64 CPU oracle for approximate
 * multiplication of matrices stored as quadtrees of dense leaf blocks
 * (Artemov, "Approximate multiplication of nearly sparse matrices with decay
 * in a fully recursive distributed task-based parallel framework").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library links or calls this file;
 * only the tests, the package smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code with the CUDA path.
 *
 * A matrix here is a list of non-null leaves: block coordinates (bi, bj) and
 * a bs x bs row-major FP64 payload each.  Everything is written as the plain
 * definition: no blocking, no fusion, no reordering beyond what the paper
 * states.  OpenMP is only used across independent output leaves, so results
 * do not depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { ORC_MODE_TRUNCATE = 0, ORC_MODE_SPAMM = 1, ORC_MODE_COMBINED = 2 };

/* Pairwise (recursive halving) sum of squares: the squared Frobenius norm
 * of a leaf (Section 2: each matrix stores its squared Frobenius norm). */
static double pairwise_sumsq(const double* x, int64_t len) {
  if (len == 0) return 0.0;
  if (len == 1) return x[0] * x[0];
  int64_t h = len / 2;
  return pairwise_sumsq(x, h) + pairwise_sumsq(x + h, len - h);
}

double orc_pairwise_sumsq(const double* x, int64_t len) { return pairwise_sumsq(x, len); }

void orc_leaf_sqnorms(int64_t m, int32_t bs, const double* data, double* out) {
  const int64_t e = (int64_t)bs * bs;
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < m; ++q) out[q] = pairwise_sumsq(data + q * e, e);
}

/* Split a dense n x n matrix into bs x bs leaves (last row/column of leaves
 * zero-padded) and keep a leaf iff it has at least one non-zero element
 * (Section 4.4).  Leaves are emitted in (bi, bj) row-major order.  With
 * out_* == NULL only the count is returned. */
int64_t orc_leaves_from_dense(int64_t n, int32_t bs, const double* a, int64_t lda, int32_t* out_bi,
                              int32_t* out_bj, double* out_data) {
  const int64_t nb = (n + bs - 1) / bs;
  int64_t cnt = 0;
  for (int64_t bi = 0; bi < nb; ++bi)
    for (int64_t bj = 0; bj < nb; ++bj) {
      int nonzero = 0;
      for (int32_t r = 0; r < bs && !nonzero; ++r)
        for (int32_t c = 0; c < bs; ++c) {
          int64_t i = bi * bs + r, j = bj * bs + c;
          if (i < n && j < n && a[i * lda + j] != 0.0) { nonzero = 1; break; }
        }
      if (!nonzero) continue;
      if (out_bi) {
        out_bi[cnt] = (int32_t)bi;
        out_bj[cnt] = (int32_t)bj;
        double* dst = out_data + cnt * (int64_t)bs * bs;
        for (int32_t r = 0; r < bs; ++r)
          for (int32_t c = 0; c < bs; ++c) {
            int64_t i = bi * bs + r, j = bj * bs + c;
            dst[r * bs + c] = (i < n && j < n) ? a[i * lda + j] : 0.0;
          }
      }
      ++cnt;
    }
  return cnt;
}

/* Quadtree norms (Section 2): level L holds the leaves on a 2^L x 2^L grid,
 * level t-1 holds the parents, with
 *     ||A^t||_F^2 = sum_{i,j in {0,1}} ||A^{t+1}_{ij}||_F^2,
 * children added in the fixed order (0,0), (0,1), (1,0), (1,1).  A node with
 * no non-null child is null (stored as -1).  `grid` holds the levels 0..L
 * back to back, level t at offset (4^t - 1) / 3, row-major within a level. */
static int64_t level_offset(int t) { return (((int64_t)1 << (2 * t)) - 1) / 3; }

void orc_tree_norms(int32_t L, int64_t m, const int32_t* bi, const int32_t* bj, const double* sq,
                    double* grid) {
  const int64_t total = level_offset(L + 1);
  for (int64_t q = 0; q < total; ++q) grid[q] = -1.0;
  const int64_t side = (int64_t)1 << L;
  double* leaf = grid + level_offset(L);
  for (int64_t q = 0; q < m; ++q) leaf[(int64_t)bi[q] * side + bj[q]] = sq[q];
  for (int t = L; t >= 1; --t) {
    const int64_t cs = (int64_t)1 << t, ps = cs / 2;
    const double* ch = grid + level_offset(t);
    double* par = grid + level_offset(t - 1);
    for (int64_t I = 0; I < ps; ++I)
      for (int64_t J = 0; J < ps; ++J) {
        double s = 0.0;
        int any = 0;
        for (int ci = 0; ci < 2; ++ci)
          for (int cj = 0; cj < 2; ++cj) {
            double v = ch[(2 * I + ci) * cs + (2 * J + cj)];
            if (v >= 0.0) { s += v; any = 1; }
          }
        par[I * ps + J] = any ? s : -1.0;
      }
  }
}

/* The norm test of Algorithm 1: the sub-product is computed iff
 * ||A_ik||_F ||B_kj||_F >= tau, with the norms taken as sqrt of the stored
 * squared norms.  Truncmul (Section 5.3) skips no product: every pair of
 * non-null blocks is multiplied. */
static int keep_pair(double sa, double sb, double tau, int mode) {
  if (mode == ORC_MODE_TRUNCATE) return 1;
  return sqrt(sa) * sqrt(sb) >= tau;
}

/* Kept leaf triples, flat form: every (i,k,j) with A_ik and B_kj non-null and
 * the leaf-level norm test passed (the test applied down to leaf pairs,
 * Section 4.4).  B leaves must be given sorted by block row (bi).  Returns the
 * count; fills out_ikj (3 per triple) when it is not NULL. */
int64_t orc_kept_flat(int64_t ma, const int32_t* a_bi, const int32_t* a_bj, const double* a_sq,
                      int64_t mb, const int32_t* b_bi, const int32_t* b_bj, const double* b_sq,
                      int32_t nbp, double tau, int32_t mode, int32_t* out_ikj) {
  int64_t* row_start = (int64_t*)calloc((size_t)nbp + 1, sizeof(int64_t));
  for (int64_t q = 0; q < mb; ++q) row_start[b_bi[q] + 1]++;
  for (int32_t r = 0; r < nbp; ++r) row_start[r + 1] += row_start[r];
  int64_t cnt = 0;
  for (int64_t p = 0; p < ma; ++p) {
    const int32_t k = a_bj[p];
    for (int64_t q = row_start[k]; q < row_start[k + 1]; ++q) {
      if (!keep_pair(a_sq[p], b_sq[q], tau, mode)) continue;
      if (out_ikj) {
        out_ikj[3 * cnt + 0] = a_bi[p];
        out_ikj[3 * cnt + 1] = k;
        out_ikj[3 * cnt + 2] = b_bj[q];
      }
      ++cnt;
    }
  }
  free(row_start);
  return cnt;
}

/* Kept leaf triples by literal recursion of Algorithm 1 over the quadtree
 * norm grids of orc_tree_norms: at the lowest level the product is recorded;
 * above it, for i, j in {0,1} and k in {0,1} the child product is entered iff
 * both children exist and pass the norm test.  The root pair is entered when
 * both roots exist. */
typedef struct {
  const double* ga;
  const double* gb;
  int32_t L;
  double tau;
  int32_t mode;
  int32_t* out;
  int64_t cnt;
} rec_state;

static double node(const double* g, int t, int64_t r, int64_t c) {
  return g[level_offset(t) + r * ((int64_t)1 << t) + c];
}

static void spamm_rec(rec_state* s, int t, int64_t I, int64_t K, int64_t J) {
  if (t == s->L) {
    if (s->out) {
      s->out[3 * s->cnt + 0] = (int32_t)I;
      s->out[3 * s->cnt + 1] = (int32_t)K;
      s->out[3 * s->cnt + 2] = (int32_t)J;
    }
    s->cnt++;
    return;
  }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      for (int k = 0; k < 2; ++k) {
        double na = node(s->ga, t + 1, 2 * I + i, 2 * K + k);
        double nb = node(s->gb, t + 1, 2 * K + k, 2 * J + j);
        if (na < 0.0 || nb < 0.0) continue; /* null sub-matrix: product is zero */
        if (keep_pair(na, nb, s->tau, s->mode)) spamm_rec(s, t + 1, 2 * I + i, 2 * K + k, 2 * J + j);
      }
}

int64_t orc_kept_recursive(int32_t L, const double* grid_a, const double* grid_b, double tau,
                           int32_t mode, int32_t* out_ikj) {
  rec_state s = {grid_a, grid_b, L, tau, mode, out_ikj, 0};
  if (grid_a[0] < 0.0 || grid_b[0] < 0.0) return 0;
  /* A single-leaf matrix (L = 0): the root pair is a leaf pair and takes the
   * leaf-level test (Section 4.4 carries the test down to leaf pairs). */
  if (L == 0 && !keep_pair(grid_a[0], grid_b[0], tau, mode)) return 0;
  spamm_rec(&s, 0, 0, 0, 0);
  return s.cnt;
}

/* Leaf products (Algorithm 1, "C = AB" at the lowest level; the batched
 * multiplication of Section 4.4): output leaf g is
 *     C_g = sum over its pairs p in [cptr[g], cptr[g+1]) of A[pa[p]] B[pb[p]],
 * pairs taken in the given order (ascending k), each leaf product a naive
 * triple loop in FP64.  Output leaves are independent and run in parallel. */
void orc_leaf_products(int32_t bs, const double* a_data, const double* b_data, int64_t nc,
                       const int64_t* cptr, const int64_t* pa, const int64_t* pb, double* c_data) {
  const int64_t e = (int64_t)bs * bs;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t g = 0; g < nc; ++g) {
    double* C = c_data + g * e;
    for (int64_t q = 0; q < e; ++q) C[q] = 0.0;
    for (int64_t p = cptr[g]; p < cptr[g + 1]; ++p) {
      const double* A = a_data + pa[p] * e;
      const double* B = b_data + pb[p] * e;
      for (int32_t r = 0; r < bs; ++r)
        for (int32_t kk = 0; kk < bs; ++kk) {
          const double av = A[r * bs + kk];
          for (int32_t c = 0; c < bs; ++c) C[r * bs + c] += av * B[kk * bs + c];
        }
    }
  }
}

/* Dense reference product C = A B (n x n, row-major), the textbook triple
 * loop; used for the tau = 0 pin on tiny inputs. */
void orc_dense_product(int64_t n, const double* a, const double* b, double* c) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    for (int64_t j = 0; j < n; ++j) c[i * n + j] = 0.0;
    for (int64_t k = 0; k < n; ++k) {
      const double av = a[i * n + k];
      for (int64_t j = 0; j < n; ++j) c[i * n + j] += av * b[k * n + j];
    }
  }
}

/* Squared Frobenius norm of the difference of two leaves: sum (x - y)^2. */
double orc_leaf_diff_sumsq(int32_t bs, const double* x, const double* y) {
  const int64_t e = (int64_t)bs * bs;
  double s = 0.0;
  for (int64_t q = 0; q < e; ++q) {
    double d = x[q] - y[q];
    s += d * d;
  }
  return s;
}

/* Threads the OpenMP loops above use (reported with the CPU baseline). */
int32_t orc_num_threads(void) {
#ifdef _OPENMP
  return (int32_t)omp_get_max_threads();
#else
  return 1;
#endif
}
