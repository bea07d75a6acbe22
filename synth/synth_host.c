/* Host build of the shared input generator (decaygen.h), exported for ctypes.
 * Compiled with -ffp-contract=off so that no multiply-add is fused and the
 * bits equal those the device build produces. */
#include "decaygen.h"

void synth_fill_dense(const synth_params* p, double* out) {
  const int64_t n = p->n;
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < n; ++j) out[i * n + j] = synth_element(p, i, j);
}

/* Leaf (bi, bj) of size bs x bs, row-major, rows bi*bs.., cols bj*bs.. */
void synth_fill_leaves(const synth_params* p, int32_t bs, int64_t nleaves, const int32_t* bi,
                       const int32_t* bj, double* out) {
#pragma omp parallel for schedule(dynamic, 4)
  for (int64_t m = 0; m < nleaves; ++m) {
    double* dst = out + m * (int64_t)bs * bs;
    for (int32_t r = 0; r < bs; ++r)
      for (int32_t c = 0; c < bs; ++c)
        dst[r * bs + c] = synth_element(p, (int64_t)bi[m] * bs + r, (int64_t)bj[m] * bs + c);
  }
}

double synth_exp_nonpos_host(double x) { return synth_exp_nonpos(x); }
double synth_uniform_host(uint64_t seed, int64_t i, int64_t j) { return synth_uniform(seed, i, j); }
double synth_distance_host(const synth_params* p, int64_t i, int64_t j) { return synth_distance(p, i, j); }
void synth_lattice_point_host(int64_t i, int32_t* xyz) { synth_lattice_point(i, xyz, xyz + 1, xyz + 2); }
double synth_leaf_bound_host(const synth_params* p, int32_t bs, int64_t bi, int64_t bj) {
  return synth_leaf_bound(p, bs, bi, bj);
}

/* The leaf bounds of leaves (bi, bj[q]), q < m: one block row at a time. */
void synth_leaf_bounds_row(const synth_params* p, int32_t bs, int64_t bi, int64_t m, const int64_t* bj, double* out) {
#pragma omp parallel for schedule(static)
  for (int64_t q = 0; q < m; ++q) out[q] = synth_leaf_bound(p, bs, bi, bj[q]);
}

/* Random block-sparse n x n matrix (the leaf-library benchmark of Section
 * 5.2): on the nb x nb grid of bs x bs blocks (nb = ceil(n / bs)), block
 * (I, J) is non-zero with probability `fill`, independently of the others
 * (uniformly distributed positions); its elements inside the matrix are
 * uniform in [-1, 1), those past row or column n (the padding of the last
 * blocks) are 0.  Position draws use the SplitMix64 stream `seed`, element
 * draws the stream `seed` + 1 (number I*nb+J, resp. i<<32|j).  Returns the
 * block count; with non-null outputs also writes the blocks in row-major
 * block order (coordinates and bs*bs row-major values each). */
int64_t synth_block_sparse(int64_t n, int32_t bs, double fill, uint64_t seed, int32_t* bi, int32_t* bj,
                           double* out) {
  const int64_t nb = (n + bs - 1) / bs;
  int64_t m = 0;
  for (int64_t I = 0; I < nb; ++I)
    for (int64_t J = 0; J < nb; ++J) {
      const double u = (double)(synth_splitmix64(seed, (uint64_t)(I * nb + J)) >> 11) * 0x1.0p-53;
      if (!(u < fill)) continue;
      if (bi) {
        bi[m] = (int32_t)I;
        bj[m] = (int32_t)J;
        double* dst = out + m * (int64_t)bs * bs;
        for (int32_t r = 0; r < bs; ++r)
          for (int32_t c = 0; c < bs; ++c) {
            const uint64_t i = (uint64_t)(I * bs + r), j = (uint64_t)(J * bs + c);
            const uint64_t h = synth_splitmix64(seed + 1ull, (i << 32) | j);
            dst[r * bs + c] = ((int64_t)i < n && (int64_t)j < n) ? (double)(h >> 11) * 0x1.0p-52 - 1.0 : 0.0;
          }
      }
      ++m;
    }
  return m;
}
