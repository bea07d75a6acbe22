// algebra.cu -- the quadtree-matrix operations a purification chain needs
// beside the multiply (Section 4.4 lists addition and rescaling among the
// leaf library's operations; density-matrix purification, Section 1, is the
// application): alpha X + beta Y, the identity, and the trace.
#include "internal.cuh"

namespace spamm {

namespace {

unsigned grid_of(spamm_ctx ctx, int64_t items, int per_block) {
  int64_t g = (items + per_block - 1) / per_block;
  const int64_t cap = (int64_t)ctx->num_sms * 32;
  if (g > cap) g = cap;
  return (unsigned)(g < 1 ? 1 : g);
}

// first index with c[index] >= key (n if none); c ascending
__device__ __forceinline__ int64_t lower_bound_code(const uint32_t* __restrict__ c, int64_t n, uint32_t key) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (c[mid] < key)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// Y leaves whose code X does not have (they become leaves of their own).
__global__ void add_ynew_kernel(const uint32_t* __restrict__ xc, int64_t nx, const uint32_t* __restrict__ yc,
                                int64_t ny, uint64_t* __restrict__ ynew) {
  for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < ny; j += (int64_t)gridDim.x * blockDim.x) {
    const int64_t lx = lower_bound_code(xc, nx, yc[j]);
    ynew[j] = (lx < nx && xc[lx] == yc[j]) ? 0u : 1u;
  }
}

// Union of the two sorted leaf sets: output position of X leaf i is i plus the
// new Y leaves before it; of new Y leaf j, the new Y leaves before it plus the
// X leaves before it.
__global__ void add_place_kernel(const uint32_t* __restrict__ xc, int64_t nx, const uint32_t* __restrict__ yc,
                                 int64_t ny, const uint64_t* __restrict__ ynew, const uint64_t* __restrict__ ypos,
                                 uint32_t* __restrict__ ocode, int64_t* __restrict__ oxi, int64_t* __restrict__ oyi) {
  const int64_t total = nx + ny;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (int64_t)gridDim.x * blockDim.x) {
    if (q < nx) {
      const uint32_t c = xc[q];
      const int64_t ly = lower_bound_code(yc, ny, c);
      const int64_t p = q + (int64_t)ypos[ly];  // ypos has ny + 1 entries
      ocode[p] = c;
      oxi[p] = q;
      oyi[p] = (ly < ny && yc[ly] == c) ? ly : -1;
    } else {
      const int64_t j = q - nx;
      if (!ynew[j]) continue;
      const int64_t p = (int64_t)ypos[j] + lower_bound_code(xc, nx, yc[j]);
      ocode[p] = yc[j];
      oxi[p] = -1;
      oyi[p] = j;
    }
  }
}

// out = alpha x + beta y element by element, an absent side taken as 0:
// fl(fl(alpha x) + fl(beta y)).  One block per output leaf.
__global__ void add_payload_kernel(int64_t nout, int64_t e, double alpha, const double* __restrict__ xpool,
                                   const int64_t* __restrict__ xslot, const int64_t* __restrict__ oxi, double beta,
                                   const double* __restrict__ ypool, const int64_t* __restrict__ yslot,
                                   const int64_t* __restrict__ oyi, double* __restrict__ out) {
  for (int64_t q = blockIdx.x; q < nout; q += gridDim.x) {
    const int64_t xi = oxi[q], yi = oyi[q];
    const double* xs = xi >= 0 ? xpool + xslot[xi] * e : nullptr;
    const double* ys = yi >= 0 ? ypool + yslot[yi] * e : nullptr;
    double* d = out + q * e;
    for (int64_t i = threadIdx.x; i < e; i += blockDim.x) {
      const double a = xs ? __dmul_rn(alpha, xs[i]) : 0.0;
      const double b = ys ? __dmul_rn(beta, ys[i]) : 0.0;
      d[i] = __dadd_rn(a, b);
    }
  }
}

// Identity leaves (i, i): ones on the diagonal rows that lie inside the matrix.
__global__ void identity_kernel(int64_t nb, int64_t n, int bs, uint32_t* __restrict__ code, double* __restrict__ pool) {
  const int64_t e = (int64_t)bs * bs;
  for (int64_t q = blockIdx.x; q < nb; q += gridDim.x) {
    if (threadIdx.x == 0) code[q] = morton2((uint32_t)q, (uint32_t)q);
    for (int64_t i = threadIdx.x; i < e; i += blockDim.x) {
      const int64_t r = i / bs, c = i % bs;
      pool[q * e + i] = (r == c && q * bs + r < n) ? 1.0 : 0.0;
    }
  }
}

// Diagonal sum of each diagonal leaf in row order (0 for the others).
__global__ void leaf_trace_kernel(const double* __restrict__ pool, const int64_t* __restrict__ slot,
                                  const uint32_t* __restrict__ code, int64_t m, int bs, double* __restrict__ part) {
  const int64_t e = (int64_t)bs * bs;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < m; q += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    if (code_row(code[q]) == code_col(code[q])) {
      const double* a = pool + slot[q] * e;
      for (int r = 0; r < bs; ++r) s = __dadd_rn(s, a[(int64_t)r * bs + r]);
    }
    part[q] = s;
  }
}

}  // namespace

spamm_mat add_scaled(double alpha, spamm_mat X, double beta, spamm_mat Y, spamm_ctx ctx) {
  const int64_t nx = X->nleaves, ny = Y->nleaves, e = (int64_t)X->bs * X->bs;
  std::unique_ptr<spamm_mat_s> out(new_mat(ctx, X->n, X->bs));
  const uint32_t* xc = P<uint32_t>(X->lv[X->L].code);
  const uint32_t* yc = P<uint32_t>(Y->lv[Y->L].code);
  BufP ynew = alloc_n<uint64_t>(ctx, ny), ypos = alloc_n<uint64_t>(ctx, ny + 1);
  if (ny > 0) {
    add_ynew_kernel<<<grid_of(ctx, ny, 256), 256, 0, ctx->stream>>>(xc, nx, yc, ny, P<uint64_t>(ynew));
    CK_LAUNCH("add_ynew_kernel");
    scan_exclusive_u64(ctx, P<uint64_t>(ynew), P<uint64_t>(ypos), ny, P<uint64_t>(ypos) + ny);
  } else {
    CK(cudaMemsetAsync(P<uint64_t>(ypos), 0, sizeof(uint64_t), ctx->stream));
  }
  const int64_t nnew = ny > 0 ? (int64_t)read_scalar<uint64_t>(ctx, P<uint64_t>(ypos) + ny) : 0;
  const int64_t nout = nx + nnew;
  BufP code = alloc_n<uint32_t>(ctx, nout), oxi = alloc_n<int64_t>(ctx, nout), oyi = alloc_n<int64_t>(ctx, nout);
  BufP sq = alloc_n<double>(ctx, nout), nz = alloc_n<uint8_t>(ctx, nout);
  out->pool = alloc_n<double>(ctx, nout * e);
  if (nout > 0) {
    add_place_kernel<<<grid_of(ctx, nx + ny, 256), 256, 0, ctx->stream>>>(
        xc, nx, yc, ny, P<uint64_t>(ynew), P<uint64_t>(ypos), P<uint32_t>(code), P<int64_t>(oxi), P<int64_t>(oyi));
    CK_LAUNCH("add_place_kernel");
    add_payload_kernel<<<grid_of(ctx, nout, 1), 256, 0, ctx->stream>>>(
        nout, e, alpha, P<double>(X->pool), P<int64_t>(X->slot), P<int64_t>(oxi), beta, P<double>(Y->pool),
        P<int64_t>(Y->slot), P<int64_t>(oyi), P<double>(out->pool));
    CK_LAUNCH("add_payload_kernel");
    leaf_sqnorms(ctx, P<double>(out->pool), nullptr, nout, X->bs, P<double>(sq), P<uint8_t>(nz), 1);
  }
  // a leaf whose sum is exactly zero is null (stored iff it has a non-zero element)
  set_leaves_compacted(out.get(), nout, P<uint32_t>(code), P<double>(sq), nullptr, P<uint8_t>(nz));
  sync_and_check(ctx);
  return out.release();
}

spamm_mat identity_mat(spamm_ctx ctx, int64_t n, int bs) {
  std::unique_ptr<spamm_mat_s> out(new_mat(ctx, n, bs));
  const int64_t nb = (n + bs - 1) / bs, e = (int64_t)bs * bs;
  BufP code = alloc_n<uint32_t>(ctx, nb), sq = alloc_n<double>(ctx, nb), nz = alloc_n<uint8_t>(ctx, nb);
  out->pool = alloc_n<double>(ctx, nb * e);
  identity_kernel<<<grid_of(ctx, nb, 1), 256, 0, ctx->stream>>>(nb, n, bs, P<uint32_t>(code), P<double>(out->pool));
  CK_LAUNCH("identity_kernel");
  leaf_sqnorms(ctx, P<double>(out->pool), nullptr, nb, bs, P<double>(sq), P<uint8_t>(nz), 0);
  set_leaves_compacted(out.get(), nb, P<uint32_t>(code), P<double>(sq), nullptr, P<uint8_t>(nz));
  sync_and_check(ctx);
  return out.release();
}

double trace_of(spamm_mat X) {
  spamm_ctx ctx = X->ctx;
  const int64_t m = X->nleaves;
  if (m == 0) return 0.0;
  BufP part = alloc_n<double>(ctx, m);
  leaf_trace_kernel<<<grid_of(ctx, m, 256), 256, 0, ctx->stream>>>(P<double>(X->pool), P<int64_t>(X->slot),
                                                                    P<uint32_t>(X->lv[X->L].code), m, X->bs,
                                                                    P<double>(part));
  CK_LAUNCH("leaf_trace_kernel");
  const double t = device_sum(ctx, P<double>(part), m);
  sync_and_check(ctx);
  return t;
}

}  // namespace spamm
