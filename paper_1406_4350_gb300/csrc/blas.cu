// Elementwise and reduction kernels of the filter and of Rayleigh-Ritz: the
// block-diagonal coefficient matrices D_V, D_S of Section 2.1, the Chebyshev three-term
// combination of Section 4.2, reorderings between the caller's plane-wave order and the
// column-sorted order of the FFT, column dot products and residual norms.
#include <algorithm>

#include "internal.cuh"
#include "kernels.cuh"

namespace chebfi {
namespace {

inline unsigned nblocks(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

template <typename R>
__global__ void k_blockdiag(int64_t nproj, int64_t nb, const int32_t* __restrict__ atom_of,
                            const int32_t* __restrict__ offs, const int64_t* __restrict__ blk_off,
                            const R* __restrict__ D, const cplx<R>* __restrict__ p, int64_t ldp,
                            cplx<R>* __restrict__ out, int64_t ldo) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nproj * nb) return;
  const int64_t i = idx % nproj, b = idx / nproj;
  const int a = atom_of[i];
  const int o = offs[a], na = offs[a + 1] - o;
  const R* row = D + blk_off[a] + (int64_t)(i - o) * na;
  const cplx<R>* pb = p + b * ldp + o;
  R sr = 0, si = 0;
  for (int j = 0; j < na; ++j) {
    sr = fma(row[j], pb[j].x, sr);
    si = fma(row[j], pb[j].y, si);
  }
  out[b * ldo + i] = cmake<cplx<R>>(sr, si);
}

template <typename R>
__global__ void k_cheb_combine(int64_t m, int64_t nb, R a, const cplx<R>* __restrict__ u, int64_t ldu, R c,
                               const cplx<R>* __restrict__ x, int64_t ldx, R b, const cplx<R>* y, int64_t ldy,
                               cplx<R>* out, int64_t ldo) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * nb) return;
  const int64_t i = idx % m, j = idx / m;
  const cplx<R> uu = u[i + j * ldu], xx = x[i + j * ldx];
  cplx<R> yy = cmake<cplx<R>>(0.0, 0.0);
  if (y) yy = y[i + j * ldy];
  cplx<R> r;
  r.x = a * (uu.x - c * xx.x) - b * yy.x;
  r.y = a * (uu.y - c * xx.y) - b * yy.y;
  out[i + j * ldo] = r;
}

template <typename R>
__global__ void k_axpby(int64_t m, int64_t nb, R alpha, const cplx<R>* x, int64_t ldx, R beta, const cplx<R>* y,
                        int64_t ldy, cplx<R>* out, int64_t ldo) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * nb) return;
  const int64_t i = idx % m, j = idx / m;
  const cplx<R> xx = x[i + j * ldx];
  cplx<R> r;
  r.x = alpha * xx.x;
  r.y = alpha * xx.y;
  if (y) {
    const cplx<R> yy = y[i + j * ldy];
    r.x += beta * yy.x;
    r.y += beta * yy.y;
  }
  out[i + j * ldo] = r;
}

template <typename A, typename B>
__global__ void k_convert(int64_t m, int64_t nb, const A* __restrict__ x, int64_t ldx, B* __restrict__ y, int64_t ldy) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * nb) return;
  const int64_t i = idx % m, j = idx / m;
  const A v = x[i + j * ldx];
  B r;
  r.x = (decltype(r.x))v.x;
  r.y = (decltype(r.y))v.y;
  y[i + j * ldy] = r;
}

__global__ void k_gather(int64_t m, int64_t nb, const int32_t* __restrict__ perm, const double2* __restrict__ src,
                         int64_t lds, double2* __restrict__ dst, int64_t ldd) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * nb) return;
  const int64_t i = idx % m, j = idx / m;
  dst[i + j * ldd] = src[perm[i] + j * lds];
}

__global__ void k_scatter(int64_t m, int64_t nb, const int32_t* __restrict__ perm, const double2* __restrict__ src,
                          int64_t lds, double2* __restrict__ dst, int64_t ldd) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * nb) return;
  const int64_t i = idx % m, j = idx / m;
  dst[perm[i] + j * ldd] = src[i + j * lds];
}

// the same reorderings with the precision change fused in (FP64 caller blocks, FP32 iterates)
__global__ void k_gather_f32(int64_t m, int64_t nb, const int32_t* __restrict__ perm, const double2* __restrict__ src,
                             int64_t lds, float2* __restrict__ dst, int64_t ldd) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * nb) return;
  const int64_t i = idx % m, j = idx / m;
  const double2 v = src[perm[i] + j * lds];
  dst[i + j * ldd] = make_float2((float)v.x, (float)v.y);
}

__global__ void k_scatter_f32(int64_t m, int64_t nb, const int32_t* __restrict__ perm, const float2* __restrict__ src,
                              int64_t lds, double2* __restrict__ dst, int64_t ldd) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * nb) return;
  const int64_t i = idx % m, j = idx / m;
  const float2 v = src[i + j * lds];
  dst[perm[i] + j * ldd] = make_double2((double)v.x, (double)v.y);
}

// one block per column; fixed-order tree reduction (deterministic)
__global__ void k_column_dots(int64_t m, const double2* __restrict__ x, int64_t ldx, const double2* __restrict__ y,
                              int64_t ldy, double* __restrict__ out, int accumulate) {
  __shared__ double red[256];
  const int64_t j = blockIdx.x;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    const double2 a = x[i + j * ldx], b = y[i + j * ldy];
    s += a.x * b.x + a.y * b.y;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = (accumulate ? out[j] : 0.0) + red[0];
}

__global__ void k_residual_norms(int64_t m, const double2* __restrict__ h, int64_t ldh, const double2* __restrict__ s,
                                 int64_t lds, const double* __restrict__ w, double* __restrict__ out) {
  __shared__ double red[256];
  const int64_t j = blockIdx.x;
  const double lam = w[j];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < m; i += blockDim.x) {
    const double2 a = h[i + j * ldh], b = s[i + j * lds];
    const double rx = a.x - lam * b.x, ry = a.y - lam * b.y;
    acc += rx * rx + ry * ry;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int hh = blockDim.x / 2; hh > 0; hh >>= 1) {
    if ((int)threadIdx.x < hh) red[threadIdx.x] += red[threadIdx.x + hh];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[j] = sqrt(red[0]);
}

__global__ void k_divide(int64_t n, const double* num, const double* den, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = num[i] / den[i];
}

__global__ void k_identity(int64_t n, double2* A, int64_t lda) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx % n, j = idx / n;
  A[i + j * lda] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}

__global__ void k_diag_of(int64_t n, const double2* A, int64_t lda, double* d) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) d[i] = A[i + i * lda].x;
}

__global__ void k_scale_sym(int64_t n, double2* A, int64_t lda, const double* d) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx % n, j = idx / n;
  const double s = 1.0 / sqrt(d[i] * d[j]);
  double2 v = A[i + j * lda];
  A[i + j * lda] = make_double2(v.x * s, v.y * s);
}

__global__ void k_scale_rows(int64_t n, int64_t m, double2* X, int64_t ldx, const double* d) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * m) return;
  const int64_t i = idx % n, j = idx / n;
  const double s = 1.0 / sqrt(d[i]);
  double2 v = X[i + j * ldx];
  X[i + j * ldx] = make_double2(v.x * s, v.y * s);
}

__global__ void k_hermitize(int64_t n, double2* A, int64_t lda) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx % n, j = idx / n;
  if (i > j) return;
  const double2 a = A[i + j * lda], b = A[j + i * lda];
  const double2 h = make_double2(0.5 * (a.x + b.x), 0.5 * (a.y - b.y));
  A[i + j * lda] = h;
  A[j + i * lda] = make_double2(h.x, -h.y);
}

__global__ void k_permute_cols(int64_t m, const int32_t* __restrict__ order, const double2* __restrict__ src,
                               double2* __restrict__ dst, int inverse) {
  const int64_t j = blockIdx.y;
  const int64_t o = order[j];
  const double2* s = src + (inverse ? j : o) * m;
  double2* d = dst + (inverse ? o : j) * m;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += (int64_t)gridDim.x * blockDim.x)
    d[i] = s[i];
}

// one thread per (projector i, band b): out_ib = sum_j B_a[i - o, j - o] p_jb over i's atom block
__global__ void k_blockdiag_apply_c(int64_t nproj, int64_t nb, const int32_t* __restrict__ atom_of,
                                    const int32_t* __restrict__ offs, const int64_t* __restrict__ cblk_off,
                                    const double2* __restrict__ B, const double2* __restrict__ p, int64_t ldp,
                                    double2* __restrict__ out, int64_t ldo) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nproj * nb) return;
  const int64_t i = idx % nproj, b = idx / nproj;
  const int a = atom_of[i];
  const int o = offs[a], na = offs[a + 1] - o;
  const double2* Ba = B + cblk_off[a];
  double re = 0.0, im = 0.0;
  for (int jl = 0; jl < na; ++jl) {
    const double2 m = Ba[(i - o) + (int64_t)jl * na], v = p[o + jl + b * ldp];
    re += m.x * v.x - m.y * v.y;
    im += m.x * v.y + m.y * v.x;
  }
  out[i + b * ldo] = make_double2(re, im);
}

// one thread per (projector i, position j within i's atom block)
template <typename C>
__global__ void k_block_outer_grad(int64_t nproj, const int32_t* __restrict__ atom_of, const int32_t* __restrict__ offs,
                                   const int64_t* __restrict__ blk_off, const C* __restrict__ q,
                                   const C* __restrict__ p, int64_t ldp, int64_t nb, double* __restrict__ gD,
                                   double scale, int accumulate) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nproj * 64) return;
  const int64_t i = idx / 64;
  const int jl = (int)(idx % 64);
  const int a = atom_of[i];
  const int o = offs[a], na = offs[a + 1] - o;
  if (jl >= na) return;
  const int64_t j = o + jl;
  double acc = 0.0;
  for (int64_t b = 0; b < nb; ++b) {
    const C u = q[i + b * ldp], v = p[j + b * ldp];
    acc += (double)u.x * (double)v.x + (double)u.y * (double)v.y;
  }
  double* g = gD + blk_off[a] + (i - o) * na + jl;
  *g = scale * acc + (accumulate ? *g : 0.0);
}

__global__ void k_mirror_lower(int64_t n, double2* A, int64_t lda) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx % n, j = idx / n;
  if (i < j) {
    const double2 v = A[j + i * lda];
    A[i + j * lda] = make_double2(v.x, -v.y);
  } else if (i == j) {
    A[i + i * lda].y = 0.0;
  }
}

__global__ void k_reduce_max(int64_t n, const double* x, double* out) {
  __shared__ double red[256];
  double m = -1e300;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, x[i]);
  red[threadIdx.x] = m;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + h]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

}  // namespace

template <typename R>
void blockdiag_apply(const chebfi_ctx* ctx, const R* Dblk, const cplx<R>* p, int64_t ldp, cplx<R>* out, int64_t ldo,
                     int64_t nb, cudaStream_t st) {
  const int64_t n = ctx->nproj * nb;
  if (n == 0) return;
  CHEBFI_LAUNCH("k_blockdiag", st, k_blockdiag<R><<<nblocks(n), 256, 0, st>>>(ctx->nproj, nb, ctx->d_atom_of.p, ctx->d_offs.p, ctx->d_blk_off.p, Dblk,
                                             p, ldp, out, ldo));
}
template void blockdiag_apply<double>(const chebfi_ctx*, const double*, const double2*, int64_t, double2*, int64_t,
                                      int64_t, cudaStream_t);
template void blockdiag_apply<float>(const chebfi_ctx*, const float*, const float2*, int64_t, float2*, int64_t,
                                     int64_t, cudaStream_t);

template <typename R>
void cheb_combine(int64_t m, int64_t nb, R a, const cplx<R>* u, int64_t ldu, R c, const cplx<R>* x, int64_t ldx, R b,
                  const cplx<R>* y, int64_t ldy, cplx<R>* out, int64_t ldo, cudaStream_t st) {
  if (m * nb == 0) return;
  CHEBFI_LAUNCH("k_cheb_combine", st, k_cheb_combine<R><<<nblocks(m * nb), 256, 0, st>>>(m, nb, a, u, ldu, c, x, ldx, b, y, ldy, out, ldo));
}
template void cheb_combine<double>(int64_t, int64_t, double, const double2*, int64_t, double, const double2*, int64_t,
                                   double, const double2*, int64_t, double2*, int64_t, cudaStream_t);
template void cheb_combine<float>(int64_t, int64_t, float, const float2*, int64_t, float, const float2*, int64_t,
                                  float, const float2*, int64_t, float2*, int64_t, cudaStream_t);

template <typename R>
void axpby(int64_t m, int64_t nb, R alpha, const cplx<R>* x, int64_t ldx, R beta, const cplx<R>* y, int64_t ldy,
           cplx<R>* out, int64_t ldo, cudaStream_t st) {
  if (m * nb == 0) return;
  CHEBFI_LAUNCH("k_axpby", st, k_axpby<R><<<nblocks(m * nb), 256, 0, st>>>(m, nb, alpha, x, ldx, beta, y, ldy, out, ldo));
}
template void axpby<double>(int64_t, int64_t, double, const double2*, int64_t, double, const double2*, int64_t,
                            double2*, int64_t, cudaStream_t);
template void axpby<float>(int64_t, int64_t, float, const float2*, int64_t, float, const float2*, int64_t, float2*,
                           int64_t, cudaStream_t);

void convert(int64_t m, int64_t nb, const double2* x, int64_t ldx, float2* y, int64_t ldy, cudaStream_t st) {
  if (m * nb == 0) return;
  CHEBFI_LAUNCH("k_convert", st, k_convert<double2, float2><<<nblocks(m * nb), 256, 0, st>>>(m, nb, x, ldx, y, ldy));
}
void convert(int64_t m, int64_t nb, const float2* x, int64_t ldx, double2* y, int64_t ldy, cudaStream_t st) {
  if (m * nb == 0) return;
  CHEBFI_LAUNCH("k_convert", st, k_convert<float2, double2><<<nblocks(m * nb), 256, 0, st>>>(m, nb, x, ldx, y, ldy));
}
void gather_rows(int64_t m, int64_t nb, const int32_t* perm, const double2* src, int64_t lds, double2* dst,
                 int64_t ldd, cudaStream_t st) {
  if (m * nb == 0) return;
  CHEBFI_LAUNCH("k_gather", st, k_gather<<<nblocks(m * nb), 256, 0, st>>>(m, nb, perm, src, lds, dst, ldd));
}
void scatter_rows(int64_t m, int64_t nb, const int32_t* perm, const double2* src, int64_t lds, double2* dst,
                  int64_t ldd, cudaStream_t st) {
  if (m * nb == 0) return;
  CHEBFI_LAUNCH("k_scatter", st, k_scatter<<<nblocks(m * nb), 256, 0, st>>>(m, nb, perm, src, lds, dst, ldd));
}
void gather_rows(int64_t m, int64_t nb, const int32_t* perm, const double2* src, int64_t lds, float2* dst, int64_t ldd,
                 cudaStream_t st) {
  if (m * nb == 0) return;
  CHEBFI_LAUNCH("k_gather", st, k_gather_f32<<<nblocks(m * nb), 256, 0, st>>>(m, nb, perm, src, lds, dst, ldd));
}
void scatter_rows(int64_t m, int64_t nb, const int32_t* perm, const float2* src, int64_t lds, double2* dst, int64_t ldd,
                  cudaStream_t st) {
  if (m * nb == 0) return;
  CHEBFI_LAUNCH("k_scatter", st, k_scatter_f32<<<nblocks(m * nb), 256, 0, st>>>(m, nb, perm, src, lds, dst, ldd));
}
void column_dots(int64_t m, int64_t nb, const double2* x, int64_t ldx, const double2* y, int64_t ldy, double* out,
                 bool accumulate, cudaStream_t st) {
  if (nb == 0) return;
  CHEBFI_LAUNCH("k_column_dots", st, k_column_dots<<<(unsigned)nb, 256, 0, st>>>(m, x, ldx, y, ldy, out, accumulate ? 1 : 0));
}
void residual_norms(int64_t m, int64_t nb, const double2* h, int64_t ldh, const double2* s, int64_t lds,
                    const double* w, double* out, cudaStream_t st) {
  if (nb == 0) return;
  CHEBFI_LAUNCH("k_residual_norms", st, k_residual_norms<<<(unsigned)nb, 256, 0, st>>>(m, h, ldh, s, lds, w, out));
}
void divide(int64_t n, const double* num, const double* den, double* out, cudaStream_t st) {
  if (n == 0) return;
  CHEBFI_LAUNCH("k_divide", st, k_divide<<<nblocks(n), 256, 0, st>>>(n, num, den, out));
}
void set_identity(int64_t n, double2* A, int64_t lda, cudaStream_t st) {
  if (n == 0) return;
  CHEBFI_LAUNCH("k_identity", st, k_identity<<<nblocks(n * n), 256, 0, st>>>(n, A, lda));
}
void diag_of(int64_t n, const double2* A, int64_t lda, double* d, cudaStream_t st) {
  if (n == 0) return;
  CHEBFI_LAUNCH("k_diag_of", st, k_diag_of<<<nblocks(n), 256, 0, st>>>(n, A, lda, d));
}
void scale_sym(int64_t n, double2* A, int64_t lda, const double* d, cudaStream_t st) {
  if (n == 0) return;
  CHEBFI_LAUNCH("k_scale_sym", st, k_scale_sym<<<nblocks(n * n), 256, 0, st>>>(n, A, lda, d));
}
void scale_rows(int64_t n, int64_t m, double2* X, int64_t ldx, const double* d, cudaStream_t st) {
  if (n * m == 0) return;
  CHEBFI_LAUNCH("k_scale_rows", st, k_scale_rows<<<nblocks(n * m), 256, 0, st>>>(n, m, X, ldx, d));
}
void hermitize(int64_t n, double2* A, int64_t lda, cudaStream_t st) {
  if (n == 0) return;
  CHEBFI_LAUNCH("k_hermitize", st, k_hermitize<<<nblocks(n * n), 256, 0, st>>>(n, A, lda));
}
template <typename C>
void block_outer_grad(const chebfi_ctx* ctx, const C* q, const C* p, int64_t ldp, int64_t nb, double* gD,
                      cudaStream_t st, double scale, bool accumulate) {
  if (ctx->nproj == 0) return;
  CHEBFI_LAUNCH("k_block_outer_grad", st,
                k_block_outer_grad<C><<<nblocks(ctx->nproj * 64), 256, 0, st>>>(ctx->nproj, ctx->d_atom_of.p, ctx->d_offs.p,
                                                                             ctx->d_blk_off.p, q, p, ldp, nb, gD,
                                                                             scale, accumulate ? 1 : 0));
}
template void block_outer_grad<double2>(const chebfi_ctx*, const double2*, const double2*, int64_t, int64_t, double*,
                                        cudaStream_t, double, bool);
template void block_outer_grad<float2>(const chebfi_ctx*, const float2*, const float2*, int64_t, int64_t, double*,
                                       cudaStream_t, double, bool);
void blockdiag_apply_c(const chebfi_ctx* ctx, const double2* Bblk, const int64_t* cblk_off, const double2* p,
                       int64_t ldp, double2* out, int64_t ldo, int64_t nb, cudaStream_t st) {
  if (ctx->nproj == 0 || nb == 0) return;
  CHEBFI_LAUNCH("k_blockdiag_apply_c", st,
                k_blockdiag_apply_c<<<nblocks(ctx->nproj * nb), 256, 0, st>>>(ctx->nproj, nb, ctx->d_atom_of.p,
                                                                            ctx->d_offs.p, cblk_off, Bblk, p, ldp,
                                                                            out, ldo));
}
void permute_cols(int64_t m, int64_t nb, const int32_t* order, const double2* src, double2* dst, bool inverse,
                  cudaStream_t st) {
  if (m == 0 || nb == 0) return;
  CHEBFI_REQUIRE(nb <= 65535, CHEBFI_ERR_ARG, "at most 65535 columns to permute");
  const unsigned gx = (unsigned)std::min<int64_t>((m + 255) / 256, 64);
  CHEBFI_LAUNCH("k_permute_cols", st, (k_permute_cols<<<dim3(gx, (unsigned)nb), 256, 0, st>>>(m, order, src, dst, inverse ? 1 : 0)));
}
void mirror_lower(int64_t n, double2* A, int64_t lda, cudaStream_t st) {
  if (n == 0) return;
  CHEBFI_LAUNCH("k_mirror_lower", st, k_mirror_lower<<<nblocks(n * n), 256, 0, st>>>(n, A, lda));
}
void reduce_max(int64_t n, const double* x, double* out, cudaStream_t st) {
  CHEBFI_LAUNCH("k_reduce_max", st, k_reduce_max<<<1, 256, 0, st>>>(n, x, out));
}

namespace {
__global__ void k_scan_nonfinite(int64_t m, int64_t nb, const double2* __restrict__ x, int64_t ldx, int* status) {
  bool bad = false;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m * nb; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 v = x[e % m + (e / m) * ldx];
    bad |= !(isfinite(v.x) && isfinite(v.y));
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicCAS(status, 0, CHEBFI_ERR_NONFINITE);
}
}  // namespace

void scan_nonfinite(int64_t m, int64_t nb, const double2* x, int64_t ldx, int* status, cudaStream_t st) {
  if (m <= 0 || nb <= 0) return;
  const int64_t blocks = std::min<int64_t>((m * nb + 255) / 256, 152 * 8);
  CHEBFI_LAUNCH("k_scan_nonfinite", st, k_scan_nonfinite<<<(unsigned)blocks, 256, 0, st>>>(m, nb, x, ldx, status));
}

}  // namespace chebfi
