// Local-potential operator of Section 2.1 (Algorithm 1, second step): the sphere
// coefficients of each band go to real space by an inverse 3D FFT, are multiplied by
// V_loc(r), and come back by a forward 3D FFT; the kinetic diagonal |k+G|^2/2 is added
// in the same epilogue.
//
// The 3D transform is pruned to the sphere and split into three passes over a
// "column space" buffer [band][z][column] that holds only the (x, y) columns in which
// the sphere has points (about 20 % of the N1 x N2 columns):
//   zinv  : sphere -> z lines of each column (zero elsewhere), inverse FFT along z;
//   plane : per (band, z) plane in shared memory: inverse FFT along y on the rows that
//           hold columns, inverse FFT along x, multiply by V_loc, forward FFT along x,
//           forward FFT along y on those rows; in place on the column buffer;
//   zfwd  : forward FFT along z, pick the sphere points, scale by 1/(N1 N2 N3), add K psi,
//           and apply the caller's epilogue (plain, or the Chebyshev three-term update).
#include <cmath>
#include <type_traits>

#include "fft_core.cuh"
#include "fft_fast.cuh"
#include "fft_fast_kernels.cuh"
#include "internal.cuh"
#include "kernels.cuh"

namespace chebfi {

void FFTAxis::build(int n_) {
  n = n_;
  CHEBFI_REQUIRE(n >= 1 && n <= kMaxN && factor_radices(n, radices), CHEBFI_ERR_ARG,
                 "FFT size " + std::to_string(n) + " is not a product of 2, 3, 5 up to 256");
  rev = digit_reversal(n, radices);
  std::vector<double2> t64(n);
  std::vector<float2> t32(n);
  for (int k = 0; k < n; ++k) {
    const double a = 2.0 * M_PI * (double)k / (double)n;
    t64[k] = make_double2(std::cos(a), -std::sin(a));
    t32[k] = make_float2((float)t64[k].x, (float)t64[k].y);
  }
  tw64.upload(t64.data(), n);
  tw32.upload(t32.data(), n);
  CHEBFI_CUDA(cudaDeviceSynchronize());
}

template <> FFTPlan<double> FFTAxis::plan<double>() const {
  FFTPlan<double> p;
  p.n = n;
  p.nst = (int)radices.size();
  for (int i = 0; i < p.nst; ++i) p.radix[i] = radices[i];
  p.tw = tw64.p;
  return p;
}
template <> FFTPlan<float> FFTAxis::plan<float>() const {
  FFTPlan<float> p;
  p.n = n;
  p.nst = (int)radices.size();
  for (int i = 0; i < p.nst; ++i) p.radix[i] = radices[i];
  p.tw = tw32.p;
  return p;
}

namespace {

constexpr int kCB = 16;       // columns per z-pass block
constexpr int kThreads = 256;

struct SphArgs {
  int ncol, n3, zpitch;
  int64_t ldt;        // complex elements per band in the column buffer (n3 * ncolp)
  int ncolp;
  const int32_t* col_start;
  const int32_t* pw_line;
  const int32_t* pw_zrev;
};

template <typename R>
__global__ void __launch_bounds__(kThreads) k_zinv(const cplx<R>* __restrict__ Y, int64_t ldy,
                                                   cplx<R>* __restrict__ T, SphArgs sa, FFTPlan<R> pz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* lines = reinterpret_cast<cplx<R>*>(smem_raw);
  const int c0 = blockIdx.x * kCB;
  const int nc = min(kCB, sa.ncol - c0);
  const int64_t b = blockIdx.y;
  const cplx<R> zero = cmake<cplx<R>>(0.0, 0.0);
  for (int i = threadIdx.x; i < kCB * sa.zpitch; i += blockDim.x) lines[i] = zero;
  __syncthreads();
  const int j0 = sa.col_start[c0], j1 = sa.col_start[c0 + nc];
  const cplx<R>* y = Y + b * ldy;
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x)
    lines[(sa.pw_line[j] - c0) * sa.zpitch + sa.pw_zrev[j]] = y[j];
  __syncthreads();
  LineMap lm;
  lm.stride = sa.zpitch;
  block_fft_dit<+1, R>(lines, nc, lm, 1, pz);
  cplx<R>* t = T + b * sa.ldt + c0;
  for (int i = threadIdx.x; i < sa.n3 * nc; i += blockDim.x) {
    const int z = i / nc, l = i - z * nc;
    t[(int64_t)z * sa.ncolp + l] = lines[l * sa.zpitch + z];
  }
}

struct PlaneArgs {
  int n1, n2, n3, ncol, nxa, pitch;
  int64_t ldt;
  int ncolp;
  const int32_t* col_off;
  const int32_t* row_off;  // rev(x) * pitch of each active x
};

template <typename R>
__global__ void __launch_bounds__(kThreads) k_plane(cplx<R>* __restrict__ T, const R* __restrict__ Vt,
                                                    PlaneArgs pa, FFTPlan<R> px, FFTPlan<R> py) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* plane = reinterpret_cast<cplx<R>*>(smem_raw);
  const int z = blockIdx.x;
  const int64_t b = blockIdx.y;
  const cplx<R> zero = cmake<cplx<R>>(0.0, 0.0);
  for (int i = threadIdx.x; i < pa.n1 * pa.pitch; i += blockDim.x) plane[i] = zero;
  __syncthreads();
  cplx<R>* t = T + b * pa.ldt + (int64_t)z * pa.ncolp;
  for (int c = threadIdx.x; c < pa.ncol; c += blockDim.x) plane[pa.col_off[c]] = t[c];
  __syncthreads();
  LineMap rows;
  rows.off = pa.row_off;
  LineMap cols;
  cols.stride = 1;
  block_fft_dit<+1, R>(plane, pa.nxa, rows, 1, py);        // along y, active rows
  block_fft_dit<+1, R>(plane, pa.n2, cols, pa.pitch, px);  // along x, every column
  const R* v = Vt + (int64_t)z * pa.n1 * pa.n2;
  for (int i = threadIdx.x; i < pa.n1 * pa.n2; i += blockDim.x) {
    const int x = i / pa.n2, yy = i - x * pa.n2;
    cplx<R>& e = plane[x * pa.pitch + yy];
    const R s = v[i];
    e.x *= s;
    e.y *= s;
  }
  __syncthreads();
  block_fft_dif<-1, R>(plane, pa.n2, cols, pa.pitch, px);  // along x
  block_fft_dif<-1, R>(plane, pa.nxa, rows, 1, py);        // along y, active rows
  for (int c = threadIdx.x; c < pa.ncol; c += blockDim.x) t[c] = plane[pa.col_off[c]];
}

template <typename R>
__global__ void __launch_bounds__(kThreads) k_zfwd(const cplx<R>* __restrict__ T, SphArgs sa, FFTPlan<R> pz,
                                                   const R* __restrict__ K, LocalEpi<R> ep) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* lines = reinterpret_cast<cplx<R>*>(smem_raw);
  const int c0 = blockIdx.x * kCB;
  const int nc = min(kCB, sa.ncol - c0);
  const int64_t b = blockIdx.y;
  const cplx<R>* t = T + b * sa.ldt + c0;
  for (int i = threadIdx.x; i < sa.n3 * nc; i += blockDim.x) {
    const int z = i / nc, l = i - z * nc;
    lines[l * sa.zpitch + z] = t[(int64_t)z * sa.ncolp + l];
  }
  __syncthreads();
  LineMap lm;
  lm.stride = sa.zpitch;
  block_fft_dif<-1, R>(lines, nc, lm, 1, pz);
  const int j0 = sa.col_start[c0], j1 = sa.col_start[c0 + nc];
  const cplx<R>* y = ep.Y + b * ep.ldy;
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    cplx<R> v = lines[(sa.pw_line[j] - c0) * sa.zpitch + sa.pw_zrev[j]];
    const cplx<R> yj = y[j];
    const R k = K[j];
    cplx<R> zj;
    zj.x = v.x * ep.inv_n3 + k * yj.x;
    zj.y = v.y * ep.inv_n3 + k * yj.y;
    if (ep.Z) ep.Z[b * ep.ldz + j] = zj;
    if (ep.Zhi) epi_split_z(ep, b, j, (float)zj.x, (float)zj.y);
    if (ep.T) {
      // three-term update without its nonlocal part: T = a (Z - c Y) - bprev Yprev
      cplx<R> tp = cmake<cplx<R>>(0.0, 0.0);
      if (ep.Yprev) tp = ep.Yprev[b * ep.ldt + j];
      cplx<R> o;
      o.x = ep.a * (zj.x - ep.c * yj.x) - ep.bprev * tp.x;
      o.y = ep.a * (zj.y - ep.c * yj.y) - ep.bprev * tp.y;
      ep.T[b * ep.ldt + j] = o;
    }
  }
}

// Real-space values on the full grid for the derivative with respect to V_loc: after the
// inverse z pass, each (band, z) plane is transformed back along y and x and written out
// as out[band][z][x][y] (natural order).
template <typename R>
__global__ void __launch_bounds__(kThreads) k_plane_real(const cplx<R>* __restrict__ T, PlaneArgs pa, FFTPlan<R> px,
                                                         FFTPlan<R> py, cplx<R>* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cplx<R>* plane = reinterpret_cast<cplx<R>*>(smem_raw);
  const int z = blockIdx.x;
  const int64_t b = blockIdx.y;
  const cplx<R> zero = cmake<cplx<R>>(0.0, 0.0);
  for (int i = threadIdx.x; i < pa.n1 * pa.pitch; i += blockDim.x) plane[i] = zero;
  __syncthreads();
  const cplx<R>* t = T + b * pa.ldt + (int64_t)z * pa.ncolp;
  for (int c = threadIdx.x; c < pa.ncol; c += blockDim.x) plane[pa.col_off[c]] = t[c];
  __syncthreads();
  LineMap rows;
  rows.off = pa.row_off;
  LineMap cols;
  cols.stride = 1;
  block_fft_dit<+1, R>(plane, pa.nxa, rows, 1, py);
  block_fft_dit<+1, R>(plane, pa.n2, cols, pa.pitch, px);
  cplx<R>* o = out + (b * pa.n3 + z) * (int64_t)pa.n1 * pa.n2;
  for (int i = threadIdx.x; i < pa.n1 * pa.n2; i += blockDim.x) {
    const int x = i / pa.n2, yy = i - x * pa.n2;
    o[i] = plane[x * pa.pitch + yy];
  }
}

// gV[(x n2 + y) n3 + z] += scale * sum_b Re(conj(g_b(r)) psi_b(r)), r = (x, y, z); fixed band order.
template <typename R>
__global__ void k_density_accum(int n1, int n2, int n3, int64_t nbc, const cplx<R>* __restrict__ psi,
                                const cplx<R>* __restrict__ g, double scale, double* __restrict__ gV) {
  const int64_t n = (int64_t)n1 * n2 * n3;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double acc = 0.0;
  for (int64_t b = 0; b < nbc; ++b) {
    const cplx<R> u = psi[b * n + r], v = g[b * n + r];
    acc += (double)v.x * (double)u.x + (double)v.y * (double)u.y;
  }
  const int64_t plane = (int64_t)n1 * n2;
  const int z = (int)(r / plane), rem = (int)(r - (int64_t)z * plane);
  const int x = rem / n2, y = rem - x * n2;
  gV[((int64_t)x * n2 + y) * n3 + z] += scale * acc;
}

// ---------------------------------------------------------------- compile-time-length path
// The pass bodies live in fft_fast_kernels.cuh; here each block finds its columns or plane
// from its grid position.
using fk::FastArgs;
using fk::kCBF;

// R: the arithmetic of the transforms (float, double, or dfl, the double-float form of the
// FP64 path); blocks, the kinetic diagonal and the epilogue's operands are stored in
// SphT<R> (double for dfl), the column buffer and the planes in cplx<R>.
template <typename R, int N3>
__global__ void __launch_bounds__(kThreads) k_zinv_f(const cplx<typename SphT<R>::type>* __restrict__ Y, int64_t ldy,
                                                     cplx<R>* __restrict__ T, FastArgs fa, const cplx<R>* __restrict__ twz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fk::zinv_body<R, N3>(Y, ldy, T, fa, twz, blockIdx.x * kCBF, blockIdx.y, smem_raw);
}

// threads of a plane block: the double-float plane (16 bytes a point, one block per SM)
// takes 16 warps to keep its FP32 pipes fed, the others 8 with three blocks per SM
template <typename R> struct PlaneThreads { static constexpr int v = kThreads; };
template <> struct PlaneThreads<dfl> { static constexpr int v = 2 * kThreads; };

template <typename R, int N>
__global__ void __launch_bounds__(PlaneThreads<R>::v) k_plane_f(cplx<R>* __restrict__ T, const R* __restrict__ Vs,
                                                                FastArgs fa, const cplx<R>* __restrict__ twxy) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  (void)twxy;
  fk::plane_body_pruned<R, N, PlaneThreads<R>::v>(T, Vs, fa, blockIdx.x, blockIdx.y, smem_raw);
}

template <typename R, int N3>
__global__ void __launch_bounds__(kThreads) k_zfwd_f(const cplx<R>* __restrict__ T, FastArgs fa,
                                                     const cplx<R>* __restrict__ twz,
                                                     const typename SphT<R>::type* __restrict__ K,
                                                     LocalEpi<typename SphT<R>::type> ep) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fk::zfwd_body<R, N3>(T, fa, twz, K, ep, blockIdx.x * kCBF, blockIdx.y, smem_raw);
}

template <typename R> void set_smem(const void* f, size_t bytes) {
  CHEBFI_CUDA(cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

}  // namespace

size_t local_workspace_elems(const chebfi_ctx* ctx, int64_t nb) {
  const int ncolp = (ctx->sph.ncol + 15) / 16 * 16;
  return (size_t)ctx->grid[2] * ncolp * (size_t)nb;
}

template <typename R> const R* vtable(const chebfi_ctx* c);
template <> const float* vtable<float>(const chebfi_ctx* c) { return c->d_vsf.p; }
template <> const double* vtable<double>(const chebfi_ctx* c) { return c->d_vs.p; }
template <> const dfl* vtable<dfl>(const chebfi_ctx* c) { return reinterpret_cast<const dfl*>(c->d_vsdf.p); }

template <typename R, int N>
void fast_launch(chebfi_ctx* ctx, const cplx<typename SphT<R>::type>* Y, int64_t ldy, int64_t nb, cplx<R>* T,
                 LocalEpi<typename SphT<R>::type> ep, cudaStream_t st, const typename SphT<R>::type* K) {
  using S = typename SphT<R>::type;
  const SphereFFT& s = ctx->sph;
  FastArgs fa;
  fa.ncol = s.ncol;
  fa.nxa = s.nxa;
  fa.pitch = s.pitch;
  fa.zpitch = s.zpitch;
  fa.ncolp = (s.ncol + 15) / 16 * 16;
  fa.ldt = (int64_t)N * fa.ncolp;
  fa.col_start = s.col_start.p;
  fa.pw_line = s.pw_line.p;
  fa.pw_z = s.pw_z.p;
  fa.col_off = s.col_off_nat.p;
  fa.row_off = s.rows_nat.p;
  fa.row_col = s.row_col.p;
  fa.act_lo = s.act_lo;
  fa.nact = s.nact;
  // ceil(2^32 / nact): exact quotients t / nact for t < 2^32 / nact (the row passes use t < 2^12)
  fa.nl_magic = s.nact > 1 ? (unsigned)(((1ull << 32) + s.nact - 1) / (unsigned long long)s.nact) : 0u;
  CHEBFI_REQUIRE(s.nxa >= 1 && s.nact >= 1, CHEBFI_ERR_STATE, "sphere without columns");
  CHEBFI_REQUIRE(s.pitch == N + 1, CHEBFI_ERR_STATE, "plane pitch of the compile-time path");
  const cplx<R>* tw = nullptr;  // the passes read their twiddles from constant tables
  const R* Vs = vtable<R>(ctx);
  const size_t zbytes = (size_t)(N + kCBF * s.zpitch) * sizeof(cplx<R>);
  const size_t pbytes = (size_t)(N + N * s.pitch) * sizeof(cplx<R>);
  fk::init_twiddles();
  set_smem<R>((const void*)k_plane_f<R, N>, pbytes);
  set_smem<R>((const void*)k_zinv_f<R, N>, zbytes);
  set_smem<R>((const void*)k_zfwd_f<R, N>, zbytes);
  for (int64_t b0 = 0; b0 < nb; b0 += 65535) {
    const int nbc = (int)std::min<int64_t>(65535, nb - b0);
    dim3 gz((s.ncol + kCBF - 1) / kCBF, nbc);
    const double esz = sizeof(cplx<R>), col = (double)N * s.ncol * nbc * esz, sph = (double)ctx->npw * nbc * esz;
    CHEBFI_LAUNCH_W("k_zinv", st, sph + col, k_zinv_f<R, N><<<gz, kThreads, zbytes, st>>>(Y + b0 * ldy, ldy, T, fa, tw));
    CHEBFI_LAUNCH_W("k_plane", st, 2.0 * col,
                    k_plane_f<R, N><<<dim3(N, nbc), PlaneThreads<R>::v, pbytes, st>>>(T, Vs, fa, tw));
    LocalEpi<S> e = ep;
    e.Y = ep.Y + b0 * ep.ldy;
    if (e.Z) e.Z = ep.Z + b0 * ep.ldz;
    if (e.Zhi) {
      e.Zhi = ep.Zhi + b0 * ep.ldzb;
      e.Zlo = ep.Zlo + b0 * ep.ldzb;
    }
    if (e.T) e.T = ep.T + b0 * ep.ldt;
    if (e.Yprev) e.Yprev = ep.Yprev + b0 * ep.ldt;
    e.inv_n3 = (S)(1.0 / ((double)N * N * N));
    const double epi = sph * (1.0 + (e.Z ? 1.0 : 0.0) + (e.T ? 1.0 : 0.0) + (e.Yprev ? 1.0 : 0.0)) +
                       (e.Zhi ? (double)ctx->npw * nbc * (e.zplane ? 12.0 : 8.0) : 0.0);
    CHEBFI_LAUNCH_W("k_zfwd", st, col + epi, k_zfwd_f<R, N><<<gz, kThreads, zbytes, st>>>(T, fa, tw, K, e));
  }
}

// Compile-time-length path for cubic grids of the supported sizes; false = not taken.
template <typename R>
bool fast_dispatch(chebfi_ctx* ctx, const cplx<typename SphT<R>::type>* Y, int64_t ldy, int64_t nb, cplx<R>* T,
                   LocalEpi<typename SphT<R>::type> ep, cudaStream_t st, const typename SphT<R>::type* K) {
  switch (ctx->grid[0]) {
    case 24: fast_launch<R, 24>(ctx, Y, ldy, nb, T, ep, st, K); return true;
    case 32: fast_launch<R, 32>(ctx, Y, ldy, nb, T, ep, st, K); return true;
    case 48: fast_launch<R, 48>(ctx, Y, ldy, nb, T, ep, st, K); return true;
    case 64: fast_launch<R, 64>(ctx, Y, ldy, nb, T, ep, st, K); return true;
    case 72: fast_launch<R, 72>(ctx, Y, ldy, nb, T, ep, st, K); return true;
    case 96: fast_launch<R, 96>(ctx, Y, ldy, nb, T, ep, st, K); return true;
    default: return false;
  }
}
// The FP64 path runs its transforms in double-float on the FP32 units unless the FP64 units
// are asked for (chebfi_set_fft64); the column buffer's complex doubles then hold
// double-float values, 16 bytes each as well.
template <typename R>
bool fast_apply(chebfi_ctx* ctx, const cplx<R>* Y, int64_t ldy, int64_t nb, cplx<R>* T, LocalEpi<R> ep,
                cudaStream_t st, const R* K) {
  if constexpr (std::is_same<R, double>::value) {
    if (ctx->fft64 == CHEBFI_FFT64_DOUBLE_FLOAT)
      return fast_dispatch<dfl>(ctx, Y, ldy, nb, reinterpret_cast<cdf*>(T), ep, st, K);
  }
  return fast_dispatch<R>(ctx, Y, ldy, nb, T, ep, st, K);
}

bool fast_fft_supported(int n1, int n2, int n3) {
  if (n1 != n2 || n1 != n3) return false;
  switch (n1) {
    case 24: case 32: case 48: case 64: case 72: case 96: return true;
    default: return false;
  }
}

int split_index(int n, int p) {
  switch (n) {
    case 24: return fast::split_index<24>(p);
    case 32: return fast::split_index<32>(p);
    case 48: return fast::split_index<48>(p);
    case 64: return fast::split_index<64>(p);
    case 72: return fast::split_index<72>(p);
    case 96: return fast::split_index<96>(p);
    default: return p;
  }
}

// (K + V_loc) applied to nb bands of sorted-order coefficients Y; the column buffer T
// must hold local_workspace_elems(ctx, nb) complex values.
template <typename R>
void local_apply(chebfi_ctx* ctx, const cplx<R>* Y, int64_t ldy, int64_t nb, cplx<R>* T,
                 LocalEpi<R> ep, cudaStream_t st) {
  if (nb <= 0) return;
  const SphereFFT& s = ctx->sph;
  SphArgs sa;
  sa.ncol = s.ncol;
  sa.n3 = s.n3;
  sa.zpitch = s.zpitch;
  sa.ncolp = (s.ncol + 15) / 16 * 16;
  sa.ldt = (int64_t)s.n3 * sa.ncolp;
  sa.col_start = s.col_start.p;
  sa.pw_line = s.pw_line.p;
  sa.pw_zrev = s.pw_zrev.p;
  PlaneArgs pa;
  pa.n1 = s.n1;
  pa.n2 = s.n2;
  pa.n3 = s.n3;
  pa.ncol = s.ncol;
  pa.nxa = s.nxa;
  pa.pitch = s.pitch;
  pa.ldt = sa.ldt;
  pa.ncolp = sa.ncolp;
  pa.col_off = s.col_off.p;
  pa.row_off = s.rows_act.p;
  const FFTPlan<R> px = ctx->ax[0].plan<R>(), py = ctx->ax[1].plan<R>(), pz = ctx->ax[2].plan<R>();
  const size_t zbytes = (size_t)kCB * s.zpitch * sizeof(cplx<R>);
  const size_t pbytes = (size_t)s.n1 * s.pitch * sizeof(cplx<R>);
  CHEBFI_REQUIRE(pbytes <= 227 * 1024, CHEBFI_ERR_ARG, "FFT plane does not fit in shared memory");
  set_smem<R>((const void*)k_plane<R>, pbytes);
  set_smem<R>((const void*)k_zinv<R>, zbytes);
  set_smem<R>((const void*)k_zfwd<R>, zbytes);
  const R* K = sizeof(R) == 8 ? (const R*)ctx->d_K.p : (const R*)ctx->d_Kf.p;
  const R* V = sizeof(R) == 8 ? (const R*)ctx->d_vt.p : (const R*)ctx->d_vtf.p;
  if (ctx->fast_fft && fast_apply<R>(ctx, Y, ldy, nb, T, ep, st, K)) return;
  // grid.y is limited to 65535: walk the bands in chunks
  for (int64_t b0 = 0; b0 < nb; b0 += 65535) {
    const int nbc = (int)std::min<int64_t>(65535, nb - b0);
    dim3 gz((s.ncol + kCB - 1) / kCB, nbc);
    const double esz = sizeof(cplx<R>), col = (double)s.n3 * s.ncol * nbc * esz, sph = (double)ctx->npw * nbc * esz;
    CHEBFI_LAUNCH_W("k_zinv", st, sph + col, k_zinv<R><<<gz, kThreads, zbytes, st>>>(Y + b0 * ldy, ldy, T, sa, pz));
    CHEBFI_LAUNCH_W("k_plane", st, 2.0 * col, k_plane<R><<<dim3(s.n3, nbc), kThreads, pbytes, st>>>(T, V, pa, px, py));
    LocalEpi<R> e = ep;
    e.Y = ep.Y + b0 * ep.ldy;
    if (e.Z) e.Z = ep.Z + b0 * ep.ldz;
    if (e.Zhi) {
      e.Zhi = ep.Zhi + b0 * ep.ldzb;
      e.Zlo = ep.Zlo + b0 * ep.ldzb;
    }
    if (e.T) e.T = ep.T + b0 * ep.ldt;
    if (e.Yprev) e.Yprev = ep.Yprev + b0 * ep.ldt;
    e.inv_n3 = (R)(1.0 / ((double)s.n1 * s.n2 * s.n3));
    // column buffer in, Y in, and the epilogue's sphere reads and writes
    const double epi = sph * (1.0 + (e.Z ? 1.0 : 0.0) + (e.T ? 1.0 : 0.0) + (e.Yprev ? 1.0 : 0.0)) +
                       (e.Zhi ? (double)ctx->npw * nbc * (e.zplane ? 12.0 : 8.0) : 0.0);
    CHEBFI_LAUNCH_W("k_zfwd", st, col + epi, k_zfwd<R><<<gz, kThreads, zbytes, st>>>(T, sa, pz, K, e));
  }
}

template <typename R>
void vloc_gradient(chebfi_ctx* ctx, const cplx<R>* Ys, const cplx<R>* Gs, int64_t nb, double* gV, cudaStream_t st,
                   DevBuf<cplx<R>>& T, DevBuf<cplx<R>>& Rb, DevBuf<cplx<R>>& Gb, double scale, bool accumulate) {
  const SphereFFT& s = ctx->sph;
  const int n1 = s.n1, n2 = s.n2, n3 = s.n3;
  const int64_t n = (int64_t)n1 * n2 * n3;
  if (!accumulate) CHEBFI_CUDA(cudaMemsetAsync(gV, 0, sizeof(double) * n, st));
  if (nb <= 0) return;
  SphArgs sa;
  sa.ncol = s.ncol;
  sa.n3 = s.n3;
  sa.zpitch = s.zpitch;
  sa.ncolp = (s.ncol + 15) / 16 * 16;
  sa.ldt = (int64_t)s.n3 * sa.ncolp;
  sa.col_start = s.col_start.p;
  sa.pw_line = s.pw_line.p;
  sa.pw_zrev = s.pw_zrev.p;
  PlaneArgs pa;
  pa.n1 = n1;
  pa.n2 = n2;
  pa.n3 = n3;
  pa.ncol = s.ncol;
  pa.nxa = s.nxa;
  pa.pitch = s.pitch;
  pa.ldt = sa.ldt;
  pa.ncolp = sa.ncolp;
  pa.col_off = s.col_off.p;
  pa.row_off = s.rows_act.p;
  const FFTPlan<R> px = ctx->ax[0].plan<R>(), py = ctx->ax[1].plan<R>(), pz = ctx->ax[2].plan<R>();
  const size_t zbytes = (size_t)kCB * s.zpitch * sizeof(cplx<R>);
  const size_t pbytes = (size_t)n1 * s.pitch * sizeof(cplx<R>);
  CHEBFI_REQUIRE(pbytes <= 227 * 1024, CHEBFI_ERR_ARG, "FFT plane does not fit in shared memory");
  set_smem<R>((const void*)k_zinv<R>, zbytes);
  set_smem<R>((const void*)k_plane_real<R>, pbytes);
  // bands per chunk: two full grids per band, at most ~512 MB of grids
  const int64_t chunk = std::max<int64_t>(1, std::min<int64_t>(nb, ((int64_t)1 << 25) / n));
  T.alloc((size_t)sa.ldt * chunk);
  Rb.alloc((size_t)n * chunk);
  Gb.alloc((size_t)n * chunk);
  for (int64_t b0 = 0; b0 < nb; b0 += chunk) {
    const int nbc = (int)std::min<int64_t>(chunk, nb - b0);
    dim3 gz((s.ncol + kCB - 1) / kCB, nbc);
    for (int which = 0; which < 2; ++which) {
      const cplx<R>* src = (which == 0 ? Ys : Gs) + b0 * ctx->npw;
      cplx<R>* dst = which == 0 ? Rb.p : Gb.p;
      CHEBFI_LAUNCH("k_zinv", st, k_zinv<R><<<gz, kThreads, zbytes, st>>>(src, ctx->npw, T.p, sa, pz));
      CHEBFI_LAUNCH("k_plane_real", st,
                    k_plane_real<R><<<dim3(n3, nbc), kThreads, pbytes, st>>>(T.p, pa, px, py, dst));
    }
    CHEBFI_LAUNCH("k_density_accum", st,
                  k_density_accum<R><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n1, n2, n3, nbc, Rb.p, Gb.p,
                                                                                    scale / (double)n, gV));
  }
}

template void vloc_gradient<double>(chebfi_ctx*, const double2*, const double2*, int64_t, double*, cudaStream_t,
                                    DevBuf<double2>&, DevBuf<double2>&, DevBuf<double2>&, double, bool);
template void vloc_gradient<float>(chebfi_ctx*, const float2*, const float2*, int64_t, double*, cudaStream_t,
                                   DevBuf<float2>&, DevBuf<float2>&, DevBuf<float2>&, double, bool);
template void local_apply<double>(chebfi_ctx*, const double2*, int64_t, int64_t, double2*, LocalEpi<double>, cudaStream_t);
template void local_apply<float>(chebfi_ctx*, const float2*, int64_t, int64_t, float2*, LocalEpi<float>, cudaStream_t);

}  // namespace chebfi
