// Bodies of the compile-time-length FFT passes of the local-potential operator (Section
// 2.1, Algorithm 1's V_loc psi): the z pass from the sphere to the column buffer, the plane
// pass (x and y transforms with the multiply by V_loc between them) and the z pass back to
// the sphere with the fused epilogue.  Shared by the single-problem kernels (fft.cu) and the
// batched k-point kernels (batch.cu), which differ only in how a block finds its problem.
//
// The inverse transforms leave real space in split order and the forward transforms read it
// back, so the z index of the column buffer and the plane's (x, y) are split positions; V_loc
// is stored in the same order.  Sphere points and columns are addressed at natural indices.
#pragma once

#include <cuda_bf16.h>

#include <cmath>
#include <vector>

#include "dfloat.cuh"
#include "fft_fast.cuh"
#include "internal.cuh"
#include "kernels.cuh"

namespace chebfi {
namespace fk {

constexpr int kThreadsF = 256;
constexpr int kCBF = 32;  // columns per z-pass block
static_assert(kThreadsF % kCBF == 0, "z-pass blocks are whole groups of kCBF threads");

struct FastArgs {
  int ncol, nxa, pitch, zpitch, ncolp;
  int64_t ldt;
  const int32_t* col_start;
  const int32_t* pw_line;
  const int32_t* pw_z;      // natural z of each sorted sphere point
  const int32_t* col_off;   // slot(x) * pitch + y of each column (plane rows cyclically shifted)
  const int32_t* row_off;   // slot(x) * pitch of each active x
  const int32_t* row_col = nullptr;            // (row act_lo + a, natural y) -> column, or -1
  int act_lo = 0, nact = 0;                    // slot range of the pruned plane pass
  unsigned nl_magic = 0;                       // t / nact == umulhi(t, nl_magic) for t < 2^16
};

template <typename R, int N>
__device__ __forceinline__ void load_tw(cplx<R>* s, const cplx<R>* g) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) s[i] = g[i];
}

// Twiddle tables tw[e] = exp(-2 pi i e / N) of the compiled line lengths, in constant memory:
// a warp of a pass reads one entry (two where it straddles two sub-transforms), which the
// constant cache broadcasts without using the shared-memory pipe that bounds these kernels.
// Each translation unit has its own copy, filled by init_twiddles before its first launch.
template <int N> struct TwOff;
template <> struct TwOff<24> { static constexpr int v = 0; };
template <> struct TwOff<32> { static constexpr int v = 24; };
template <> struct TwOff<48> { static constexpr int v = 56; };
template <> struct TwOff<64> { static constexpr int v = 104; };
template <> struct TwOff<72> { static constexpr int v = 168; };
template <> struct TwOff<96> { static constexpr int v = 240; };
constexpr int kTwTotal = 336;
static __constant__ float2 c_twf[kTwTotal];
static __constant__ double2 c_twd[kTwTotal];
static __constant__ float4 c_twdf[kTwTotal];  // double-float: (re.h, re.l, im.h, im.l)

template <typename R, int N> struct ConstTw;
template <int N> struct ConstTw<float, N> {
  __device__ __forceinline__ float2 operator()(int e) const { return c_twf[TwOff<N>::v + e]; }
};
template <int N> struct ConstTw<double, N> {
  __device__ __forceinline__ double2 operator()(int e) const { return c_twd[TwOff<N>::v + e]; }
};
template <int N> struct ConstTw<dfl, N> {
  __device__ __forceinline__ cdf operator()(int e) const {
    const float4 w = c_twdf[TwOff<N>::v + e];
    return cdf{dfl(w.x, w.y), dfl(w.z, w.w)};
  }
};

// Fill this translation unit's tables on the current device (once per device; not inside a
// stream capture).
static inline void init_twiddles() {
  static bool done[64] = {false};
  int dev = 0;
  CHEBFI_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64 || done[dev]) return;
  const int lens[6] = {24, 32, 48, 64, 72, 96};
  std::vector<float2> f;
  std::vector<double2> d;
  std::vector<float4> df;
  for (int n : lens)
    for (int k = 0; k < n; ++k) {
      const double a = 2.0 * M_PI * (double)k / (double)n;
      d.push_back(make_double2(std::cos(a), -std::sin(a)));
      f.push_back(make_float2((float)d.back().x, (float)d.back().y));
      const dfl re(d.back().x), im(d.back().y);
      df.push_back(make_float4(re.h, re.l, im.h, im.l));
    }
  CHEBFI_CUDA(cudaMemcpyToSymbol(c_twf, f.data(), sizeof(float2) * f.size()));
  CHEBFI_CUDA(cudaMemcpyToSymbol(c_twd, d.data(), sizeof(double2) * d.size()));
  CHEBFI_CUDA(cudaMemcpyToSymbol(c_twdf, df.data(), sizeof(float4) * df.size()));
  done[dev] = true;
}

// sphere block b, columns [c0, c0 + kCBF) -> inverse z transform -> column buffer T
template <typename R, int N3>
__device__ __forceinline__ void zinv_body(const cplx<typename SphT<R>::type>* __restrict__ Y, int64_t ldy,
                                          cplx<R>* __restrict__ T, const FastArgs& fa,
                                          const cplx<R>* __restrict__ twz, int c0, int64_t b,
                                          unsigned char* smem_raw) {
  (void)twz;
  const ConstTw<R, N3> tw;
  cplx<R>* lines = reinterpret_cast<cplx<R>*>(smem_raw) + N3;
  const int nc = min(kCBF, fa.ncol - c0);
  const cplx<R> zero = cmake<cplx<R>>(0.0, 0.0);
  for (int i = threadIdx.x; i < kCBF * fa.zpitch; i += blockDim.x) lines[i] = zero;
  __syncthreads();
  const int j0 = fa.col_start[c0], j1 = fa.col_start[c0 + nc];
  const auto* y = Y + b * ldy;
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x)
    lines[(fa.pw_line[j] - c0) * fa.zpitch + fa.pw_z[j]] = to_compute<cplx<R>>(y[j]);
  __syncthreads();
  LineMap lm;
  lm.stride = fa.zpitch;
  // a full block's line count is the compile-time kCBF (the passes' item decode divides by it)
  if (nc == kCBF) fast::lines_F<N3, +1>(lines, kCBF, lm, 1, tw);
  else fast::lines_F<N3, +1>(lines, nc, lm, 1, tw);
  cplx<R>* t = T + b * fa.ldt + c0;
  // lane l of each group of kCBF threads writes column l (blockDim.x is a multiple of kCBF)
  const int l = threadIdx.x % kCBF;
  if (l < nc)
    for (int z = threadIdx.x / kCBF; z < N3; z += blockDim.x / kCBF)
      t[(int64_t)z * fa.ncolp + l] = lines[l * fa.zpitch + z];
}

// plane z of block b: inverse y and x transforms, multiply by V_loc, forward x and y
template <typename R, int N>
__device__ __forceinline__ void plane_body(cplx<R>* __restrict__ T, const R* __restrict__ Vs, const FastArgs& fa,
                                           const cplx<R>* __restrict__ twxy, int z, int64_t b,
                                           unsigned char* smem_raw) {
  (void)twxy;
  const ConstTw<R, N> tw;
  cplx<R>* plane = reinterpret_cast<cplx<R>*>(smem_raw) + N;
  const cplx<R> zero = cmake<cplx<R>>(0.0, 0.0);
  for (int i = threadIdx.x; i < N * fa.pitch; i += blockDim.x) plane[i] = zero;
  __syncthreads();
  cplx<R>* t = T + b * fa.ldt + (int64_t)z * fa.ncolp;
  for (int c = threadIdx.x; c < fa.ncol; c += blockDim.x) plane[fa.col_off[c]] = t[c];
  __syncthreads();
  LineMap rows;
  rows.off = fa.row_off;
  LineMap cols;
  cols.stride = 1;
  fast::lines_F<N, +1>(plane, fa.nxa, rows, 1, tw);       // along y on the rows that hold columns
  // along x on every y: F's pass A; then, per contiguous group, F's pass B, the multiply by
  // V_loc and G's pass B in registers; then G's pass A
  fast::F_passA<N, +1>(plane, N, cols, fa.pitch, tw, threadIdx.x, blockDim.x);
  __syncthreads();
  {
    constexpr int NA = fast::Plan<N>::NA, NB = fast::Plan<N>::NB;
    const R* v = Vs + (int64_t)z * N * N;
    for (int it = threadIdx.x; it < N * NA; it += blockDim.x) {
      const int ka = it / N, yy = it - ka * N;
      cplx<R>* a = plane + yy + NB * ka * fa.pitch;
      const R* vv = v + (NB * ka) * N + yy;
      cplx<R> u[NB];
#pragma unroll
      for (int nb = 0; nb < NB; ++nb) u[nb] = a[nb * fa.pitch];
      fast::dft<NB, +1>(u);
#pragma unroll
      for (int kb = 0; kb < NB; ++kb) {
        const R s = vv[kb * N];
        u[kb] = cscale(u[kb], s);
      }
      fast::dft<NB, -1>(u);
#pragma unroll
      for (int nb = 0; nb < NB; ++nb)
        a[nb * fa.pitch] = (ka == 0 || nb == 0) ? u[nb] : u[nb] * fast::twN<-1>(tw, nb * ka);
    }
  }
  __syncthreads();
  fast::G_passA<N, -1>(plane, N, cols, fa.pitch, threadIdx.x, blockDim.x);
  __syncthreads();
  fast::lines_G<N, -1>(plane, fa.nxa, rows, 1, tw);       // along y on the needed rows
  for (int c = threadIdx.x; c < fa.ncol; c += blockDim.x) t[c] = plane[fa.col_off[c]];
}

// The plane pass of plane_body with its zero rows pruned and its scatter / gather fused:
// the first y pass reads the sphere columns straight from the column buffer (no zeroed
// plane, no scatter), the x passes skip the loads of rows outside the active slot range
// [act_lo, act_lo + nact) (they are zero) and the stores of rows no later pass reads, and
// the last y pass stores the columns straight to the column buffer (no gather).  Same
// arithmetic, in the same order.  The row pitch is the compile-time N + 1 (odd: the
// row-wise passes meet no bank conflicts), so every shared-memory offset of a pass is an
// immediate; where the block's NT / 32 warps are a multiple of NB (N = 64, 96) each warp of
// an x pass keeps one nb and its twiddles in registers.
template <typename R, int N, int NT = kThreadsF>
__device__ __forceinline__ void plane_body_pruned(cplx<R>* __restrict__ T, const R* __restrict__ Vs,
                                                  const FastArgs& fa, int z, int64_t b, unsigned char* smem_raw) {
  using C = cplx<R>;
  constexpr int NA = fast::Plan<N>::NA, NB = fast::Plan<N>::NB, P = N + 1, W = NT / 32;
  constexpr bool kWarpNb = N % 32 == 0 && W % NB == 0;
  const ConstTw<R, N> tw;
  C* plane = reinterpret_cast<C*>(smem_raw) + N;
  const C zero = cmake<C>(0.0, 0.0);
  C* t = T + b * fa.ldt + (int64_t)z * fa.ncolp;
  const int nl = fa.nact, lo = fa.act_lo;
  C* rows = plane + lo * P;  // row a of the active range
  // y, inverse: F's pass A on the active rows, its inputs read from the column buffer;
  // consecutive threads take consecutive y of one row, so they read consecutive columns
  if constexpr (NT % NB == 0) {
    // blockDim.x (NT) is a multiple of NB, so every item of this thread has the same nb: its
    // twiddles are read once (a warp's threads hold NB different nb)
    const int nb = threadIdx.x % NB;
    C w[NA];
#pragma unroll
    for (int ka = 1; ka < NA; ++ka) w[ka] = fast::twN<+1>(tw, nb * ka);
    for (int it = threadIdx.x; it < nl * NB; it += blockDim.x) {
      const int a = it / NB;
      C* row = rows + a * P + nb;
      const int32_t* rc = fa.row_col + a * N + nb;
      C v[NA];
#pragma unroll
      for (int na = 0; na < NA; ++na) {
        const int c = __ldg(rc + NB * na);
        v[na] = c >= 0 ? t[c] : zero;
      }
      fast::dft<NA, +1>(v);
      row[0] = v[0];
#pragma unroll
      for (int ka = 1; ka < NA; ++ka) row[NB * ka] = v[ka] * w[ka];
    }
  } else {
    // NB = 6 with a 256-thread block: an item's nb and twiddles are its own
    for (int it = threadIdx.x; it < nl * NB; it += blockDim.x) {
      const int a = it / NB, nb = it - a * NB;
      C* row = rows + a * P + nb;
      const int32_t* rc = fa.row_col + a * N + nb;
      C v[NA];
#pragma unroll
      for (int na = 0; na < NA; ++na) {
        const int c = __ldg(rc + NB * na);
        v[na] = c >= 0 ? t[c] : zero;
      }
      fast::dft<NA, +1>(v);
      row[0] = v[0];
#pragma unroll
      for (int ka = 1; ka < NA; ++ka) row[NB * ka] = v[ka] * fast::twN<+1>(tw, nb * ka);
    }
  }
  __syncthreads();
  // F's pass B on the active rows: item t = (ka, row) with the row fastest (rows are an odd
  // pitch apart: no bank conflicts); ka = t / nl by the multiplier of fa.nl_magic
  for (int it = threadIdx.x; it < nl * NA; it += blockDim.x) {
    const int ka = nl == 1 ? it : (int)__umulhi((unsigned)it, fa.nl_magic), a = it - ka * nl;
    C* g = rows + a * P + NB * ka;
    C u[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) u[q] = g[q];
    fast::dft<NB, +1>(u);
#pragma unroll
    for (int q = 0; q < NB; ++q) g[q] = u[q];
  }
  __syncthreads();
  // x, inverse: F's pass A on every y line, slots outside the active range are zero
  if constexpr (kWarpNb) {
    const int warp = threadIdx.x / 32, nb = warp % NB, d = nb - lo;
    C w[NA];
#pragma unroll
    for (int ka = 1; ka < NA; ++ka) w[ka] = fast::twN<+1>(tw, nb * ka);
#pragma unroll 1
    for (int yy = threadIdx.x % 32 + 32 * (warp / NB); yy < N; yy += 32 * (W / NB)) {
      C* a = plane + yy + nb * P;
      C v[NA];
#pragma unroll
      for (int na = 0; na < NA; ++na) v[na] = (unsigned)(d + NB * na) < (unsigned)nl ? a[NB * na * P] : zero;
      fast::dft<NA, +1>(v);
      a[0] = v[0];
#pragma unroll
      for (int ka = 1; ka < NA; ++ka) a[NB * ka * P] = v[ka] * w[ka];
    }
  } else {
    for (int it = threadIdx.x; it < N * NB; it += blockDim.x) {
      const int nb = it / N, yy = it - nb * N, d = nb - lo;
      C* a = plane + yy + nb * P;
      C v[NA];
#pragma unroll
      for (int na = 0; na < NA; ++na) v[na] = (unsigned)(d + NB * na) < (unsigned)nl ? a[NB * na * P] : zero;
      fast::dft<NA, +1>(v);
#pragma unroll
      for (int ka = 0; ka < NA; ++ka) a[NB * ka * P] = ka == 0 ? v[0] : v[ka] * fast::twN<+1>(tw, nb * ka);
    }
  }
  __syncthreads();
  {
    // F's pass B, the multiply by V_loc and G's pass B, in registers per contiguous group
    const R* v = Vs + (int64_t)z * N * N;
    for (int it = threadIdx.x; it < N * NA; it += blockDim.x) {
      const int ka = it / N, yy = it - ka * N;
      C* a = plane + yy + NB * ka * P;
      const R* vv = v + (NB * ka) * N + yy;
      C u[NB];
#pragma unroll
      for (int nb = 0; nb < NB; ++nb) u[nb] = a[nb * P];
      fast::dft<NB, +1>(u);
#pragma unroll
      for (int kb = 0; kb < NB; ++kb) {
        const R s = vv[kb * N];
        u[kb] = cscale(u[kb], s);
      }
      fast::dft<NB, -1>(u);
#pragma unroll
      for (int nb = 0; nb < NB; ++nb)
        a[nb * P] = (ka == 0 || nb == 0) ? u[nb] : u[nb] * fast::twN<-1>(tw, nb * ka);
    }
  }
  __syncthreads();
  // x, forward: G's pass A, storing only the rows the y pass reads
  if constexpr (kWarpNb) {
    const int warp = threadIdx.x / 32, nb = warp % NB, d = nb - lo;
#pragma unroll 1
    for (int yy = threadIdx.x % 32 + 32 * (warp / NB); yy < N; yy += 32 * (W / NB)) {
      C* a = plane + yy + nb * P;
      C v[NA];
#pragma unroll
      for (int ka = 0; ka < NA; ++ka) v[ka] = a[NB * ka * P];
      fast::dft<NA, -1>(v);
#pragma unroll
      for (int na = 0; na < NA; ++na)
        if ((unsigned)(d + NB * na) < (unsigned)nl) a[NB * na * P] = v[na];
    }
  } else {
    for (int it = threadIdx.x; it < N * NB; it += blockDim.x) {
      const int nb = it / N, yy = it - nb * N, d = nb - lo;
      C* a = plane + yy + nb * P;
      C v[NA];
#pragma unroll
      for (int ka = 0; ka < NA; ++ka) v[ka] = a[NB * ka * P];
      fast::dft<NA, -1>(v);
#pragma unroll
      for (int na = 0; na < NA; ++na)
        if ((unsigned)(d + NB * na) < (unsigned)nl) a[NB * na * P] = v[na];
    }
  }
  __syncthreads();
  // y, forward: G's pass B, then G's pass A storing the columns to the column buffer
  for (int it = threadIdx.x; it < nl * NA; it += blockDim.x) {
    const int ka = nl == 1 ? it : (int)__umulhi((unsigned)it, fa.nl_magic), a = it - ka * nl;
    C* g = rows + a * P + NB * ka;
    C u[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) u[q] = g[q];
    fast::dft<NB, -1>(u);
#pragma unroll
    for (int q = 0; q < NB; ++q) g[q] = (ka == 0 || q == 0) ? u[q] : u[q] * fast::twN<-1>(tw, q * ka);
  }
  __syncthreads();
  for (int it = threadIdx.x; it < nl * NB; it += blockDim.x) {
    const int a = it / NB, nb = it - a * NB;  // consecutive columns per warp, as above
    const C* row = rows + a * P + nb;
    const int32_t* rc = fa.row_col + a * N + nb;
    C v[NA];
#pragma unroll
    for (int ka = 0; ka < NA; ++ka) v[ka] = row[NB * ka];
    fast::dft<NA, -1>(v);
#pragma unroll
    for (int na = 0; na < NA; ++na) {
      const int c = __ldg(rc + NB * na);
      if (c >= 0) t[c] = v[na];
    }
  }
}

// columns [c0, c0 + kCBF) of block b: forward z transform, back to the sphere, + K psi and
// the epilogue (Z, its bf16 planes, and the Chebyshev combination T = a (Z - c Y) - b Yprev)
template <typename R, int N3>
__device__ __forceinline__ void zfwd_body(const cplx<R>* __restrict__ T, const FastArgs& fa,
                                          const cplx<R>* __restrict__ twz,
                                          const typename SphT<R>::type* __restrict__ K,
                                          const LocalEpi<typename SphT<R>::type>& ep, int c0, int64_t b,
                                          unsigned char* smem_raw) {
  using CS = cplx<typename SphT<R>::type>;
  (void)twz;
  const ConstTw<R, N3> tw;
  cplx<R>* lines = reinterpret_cast<cplx<R>*>(smem_raw) + N3;
  const int nc = min(kCBF, fa.ncol - c0);
  const cplx<R>* t = T + b * fa.ldt + c0;
  {
    const int l = threadIdx.x % kCBF;  // as in the inverse pass
    if (l < nc)
      for (int z = threadIdx.x / kCBF; z < N3; z += blockDim.x / kCBF)
        lines[l * fa.zpitch + z] = t[(int64_t)z * fa.ncolp + l];
  }
  __syncthreads();
  LineMap lm;
  lm.stride = fa.zpitch;
  if (nc == kCBF) fast::lines_G<N3, -1>(lines, kCBF, lm, 1, tw);
  else fast::lines_G<N3, -1>(lines, nc, lm, 1, tw);
  const int j0 = fa.col_start[c0], j1 = fa.col_start[c0 + nc];
  const CS* y = ep.Y + b * ep.ldy;
  const R inv_n3 = to_compute<R>(ep.inv_n3), ea = to_compute<R>(ep.a), ec = to_compute<R>(ep.c),
          eb = to_compute<R>(ep.bprev);
  for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const cplx<R> v = lines[(fa.pw_line[j] - c0) * fa.zpitch + fa.pw_z[j]];
    const cplx<R> yj = to_compute<cplx<R>>(y[j]);
    const R k = to_compute<R>(K[j]);
    cplx<R> zj;
    zj.x = v.x * inv_n3 + k * yj.x;
    zj.y = v.y * inv_n3 + k * yj.y;
    if (ep.Z) ep.Z[b * ep.ldz + j] = to_store<CS>(zj);
    if (ep.Zhi) epi_split_z(ep, b, j, to_f32(zj.x), to_f32(zj.y));
    if (ep.T) {
      cplx<R> tp = cmake<cplx<R>>(0.0, 0.0);
      if (ep.Yprev) tp = to_compute<cplx<R>>(ep.Yprev[b * ep.ldt + j]);
      cplx<R> o;
      o.x = ea * (zj.x - ec * yj.x) - eb * tp.x;
      o.y = ea * (zj.y - ec * yj.y) - eb * tp.y;
      ep.T[b * ep.ldt + j] = to_store<CS>(o);
    }
  }
}

}  // namespace fk
}  // namespace chebfi
