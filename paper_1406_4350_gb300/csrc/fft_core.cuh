// In-place mixed-radix (2, 3, 4, 5) FFT stages on complex lines held in shared memory.
//
// Used by the local-potential operator of Section 2.1 (inverse FFT to real space,
// multiply by V_loc, forward FFT back).  Two in-place schemes, chosen so that neither
// needs a separate reordering pass:
//   * decimation in time (DIT) reads its input in digit-reversed order and writes the
//     transform in natural order;
//   * decimation in frequency (DIF) reads natural order and writes digit-reversed order.
// With radices r_1..r_k (DIT stage order, DIF runs them backwards) the digit-reversed
// position of index i puts the base-r_k digit of i (least significant) at weight
// N/r_k, the base-r_{k-1} digit at weight N/(r_k r_{k-1}), ..., the base-r_1 digit at 1.
//
// One stage is a loop over (line, butterfly) pairs, written as a function of
// (thread id, thread count) so the same code runs inside a kernel (followed by a block
// barrier) and on the host for index checks.
#pragma once

#include "internal.cuh"

namespace chebfi {

__host__ __device__ __forceinline__ float half_of(float v) { return 0.5f * v; }
__host__ __device__ __forceinline__ double half_of(double v) { return 0.5 * v; }

// Component-wise helpers of the codelets; the double-float complex type overloads them
// (dfloat.cuh) with packed FP32x2 arithmetic on its (Re, Im) pairs.
template <typename C> __host__ __device__ __forceinline__ C chalf(C a) {  // a / 2, exact
  C r;
  r.x = half_of(a.x);
  r.y = half_of(a.y);
  return r;
}
template <int SIGN, typename C, typename R> __host__ __device__ __forceinline__ C cmul_i(C d, R h) {  // SIGN i h d
  C u;
  u.x = h * d.y;
  u.y = h * d.x;
  if (SIGN > 0) u.x = -u.x;
  else u.y = -u.y;
  return u;
}
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) {  // s a, s real
  a.x *= s;
  a.y *= s;
  return a;
}

// r-point DFT out_p = sum_q x_q w^{pq}, w = exp(SIGN 2 pi i / r), in place.
template <int SIGN, typename C>
__host__ __device__ __forceinline__ void small_dft(C* x, int r) {
  using R = decltype(x[0].x);
  if (r == 2) {
    C a = x[0], b = x[1];
    x[0] = a + b;
    x[1] = a - b;
  } else if (r == 4) {
    C a = x[0] + x[2], b = x[0] - x[2], c = x[1] + x[3], d = x[1] - x[3];
    // w d with w = SIGN i
    C wd;
    if (SIGN > 0) {
      wd.x = -d.y;
      wd.y = d.x;
    } else {
      wd.x = d.y;
      wd.y = -d.x;
    }
    x[0] = a + c;
    x[2] = a - c;
    x[1] = b + wd;
    x[3] = b - wd;
  } else if (r == 3) {
    const R h = (R)0.86602540378443864676;  // sqrt(3)/2
    C s = x[1] + x[2], d = x[1] - x[2];
    const C t = x[0] - chalf(s);
    const C u = cmul_i<SIGN>(d, h);  // SIGN i sqrt(3)/2 d
    x[0] = x[0] + s;
    x[1] = t + u;
    x[2] = t - u;
  } else {  // r == 5
    const R c1 = (R)0.30901699437494742410, c2 = (R)-0.80901699437494742410;
    const R s1 = (R)0.95105651629515357212, s2 = (R)0.58778525229247312917;
    C a1 = x[1] + x[4], b1 = x[1] - x[4], a2 = x[2] + x[3], b2 = x[2] - x[3];
    C t1, t2, u1, u2;
    t1.x = x[0].x + c1 * a1.x + c2 * a2.x;
    t1.y = x[0].y + c1 * a1.y + c2 * a2.y;
    t2.x = x[0].x + c2 * a1.x + c1 * a2.x;
    t2.y = x[0].y + c2 * a1.y + c1 * a2.y;
    // u1 = SIGN i (s1 b1 + s2 b2), u2 = SIGN i (s2 b1 - s1 b2)
    R v1x = s1 * b1.x + s2 * b2.x, v1y = s1 * b1.y + s2 * b2.y;
    R v2x = s2 * b1.x - s1 * b2.x, v2y = s2 * b1.y - s1 * b2.y;
    if (SIGN > 0) {
      u1.x = -v1y;
      u1.y = v1x;
      u2.x = -v2y;
      u2.y = v2x;
    } else {
      u1.x = v1y;
      u1.y = -v1x;
      u2.x = v2y;
      u2.y = -v2x;
    }
    x[0] = x[0] + a1 + a2;
    x[1] = t1 + u1;
    x[4] = t1 - u1;
    x[2] = t2 + u2;
    x[3] = t2 - u2;
  }
}

template <int SIGN, typename C>
__host__ __device__ __forceinline__ C twiddle(const C* tw, int k) {
  C w = tw[k];
  if (SIGN > 0) w.y = -w.y;
  return w;
}

// Lines: line l starts at buf + loff(l); element i of a line is at + i*es.
struct LineMap {
  const int* off = nullptr;  // explicit offsets, or
  int stride = 0;            // regular stride between lines
  __host__ __device__ __forceinline__ int operator()(int l) const { return off ? off[l] : l * stride; }
};

// One DIT stage s (0-based, radix plan.radix[s]).
template <int SIGN, typename R>
__host__ __device__ __forceinline__ void dit_stage(cplx<R>* buf, int nlines, LineMap lm, int es,
                                                   const FFTPlan<R>& pl, int s, int tid, int nthr) {
  int Lp = 1;
  for (int i = 0; i < s; ++i) Lp *= pl.radix[i];
  const int r = pl.radix[s], L = Lp * r, nbf = pl.n / r, tws = pl.n / L;
  const int total = nlines * nbf;
  for (int t = tid; t < total; t += nthr) {
    const int line = t % nlines, b = t / nlines;
    const int blk = b / Lp, j = b - blk * Lp;
    cplx<R>* a = buf + lm(line) + (blk * L + j) * es;
    cplx<R> x[5];
    x[0] = a[0];
    for (int q = 1; q < r; ++q) x[q] = a[q * Lp * es] * twiddle<SIGN>(pl.tw, q * j * tws);
    small_dft<SIGN>(x, r);
    for (int p = 0; p < r; ++p) a[p * Lp * es] = x[p];
  }
}

// One DIF stage; stages run s = nst-1 .. 0.
template <int SIGN, typename R>
__host__ __device__ __forceinline__ void dif_stage(cplx<R>* buf, int nlines, LineMap lm, int es,
                                                   const FFTPlan<R>& pl, int s, int tid, int nthr) {
  int L = pl.n;
  for (int i = pl.nst - 1; i > s; --i) L /= pl.radix[i];
  const int r = pl.radix[s], Ln = L / r, nbf = pl.n / r, tws = pl.n / L;
  const int total = nlines * nbf;
  for (int t = tid; t < total; t += nthr) {
    const int line = t % nlines, b = t / nlines;
    const int blk = b / Ln, j = b - blk * Ln;
    cplx<R>* a = buf + lm(line) + (blk * L + j) * es;
    cplx<R> x[5];
    for (int q = 0; q < r; ++q) x[q] = a[q * Ln * es];
    small_dft<SIGN>(x, r);
    a[0] = x[0];
    for (int p = 1; p < r; ++p) a[p * Ln * es] = x[p] * twiddle<SIGN>(pl.tw, p * j * tws);
  }
}

#ifdef __CUDACC__
// Whole transforms by the thread block (every thread must call; ends with a barrier).
template <int SIGN, typename R>
__device__ __forceinline__ void block_fft_dit(cplx<R>* buf, int nlines, LineMap lm, int es, const FFTPlan<R>& pl) {
  for (int s = 0; s < pl.nst; ++s) {
    dit_stage<SIGN, R>(buf, nlines, lm, es, pl, s, threadIdx.x, blockDim.x);
    __syncthreads();
  }
}
template <int SIGN, typename R>
__device__ __forceinline__ void block_fft_dif(cplx<R>* buf, int nlines, LineMap lm, int es, const FFTPlan<R>& pl) {
  for (int s = pl.nst - 1; s >= 0; --s) {
    dif_stage<SIGN, R>(buf, nlines, lm, es, pl, s, threadIdx.x, blockDim.x);
    __syncthreads();
  }
}
#endif

// Host helpers: radix plan and digit reversal (shared by the kernels' setup and the
// host-side index checks).
inline bool factor_radices(int n, std::vector<int>& rad) {
  rad.clear();
  int m = n;
  while (m % 4 == 0) { rad.push_back(4); m /= 4; }
  while (m % 2 == 0) { rad.push_back(2); m /= 2; }
  while (m % 3 == 0) { rad.push_back(3); m /= 3; }
  while (m % 5 == 0) { rad.push_back(5); m /= 5; }
  return m == 1 && (int)rad.size() <= kMaxStages;
}

inline std::vector<int> digit_reversal(int n, const std::vector<int>& rad) {
  std::vector<int> rev(n);
  for (int i = 0; i < n; ++i) {
    int m = i, w = n, pos = 0;
    for (int s = (int)rad.size() - 1; s >= 0; --s) {
      const int r = rad[s];
      const int d = m % r;
      m /= r;
      w /= r;
      pos += d * w;
    }
    rev[i] = pos;
  }
  return rev;
}

}  // namespace chebfi
