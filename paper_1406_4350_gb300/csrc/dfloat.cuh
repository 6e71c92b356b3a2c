// Double-float ("double-word") arithmetic on the FP32 units, for the FFT of the FP64 form.
//
// GB300 issues FP64 FMAs at about 1/64 of its FP32 rate, so an FFT in FP64 is bound by the
// FP64 units.  A value here is the unevaluated sum h + l of two floats with |l| <= ulp(h)/2
// (a 48-bit significand with float's exponent range); the operations are the classical
// error-free transformations:
//   TwoSum (Knuth, TAOCP vol. 2, 4.2.2): s = fl(a + b) and the exact error e, a + b = s + e;
//   Fast2Sum (Dekker 1971): the same when |a| >= |b|, three operations;
//   TwoProd by FMA: p = fl(a b), e = fma(a, b, -p), a b = p + e exactly;
// combined into double-word addition (the "sloppy" variant: TwoSum of the high parts, the
// low parts added, one Fast2Sum; error at most about 2 u^2 (|a| + |b|), u = 2^-24) and
// multiplication (TwoProd of the high parts plus the two cross products, one Fast2Sum;
// relative error below 5 u^2), as analysed by Joldes, Muller and Popescu (2017).  An FFT is
// stable in the norm-wise sense, so the additions' bound in terms of |a| + |b| is the one
// that matters: a 96-point line transform keeps about 2^-44 of the line's norm.
// Every operation uses the _rn intrinsics, which the compiler neither contracts into FMAs
// nor reorders, so the transformations stay exact.
#pragma once

#include <cuda_runtime.h>

#include "internal.cuh"

namespace chebfi {

struct dfl {
  float h, l;
  dfl() = default;
  __host__ __device__ constexpr dfl(float hi, float lo) : h(hi), l(lo) {}
  // the nearest double-float to v (exact for |v| well inside float's range, up to 2^-48 v)
  __host__ __device__ constexpr dfl(double v) : h((float)v), l((float)(v - (double)(float)v)) {}
  __host__ __device__ constexpr dfl(int v) : h((float)v), l(0.f) {}
};

struct cdf {
  dfl x, y;
};
template <> struct cplx_t<dfl> { using type = cdf; };
template <> __host__ __device__ __forceinline__ cdf cmake<cdf>(double re, double im) {
  cdf z;
  z.x = dfl(re);
  z.y = dfl(im);
  return z;
}

#ifdef __CUDACC__
__device__ __forceinline__ dfl df_fast2sum(float a, float b) {  // |a| >= |b| (or a = 0)
  const float s = __fadd_rn(a, b);
  return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ dfl df_twosum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return dfl(s, e);
}
__device__ __forceinline__ dfl operator+(dfl a, dfl b) {
  const dfl s = df_twosum(a.h, b.h);
  return df_fast2sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dfl operator-(dfl a) { return dfl(-a.h, -a.l); }
__device__ __forceinline__ dfl operator-(dfl a, dfl b) { return a + (-b); }
__device__ __forceinline__ dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return df_fast2sum(p, e);
}
__device__ __forceinline__ dfl& operator*=(dfl& a, dfl b) { return a = a * b; }
__device__ __forceinline__ dfl& operator+=(dfl& a, dfl b) { return a = a + b; }
// exact scaling by 1/2
__device__ __forceinline__ dfl df_half(dfl a) { return dfl(0.5f * a.h, 0.5f * a.l); }

__device__ __forceinline__ cdf operator+(cdf a, cdf b) { return cdf{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cdf operator-(cdf a, cdf b) { return cdf{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cdf operator*(cdf a, cdf b) { return cdf{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ cdf conjg(cdf a) { return cdf{a.x, -a.y}; }

// conversions at the FP64 storage boundary (one FP64 add each way)
__device__ __forceinline__ dfl df_from(double v) {
  const float h = __double2float_rn(v);
  return dfl(h, __double2float_rn(v - (double)h));
}
__device__ __forceinline__ double df_to(dfl a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ cdf df_from(double2 v) { return cdf{df_from(v.x), df_from(v.y)}; }
__device__ __forceinline__ double2 df_to(cdf a) { return make_double2(df_to(a.x), df_to(a.y)); }
#endif

// Storage type of sphere-side data (wavefunction blocks, the kinetic diagonal) for an FFT
// computed in R: the same type, except FP64 blocks for the double-float FFT.
template <typename R> struct SphT { using type = R; };
template <> struct SphT<dfl> { using type = double; };

#ifdef __CUDACC__
// value conversions between the sphere storage type and the compute type
template <typename C, typename S> __device__ __forceinline__ C to_compute(S v) { return v; }
template <> __device__ __forceinline__ cdf to_compute<cdf, double2>(double2 v) { return df_from(v); }
template <> __device__ __forceinline__ dfl to_compute<dfl, double>(double v) { return df_from(v); }
template <typename S, typename C> __device__ __forceinline__ S to_store(C v) { return v; }
template <> __device__ __forceinline__ double2 to_store<double2, cdf>(cdf v) { return df_to(v); }
// the nearest float (the bf16 split of the mixed form reads its inputs as floats)
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(double v) { return (float)v; }
__device__ __forceinline__ float to_f32(dfl v) { return v.h; }
// exact halving (the float and double forms are in fft_core.cuh)
__device__ __forceinline__ dfl half_of(dfl v) { return df_half(v); }
#endif

}  // namespace chebfi
