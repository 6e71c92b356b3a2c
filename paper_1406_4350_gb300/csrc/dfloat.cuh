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

#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
// The complex operations with the (Re, Im) pair of each part in one packed FP32x2 register
// pair: the same error-free transformations, in the same order, with one packed instruction
// for the two components (a difference is b (-1) + a, exact product, one rounding).
struct dfl2 {
  float2 h, l;  // (Re.h, Im.h), (Re.l, Im.l)
};
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ dfl2 pk(cdf a) { return dfl2{make_float2(a.x.h, a.y.h), make_float2(a.x.l, a.y.l)}; }
__device__ __forceinline__ cdf upk(dfl2 a) { return cdf{dfl(a.h.x, a.l.x), dfl(a.h.y, a.l.y)}; }
__device__ __forceinline__ dfl2 fast2sum2(float2 a, float2 b) {
  const float2 s = __fadd2_rn(a, b);
  return dfl2{s, f2sub(b, f2sub(s, a))};
}
__device__ __forceinline__ dfl2 add2(dfl2 a, dfl2 b) {
  const float2 s = __fadd2_rn(a.h, b.h);
  const float2 bb = f2sub(s, a.h);
  const float2 e = __fadd2_rn(f2sub(a.h, f2sub(s, bb)), f2sub(b.h, bb));
  return fast2sum2(s, __fadd2_rn(e, __fadd2_rn(a.l, b.l)));
}
__device__ __forceinline__ dfl2 mul2(dfl2 a, dfl2 b) {
  const float2 p = __fmul2_rn(a.h, b.h);
  float2 e = __ffma2_rn(a.h, b.h, make_float2(-p.x, -p.y));
  e = __ffma2_rn(a.h, b.l, e);
  e = __ffma2_rn(a.l, b.h, e);
  return fast2sum2(p, e);
}
__device__ __forceinline__ cdf operator+(cdf a, cdf b) { return upk(add2(pk(a), pk(b))); }
__device__ __forceinline__ cdf operator-(cdf a, cdf b) { return upk(add2(pk(a), pk(cdf{-b.x, -b.y}))); }
// (a.x b.x - a.y b.y, a.x b.y + a.y b.x): the products (a.x b.x, a.x b.y) and (a.y b.y, a.y b.x)
// as two packed products, then one packed sum with the first lane's sign flipped
__device__ __forceinline__ cdf operator*(cdf a, cdf b) {
  const dfl2 p1 = mul2(dfl2{make_float2(a.x.h, a.x.h), make_float2(a.x.l, a.x.l)}, pk(b));
  const dfl2 p2 = mul2(dfl2{make_float2(a.y.h, a.y.h), make_float2(a.y.l, a.y.l)},
                       dfl2{make_float2(b.y.h, b.x.h), make_float2(b.y.l, b.x.l)});
  return upk(add2(p1, dfl2{make_float2(-p2.h.x, p2.h.y), make_float2(-p2.l.x, p2.l.y)}));
}
// the codelets' helpers (fft_core.cuh): a / 2 (exact), SIGN i h d, s a
__device__ __forceinline__ cdf chalf(cdf a) {
  const dfl2 v = pk(a);
  return upk(dfl2{__fmul2_rn(v.h, make_float2(0.5f, 0.5f)), __fmul2_rn(v.l, make_float2(0.5f, 0.5f))});
}
template <int SIGN> __device__ __forceinline__ cdf cmul_i(cdf d, dfl h) {
  // (h d.y, h d.x), then the sign of one lane: (-h d.y, h d.x) = i h d, (h d.y, -h d.x) = -i h d
  const dfl2 q = mul2(dfl2{make_float2(h.h, h.h), make_float2(h.l, h.l)},
                      dfl2{make_float2(d.y.h, d.x.h), make_float2(d.y.l, d.x.l)});
  return SIGN > 0 ? cdf{dfl(-q.h.x, -q.l.x), dfl(q.h.y, q.l.y)} : cdf{dfl(q.h.x, q.l.x), dfl(-q.h.y, -q.l.y)};
}
__device__ __forceinline__ cdf cscale(cdf a, dfl s) {
  return upk(mul2(pk(a), dfl2{make_float2(s.h, s.h), make_float2(s.l, s.l)}));  // a.x s, a.y s
}
#else
__device__ __forceinline__ cdf operator+(cdf a, cdf b) { return cdf{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ cdf operator-(cdf a, cdf b) { return cdf{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ cdf operator*(cdf a, cdf b) { return cdf{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
#endif
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
