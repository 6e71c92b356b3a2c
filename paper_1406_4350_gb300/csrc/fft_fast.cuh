// Two-pass line FFTs with compile-time lengths (register codelets), for the common grid
// sizes of the local-potential operator (Section 2.1).
//
// A line of length N = NA * NB is transformed in two in-place passes over shared memory:
//   F (natural in, "split" order out):  pass A does length-NA DFTs over the stride-NB
//     subsequences x[NB*na + nb] and multiplies by w^(nb*ka); pass B does length-NB DFTs over
//     the contiguous groups; position NB*ka + kb then holds X[ka + NA*kb].
//   G (split order in, natural out): the same passes in reverse order with the same twiddles
//     (the transpose of F, hence the DFT read from split order).
// The inverse transform to real space uses F and the forward transform back uses G, so every
// pass is in place and needs one barrier; the permutation only changes where real-space
// values sit, which the potential table accounts for (it is stored in split order).
#pragma once

#include "fft_core.cuh"

namespace chebfi {
namespace fast {

// cos(2 pi m / L), sin(2 pi m / L) for the composite codelet lengths
template <int L> struct SmallTw;
#define CHEBFI_R32 0.86602540378443864676
#define CHEBFI_R22 0.70710678118654752440
#define CHEBFI_C8 0.92387953251128675613
#define CHEBFI_S8 0.38268343236508977173
#define CHEBFI_C5a 0.30901699437494742410
#define CHEBFI_S5a 0.95105651629515357212
#define CHEBFI_C5b 0.80901699437494742410
#define CHEBFI_S5b 0.58778525229247312917
template <> struct SmallTw<6> {
  __host__ __device__ static double c(int m) {
    const double t[6] = {1, 0.5, -0.5, -1, -0.5, 0.5};
    return t[m];
  }
  __host__ __device__ static double s(int m) {
    const double t[6] = {0, CHEBFI_R32, CHEBFI_R32, 0, -CHEBFI_R32, -CHEBFI_R32};
    return t[m];
  }
};
template <> struct SmallTw<8> {
  __host__ __device__ static double c(int m) {
    const double t[8] = {1, CHEBFI_R22, 0, -CHEBFI_R22, -1, -CHEBFI_R22, 0, CHEBFI_R22};
    return t[m];
  }
  __host__ __device__ static double s(int m) {
    const double t[8] = {0, CHEBFI_R22, 1, CHEBFI_R22, 0, -CHEBFI_R22, -1, -CHEBFI_R22};
    return t[m];
  }
};
template <> struct SmallTw<10> {
  __host__ __device__ static double c(int m) {
    const double t[10] = {1, CHEBFI_C5b, CHEBFI_C5a, -CHEBFI_C5a, -CHEBFI_C5b, -1, -CHEBFI_C5b, -CHEBFI_C5a, CHEBFI_C5a, CHEBFI_C5b};
    return t[m];
  }
  __host__ __device__ static double s(int m) {
    const double t[10] = {0, CHEBFI_S5b, CHEBFI_S5a, CHEBFI_S5a, CHEBFI_S5b, 0, -CHEBFI_S5b, -CHEBFI_S5a, -CHEBFI_S5a, -CHEBFI_S5b};
    return t[m];
  }
};
template <> struct SmallTw<12> {
  __host__ __device__ static double c(int m) {
    const double t[12] = {1, CHEBFI_R32, 0.5, 0, -0.5, -CHEBFI_R32, -1, -CHEBFI_R32, -0.5, 0, 0.5, CHEBFI_R32};
    return t[m];
  }
  __host__ __device__ static double s(int m) {
    const double t[12] = {0, 0.5, CHEBFI_R32, 1, CHEBFI_R32, 0.5, 0, -0.5, -CHEBFI_R32, -1, -CHEBFI_R32, -0.5};
    return t[m];
  }
};
template <> struct SmallTw<16> {
  __host__ __device__ static double c(int m) {
    const double t[16] = {1, CHEBFI_C8, CHEBFI_R22, CHEBFI_S8, 0, -CHEBFI_S8, -CHEBFI_R22, -CHEBFI_C8,
                          -1, -CHEBFI_C8, -CHEBFI_R22, -CHEBFI_S8, 0, CHEBFI_S8, CHEBFI_R22, CHEBFI_C8};
    return t[m];
  }
  __host__ __device__ static double s(int m) {
    const double t[16] = {0, CHEBFI_S8, CHEBFI_R22, CHEBFI_C8, 1, CHEBFI_C8, CHEBFI_R22, CHEBFI_S8,
                          0, -CHEBFI_S8, -CHEBFI_R22, -CHEBFI_C8, -1, -CHEBFI_C8, -CHEBFI_R22, -CHEBFI_S8};
    return t[m];
  }
};

template <int L> struct Split;  // L = A * B for the composite codelets
template <> struct Split<6> { static constexpr int A = 2, B = 3; };
template <> struct Split<8> { static constexpr int A = 2, B = 4; };
template <> struct Split<10> { static constexpr int A = 2, B = 5; };
template <> struct Split<12> { static constexpr int A = 4, B = 3; };
template <> struct Split<16> { static constexpr int A = 4, B = 4; };

// In-register DFT of length L, natural order in and out: X[k] = sum_n x[n] exp(SIGN 2 pi i nk/L).
template <int L, int SIGN, typename C> __host__ __device__ __forceinline__ void dft(C* x) {
  if constexpr (L == 1) {
  } else if constexpr (L <= 5) {
    small_dft<SIGN>(x, L);
  } else {
    constexpr int A = Split<L>::A, B = Split<L>::B;
    C y[L];
#pragma unroll
    for (int nb = 0; nb < B; ++nb) {
      C t[A];
#pragma unroll
      for (int na = 0; na < A; ++na) t[na] = x[B * na + nb];
      dft<A, SIGN>(t);
#pragma unroll
      for (int ka = 0; ka < A; ++ka) {
        const int e = (nb * ka) % L;
        if (e == 0) {
          y[ka * B + nb] = t[ka];
        } else if ((4 * e) % L == 0) {  // a quarter turn: w = (SIGN i)^q, a rotation
          const int q = (((4 * e) / L) * (SIGN > 0 ? 1 : 3)) % 4;
          const C v = t[ka];
          C r;
          if (q == 1) {
            r.x = -v.y;
            r.y = v.x;
          } else if (q == 2) {
            r.x = -v.x;
            r.y = -v.y;
          } else {
            r.x = v.y;
            r.y = -v.x;
          }
          y[ka * B + nb] = r;
        } else {
          const C w = cmake<C>(SmallTw<L>::c(e), SIGN * SmallTw<L>::s(e));
          y[ka * B + nb] = t[ka] * w;
        }
      }
    }
#pragma unroll
    for (int ka = 0; ka < A; ++ka) {
      C u[B];
#pragma unroll
      for (int nb = 0; nb < B; ++nb) u[nb] = y[ka * B + nb];
      dft<B, SIGN>(u);
#pragma unroll
      for (int kb = 0; kb < B; ++kb) x[ka + A * kb] = u[kb];
    }
  }
}

// Two-factor plan of a line length.
template <int N> struct Plan;
template <> struct Plan<16> { static constexpr int NA = 4, NB = 4; };
template <> struct Plan<24> { static constexpr int NA = 4, NB = 6; };
template <> struct Plan<32> { static constexpr int NA = 8, NB = 4; };
template <> struct Plan<48> { static constexpr int NA = 8, NB = 6; };
template <> struct Plan<64> { static constexpr int NA = 8, NB = 8; };
template <> struct Plan<72> { static constexpr int NA = 12, NB = 6; };
template <> struct Plan<96> { static constexpr int NA = 12, NB = 8; };
template <> struct Plan<120> { static constexpr int NA = 12, NB = 10; };
template <> struct Plan<128> { static constexpr int NA = 16, NB = 8; };
template <> struct Plan<144> { static constexpr int NA = 12, NB = 12; };

// twiddle w^e = exp(SIGN 2 pi i e / N) from the table tw[e] = exp(-2 pi i e / N), held in
// memory (a pointer) or behind an accessor object tw(e)
template <int SIGN, typename C> __host__ __device__ __forceinline__ C twN(const C* tw, int e) {
  C w = tw[e];
  if (SIGN > 0) w.y = -w.y;
  return w;
}
template <int SIGN, typename T>
__host__ __device__ __forceinline__ auto twN(const T& tw, int e) -> decltype(tw(e)) {
  auto w = tw(e);
  if (SIGN > 0) w.y = -w.y;
  return w;
}

// F: natural in, split order out (position NB*ka + kb holds X[ka + NA*kb]).
// Each pass is a loop over (line, sub-DFT) items of thread `tid` of `nthr`.
template <int N, int SIGN, typename C, typename TW>
__host__ __device__ __forceinline__ void F_passA(C* buf, int nlines, LineMap lm, int es, const TW& tw, int tid,
                                                 int nthr) {
  constexpr int NA = Plan<N>::NA, NB = Plan<N>::NB;
  for (int t = tid; t < nlines * NB; t += nthr) {
    const int nb = t / nlines, line = t - nb * nlines;
    C* a = buf + lm(line) + nb * es;
    C v[NA];
#pragma unroll
    for (int na = 0; na < NA; ++na) v[na] = a[NB * na * es];
    dft<NA, SIGN>(v);
#pragma unroll
    for (int ka = 0; ka < NA; ++ka) a[NB * ka * es] = ka == 0 ? v[0] : v[ka] * twN<SIGN>(tw, nb * ka);
  }
}
template <int N, int SIGN, typename C>
__host__ __device__ __forceinline__ void F_passB(C* buf, int nlines, LineMap lm, int es, int tid, int nthr) {
  constexpr int NA = Plan<N>::NA, NB = Plan<N>::NB;
  for (int t = tid; t < nlines * NA; t += nthr) {
    const int ka = t / nlines, line = t - ka * nlines;
    C* a = buf + lm(line) + NB * ka * es;
    C u[NB];
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) u[nb] = a[nb * es];
    dft<NB, SIGN>(u);
#pragma unroll
    for (int kb = 0; kb < NB; ++kb) a[kb * es] = u[kb];
  }
}
// G: split order in, natural out (the transpose of F: pass B, twiddles, pass A).
template <int N, int SIGN, typename C, typename TW>
__host__ __device__ __forceinline__ void G_passB(C* buf, int nlines, LineMap lm, int es, const TW& tw, int tid,
                                                 int nthr) {
  constexpr int NA = Plan<N>::NA, NB = Plan<N>::NB;
  for (int t = tid; t < nlines * NA; t += nthr) {
    const int ka = t / nlines, line = t - ka * nlines;
    C* a = buf + lm(line) + NB * ka * es;
    C u[NB];
#pragma unroll
    for (int kb = 0; kb < NB; ++kb) u[kb] = a[kb * es];
    dft<NB, SIGN>(u);
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) a[nb * es] = (ka == 0 || nb == 0) ? u[nb] : u[nb] * twN<SIGN>(tw, nb * ka);
  }
}
template <int N, int SIGN, typename C>
__host__ __device__ __forceinline__ void G_passA(C* buf, int nlines, LineMap lm, int es, int tid, int nthr) {
  constexpr int NA = Plan<N>::NA, NB = Plan<N>::NB;
  for (int t = tid; t < nlines * NB; t += nthr) {
    const int nb = t / nlines, line = t - nb * nlines;
    C* a = buf + lm(line) + nb * es;
    C v[NA];
#pragma unroll
    for (int ka = 0; ka < NA; ++ka) v[ka] = a[NB * ka * es];
    dft<NA, SIGN>(v);
#pragma unroll
    for (int na = 0; na < NA; ++na) a[NB * na * es] = v[na];
  }
}

#ifdef __CUDACC__
template <int N, int SIGN, typename C, typename TW>
__device__ __forceinline__ void lines_F(C* buf, int nlines, LineMap lm, int es, const TW& tw) {
  F_passA<N, SIGN>(buf, nlines, lm, es, tw, threadIdx.x, blockDim.x);
  __syncthreads();
  F_passB<N, SIGN>(buf, nlines, lm, es, threadIdx.x, blockDim.x);
  __syncthreads();
}
template <int N, int SIGN, typename C, typename TW>
__device__ __forceinline__ void lines_G(C* buf, int nlines, LineMap lm, int es, const TW& tw) {
  G_passB<N, SIGN>(buf, nlines, lm, es, tw, threadIdx.x, blockDim.x);
  __syncthreads();
  G_passA<N, SIGN>(buf, nlines, lm, es, threadIdx.x, blockDim.x);
  __syncthreads();
}
#endif

// position -> frequency/space index of the split order: p = NB*ka + kb holds index ka + NA*kb
template <int N> __host__ __device__ inline int split_index(int p) {
  constexpr int NA = Plan<N>::NA, NB = Plan<N>::NB;
  return (p / NB) + NA * (p % NB);
}

}  // namespace fast
}  // namespace chebfi
