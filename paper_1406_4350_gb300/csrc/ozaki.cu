// FP64-accurate complex GEMM on the tcgen05 tensor cores by modular arithmetic.
//
// GB300 runs FP64 FMAs at about 2 per clock per SM, so the subspace matrices, rotations and
// projector products of Algorithm 2 (Section 4.2) in FP64 would be bound by that unit.
// This file emulates them on the bf16 tensor pipe with the integer-modular scheme of Ozaki,
// Uchino and Imamura ("Ozaki scheme II", 2025), written here from its mathematics:
//
//  1. each row r of op(A) and each column n of op(B) is scaled by a power of two 2^s so
//     that its 2-norm lies in [2^(E-1), 2^E), and rounded to integers: A_int, B_int;
//     by Cauchy-Schwarz every entry of C_int = A_int B_int then satisfies |C_int| < 2^(2E);
//  2. for pairwise coprime moduli m_1..m_n <= 256 with M = prod m_i >= 2^(2E+3), the
//     symmetric residues of A_int and B_int (|r| <= 128) are exact in bf16 and their
//     products exact in FP32; one tensor-core GEMM per modulus sums them in FP32 in chunks
//     of 512 products (|partial| <= 2^23, so every partial sum is an exact integer), and the
//     epilogue reduces each chunk modulo m_i on the FP32 units;
//  3. C_int mod M follows from the n residue matrices by the Chinese remainder theorem,
//     evaluated exactly in 128-bit integers, and C = 2^-(s_r + s_n) C_int.
// The only rounding is step 1's: each scaled entry is within 1/2 of its integer, so an
// entry of C is within about 2^-E ||a_r|| ||b_n|| (times a small constant) of the exact
// product - with 14 moduli, E = 53, at or below the error of an FP64 dot product.
//
// Complex products use the real embedding of interleaved data: the A operand holds two
// real rows per complex row, (Re a, -Im a) and (Im a, Re a), the B operand one, (Re b, Im b),
// so the real GEMM's output rows 2m and 2m+1 are Re and Im of C[m, n] and the output is the
// interleaved complex matrix itself.
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace chebfi {
namespace oz {

// pairwise coprime moduli, largest first; a set uses the first n of them
constexpr int kMods[kOzMaxMod] = {256, 255, 253, 251, 247, 241, 239, 233, 229, 227, 223, 217, 211, 199, 197};

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 6;
constexpr int CHUNK = 8;                      // k-tiles (512 products) per exact TMEM accumulation
constexpr int A_BYTES = BM * BK * 2;          // 16 KB
constexpr int B_BYTES = BN * BK * 2;          // 16 KB
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int THREADS = 192;
constexpr int NACC = 4;
constexpr uint32_t TMEM_COLS = NACC * BN;

struct GemmArgs {
  int M, N, K;      // real GEMM: M x N output, K-major operands of K reals
  int nmod;
  int lower;        // complex lower triangle only: tiles whose complex rows reach the diagonal
  int tiles_m, tiles_n, tiles;  // tiles = valid tiles per modulus
  signed char* R;   // residues: R[mod * rstride + n * M + m]
  int64_t rstride;
  int* status;
  float m[kOzMaxMod], inv[kOzMaxMod];
};

// number of column tiles of row tile tm that touch the complex lower triangle (complex rows
// [64 tm, 64 tm + 64) against complex columns [128 tn, 128 tn + 128))
__host__ __device__ __forceinline__ int lower_count(int tm, int tiles_n) { return min(tiles_n, (64 * tm + 63) / 128 + 1); }

__device__ __forceinline__ void unit_tile(const GemmArgs& a, int t, int& tm, int& tn) {
  if (!a.lower) {
    tm = t / a.tiles_n;
    tn = t % a.tiles_n;
    return;
  }
  int cum = 0;
  for (tm = 0; tm < a.tiles_m; ++tm) {
    const int c = lower_count(tm, a.tiles_n);
    if (t < cum + c) break;
    cum += c;
  }
  tn = t - cum;
}

// One persistent CTA per SM over (modulus, tile) units, modulus-major so that the CTAs in
// flight share operand k-slices in L2.  Warp 0: TMA loads of the residue tiles (6-stage
// ring); warp 1: one tcgen05 MMA chain per k-tile into one of four TMEM accumulators (one
// per 512-product chunk); warps 2-5: per chunk, add the exact FP32 sums into register
// accumulators reduced modulo m, then store the tile's residues as int8.
__global__ void __launch_bounds__(THREADS, 1)
    k_oz_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
              const __grid_constant__ GemmArgs args) {
  using namespace tc;
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + NACC;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + NACC);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int num_k = (args.K + BK - 1) / BK;
  const int num_chunks = (num_k + CHUNK - 1) / CHUNK;
  const int units = args.tiles * args.nmod;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int q = 0; q < NACC; ++q) {
      mbar_init(&acc_full[q], 1);
      mbar_init(&acc_empty[q], 4);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, TMEM_COLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const int mod = u / args.tiles;
        int tm, tn;
        unit_tile(args, u % args.tiles, tm, tn);
        for (int kt = 0; kt < num_k; ++kt, ++g) {
          const int s = g % STAGES;
          const uint32_t par = (g / STAGES) & 1;
          if (g >= STAGES && !mbar_wait(&empty[s], par ^ 1)) {
            flag(args.status, CHEBFI_ERR_CUDA);
            ok = false;
            break;
          }
          uint8_t* st = smem + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          tma_load_3d(st, &tmA, kt * BK, tm * BM, mod, &full[s]);
          tma_load_3d(st + A_BYTES, &tmB, kt * BK, tn * BN, mod, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(BM, BN);
      bool ok = true;
      int g = 0, gch = 0;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        int kt = 0;
        for (int ch = 0; ch < num_chunks && ok; ++ch, ++gch) {
          const int acc = gch % NACC;
          if (gch >= NACC && !mbar_wait(&acc_empty[acc], ((gch / NACC) - 1) & 1)) {
            flag(args.status, CHEBFI_ERR_CUDA);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(acc * BN);
          const int kend = min(num_k, (ch + 1) * CHUNK);
          for (; kt < kend; ++kt, ++g) {
            const int s = g % STAGES;
            const uint32_t par = (g / STAGES) & 1;
            if (!mbar_wait(&full[s], par)) {
              flag(args.status, CHEBFI_ERR_CUDA);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
            const bool first = kt == ch * CHUNK;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t off = kk * 32;  // 16 bf16 along K
              mma_bf16(d, sw128_desc(base + off), sw128_desc(base + A_BYTES + off), idesc,
                       (first && kk == 0) ? 0u : 1u);
            }
            mma_commit(&empty[s]);
          }
          mma_commit(&acc_full[acc]);
        }
      }
    }
  } else {
    const int lane_base = 32 * (warp % 4);
    bool ok = true;
    int gch = 0;
    for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const int mod = u / args.tiles;
      int tm, tn;
      unit_tile(args, u % args.tiles, tm, tn);
      const float mm = args.m[mod], inv = args.inv[mod];
      const int m = tm * BM + lane_base + lane;
      float racc[BN];
#pragma unroll
      for (int j = 0; j < BN; ++j) racc[j] = 0.f;
      for (int ch = 0; ch < num_chunks; ++ch, ++gch) {
        const int acc = gch % NACC;
        if (!mbar_wait(&acc_full[acc], (gch / NACC) & 1)) {
          flag(args.status, CHEBFI_ERR_CUDA);
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < BN; c += 32) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(acc * BN + c), v);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            // exact: |racc| < 1.5 m and |v| <= 2^23, so the sum and the product q m are integers below 2^24
            const float s = racc[c + j] + v[j];
            racc[c + j] = fmaf(-mm, rintf(s * inv), s);
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[acc]);
      }
      if (ok && m < args.M) {
        const int n0 = tn * BN, nvalid = min(BN, args.N - n0);
        signed char* out = args.R + (int64_t)mod * args.rstride + (int64_t)n0 * args.M + m;
#pragma unroll
        for (int j = 0; j < BN; ++j) {
          if (j < nvalid) {
            float r = fmaf(-mm, rintf(racc[j] * inv), racc[j]);  // |r| <= m / 2
            if (r > 127.f) r -= mm;                              // +128 (m = 256) as -128
            out[(int64_t)j * args.M] = (signed char)(int)r;
          }
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    tmem_dealloc(tmem, TMEM_COLS);
  }
}

// ---------------------------------------------------------------- operand preparation
// 2-norm of each row of op(X) -> scale exponent s with ||row|| 2^s in [2^(E-1), 2^E);
// 0 for a zero row, kOzBadShift for a non-finite one (its products come out NaN).
__device__ __forceinline__ int shift_for(double sumsq, int E) {
  if (!(sumsq < INFINITY)) return kOzBadShift;  // inf or NaN
  if (sumsq == 0.0) return 0;
  return E - 1 - ilogb(sqrt(sumsq));
}

// rows of op(X) are the columns of X (contiguous): one block per row
__global__ void k_oz_norm_cols(int64_t nrows, int64_t K, const double2* __restrict__ X, int64_t ldx, int E,
                               int* __restrict__ shift) {
  __shared__ double red[256];
  const int64_t r = blockIdx.x;
  const double2* x = X + r * ldx;
  double s = 0.0;
  for (int64_t k = threadIdx.x; k < K; k += blockDim.x) {
    const double2 v = x[k];
    s = fma(v.x, v.x, fma(v.y, v.y, s));
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) shift[r] = shift_for(red[0], E);
}

// rows of op(X) are the rows of X (strided): 32 rows per block, eight threads per row
// summing every eighth column, their partial sums added in a fixed order
__global__ void __launch_bounds__(256) k_oz_norm_rows(int64_t nrows, int64_t K, const double2* __restrict__ X,
                                                      int64_t ldx, int E, int* __restrict__ shift) {
  __shared__ double part[8][33];
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;
  const int64_t r = (int64_t)blockIdx.x * 32 + tx;
  double s = 0.0;
  if (r < nrows) {
    for (int64_t k = ty; k < K; k += 8) {
      const double2 v = X[r + k * ldx];
      s = fma(v.x, v.x, fma(v.y, v.y, s));
    }
  }
  part[ty][tx] = s;
  __syncthreads();
  if (ty == 0 && r < nrows) {
    double t = part[0][tx];
#pragma unroll
    for (int j = 1; j < 8; ++j) t += part[j][tx];
    shift[r] = shift_for(t, E);
  }
}

// round(x 2^s) for |x 2^s| <= 2^62 by integer operations on the bits (ties to even)
__device__ __forceinline__ long long scaled_int(double x, int s) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0 || e == 0x7FF) return 0;  // zero, subnormal (below 2^-1022: dropped), non-finite (flagged by the norm)
  const long long mant = (long long)((b & 0xFFFFFFFFFFFFFull) | (1ull << 52));
  const int sh = e - 1075 + s;  // x 2^s = mant 2^sh
  long long q;
  if (sh >= 0) {
    q = mant << min(sh, 10);
  } else if (sh < -63) {
    q = 0;
  } else {
    const int k = -sh;
    q = mant >> k;
    const unsigned long long rem = (unsigned long long)mant & ((1ull << k) - 1), half = 1ull << (k - 1);
    if (rem > half || (rem == half && (q & 1))) ++q;
  }
  return (b >> 63) ? -q : q;
}

// Symmetric residues of v modulo kMods[I], from 19-bit limbs of |v| (|v| <= 2^57):
// |v| = a 2^38 + b 2^19 + c, so
// |v| mod m = (a (2^38 mod m) + b (2^19 mod m) + c) mod m with every term below 2^28 -- one
// 32-bit remainder by a constant per modulus; then the symmetric representative (|r| <= m/2)
// and v's sign.  Any representative with |r| <= 128 serves the products' exactness.
template <int I> __device__ __forceinline__ int sres_limbs(unsigned a, unsigned b, unsigned c, bool neg) {
  constexpr unsigned m = (unsigned)kMods[I];
  constexpr unsigned c38 = (unsigned)((1ull << 38) % m), c19 = (unsigned)((1ull << 19) % m);
  unsigned x = (a * c38 + b * c19 + c) % m;
  int r = (int)x;
  if (x > m / 2) r -= (int)m;
  return neg ? -r : r;
}

// the 19-bit limbs of |v| and v's sign
struct Limbs {
  unsigned a, b, c;
  bool neg;
};
__device__ __forceinline__ Limbs limbs_of(long long v) {
  const bool neg = v < 0;
  const unsigned long long u = (unsigned long long)(neg ? -v : v);
  return Limbs{(unsigned)(u >> 38), (unsigned)((u >> 19) & 0x7FFFFu), (unsigned)(u & 0x7FFFFu), neg};
}

// the float bits of a small integer (|n| < 2^22) without a conversion instruction: 1.5 2^23 + n
// has n in its low mantissa bits, and subtracting 1.5 2^23 is exact
__device__ __forceinline__ unsigned small_int_float_bits(int n) {
  return (unsigned)__float_as_int(__fsub_rn(__int_as_float(0x4B400000 + n), 12582912.0f));
}
// two residues (|r| <= 128, exact in bf16) as a bf16 pair: the high halves of their float bits
__device__ __forceinline__ unsigned bf16_pair(unsigned lo_bits, unsigned hi_bits) {
  return __byte_perm(lo_bits, hi_bits, 0x7632);
}

// Writes the residues of NE consecutive complex entries a_e = op(X)[r][k + e] (after the
// optional conjugation) for moduli I.. into their matrices, one modulus at a time so that no
// residue outlives its store: plain (row r: Re, Im) or doubled (row 2r: Re, -Im; row 2r+1:
// Im, Re).  o0 / o1 point at entry k of those rows in modulus I's matrix.
template <int I, int NE>
__device__ __forceinline__ void put_mods(const Limbs (&re)[NE], const Limbs (&im)[NE], int nmod, bool doubled,
                                         __nv_bfloat16* o0, __nv_bfloat16* o1, int64_t mstride) {
  if constexpr (I < kOzMaxMod) {
    if (I < nmod) {
      unsigned fr[NE], fi[NE];
#pragma unroll
      for (int e = 0; e < NE; ++e) {
        fr[e] = small_int_float_bits(sres_limbs<I>(re[e].a, re[e].b, re[e].c, re[e].neg));
        fi[e] = small_int_float_bits(sres_limbs<I>(im[e].a, im[e].b, im[e].c, im[e].neg));
      }
      if constexpr (NE == 2) {
        if (doubled) {
          *reinterpret_cast<uint2*>(o0) =
              make_uint2(bf16_pair(fr[0], fi[0] ^ 0x80000000u), bf16_pair(fr[1], fi[1] ^ 0x80000000u));
          *reinterpret_cast<uint2*>(o1) = make_uint2(bf16_pair(fi[0], fr[0]), bf16_pair(fi[1], fr[1]));
        } else {
          *reinterpret_cast<uint2*>(o0) = make_uint2(bf16_pair(fr[0], fi[0]), bf16_pair(fr[1], fi[1]));
        }
      } else {
        if (doubled) {
          *reinterpret_cast<unsigned*>(o0) = bf16_pair(fr[0], fi[0] ^ 0x80000000u);
          *reinterpret_cast<unsigned*>(o1) = bf16_pair(fi[0], fr[0]);
        } else {
          *reinterpret_cast<unsigned*>(o0) = bf16_pair(fr[0], fi[0]);
        }
      }
      put_mods<I + 1, NE>(re, im, nmod, doubled, o0 + mstride, o1 + mstride, mstride);
    }
  }
}

// the residues of entries a[0..NE) = op(X)[r][k..k+NE) with row shift s
template <int NE>
__device__ __forceinline__ void put_entries(const double2 (&a)[NE], int s, int nmod, bool doubled,
                                            __nv_bfloat16* __restrict__ out, int64_t mstride, int64_t ld, int64_t r,
                                            int64_t k) {
  Limbs re[NE], im[NE];
#pragma unroll
  for (int e = 0; e < NE; ++e) {
    re[e] = limbs_of(s == kOzBadShift ? 0ll : scaled_int(a[e].x, s));
    im[e] = limbs_of(s == kOzBadShift ? 0ll : scaled_int(a[e].y, s));
  }
  __nv_bfloat16* o0 = out + (doubled ? 2 * r : r) * ld + 2 * k;
  put_mods<0, NE>(re, im, nmod, doubled, o0, o0 + ld, mstride);
}

// rows of op(X) = columns of X: grid (k blocks, rows); two consecutive entries per thread
// (ld and the modulus stride are multiples of 8 bf16 values, so the pairs' 8-byte stores
// are aligned)
__global__ void __launch_bounds__(256) k_oz_res_cols(int64_t K, const double2* __restrict__ X, int64_t ldx,
                                                     const int* __restrict__ shift, int conj, int doubled, int nmod,
                                                     __nv_bfloat16* __restrict__ out, int64_t mstride, int64_t ld) {
  const int64_t r = blockIdx.y;
  const int64_t k = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  if (k >= K) return;
  const int s = shift[r];
  const double2* x = X + r * ldx;
  if (k + 1 < K) {
    double2 a[2] = {x[k], x[k + 1]};
    if (conj) {
      a[0].y = -a[0].y;
      a[1].y = -a[1].y;
    }
    put_entries<2>(a, s, nmod, doubled != 0, out, mstride, ld, r, k);
  } else {
    double2 a[1] = {x[k]};
    if (conj) a[0].y = -a[0].y;
    put_entries<1>(a, s, nmod, doubled != 0, out, mstride, ld, r, k);
  }
}

// rows of op(X) = rows of X: 32-row x 64-k tiles through shared memory so that both the
// reads (along rows of X) and the writes (along k, two entries per thread) are coalesced
__global__ void __launch_bounds__(256) k_oz_res_rows(int64_t nrows, int64_t K, const double2* __restrict__ X,
                                                     int64_t ldx, const int* __restrict__ shift, int conj,
                                                     int doubled, int nmod, __nv_bfloat16* __restrict__ out,
                                                     int64_t mstride, int64_t ld) {
  __shared__ double2 t[32][65];  // [row][k], odd pitch
  const int64_t r0 = (int64_t)blockIdx.x * 32, k0 = (int64_t)blockIdx.y * 64;
  const int tx = threadIdx.x % 32, ty = threadIdx.x / 32;  // 256 threads: 8 rows of 32
  for (int j = ty; j < 64; j += 8) {
    const int64_t r = r0 + tx, k = k0 + j;
    t[tx][j] = (r < nrows && k < K) ? X[r + k * ldx] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int j = ty; j < 32; j += 8) {
    const int64_t r = r0 + j, k = k0 + 2 * tx;
    if (r >= nrows || k >= K) continue;
    const int s = shift[r];
    if (k + 1 < K) {
      double2 a[2] = {t[j][2 * tx], t[j][2 * tx + 1]};
      if (conj) {
        a[0].y = -a[0].y;
        a[1].y = -a[1].y;
      }
      put_entries<2>(a, s, nmod, doubled != 0, out, mstride, ld, r, k);
    } else {
      double2 a[1] = {t[j][2 * tx]};
      if (conj) a[0].y = -a[0].y;
      put_entries<1>(a, s, nmod, doubled != 0, out, mstride, ld, r, k);
    }
  }
}

// ---------------------------------------------------------------- reconstruction
struct CrtArgs {
  int nmod;
  float m[kOzMaxMod], inv[kOzMaxMod], y[kOzMaxMod];  // y_i = (M / m_i)^-1 mod m_i
  int L[kOzMaxMod][4];                               // M / m_i in 30-bit limbs, least significant first
  int ML[4];                                         // M in 30-bit limbs
};

// M < 2^120 for every modulus count: four 30-bit limbs hold M and each M / m_i
constexpr bool mods_fit_limbs() {
  unsigned __int128 M = 1;
  for (int i = 0; i < kOzMaxMod; ++i) M *= (unsigned)kMods[i];
  return (M >> 120) == 0;
}
static_assert(mods_fit_limbs(), "CRT modulus too large for four 30-bit limbs");

// 1.5 2^23: for |x| < 2^22, x + kMagic rounds x to an integer held in the low mantissa bits
constexpr float kMagic = 12582912.0f;

// one modulus' term of the CRT sum for residue r: t = r y_i mod m_i (symmetric, exact in
// float), its share t / m_i of S / M added to f.  The float conversions go through kMagic
// (one integer and one float addition each) instead of conversion instructions.
__device__ __forceinline__ int crt_term(int r, float y, float m, float inv, float& f) {
  const float p = __fmul_rn(__fsub_rn(__int_as_float(0x4B400000 + r), kMagic), y);  // r y, exact (< 2^15)
  const float q = __fsub_rn(__fmaf_rn(p, inv, kMagic), kMagic);                     // round(p / m_i)
  const float t = __fmaf_rn(-m, q, p);                                               // exact, |t| <= m_i / 2 + 1
  f = __fmaf_rn(t, inv, f);
  return __float_as_int(__fadd_rn(t, kMagic)) - 0x4B400000;
}

// sum_j a_j 2^(30 j) in 128-bit two's complement (the true sum fits)
__device__ __forceinline__ __int128 limb_sum(const long long (&a)[4]) {
  using u128 = unsigned __int128;
  const u128 u = (u128)(__int128)a[0] + ((u128)(__int128)a[1] << 30) + ((u128)(__int128)a[2] << 60) +
                 ((u128)(__int128)a[3] << 90);
  return (__int128)u;
}

// C_int of the two adjacent values (Re, Im) at r[0], r[1] of every modulus' residue matrix
// (modulus stride rs): t_i = r_i y_i mod m_i, S = sum t_i (M / m_i) = C_int (mod M), and
// C_int = S - M round(S / M) with S / M = sum t_i / m_i (FP32 suffices: |C_int| <= M / 8 keeps
// S / M at least 3/8 away from a half-integer).  The products t_i (M / m_i) accumulate per
// 30-bit limb of M / m_i in 64-bit integers (one 32 x 32 -> 64-bit multiply-add each, sums
// below 2^43), combined once into 128 bits: exact.
// NM moduli (a compile-time count, so that all NM loads are in flight at once).
template <int NM>
__device__ __forceinline__ void crt_pair(const signed char* r, int64_t rs, const CrtArgs& c, __int128& S0,
                                         __int128& S1) {
  unsigned v[NM];
#pragma unroll
  for (int i = 0; i < NM; ++i) v[i] = *reinterpret_cast<const unsigned short*>(r + i * rs);
  long long a0[4] = {0, 0, 0, 0}, a1[4] = {0, 0, 0, 0};
  float f0 = 0.f, f1 = 0.f;
#pragma unroll
  for (int i = 0; i < NM; ++i) {
    const int t0 = crt_term((int)(signed char)(v[i] & 0xFFu), c.y[i], c.m[i], c.inv[i], f0);
    const int t1 = crt_term((int)(signed char)(v[i] >> 8), c.y[i], c.m[i], c.inv[i], f1);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      a0[j] += (long long)t0 * (long long)c.L[i][j];
      a1[j] += (long long)t1 * (long long)c.L[i][j];
    }
  }
  const int k0 = __float_as_int(__fadd_rn(f0, kMagic)) - 0x4B400000;
  const int k1 = __float_as_int(__fadd_rn(f1, kMagic)) - 0x4B400000;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    a0[j] -= (long long)k0 * (long long)c.ML[j];
    a1[j] -= (long long)k1 * (long long)c.ML[j];
  }
  S0 = limb_sum(a0);
  S1 = limb_sum(a1);
}

// S 2^-sh as the nearest double (ties to even), by integer operations on the bits: GB300's
// FP64 pipe is its slowest, and a conversion plus a scaling there per value bound this
// kernel.  Results outside the normal range go through ldexp.
__device__ __forceinline__ double scaled_double(__int128 S, int sh) {
  if (S == 0) return 0.0;
  const bool neg = S < 0;
  unsigned __int128 u = neg ? (unsigned __int128)(-S) : (unsigned __int128)S;
  const unsigned long long h = (unsigned long long)(u >> 64), l = (unsigned long long)u;
  const int lz = h ? __clzll((long long)h) : 64 + __clzll((long long)l);
  u <<= lz;  // leading one at bit 127
  const unsigned long long top = (unsigned long long)(u >> 64), rest = (unsigned long long)u;
  unsigned long long mant = top >> 11;  // 53 bits, bit 52 set
  const unsigned long long rb = top & 0x7FFull;
  if (rb > 0x400ull || (rb == 0x400ull && (rest != 0 || (mant & 1ull)))) ++mant;
  int e = 127 - lz;
  if (mant >> 53) {
    mant >>= 1;
    ++e;
  }
  e -= sh;
  if (e < -1022 || e > 1023) {  // subnormal or overflow: the library's ldexp
    const double v = __longlong_as_double((long long)((1023ull << 52) | (mant & ((1ull << 52) - 1))));
    return ldexp(neg ? -v : v, e);
  }
  const unsigned long long bits =
      ((unsigned long long)neg << 63) | ((unsigned long long)(e + 1023) << 52) | (mant & ((1ull << 52) - 1));
  return __longlong_as_double((long long)bits);
}

// C[m, n] = alpha 2^-(sa_m + sb_n) C_int[m, n] + beta C[m, n]; one thread per complex entry,
// grid (m blocks, columns n strided); NM = crt.nmod
template <int NM>
__global__ void __launch_bounds__(256) k_oz_recon(int64_t M, int64_t N, const signed char* __restrict__ R, int64_t rstride,
                           const int* __restrict__ sa, const int* __restrict__ sb, double alpha, double beta,
                           double2* C, int64_t ldc, int lower, const __grid_constant__ CrtArgs crt) {
  const int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M) return;
  const int s1 = sa[m];
  for (int64_t n = blockIdx.y; n < N; n += gridDim.y) {
    if (lower && m < n) continue;
    const int s2 = sb[n];
    double re, im;
    if (s1 == kOzBadShift || s2 == kOzBadShift) {
      re = im = __longlong_as_double(0x7FF8000000000000ll);
    } else {
      __int128 S0, S1;
      crt_pair<NM>(R + n * (2 * M) + 2 * m, rstride, crt, S0, S1);
      re = scaled_double(S0, s1 + s2);
      im = scaled_double(S1, s1 + s2);
    }
    double2 v = alpha == 1.0 ? make_double2(re, im) : make_double2(alpha * re, alpha * im);
    double2* c = C + m + n * ldc;
    if (beta != 0.0) {
      const double2 o = *c;
      v.x = fma(beta, o.x, v.x);
      v.y = fma(beta, o.y, v.y);
    }
    *c = v;
  }
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// 3-D bf16 map over the residue stack [nmod][rows][ld], boxes of 64 x 128 x 1, 128-byte swizzle
CUtensorMap make_map3(const __nv_bfloat16* base, int64_t k, int64_t rows, int64_t ld, int nmod, int64_t mstride) {
  CHEBFI_REQUIRE(ld % 8 == 0 && mstride % 8 == 0 && (reinterpret_cast<uintptr_t>(base) % 16) == 0, CHEBFI_ERR_ARG,
                 "residue operand must be 16-byte aligned with strides multiple of 8 elements");
  CUtensorMap mp;
  cuuint64_t dims[3] = {(cuuint64_t)k, (cuuint64_t)rows, (cuuint64_t)nmod};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * 2), (cuuint64_t)(mstride * 2)};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)BM, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = tc::encode_fn()(&mp, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, (void*)base, dims, strides, box, estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CHEBFI_REQUIRE(r == CUDA_SUCCESS, CHEBFI_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return mp;
}

struct ModSet {
  int n = 0, E = 0;
  CrtArgs crt;
};

// moduli, E and the CRT constants of the first n moduli (host, 128-bit arithmetic)
const ModSet& modset(int n) {
  static ModSet sets[kOzMaxMod + 1];
  ModSet& s = sets[n];
  if (s.n == n) return s;
  unsigned __int128 M = 1;
  double l2 = 0.0;
  for (int i = 0; i < n; ++i) {
    M *= (unsigned)kMods[i];
    l2 += std::log2((double)kMods[i]);
  }
  s.crt.nmod = n;
  for (int i = 0; i < n; ++i) {
    const int m = kMods[i];
    const unsigned __int128 Mi = M / (unsigned)m;
    const int a = (int)(Mi % (unsigned)m);
    int y = 1;
    while ((a * y) % m != 1) ++y;  // m <= 256: direct search of the inverse
    s.crt.m[i] = (float)m;
    s.crt.inv[i] = 1.0f / (float)m;
    s.crt.y[i] = (float)y;
    for (int j = 0; j < 4; ++j) s.crt.L[i][j] = (int)((Mi >> (30 * j)) & ((1u << 30) - 1));
  }
  for (int j = 0; j < 4; ++j) s.crt.ML[j] = (int)((M >> (30 * j)) & ((1u << 30) - 1));
  s.E = std::min(62, (int)std::floor((l2 - 3.0) / 2.0));
  s.n = n;
  return s;
}

}  // namespace oz

int oz_precision_bits(int nmod) {
  CHEBFI_REQUIRE(nmod >= kOzMinMod && nmod <= kOzMaxMod, CHEBFI_ERR_ARG, "modulus count out of range");
  return oz::modset(nmod).E;
}

void oz_prepare(const double2* X, int64_t ldx, int64_t nrows, int64_t K, bool rows_are_columns, bool conj,
                bool doubled, int nmod, OzOperand& out, cudaStream_t st) {
  const oz::ModSet& ms = oz::modset(nmod);
  out.nmod = nmod;
  out.crows = nrows;
  out.rows = doubled ? 2 * nrows : nrows;
  out.kreal = 2 * K;
  out.ld = (out.kreal + 7) / 8 * 8;
  out.mstride = out.rows * out.ld;
  out.res.alloc((size_t)nmod * out.mstride);
  out.shift.alloc((size_t)std::max<int64_t>(nrows, 1));
  if (nrows == 0 || K == 0) return;
  if (rows_are_columns) {
    CHEBFI_LAUNCH("k_oz_norm", st, oz::k_oz_norm_cols<<<(unsigned)nrows, 256, 0, st>>>(nrows, K, X, ldx, ms.E, out.shift.p));
    const unsigned kb = (unsigned)((K + 511) / 512);  // one pair of entries per thread
    CHEBFI_REQUIRE(nrows <= 65535, CHEBFI_ERR_ARG, "too many rows for the residue kernel");
    CHEBFI_LAUNCH("k_oz_res", st,
                  oz::k_oz_res_cols<<<dim3(kb, (unsigned)nrows), 256, 0, st>>>(K, X, ldx, out.shift.p, conj ? 1 : 0,
                                                                               doubled ? 1 : 0, nmod, out.res.p,
                                                                               out.mstride, out.ld));
  } else {
    CHEBFI_LAUNCH("k_oz_norm", st, oz::k_oz_norm_rows<<<oz::nblk(nrows, 32), 256, 0, st>>>(nrows, K, X, ldx, ms.E, out.shift.p));
    CHEBFI_REQUIRE((K + 63) / 64 <= 65535, CHEBFI_ERR_ARG, "inner dimension too large for the residue kernel");
    CHEBFI_LAUNCH("k_oz_res", st,
                  oz::k_oz_res_rows<<<dim3((unsigned)((nrows + 31) / 32), (unsigned)((K + 63) / 64)), 256, 0, st>>>(
                      nrows, K, X, ldx, out.shift.p, conj ? 1 : 0, doubled ? 1 : 0, nmod, out.res.p, out.mstride,
                      out.ld));
  }
}

void oz_gemm(const OzOperand& A, const OzOperand& B, double alpha, double beta, double2* C, int64_t ldc, bool lower,
             DevBuf<signed char>& R, int* status, cudaStream_t st, const char* tag) {
  const int64_t M = A.crows, N = B.crows;
  if (M <= 0 || N <= 0) return;
  CHEBFI_REQUIRE(A.rows == 2 * M && B.rows == N && A.kreal == B.kreal && A.nmod == B.nmod, CHEBFI_ERR_ARG,
                 "modular GEMM operands do not match");
  CHEBFI_REQUIRE(!lower || M == N, CHEBFI_ERR_ARG, "lower-triangle GEMM needs a square result");
  CHEBFI_REQUIRE(2 * M < (1ll << 31) && N < (1ll << 31) && A.kreal < (1ll << 31), CHEBFI_ERR_ARG, "GEMM too large");
  const int nmod = A.nmod;
  const oz::ModSet& ms = oz::modset(nmod);
  oz::GemmArgs a;
  a.M = (int)(2 * M);
  a.N = (int)N;
  a.K = (int)A.kreal;
  a.nmod = nmod;
  a.lower = lower ? 1 : 0;
  a.tiles_m = (a.M + oz::BM - 1) / oz::BM;
  a.tiles_n = (a.N + oz::BN - 1) / oz::BN;
  if (lower) {
    int64_t t = 0;
    for (int tm = 0; tm < a.tiles_m; ++tm) t += oz::lower_count(tm, a.tiles_n);
    a.tiles = (int)t;
  } else {
    a.tiles = a.tiles_m * a.tiles_n;
  }
  a.rstride = (int64_t)a.M * a.N;
  R.alloc((size_t)nmod * a.rstride);
  a.R = R.p;
  a.status = status;
  for (int i = 0; i < kOzMaxMod; ++i) {
    a.m[i] = ms.crt.m[i];
    a.inv[i] = ms.crt.inv[i];
  }
  const CUtensorMap ta = oz::make_map3(A.res.p, A.kreal, A.rows, A.ld, nmod, A.mstride);
  const CUtensorMap tb = oz::make_map3(B.res.p, B.kreal, B.rows, B.ld, nmod, B.mstride);
  CHEBFI_CUDA(cudaFuncSetAttribute(oz::k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, oz::SMEM_BYTES));
  int dev = 0, sms = 0;
  CHEBFI_CUDA(cudaGetDevice(&dev));
  CHEBFI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int64_t units = (int64_t)a.tiles * nmod;
  // recorded work: the FP64 product's algorithmic flops (8 M N K complex); the tensor pipe
  // executes nmod times as many (one bf16 GEMM per modulus)
  const double tiles_done = (double)a.tiles / (double)(a.tiles_m * a.tiles_n);
  (void)tag;  // every modular GEMM is timed under one name, so its engine is unambiguous
  CHEBFI_LAUNCH_W("k_oz_gemm", st, 2.0 * (double)a.M * (double)a.N * (double)a.K * tiles_done,
                  oz::k_oz_gemm<<<(unsigned)std::min<int64_t>(units, sms), oz::THREADS, oz::SMEM_BYTES, st>>>(ta, tb, a));
  const dim3 rgrid(oz::nblk(M), (unsigned)std::min<int64_t>(N, 65535));
  auto recon = [&](auto kernel) {
    CHEBFI_LAUNCH("k_oz_recon", st,
                  kernel<<<rgrid, 256, 0, st>>>(M, N, R.p, a.rstride, A.shift.p, B.shift.p, alpha, beta, C, ldc,
                                                lower ? 1 : 0, ms.crt));
  };
  static_assert(kOzMinMod == 8 && kOzMaxMod == 15, "one reconstruction kernel per modulus count");
  switch (nmod) {
    case 8: recon(oz::k_oz_recon<8>); break;
    case 9: recon(oz::k_oz_recon<9>); break;
    case 10: recon(oz::k_oz_recon<10>); break;
    case 11: recon(oz::k_oz_recon<11>); break;
    case 12: recon(oz::k_oz_recon<12>); break;
    case 13: recon(oz::k_oz_recon<13>); break;
    case 14: recon(oz::k_oz_recon<14>); break;
    default: recon(oz::k_oz_recon<15>); break;
  }
}

}  // namespace chebfi
