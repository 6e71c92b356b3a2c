// Tensor-core GEMM of the mixed-precision filter on sm_103a (tcgen05 + TMA + TMEM).
//
// Computes D = alpha * A B (+ beta * C) for real matrices with FP32 accumulation, where
// A (M x K) and B (K x N) are both K-major (K contiguous) and given as bf16 pairs
// (hi, lo) with x ~= hi + lo; the product uses the three terms
//     A_hi B_hi + A_hi B_lo + A_lo B_hi
// (the lo * lo term is below the FP32 accumulation error), which carries about 16
// significant bits per operand instead of bf16's 8.  D and C are FP32 column-major.
//
// Complex projector products of Section 5.1 map onto it through the real embedding of
// interleaved complex data: with z stored as (re, im) pairs, P^H z and P w become real
// GEMMs whose A matrices (built once from P at setup) hold the 2 x 2 blocks
// [[Re, Im], [-Im, Re]] and [[Re, -Im], [Im, Re]].
//
// Persistent kernel, one CTA per SM looping over 128 x 128 tiles: warp 0 issues the TMA
// loads (128-byte swizzle,
// three-stage mbarrier ring), warp 1 allocates all 512 TMEM columns and issues the MMAs
// (tcgen05.mma cta_group::1 kind::f16, M = 128, N = 128, K = 16), warps 2-5 read the
// accumulator with tcgen05.ld.  The long contractions of the projector products (K up to
// 1.2e5) would lose accuracy in one tensor-core accumulator, so K is cut into chunks of
// 8 k-tiles (96 MMAs): each chunk accumulates in one of four TMEM buffers while the
// epilogue warps add finished ones into FP32 registers; the alpha/beta epilogue writes the
// register sums.  Four buffers let the MMAs run three chunks ahead while the epilogue
// reads C and stores D for a finished tile.  Every wait on an mbarrier gives up after a fixed time,
// records an error code and lets the CTA finish (the TMEM is released on every path).
#include <cuda.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <mutex>

#include "internal.cuh"
#include "kernels.cuh"
#include "tc_ptx.cuh"

namespace chebfi {
namespace tc {

constexpr int BM = 128, BN = 128, BK = 64, STAGES = 3;
constexpr int CHUNK = 8;                                 // k-tiles per TMEM accumulation
constexpr int A_BYTES = BM * BK * 2;                     // 16 KB
constexpr int B_BYTES = BN * BK * 2;                     // 16 KB
constexpr int STAGE_BYTES = 2 * A_BYTES + 2 * B_BYTES;   // hi + lo of both: 64 KB
constexpr int SMEM_BYTES = STAGES * STAGE_BYTES + 1024 + 256;
constexpr int THREADS = 192;
constexpr int NACC = 4;                                  // TMEM accumulators (chunks in flight)
constexpr uint32_t TMEM_COLS = NACC * BN;                // all 512 columns

struct Args {
  int M, N, K;
  float alpha, beta;
  float* D;
  int64_t ldd;
  const float* C;
  int64_t ldc;
  int* status;
  int splits;  // K split over this many work units per tile (partial sums go to ws)
  float* ws;   // splits x M x N column-major partial sums when splits > 1
};

__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gemm(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
              const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl, Args args) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;   // [NACC]: MMAs of a chunk done
  uint64_t* acc_empty = acc_full + NACC; // [NACC]: epilogue has drained the buffer
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + NACC);

  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int num_k = (args.K + BK - 1) / BK;
  const int tiles_n = (args.N + BN - 1) / BN;
  const int tiles = tiles_n * ((args.M + BM - 1) / BM);
  // work unit u: tile u % tiles, k-tiles [kb, ke) of split u / tiles
  const int units = tiles * args.splits;
  const int kpt = (num_k + args.splits - 1) / args.splits;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < NACC; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);  // one arrival per epilogue warp
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // Persistent: CTA b takes tiles b, b + gridDim.x, ...; tiles are numbered n-fastest so
  // the CTAs running together share rows of A (L2 reuse).  The k-tile and chunk counters
  // run on across tiles and give the ring slots and the mbarrier phases.
  if (warp == 0) {
    if (lane == 0) {
      int g = 0;
      bool ok = true;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const int tile = u % tiles, kb = (u / tiles) * kpt, ke = min(num_k, kb + kpt);
        const int n0 = (tile % tiles_n) * BN, m0 = (tile / tiles_n) * BM;
        for (int kt = kb; kt < ke; ++kt, ++g) {
          const int s = g % STAGES;
          const uint32_t par = (g / STAGES) & 1;
          if (g >= STAGES && !mbar_wait(&empty[s], par ^ 1)) {
            flag(args.status, CHEBFI_ERR_CUDA);
            ok = false;
            break;
          }
          uint8_t* st = smem + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          const int x = kt * BK;
          tma_load_2d(st, &tmAh, x, m0, &full[s]);
          tma_load_2d(st + A_BYTES, &tmAl, x, m0, &full[s]);
          tma_load_2d(st + 2 * A_BYTES, &tmBh, x, n0, &full[s]);
          tma_load_2d(st + 2 * A_BYTES + B_BYTES, &tmBl, x, n0, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(BM, BN);
      bool ok = true;
      int g = 0, gch = 0;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const int kb = (u / tiles) * kpt, ke = min(num_k, kb + kpt);
        const int num_chunks = (ke - kb + CHUNK - 1) / CHUNK;
        int kt = kb;
        for (int ch = 0; ch < num_chunks && ok; ++ch, ++gch) {
          const int acc = gch % NACC;
          if (gch >= NACC && !mbar_wait(&acc_empty[acc], ((gch / NACC) - 1) & 1)) {
            flag(args.status, CHEBFI_ERR_CUDA);
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(acc * BN);
          const int kend = min(ke, kb + (ch + 1) * CHUNK);
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
            const bool first = kt == kb + ch * CHUNK;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t off = kk * 32;  // 16 bf16 along K
              const uint64_t ah = sw128_desc(base + off), al = sw128_desc(base + A_BYTES + off);
              const uint64_t bh = sw128_desc(base + 2 * A_BYTES + off),
                             bl = sw128_desc(base + 2 * A_BYTES + B_BYTES + off);
              mma_bf16(d, ah, bh, idesc, (first && kk == 0) ? 0u : 1u);
              mma_bf16(d, ah, bl, idesc, 1);
              mma_bf16(d, al, bh, idesc, 1);
            }
            mma_commit(&empty[s]);
          }
          mma_commit(&acc_full[acc]);
        }
      }
    }
  } else {
    // epilogue: warp w owns TMEM lanes 32 (w % 4) .. +31, i.e. tile rows
    const int lane_base = 32 * (warp % 4);
    bool ok = true;
    int gch = 0;
    for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const int tile = u % tiles, split = u / tiles, kb = split * kpt, ke = min(num_k, kb + kpt);
      const int num_chunks = (ke - kb + CHUNK - 1) / CHUNK;
      const int n0 = (tile % tiles_n) * BN, m0 = (tile / tiles_n) * BM;
      const int m = m0 + lane_base + lane;
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
          for (int j = 0; j < 32; ++j) racc[c + j] += v[j];
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[acc]);
      }
      if (ok && m < args.M && args.splits > 1) {
        // partial sum of this K split; k_tc_reduce applies alpha and beta
        const int nvalid = min(BN, args.N - n0);
        float* w = args.ws + (int64_t)split * args.M * args.N + (int64_t)m + (int64_t)n0 * args.M;
#pragma unroll
        for (int j = 0; j < BN; ++j)
          if (j < nvalid) w[(int64_t)j * args.M] = racc[j];
      } else if (ok && m < args.M) {
        // C may be D itself: read every C value of the row first (no store in between, so
        // the loads can all be in flight together), then store
        const int nvalid = min(BN, args.N - n0);
        if (args.beta != 0.f) {
          const float* c = args.C + (int64_t)m + (int64_t)n0 * args.ldc;
#pragma unroll
          for (int j = 0; j < BN; ++j)
            if (j < nvalid) racc[j] = fmaf(args.beta, c[(int64_t)j * args.ldc], args.alpha * racc[j]);
        } else {
#pragma unroll
          for (int j = 0; j < BN; ++j) racc[j] *= args.alpha;
        }
        float* d = args.D + (int64_t)m + (int64_t)n0 * args.ldd;
#pragma unroll
        for (int j = 0; j < BN; ++j)
          if (j < nvalid) d[(int64_t)j * args.ldd] = racc[j];
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS) : "memory");
  }
}

// Grouped form for many independent problems of different sizes (the batched k-points):
// work item i = (problem, output tile), CTA b taking items b, b + gridDim.x, ... (ordered by
// the caller, longest contraction first).  The four bf16 tensor maps of each problem (A hi,
// A lo, B hi, B lo) live in a device table, written before the launch; the pipeline is
// k_tc_gemm's (TMA warp, MMA warp, four epilogue warps, chunked TMEM accumulation).
__global__ void __launch_bounds__(THREADS, 1)
    k_tc_gemm_grouped(const CUtensorMap* __restrict__ maps, const TcGroupProb* __restrict__ probs,
                      const int2* __restrict__ items, int nitems, float alpha_mul, int* status) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + NACC;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + NACC);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < NACC; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], 4);
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
      for (int u = blockIdx.x; u < nitems && ok; u += gridDim.x) {
        const int2 it = items[u];
        const TcGroupProb& p = probs[it.x];
        const CUtensorMap* mp = maps + 4 * p.map;
        const int tiles_n = (p.N + BN - 1) / BN;
        const int n0 = (it.y % tiles_n) * BN, m0 = (it.y / tiles_n) * BM;
        const int num_k = (p.K + BK - 1) / BK;
        for (int kt = 0; kt < num_k; ++kt, ++g) {
          const int s = g % STAGES;
          const uint32_t par = (g / STAGES) & 1;
          if (g >= STAGES && !mbar_wait(&empty[s], par ^ 1)) {
            flag(status, CHEBFI_ERR_CUDA);
            ok = false;
            break;
          }
          uint8_t* st = smem + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          const int x = kt * BK;
          tma_load_2d(st, mp + 0, x, m0, &full[s]);
          tma_load_2d(st + A_BYTES, mp + 1, x, m0, &full[s]);
          tma_load_2d(st + 2 * A_BYTES, mp + 2, x, n0, &full[s]);
          tma_load_2d(st + 2 * A_BYTES + B_BYTES, mp + 3, x, n0, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(BM, BN);
      bool ok = true;
      int g = 0, gch = 0;
      for (int u = blockIdx.x; u < nitems && ok; u += gridDim.x) {
        const TcGroupProb& p = probs[items[u].x];
        const int num_k = (p.K + BK - 1) / BK;
        const int num_chunks = (num_k + CHUNK - 1) / CHUNK;
        int kt = 0;
        for (int ch = 0; ch < num_chunks && ok; ++ch, ++gch) {
          const int acc = gch % NACC;
          if (gch >= NACC && !mbar_wait(&acc_empty[acc], ((gch / NACC) - 1) & 1)) {
            flag(status, CHEBFI_ERR_CUDA);
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
              flag(status, CHEBFI_ERR_CUDA);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t base = smem_u32(smem + s * STAGE_BYTES);
            const bool first = kt == ch * CHUNK;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t off = kk * 32;
              const uint64_t ah = sw128_desc(base + off), al = sw128_desc(base + A_BYTES + off);
              const uint64_t bh = sw128_desc(base + 2 * A_BYTES + off),
                             bl = sw128_desc(base + 2 * A_BYTES + B_BYTES + off);
              mma_bf16(d, ah, bh, idesc, (first && kk == 0) ? 0u : 1u);
              mma_bf16(d, ah, bl, idesc, 1);
              mma_bf16(d, al, bh, idesc, 1);
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
    for (int u = blockIdx.x; u < nitems && ok; u += gridDim.x) {
      const int2 it = items[u];
      const TcGroupProb& p = probs[it.x];
      const int tiles_n = (p.N + BN - 1) / BN;
      const int n0 = (it.y % tiles_n) * BN, m0 = (it.y / tiles_n) * BM;
      const int num_chunks = ((p.K + BK - 1) / BK + CHUNK - 1) / CHUNK;
      const int m = m0 + lane_base + lane;
      float racc[BN];
#pragma unroll
      for (int j = 0; j < BN; ++j) racc[j] = 0.f;
      for (int ch = 0; ch < num_chunks; ++ch, ++gch) {
        const int acc = gch % NACC;
        if (!mbar_wait(&acc_full[acc], (gch / NACC) & 1)) {
          flag(status, CHEBFI_ERR_CUDA);
          ok = false;
          break;
        }
        tc_fence_after();
#pragma unroll
        for (int c = 0; c < BN; c += 32) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(acc * BN + c), v);
#pragma unroll
          for (int j = 0; j < 32; ++j) racc[c + j] += v[j];
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&acc_empty[acc]);
      }
      if (ok && m < p.M) {
        const int nvalid = min(BN, p.N - n0);
        const float alpha = p.alpha * (p.scale_alpha ? alpha_mul : 1.f);
        if (p.beta != 0.f) {
          const float* c = p.C + (int64_t)m + (int64_t)n0 * p.ldc;
#pragma unroll
          for (int j = 0; j < BN; ++j)
            if (j < nvalid) racc[j] = fmaf(p.beta, c[(int64_t)j * p.ldc], alpha * racc[j]);
        } else {
#pragma unroll
          for (int j = 0; j < BN; ++j) racc[j] *= alpha;
        }
        float* dd = p.D + (int64_t)m + (int64_t)n0 * p.ldd;
#pragma unroll
        for (int j = 0; j < BN; ++j)
          if (j < nvalid) dd[(int64_t)j * p.ldd] = racc[j];
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

// Complex product by three real multiplications (Gauss's form).  With A = Ar + i Ai and
// B = Br + i Bi, the real products T1 = A1 B1, T2 = A2 B2, T3 = A3 B3 of the planes
// (A1, A2, A3) = (Ar, Ai, Ar -+ Ai) and (B1, B2, B3) = (Br, Bi, Br + Bi) give
//   C^H-type product (P^H z):  re = T1 + T2,  im = T3 - T1 + T2   with A3 = Ar - Ai, A = P^T
//   plain product (P w):       re = T1 - T2,  im = T3 - T1 - T2   with A3 = Ar + Ai
// (the signs come in as sre / sim), three quarters of the four real products of the real
// embedding.  The pipeline is k_tc_gemm's: per work unit the TMA warp streams the k-tiles of
// product 1, then 2, then 3; every chunk of 8 k-tiles accumulates in one of four TMEM buffers
// and the epilogue adds it, with the product's two signs, into register sums of re and im.
// Eight epilogue warps: warp w reads TMEM lanes 32 (w % 4) .. +31 and columns
// 64 ((w - 2) / 4) .. +63 of each buffer.  D and C are complex (interleaved FP32).
constexpr int THREADS3 = 320;
constexpr int EPI_WARPS3 = 8;
constexpr int HALF3 = BN / 2;

struct TmSet3 {
  CUtensorMap a[6];  // plane q: a[2q] hi, a[2q + 1] lo
  CUtensorMap b[6];
};
struct CArgs {
  int M, N, K;
  float alpha, beta;
  float2* D;
  int64_t ldd;
  const float2* C;
  int64_t ldc;
  int* status;
  int splits;
  float2* ws;  // splits x M x N partial sums when splits > 1
  float sre[3], sim[3];
};

__global__ void __launch_bounds__(THREADS3, 1) k_tc_cgemm3(const __grid_constant__ TmSet3 tm, CArgs args) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + NACC;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + NACC);
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  const int num_k = (args.K + BK - 1) / BK;
  const int tiles_n = (args.N + BN - 1) / BN;
  const int tiles = tiles_n * ((args.M + BM - 1) / BM);
  const int units = tiles * args.splits;
  const int kpt = (num_k + args.splits - 1) / args.splits;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int a = 0; a < NACC; ++a) {
      mbar_init(&acc_full[a], 1);
      mbar_init(&acc_empty[a], EPI_WARPS3);
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
        const int tile = u % tiles, kb = (u / tiles) * kpt, ke = min(num_k, kb + kpt);
        const int n0 = (tile % tiles_n) * BN, m0 = (tile / tiles_n) * BM;
        for (int c0 = kb; c0 < ke && ok; c0 += CHUNK) {
          for (int q = 0; q < 3 && ok; ++q) {
            for (int kt = c0; kt < min(ke, c0 + CHUNK); ++kt, ++g) {
              const int s = g % STAGES;
              const uint32_t par = (g / STAGES) & 1;
              if (g >= STAGES && !mbar_wait(&empty[s], par ^ 1)) {
                flag(args.status, CHEBFI_ERR_CUDA);
                ok = false;
                break;
              }
              uint8_t* st = smem + s * STAGE_BYTES;
              mbar_expect_tx(&full[s], STAGE_BYTES);
              const int x = kt * BK;
              tma_load_2d(st, &tm.a[2 * q], x, m0, &full[s]);
              tma_load_2d(st + A_BYTES, &tm.a[2 * q + 1], x, m0, &full[s]);
              tma_load_2d(st + 2 * A_BYTES, &tm.b[2 * q], x, n0, &full[s]);
              tma_load_2d(st + 2 * A_BYTES + B_BYTES, &tm.b[2 * q + 1], x, n0, &full[s]);
            }
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_bf16_f32(BM, BN);
      bool ok = true;
      int g = 0, gch = 0;
      for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
        const int kb = (u / tiles) * kpt, ke = min(num_k, kb + kpt);
        const int num_chunks = (ke - kb + CHUNK - 1) / CHUNK;
        for (int ch = 0; ch < num_chunks && ok; ++ch) {
          for (int q = 0; q < 3 && ok; ++q, ++gch) {
            int kt = kb + ch * CHUNK;
            const int acc = gch % NACC;
            if (gch >= NACC && !mbar_wait(&acc_empty[acc], ((gch / NACC) - 1) & 1)) {
              flag(args.status, CHEBFI_ERR_CUDA);
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(acc * BN);
            const int kend = min(ke, kb + (ch + 1) * CHUNK);
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
              const bool first = kt == kb + ch * CHUNK;
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk) {
                const uint32_t off = kk * 32;
                const uint64_t ah = sw128_desc(base + off), al = sw128_desc(base + A_BYTES + off);
                const uint64_t bh = sw128_desc(base + 2 * A_BYTES + off),
                               bl = sw128_desc(base + 2 * A_BYTES + B_BYTES + off);
                mma_bf16(d, ah, bh, idesc, (first && kk == 0) ? 0u : 1u);
                mma_bf16(d, ah, bl, idesc, 1);
                mma_bf16(d, al, bh, idesc, 1);
              }
              mma_commit(&empty[s]);
            }
            mma_commit(&acc_full[acc]);
          }
        }
      }
    }
  } else {
    const int lane_base = 32 * (warp % 4), col0 = HALF3 * ((warp - 2) / 4);
    bool ok = true;
    int gch = 0;
    for (int u = blockIdx.x; u < units && ok; u += gridDim.x) {
      const int tile = u % tiles, split = u / tiles, kb = split * kpt, ke = min(num_k, kb + kpt);
      const int num_chunks = (ke - kb + CHUNK - 1) / CHUNK;
      const int n0 = (tile % tiles_n) * BN + col0, m0 = (tile / tiles_n) * BM;
      const int m = m0 + lane_base + lane;
      float re[HALF3], im[HALF3];
#pragma unroll
      for (int j = 0; j < HALF3; ++j) re[j] = im[j] = 0.f;
      for (int ch = 0; ch < num_chunks && ok; ++ch) {
        for (int q = 0; q < 3; ++q, ++gch) {
          const float sr = args.sre[q], si = args.sim[q];
          const int acc = gch % NACC;
          if (!mbar_wait(&acc_full[acc], (gch / NACC) & 1)) {
            flag(args.status, CHEBFI_ERR_CUDA);
            ok = false;
            break;
          }
          tc_fence_after();
#pragma unroll
          for (int c = 0; c < HALF3; c += 32) {
            float v[32];
            tmem_ld32(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(acc * BN + col0 + c), v);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              re[c + j] = fmaf(sr, v[j], re[c + j]);
              im[c + j] = fmaf(si, v[j], im[c + j]);
            }
          }
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&acc_empty[acc]);
        }
      }
      const int nvalid = min(HALF3, args.N - n0);
      if (ok && m < args.M && nvalid > 0) {
        if (args.splits > 1) {
          float2* w = args.ws + (int64_t)split * args.M * args.N + (int64_t)m + (int64_t)n0 * args.M;
#pragma unroll
          for (int j = 0; j < HALF3; ++j)
            if (j < nvalid) w[(int64_t)j * args.M] = make_float2(re[j], im[j]);
        } else {
          if (args.beta != 0.f) {
            const float2* c = args.C + (int64_t)m + (int64_t)n0 * args.ldc;
#pragma unroll
            for (int j = 0; j < HALF3; ++j)
              if (j < nvalid) {
                const float2 cv = c[(int64_t)j * args.ldc];
                re[j] = fmaf(args.beta, cv.x, args.alpha * re[j]);
                im[j] = fmaf(args.beta, cv.y, args.alpha * im[j]);
              }
          } else {
#pragma unroll
            for (int j = 0; j < HALF3; ++j) {
              re[j] *= args.alpha;
              im[j] *= args.alpha;
            }
          }
          float2* dd = args.D + (int64_t)m + (int64_t)n0 * args.ldd;
#pragma unroll
          for (int j = 0; j < HALF3; ++j)
            if (j < nvalid) dd[(int64_t)j * args.ldd] = make_float2(re[j], im[j]);
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

// D = alpha * (sum of the K-split complex partial sums, in split order) + beta * C
__global__ void k_tc_creduce(int M, int N, int splits, const float2* __restrict__ ws, float alpha, float beta,
                             const float2* C, int64_t ldc, float2* D, int64_t ldd) {
  const int64_t mn = (int64_t)M * N;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= mn) return;
  const int64_t n = i / M, m = i - n * M;
  float2 acc = ws[i];
  for (int sp = 1; sp < splits; ++sp) {
    const float2 v = ws[sp * mn + i];
    acc.x += v.x;
    acc.y += v.y;
  }
  float2 r = make_float2(alpha * acc.x, alpha * acc.y);
  if (beta != 0.f) {
    const float2 c = C[m + n * ldc];
    r.x = fmaf(beta, c.x, r.x);
    r.y = fmaf(beta, c.y, r.y);
  }
  D[m + n * ldd] = r;
}

// D = alpha * (sum of the K-split partial sums, in split order) + beta * C; C may be D
// (M x N <= 2^26 in split mode, so 32-bit indices; one thread per 4 consecutive rows)
__global__ void k_tc_reduce(int M, int N, int splits, const float* __restrict__ ws, float alpha, float beta,
                            const float* C, int64_t ldc, float* D, int64_t ldd) {
  const int mn = M * N;
  const int i0 = 4 * (blockIdx.x * blockDim.x + threadIdx.x);
  if (i0 >= mn) return;
  const int n = i0 / M;
  int m = i0 - n * M;
  const float* c = C + (int64_t)n * ldc;
  float* d = D + (int64_t)n * ldd;
  for (int q = 0; q < 4 && i0 + q < mn; ++q, ++m) {
    if (m == M) {  // the four rows ran into the next column
      m = 0;
      c += ldc;
      d += ldd;
    }
    const int i = i0 + q;
    float acc = ws[i];
    for (int sp = 1; sp < splits; ++sp) acc += ws[sp * mn + i];
    float r = alpha * acc;
    if (beta != 0.f) r = fmaf(beta, c[m], r);
    d[m] = r;
  }
}

// ---------------------------------------------------------------- host side
EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  CHEBFI_REQUIRE(fn != nullptr, CHEBFI_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
  return fn;
}

// 2-D bf16 map over a K-major matrix with `rows` rows of `k` elements (row stride ld
// elements, a multiple of 8), boxes of BK x box_rows, 128-byte swizzle, zero fill.
CUtensorMap make_map(const __nv_bfloat16* base, int64_t k, int64_t rows, int64_t ld, int box_rows) {
  CHEBFI_REQUIRE(ld % 8 == 0 && (reinterpret_cast<uintptr_t>(base) % 16) == 0, CHEBFI_ERR_ARG,
                 "tensor-core operand must be 16-byte aligned with a row stride multiple of 8");
  CUtensorMap m;
  cuuint64_t dims[2] = {(cuuint64_t)k, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode_fn()(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  CHEBFI_REQUIRE(r == CUDA_SUCCESS, CHEBFI_ERR_CUDA, "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")");
  return m;
}

}  // namespace tc

void tc_gemm(const SplitBF16& A, const SplitBF16& B, int64_t M, int64_t N, int64_t K, float alpha, float beta,
             const float* C, int64_t ldc, float* D, int64_t ldd, int* status, cudaStream_t st, const char* tag,
             DevBuf<float>* ws) {
  if (M <= 0 || N <= 0) return;
  CHEBFI_REQUIRE(K > 0, CHEBFI_ERR_ARG, "tensor-core GEMM with K = 0");
  CHEBFI_REQUIRE(M < (1ll << 31) && N < (1ll << 31) && K < (1ll << 31), CHEBFI_ERR_ARG, "GEMM too large");
  CHEBFI_REQUIRE(A.ld >= K && B.ld >= K, CHEBFI_ERR_ARG, "operand leading dimension below K");
  const CUtensorMap ah = tc::make_map(A.hi, K, M, A.ld, tc::BM), al = tc::make_map(A.lo, K, M, A.ld, tc::BM);
  const CUtensorMap bh = tc::make_map(B.hi, K, N, B.ld, tc::BN), bl = tc::make_map(B.lo, K, N, B.ld, tc::BN);
  tc::Args a;
  a.M = (int)M;
  a.N = (int)N;
  a.K = (int)K;
  a.alpha = alpha;
  a.beta = beta;
  a.D = D;
  a.ldd = ldd;
  a.C = C;
  a.ldc = ldc;
  a.status = status;
  CHEBFI_CUDA(cudaFuncSetAttribute(tc::k_tc_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
  // persistent grid: one CTA per SM (the shared-memory ring admits one per SM)
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    CHEBFI_CUDA(cudaGetDevice(&dev));
    CHEBFI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const int64_t tiles = ((N + tc::BN - 1) / tc::BN) * ((M + tc::BM - 1) / tc::BM);
  CHEBFI_REQUIRE(tiles < (1ll << 31), CHEBFI_ERR_ARG, "GEMM too large");
  // K split: when the tiles fill the SMs in a whole number of rounds poorly (e.g. 512 tiles
  // on 152 SMs: 4 rounds, the last one 1/3 full), more and shorter work units balance better;
  // the split with the fewest rounds x k-tiles per unit wins if it saves at least 5 %, each
  // unit keeping at least one full accumulation chunk, and only for outputs small enough
  // (at most 2^26 elements) and contractions long enough (at least 16 chunks) that the
  // extra pass over the partial sums costs little next to the GEMM
  const int64_t num_k = (K + tc::BK - 1) / tc::BK;
  int splits = 1;
  if (ws && M * N <= (int64_t(1) << 26) && num_k >= 16 * tc::CHUNK) {
    const int64_t single = ((tiles + sms - 1) / sms) * num_k;
    int64_t best = single;
    for (int sp = 2; sp <= 8; ++sp) {
      const int64_t kpt = (num_k + sp - 1) / sp;
      if (kpt < tc::CHUNK || (sp - 1) * kpt >= num_k) break;
      const int64_t cost = ((tiles * sp + sms - 1) / sms) * kpt;
      if (cost < best && cost * 20 <= single * 19) {
        best = cost;
        splits = sp;
      }
    }
  }
  a.splits = splits;
  a.ws = nullptr;
  if (splits > 1) {
    ws->alloc((size_t)splits * M * N);
    a.ws = ws->p;
  }
  const int64_t units = tiles * splits;
  dim3 grid((unsigned)std::min<int64_t>(units, sms));
  CHEBFI_LAUNCH_W(tag, st, 2.0 * (double)M * (double)N * (double)K, tc::k_tc_gemm<<<grid, tc::THREADS, tc::SMEM_BYTES, st>>>(ah, al, bh, bl, a));
  if (splits > 1) {
    const int64_t n4 = (M * N + 3) / 4;
    CHEBFI_LAUNCH("k_tc_reduce", st, tc::k_tc_reduce<<<(unsigned)((n4 + 255) / 256), 256, 0, st>>>((int)M, (int)N, splits, a.ws, alpha, beta, C, ldc, D, ldd));
  }
}

void tc_cgemm3(const SplitBF16x3& A, const SplitBF16x3& B, bool conjA, int64_t M, int64_t N, int64_t K, float alpha,
               float beta, const float2* C, int64_t ldc, float2* D, int64_t ldd, int* status, cudaStream_t st,
               const char* tag, DevBuf<float>* ws) {
  if (M <= 0 || N <= 0) return;
  CHEBFI_REQUIRE(K > 0, CHEBFI_ERR_ARG, "tensor-core GEMM with K = 0");
  CHEBFI_REQUIRE(M < (1ll << 31) && N < (1ll << 31) && K < (1ll << 31), CHEBFI_ERR_ARG, "GEMM too large");
  CHEBFI_REQUIRE(A.ld >= K && B.ld >= K && A.plane >= A.ld * M && B.plane >= B.ld * N, CHEBFI_ERR_ARG,
                 "operand planes below the product's size");
  tc::TmSet3 tm;
  for (int q = 0; q < 3; ++q) {
    const SplitBF16 a = A.view(q), b = B.view(q);
    tm.a[2 * q] = tc::make_map(a.hi, K, M, a.ld, tc::BM);
    tm.a[2 * q + 1] = tc::make_map(a.lo, K, M, a.ld, tc::BM);
    tm.b[2 * q] = tc::make_map(b.hi, K, N, b.ld, tc::BN);
    tm.b[2 * q + 1] = tc::make_map(b.lo, K, N, b.ld, tc::BN);
  }
  tc::CArgs a;
  a.M = (int)M;
  a.N = (int)N;
  a.K = (int)K;
  a.alpha = alpha;
  a.beta = beta;
  a.D = D;
  a.ldd = ldd;
  a.C = C;
  a.ldc = ldc;
  a.status = status;
  // A^H B (A's planes from P^H: Ar, Ai, Ar - Ai) or A B (from P: Ar, Ai, Ar + Ai)
  const float sre[3] = {1.f, conjA ? 1.f : -1.f, 0.f}, sim[3] = {-1.f, conjA ? 1.f : -1.f, 1.f};
  for (int q = 0; q < 3; ++q) {
    a.sre[q] = sre[q];
    a.sim[q] = sim[q];
  }
  CHEBFI_CUDA(cudaFuncSetAttribute(tc::k_tc_cgemm3, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    CHEBFI_CUDA(cudaGetDevice(&dev));
    CHEBFI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  const int64_t tiles = ((N + tc::BN - 1) / tc::BN) * ((M + tc::BM - 1) / tc::BM);
  CHEBFI_REQUIRE(tiles < (1ll << 31), CHEBFI_ERR_ARG, "GEMM too large");
  // K split as in tc_gemm (rounds x k-tiles per unit, at least 5 % saved)
  const int64_t num_k = (K + tc::BK - 1) / tc::BK;
  int splits = 1;
  if (ws && M * N <= (int64_t(1) << 25) && num_k >= 16 * tc::CHUNK) {
    const int64_t single = ((tiles + sms - 1) / sms) * num_k;
    int64_t best = single;
    for (int sp = 2; sp <= 8; ++sp) {
      const int64_t kpt = (num_k + sp - 1) / sp;
      if (kpt < tc::CHUNK || (sp - 1) * kpt >= num_k) break;
      const int64_t cost = ((tiles * sp + sms - 1) / sms) * kpt;
      if (cost < best && cost * 20 <= single * 19) {
        best = cost;
        splits = sp;
      }
    }
  }
  a.splits = splits;
  a.ws = nullptr;
  if (splits > 1) {
    ws->alloc((size_t)splits * M * N * 2);
    a.ws = reinterpret_cast<float2*>(ws->p);
  }
  const int64_t units = tiles * splits;
  dim3 grid((unsigned)std::min<int64_t>(units, sms));
  CHEBFI_LAUNCH_W(tag, st, 8.0 * (double)M * (double)N * (double)K,
                  tc::k_tc_cgemm3<<<grid, tc::THREADS3, tc::SMEM_BYTES, st>>>(tm, a));
  if (splits > 1) {
    const int64_t mn = M * N;
    CHEBFI_LAUNCH("k_tc_reduce", st, tc::k_tc_creduce<<<(unsigned)((mn + 255) / 256), 256, 0, st>>>((int)M, (int)N, splits, a.ws, alpha, beta, C, ldc, D, ldd));
  }
}

CUtensorMap tc_map(const __nv_bfloat16* base, int64_t k, int64_t rows, int64_t ld) {
  return tc::make_map(base, k, rows, ld, tc::BM);
}

void tc_gemm_grouped(const CUtensorMap* maps, const TcGroupProb* probs, const int2* items, int nitems, float alpha_mul,
                     int* status, cudaStream_t st, const char* tag, double work) {
  if (nitems <= 0) return;
  CHEBFI_CUDA(cudaFuncSetAttribute(tc::k_tc_gemm_grouped, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::SMEM_BYTES));
  int dev = 0, sms = 0;
  CHEBFI_CUDA(cudaGetDevice(&dev));
  CHEBFI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned grid = (unsigned)std::min(nitems, sms);
  CHEBFI_LAUNCH_W(tag, st, work,
                  tc::k_tc_gemm_grouped<<<grid, tc::THREADS, tc::SMEM_BYTES, st>>>(maps, probs, items, nitems, alpha_mul,
                                                                                 status));
}

}  // namespace chebfi

// ---------------------------------------------------------------- operand preparation
namespace chebfi {
namespace {

__device__ __forceinline__ void split2(double v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __double2bfloat16(v);
  lo = __double2bfloat16(v - (double)__bfloat162float(hi));
}
__device__ __forceinline__ void split2f(float v, __nv_bfloat16& hi, __nv_bfloat16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// Real embedding of y = P^H x (P: npw x nq complex, column-major, ld = npw):
// row 2i holds (Re P_gi, Im P_gi) at columns (2g, 2g+1); row 2i+1 holds (-Im P_gi, Re P_gi).
__global__ void k_embed_ph(int64_t npw, int64_t nq, const double2* __restrict__ P, int64_t ldp,
                           __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int64_t ld) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npw * nq) return;
  const int64_t g = idx % npw, i = idx / npw;
  const double2 p = P[g + i * ldp];
  const int64_t r0 = (2 * i) * ld + 2 * g, r1 = (2 * i + 1) * ld + 2 * g;
  split2(p.x, hi[r0], lo[r0]);
  split2(p.y, hi[r0 + 1], lo[r0 + 1]);
  split2(-p.y, hi[r1], lo[r1]);
  split2(p.x, hi[r1 + 1], lo[r1 + 1]);
}

// Real embedding of y = A x for a complex A (m x k, column-major, ld = lda):
// row 2g holds (Re A_gj, -Im A_gj) at columns (2j, 2j+1); row 2g+1 holds (Im A_gj, Re A_gj).
__global__ void k_embed_n(int64_t m, int64_t k, const double2* __restrict__ A, int64_t lda,
                          __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int64_t ld) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * k) return;
  const int64_t g = idx % m, j = idx / m;
  const double2 a = A[g + j * lda];
  const int64_t r0 = (2 * g) * ld + 2 * j, r1 = (2 * g + 1) * ld + 2 * j;
  split2(a.x, hi[r0], lo[r0]);
  split2(-a.y, hi[r0 + 1], lo[r0 + 1]);
  split2(a.y, hi[r1], lo[r1]);
  split2(a.x, hi[r1 + 1], lo[r1 + 1]);
}

// Complex FP32 block (m x nb, column-major) -> bf16 (hi, lo) K-major operand: column b holds
// the 2m interleaved reals.
__global__ void k_split_block(int64_t m, int64_t nb, const float2* __restrict__ x, int64_t ldx,
                              __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int64_t ld) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * nb) return;
  const int64_t i = idx % m, b = idx / m;
  const float2 v = x[i + b * ldx];
  const int64_t o = b * ld + 2 * i;
  split2f(v.x, hi[o], lo[o]);
  split2f(v.y, hi[o + 1], lo[o + 1]);
}

// The three planes of P for the three-multiplication products (element (g, i) of the
// npw x nq matrix P): PH (rows i, K = g) holds Re, Im, Re - Im for P^H z; otherwise (rows g,
// K = i) Re, Im, Re + Im for P w.
template <bool PH>
__global__ void k_embed3(int64_t npw, int64_t nq, const double2* __restrict__ P, int64_t ldp,
                         __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int64_t ld, int64_t plane) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= npw * nq) return;
  const int64_t g = idx % npw, i = idx / npw;
  const double2 p = P[g + i * ldp];
  const int64_t o = PH ? i * ld + g : g * ld + i;
  split2(p.x, hi[o], lo[o]);
  split2(p.y, hi[o + plane], lo[o + plane]);
  split2(PH ? p.x - p.y : p.x + p.y, hi[o + 2 * plane], lo[o + 2 * plane]);
}

// The same planes from a complex FP32 matrix A (rows x cols, column-major): PH takes row
// index = column j of A and K = row g (planes Re, Im, Re - Im of A^H's real parts), else
// row index = row g and K = column j (Re, Im, Re + Im).
template <bool PH>
__global__ void k_embed3f(int64_t rows, int64_t cols, const float2* __restrict__ A, int64_t lda,
                          __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int64_t ld, int64_t plane) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= rows * cols) return;
  const int64_t g = idx % rows, j = idx / rows;
  const float2 a = A[g + j * lda];
  const int64_t o = PH ? j * ld + g : g * ld + j;
  split2f(a.x, hi[o], lo[o]);
  split2f(a.y, hi[o + plane], lo[o + plane]);
  split2f(PH ? a.x - a.y : a.x + a.y, hi[o + 2 * plane], lo[o + 2 * plane]);
}

// Complex FP32 block (m x nb) -> the (re, im, re + im) planes, row b = column b of the block
__global__ void k_split3(int64_t m, int64_t nb, const float2* __restrict__ x, int64_t ldx,
                         __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo, int64_t ld, int64_t plane) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= m * nb) return;
  const int64_t i = idx % m, b = idx / m;
  const float2 v = x[i + b * ldx];
  const int64_t o = b * ld + i;
  split2f(v.x, hi[o], lo[o]);
  split2f(v.y, hi[o + plane], lo[o + plane]);
  split2f(v.x + v.y, hi[o + 2 * plane], lo[o + 2 * plane]);
}

inline unsigned nblk(int64_t n) { return (unsigned)std::max<int64_t>(1, (n + 255) / 256); }

}  // namespace

void embed_ph(int64_t npw, int64_t nq, const double2* P, int64_t ldp, SplitBF16Buf& out, cudaStream_t st) {
  out.ld = (2 * npw + 7) / 8 * 8;
  out.alloc((size_t)out.ld * 2 * nq);
  CHEBFI_CUDA(cudaMemsetAsync(out.hi.p, 0, out.hi.n * sizeof(__nv_bfloat16), st));
  CHEBFI_CUDA(cudaMemsetAsync(out.lo.p, 0, out.lo.n * sizeof(__nv_bfloat16), st));
  CHEBFI_LAUNCH("k_embed_ph", st, k_embed_ph<<<nblk(npw * nq), 256, 0, st>>>(npw, nq, P, ldp, out.hi.p, out.lo.p, out.ld));
}

void embed_n(int64_t m, int64_t k, const double2* A, int64_t lda, SplitBF16Buf& out, cudaStream_t st) {
  out.ld = (2 * k + 7) / 8 * 8;
  out.alloc((size_t)out.ld * 2 * m);
  CHEBFI_CUDA(cudaMemsetAsync(out.hi.p, 0, out.hi.n * sizeof(__nv_bfloat16), st));
  CHEBFI_CUDA(cudaMemsetAsync(out.lo.p, 0, out.lo.n * sizeof(__nv_bfloat16), st));
  CHEBFI_LAUNCH("k_embed_n", st, k_embed_n<<<nblk(m * k), 256, 0, st>>>(m, k, A, lda, out.hi.p, out.lo.p, out.ld));
}

void embed3_n(int64_t npw, int64_t nq, const double2* P, int64_t ldp, SplitBF16x3& out, cudaStream_t st) {
  out.alloc(npw, nq);
  CHEBFI_CUDA(cudaMemsetAsync(out.hi.p, 0, out.hi.n * sizeof(__nv_bfloat16), st));
  CHEBFI_CUDA(cudaMemsetAsync(out.lo.p, 0, out.lo.n * sizeof(__nv_bfloat16), st));
  CHEBFI_LAUNCH("k_embed3", st, k_embed3<false><<<nblk(npw * nq), 256, 0, st>>>(npw, nq, P, ldp, out.hi.p, out.lo.p, out.ld, out.plane));
}

void embed3f(bool conj, int64_t rows, int64_t cols, const float2* A, int64_t lda, SplitBF16x3& out, cudaStream_t st) {
  if (conj) out.alloc(cols, rows);
  else out.alloc(rows, cols);
  CHEBFI_CUDA(cudaMemsetAsync(out.hi.p, 0, out.hi.n * sizeof(__nv_bfloat16), st));
  CHEBFI_CUDA(cudaMemsetAsync(out.lo.p, 0, out.lo.n * sizeof(__nv_bfloat16), st));
  if (conj)
    CHEBFI_LAUNCH("k_embed3", st, k_embed3f<true><<<nblk(rows * cols), 256, 0, st>>>(rows, cols, A, lda, out.hi.p, out.lo.p, out.ld, out.plane));
  else
    CHEBFI_LAUNCH("k_embed3", st, k_embed3f<false><<<nblk(rows * cols), 256, 0, st>>>(rows, cols, A, lda, out.hi.p, out.lo.p, out.ld, out.plane));
}

void split3_block(int64_t m, int64_t nb, const float2* x, int64_t ldx, SplitBF16x3& out, cudaStream_t st) {
  out.alloc(nb, m);
  CHEBFI_LAUNCH("k_split_block", st, k_split3<<<nblk(m * nb), 256, 0, st>>>(m, nb, x, ldx, out.hi.p, out.lo.p, out.ld, out.plane));
}

void split_block(int64_t m, int64_t nb, const float2* x, int64_t ldx, SplitBF16Buf& out, cudaStream_t st) {
  out.ld = (2 * m + 7) / 8 * 8;
  out.alloc((size_t)out.ld * nb);
  CHEBFI_LAUNCH("k_split_block", st, k_split_block<<<nblk(m * nb), 256, 0, st>>>(m, nb, x, ldx, out.hi.p, out.lo.p, out.ld));
}

}  // namespace chebfi
