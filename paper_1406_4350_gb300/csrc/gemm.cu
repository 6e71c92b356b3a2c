// Complex GEMM on the CUDA cores (FP64 DFMA or FP32 FFMA), C = alpha op(A) op(B) + beta C.
//
// Used for the FP64 and FP32 forms of the projector products P^H psi and P W
// (Algorithm 1, Section 5.1), the Woodbury core products, and the subspace matrices and
// rotations of Algorithm 2.  64 x 64 output tiles, 256 threads, 4 x 4 complex outputs per
// thread; split-K with a deterministic second pass when the output has too few tiles to
// fill the 152 SMs.
#include <algorithm>

#include "internal.cuh"
#include "kernels.cuh"

namespace chebfi {
namespace {

constexpr int BM = 64, BN = 64, BK = 8;

template <typename C> __device__ __forceinline__ C ld_op(const C* p, bool conj_) {
  C v = *p;
  if (conj_) v.y = -v.y;
  return v;
}

template <typename R, bool CA, bool CB>
__global__ void __launch_bounds__(256) k_gemm(int64_t M, int64_t N, int64_t K, R alpha, const cplx<R>* __restrict__ A,
                                              int64_t lda, const cplx<R>* __restrict__ B, int64_t ldb, R beta,
                                              cplx<R>* __restrict__ Cm, int64_t ldc, int64_t kchunk,
                                              cplx<R>* __restrict__ ws, int lower, int n_fastest) {
  using C = cplx<R>;
  // n_fastest: blockIdx.x walks the column tiles, so CTAs launched together share a row
  // tile of A (the large operand when M >> N) in L2
  const int64_t tile_i = n_fastest ? blockIdx.y : blockIdx.x, tile_j = n_fastest ? blockIdx.x : blockIdx.y;
  if (lower && tile_i < tile_j) return;  // tile strictly above the diagonal
  __shared__ C As[BK][BM + 1];
  __shared__ C Bs[BK][BN + 1];
  const int tid = threadIdx.x;
  const int tx = tid % 16, ty = tid / 16;
  const int64_t i0 = tile_i * BM, j0 = tile_j * BN;
  const int64_t kbeg = (int64_t)blockIdx.z * kchunk;
  const int64_t kend = min(K, kbeg + kchunk);
  R accr[4][4], acci[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) accr[a][b] = acci[a][b] = (R)0;
  const C zero = cmake<C>(0.0, 0.0);
  for (int64_t k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int e0 = 0; e0 < BM * BK; e0 += 256) {
      const int e = e0 + tid;
      int i, k;
      if (!CA) { i = e % BM; k = e / BM; } else { k = e % BK; i = e / BK; }
      const int64_t gi = i0 + i, gk = k0 + k;
      C v = zero;
      if (gi < M && gk < kend) v = CA ? ld_op(A + gk + gi * lda, true) : A[gi + gk * lda];
      As[k][i] = v;
    }
#pragma unroll
    for (int e0 = 0; e0 < BN * BK; e0 += 256) {
      const int e = e0 + tid;
      int j, k;
      if (!CB) { k = e % BK; j = e / BK; } else { j = e % BN; k = e / BN; }
      const int64_t gj = j0 + j, gk = k0 + k;
      C v = zero;
      if (gj < N && gk < kend) v = CB ? ld_op(B + gj + gk * ldb, true) : B[gk + gj * ldb];
      Bs[k][j] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      C av[4], bv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) av[a] = As[k][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) bv[b] = Bs[k][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          accr[a][b] = fma(av[a].x, bv[b].x, accr[a][b]);
          accr[a][b] = fma(-av[a].y, bv[b].y, accr[a][b]);
          acci[a][b] = fma(av[a].x, bv[b].y, acci[a][b]);
          acci[a][b] = fma(av[a].y, bv[b].x, acci[a][b]);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int64_t gj = j0 + ty + 16 * b;
    if (gj >= N) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int64_t gi = i0 + tx + 16 * a;
      if (gi >= M) continue;
      C r;
      r.x = alpha * accr[a][b];
      r.y = alpha * acci[a][b];
      if (ws) {
        ws[(int64_t)blockIdx.z * M * N + gi + gj * M] = r;
      } else {
        if (beta != (R)0) {
          const C c = Cm[gi + gj * ldc];
          r.x = fma(beta, c.x, r.x);
          r.y = fma(beta, c.y, r.y);
        }
        Cm[gi + gj * ldc] = r;
      }
    }
  }
}

template <typename R>
__global__ void k_splitk_reduce(int64_t M, int64_t N, int splits, const cplx<R>* __restrict__ ws, R beta,
                                cplx<R>* __restrict__ Cm, int64_t ldc) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= M * N) return;
  const int64_t i = idx % M, j = idx / M;
  cplx<R> r = cmake<cplx<R>>(0.0, 0.0);
  for (int z = 0; z < splits; ++z) {
    const cplx<R> v = ws[(int64_t)z * M * N + idx];
    r.x += v.x;
    r.y += v.y;
  }
  if (beta != (R)0) {
    const cplx<R> c = Cm[i + j * ldc];
    r.x = fma(beta, c.x, r.x);
    r.y = fma(beta, c.y, r.y);
  }
  Cm[i + j * ldc] = r;
}

template <typename R, bool CA, bool CB>
void launch(int64_t M, int64_t N, int64_t K, double alpha, const cplx<R>* A, int64_t lda, const cplx<R>* B,
            int64_t ldb, double beta, cplx<R>* Cm, int64_t ldc, cudaStream_t st, DevBuf<cplx<R>>* ws,
            const char* tag, bool lower) {
  const int64_t tm = (M + BM - 1) / BM, tn = (N + BN - 1) / BN;
  int splits = 1;
  const int64_t tiles = tm * tn;
  if (ws && tiles < 304 && K >= 2048) {
    splits = (int)std::min<int64_t>((304 + tiles - 1) / tiles, K / 1024);
    splits = std::max(1, std::min(splits, 64));
  }
  int64_t kchunk = (K + splits - 1) / splits;
  kchunk = (kchunk + BK - 1) / BK * BK;
  splits = (int)((K + kchunk - 1) / kchunk);
  if (K == 0) { splits = 1; kchunk = BK; }

  cplx<R>* wsp = nullptr;
  if (splits > 1) {
    ws->alloc((size_t)splits * M * N);
    wsp = ws->p;
  }
  const bool n_fastest = tm > 4 * tn;
  CHEBFI_REQUIRE((n_fastest ? tm : tn) <= 65535, CHEBFI_ERR_ARG, "GEMM too large");
  dim3 grid(n_fastest ? (unsigned)tn : (unsigned)tm, n_fastest ? (unsigned)tm : (unsigned)tn, (unsigned)splits);
  const double tiles_done = lower ? (double)(tm * (tm + 1) / 2) / (double)(tm * tn) : 1.0;
  CHEBFI_LAUNCH_W(tag, st, 8.0 * (double)M * (double)N * (double)K * tiles_done,
                  k_gemm<R, CA, CB><<<grid, 256, 0, st>>>(M, N, K, (R)alpha, A, lda, B, ldb, (R)beta, Cm, ldc, kchunk,
                                                          wsp, lower ? 1 : 0, n_fastest ? 1 : 0));
  if (splits > 1) {
    const int64_t tot = M * N;
    CHEBFI_LAUNCH("k_splitk_reduce", st, k_splitk_reduce<R><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(M, N, splits, wsp, (R)beta, Cm, ldc));
  }
}

}  // namespace

template <typename R>
void gemm(bool conjA, bool conjB, int64_t M, int64_t N, int64_t K, double alpha, const cplx<R>* A, int64_t lda,
          const cplx<R>* B, int64_t ldb, double beta, cplx<R>* C, int64_t ldc, cudaStream_t st,
          DevBuf<cplx<R>>* ws, const char* tag, bool lower) {
  if (M <= 0 || N <= 0) return;
  CHEBFI_REQUIRE(!lower || M == N, CHEBFI_ERR_ARG, "lower-triangle GEMM needs a square result");
  if (conjA && conjB) launch<R, true, true>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, ws, tag, lower);
  else if (conjA) launch<R, true, false>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, ws, tag, lower);
  else if (conjB) launch<R, false, true>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, ws, tag, lower);
  else launch<R, false, false>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, ws, tag, lower);
}

template void gemm<double>(bool, bool, int64_t, int64_t, int64_t, double, const double2*, int64_t, const double2*,
                           int64_t, double, double2*, int64_t, cudaStream_t, DevBuf<double2>*, const char*, bool);
template void gemm<float>(bool, bool, int64_t, int64_t, int64_t, double, const float2*, int64_t, const float2*,
                          int64_t, double, float2*, int64_t, cudaStream_t, DevBuf<float2>*, const char*, bool);

}  // namespace chebfi
