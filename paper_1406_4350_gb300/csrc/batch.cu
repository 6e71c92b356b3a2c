// Batched k-points: Algorithm 2's filter for many Bloch vectors k of one cell at once.
//
// Section 2.1: sampling the Brillouin zone gives one independent eigenproblem per k; all of
// them share the cell, the grid, V_loc and the atoms (hence D and Q), while the G-sphere, the
// kinetic diagonal |k+G|^2/2 and the projector matrix P_k (so G_k = P_k^H P_k and the Woodbury
// core M_k) depend on k.  The spheres are uneven, and one k-point of a few thousand plane
// waves and 128 bands is too small to fill the GPU, so the batch runs every stage of the
// filter as ONE grouped launch over all k-points:
//
//   * the three FFT passes find their k-point and columns (or plane) from a block table;
//   * the projector GEMMs are persistent kernels that take (k, output tile) items from a
//     device work queue (an atomic counter; items ordered longest first), with tile shapes
//     picked by a built-in autotuner that times every candidate on the batch itself;
//   * the elementwise steps run flat over the concatenated blocks.
//
// The whole degree-n filter (gather, n steps, scatter) is captured once per (degree, form)
// in a CUDA graph and replayed; per-call values (block pointers, c and r of each k-point)
// live in a device descriptor table updated before each replay.  No kernel waits on another
// block, so the batch has no device-side spin.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <vector>

#include "fft_fast_kernels.cuh"
#include "internal.cuh"
#include "kernels.cuh"

namespace chebfi {
namespace {

using fk::FastArgs;
using fk::kCBF;
constexpr int kT = fk::kThreadsF;

// per k-point descriptor (device); user, ld, c, r are per call
template <typename R> struct KDesc {
  FastArgs fa;
  const R* K;
  const cplx<R>* P;  // npw x nq, sorted rows
  const cplx<R>* G;  // nq x nq
  const cplx<R>* M;  // nq x nq (PAW)
  const int32_t* perm;  // sorted row -> caller row
  int64_t npw, y_off, t_off;
  double2* user;
  int64_t ld;
  R c, r;
};

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// ---------------------------------------------------------------- gather / scatter
template <typename R>
__global__ void k_bgather(const KDesc<R>* __restrict__ ks, int64_t nb, cplx<R>* __restrict__ Y) {
  const int64_t kb = blockIdx.y, k = kb / nb, b = kb - k * nb;
  const KDesc<R>& d = ks[k];
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d.npw) return;
  const double2 v = d.user[d.perm[j] + b * d.ld];
  Y[d.y_off + b * d.npw + j] = cmake<cplx<R>>(v.x, v.y);
}

template <typename R>
__global__ void k_bscatter(const KDesc<R>* __restrict__ ks, int64_t nb, const cplx<R>* __restrict__ Y) {
  const int64_t kb = blockIdx.y, k = kb / nb, b = kb - k * nb;
  const KDesc<R>& d = ks[k];
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d.npw) return;
  const cplx<R> v = Y[d.y_off + b * d.npw + j];
  d.user[d.perm[j] + b * d.ld] = make_double2((double)v.x, (double)v.y);
}

// ---------------------------------------------------------------- FFT passes
template <typename R, int N>
__global__ void __launch_bounds__(kT) k_bzinv(const KDesc<R>* __restrict__ ks, const cplx<R>* __restrict__ Y,
                                              cplx<R>* __restrict__ T, const cplx<R>* __restrict__ tw,
                                              const int32_t* __restrict__ cb_k, const int32_t* __restrict__ cb_c0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = cb_k[blockIdx.x];
  const KDesc<R>& d = ks[k];
  const FastArgs fa = d.fa;
  fk::zinv_body<R, N>(Y + d.y_off, d.npw, T + d.t_off, fa, tw, cb_c0[blockIdx.x], blockIdx.y, smem_raw);
}

template <typename R, int N>
__global__ void __launch_bounds__(kT) k_bplane(const KDesc<R>* __restrict__ ks, int64_t nb, cplx<R>* __restrict__ T,
                                               const R* __restrict__ Vs, const cplx<R>* __restrict__ tw) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t kb = blockIdx.y, k = kb / nb, b = kb - k * nb;
  const KDesc<R>& d = ks[k];
  const FastArgs fa = d.fa;
  fk::plane_body<R, N>(T + d.t_off, Vs, fa, tw, blockIdx.x, b, smem_raw);
}

// z pass back with the Chebyshev epilogue of step `first` (0: later steps, 1: the first):
// Z_k = (K + V_loc) Y_k and T_k = a_k (Z_k - c_k Y_k) - b Yprev_k written over Yprev_k
template <typename R, int N>
__global__ void __launch_bounds__(kT) k_bzfwd(const KDesc<R>* __restrict__ ks, const cplx<R>* __restrict__ T,
                                              const cplx<R>* __restrict__ tw, const int32_t* __restrict__ cb_k,
                                              const int32_t* __restrict__ cb_c0, const cplx<R>* Ycur, cplx<R>* Z,
                                              cplx<R>* Yprev, int first) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = cb_k[blockIdx.x];
  const KDesc<R>& d = ks[k];
  const FastArgs fa = d.fa;
  LocalEpi<R> ep;
  ep.Y = Ycur + d.y_off;
  ep.ldy = d.npw;
  ep.Z = Z ? Z + d.y_off : nullptr;
  ep.ldz = d.npw;
  ep.T = Yprev + d.y_off;
  ep.Yprev = first ? nullptr : Yprev + d.y_off;
  ep.ldt = d.npw;
  ep.a = (first ? (R)1 : (R)2) / d.r;
  ep.c = d.c;
  ep.bprev = first ? (R)0 : (R)1;
  ep.inv_n3 = (R)(1.0 / ((double)N * N * N));
  fk::zfwd_body<R, N>(T + d.t_off, fa, tw, d.K, ep, cb_c0[blockIdx.x], blockIdx.y, smem_raw);
}

// ---------------------------------------------------------------- projection-space combination
// p_next = a_k (pz - c_k pcur) - b pprev, written over pprev (flat over nk x nq x nb)
// bf16 (hi, lo) pair of every k-point's Z block: row b of k-point k holds its 2 npw_k reals
template <typename R>
__global__ void k_bsplit_z(const KDesc<R>* __restrict__ ks, int64_t nb, const cplx<R>* __restrict__ Z,
                           const int64_t* __restrict__ zb_off, const int64_t* __restrict__ zb_ld,
                           __nv_bfloat16* __restrict__ hi, __nv_bfloat16* __restrict__ lo) {
  const int64_t kb = blockIdx.y, k = kb / nb, b = kb - k * nb;
  const KDesc<R>& d = ks[k];
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= d.npw) return;
  const float2 v = Z[d.y_off + b * d.npw + j];
  const int64_t o = zb_off[k] + b * zb_ld[k] + 2 * j;
  const __nv_bfloat16 hr = __float2bfloat16_rn(v.x), hi_ = __float2bfloat16_rn(v.y);
  hi[o] = hr;
  hi[o + 1] = hi_;
  lo[o] = __float2bfloat16_rn(v.x - __bfloat162float(hr));
  lo[o + 1] = __float2bfloat16_rn(v.y - __bfloat162float(hi_));
}

template <typename R>
__global__ void k_bcombine(const KDesc<R>* __restrict__ ks, int64_t per_k, int64_t n, const cplx<R>* __restrict__ pz,
                           const cplx<R>* __restrict__ pcur, cplx<R>* pprev, int first) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const KDesc<R>& d = ks[i / per_k];
  const R a = (first ? (R)1 : (R)2) / d.r;
  const cplx<R> u = pz[i], x = pcur[i];
  cplx<R> o;
  o.x = a * (u.x - d.c * x.x);
  o.y = a * (u.y - d.c * x.y);
  if (!first) {
    const cplx<R> y = pprev[i];
    o.x -= y.x;
    o.y -= y.y;
  }
  pprev[i] = o;
}

// ---------------------------------------------------------------- grouped GEMM
enum BOp : int { OP_PHY = 0, OP_G = 1, OP_M = 2, OP_GNEG = 3, OP_PW = 4 };

// One problem of the group: C = alpha op(A) B + beta C, complex, column-major.
template <typename R> struct Prob {
  int64_t M, N, K, lda, ldb, ldc;
  const cplx<R>* A;
  const cplx<R>* B;
  cplx<R>* C;
  R alpha, beta;
};

template <typename R>
__device__ __forceinline__ Prob<R> make_prob(const KDesc<R>& d, int op, int first, int64_t k, int64_t nq, int64_t nb,
                                             const cplx<R>* Bb, cplx<R>* Cb) {
  Prob<R> p;
  p.N = nb;
  if (op == OP_PHY) {  // p_k = P_k^H Z_k
    p.M = nq; p.K = d.npw; p.A = d.P; p.lda = d.npw; p.B = Bb + d.y_off; p.ldb = d.npw;
    p.C = Cb + k * nq * nb; p.ldc = nq; p.alpha = 1; p.beta = 0;
  } else if (op == OP_PW) {  // Y_k += a_k P_k W_k
    p.M = d.npw; p.K = nq; p.A = d.P; p.lda = d.npw; p.B = Bb + k * nq * nb; p.ldb = nq;
    p.C = Cb + d.y_off; p.ldc = d.npw; p.alpha = (first ? (R)1 : (R)2) / d.r; p.beta = 1;
  } else {  // G_k or M_k times a projection block
    p.M = nq; p.K = nq; p.A = op == OP_M ? d.M : d.G; p.lda = nq; p.B = Bb + k * nq * nb; p.ldb = nq;
    p.C = Cb + k * nq * nb; p.ldc = nq;
    p.alpha = op == OP_GNEG ? (R)-1 : (R)1;
    p.beta = op == OP_M ? (R)0 : (R)1;
  }
  return p;
}

// Persistent CTAs take (k, tile) items from the queue until it is empty.  Tile BM x BN with
// BM = 16 TM, BN = 16 TN; 256 threads, TM x TN complex outputs per thread.  CA: op(A) = A^H.
// The K loop is double-buffered: the next BKb-deep slices of A and B are fetched into
// registers while the current ones are multiplied from shared memory (one barrier per slice).
// With nsplit > 1 (the P^H Z class, whose inner dimension is a whole sphere) an item is
// (k, tile * nsplit + chunk): it sums one K-chunk into its own slice of ws, and
// k_bsplit_reduce adds the slices in chunk order (deterministic).
constexpr int BKb = 16;

template <typename R, int TM, int TN>
constexpr size_t bgemm_smem() {
  return (size_t)2 * BKb * (16 * TM + 1 + 16 * TN + 1) * sizeof(cplx<R>);
}

template <typename R, int TM, int TN, bool CA>
__global__ void __launch_bounds__(256) k_bgemm(const KDesc<R>* __restrict__ ks, int op, int first, int64_t nq,
                                               int64_t nb, const int2* __restrict__ items, int nitems,
                                               int* __restrict__ counter, const cplx<R>* Bb, cplx<R>* Cb,
                                               int nsplit, cplx<R>* __restrict__ ws) {
  using C = cplx<R>;
  constexpr int BM = 16 * TM, BN = 16 * TN;
  constexpr int LA = BM * BKb / 256, LB = BN * BKb / 256;
  static_assert(LA * 256 == BM * BKb && LB * 256 == BN * BKb, "tile slices must split evenly over 256 threads");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* As = reinterpret_cast<C*>(smem_raw);  // [2][BKb][BM + 1]
  C* Bs = As + 2 * BKb * (BM + 1);         // [2][BKb][BN + 1]
  __shared__ int s_item;
  const int tid = threadIdx.x, tx = tid % 16, ty = tid / 16;
  const C zero = cmake<C>(0.0, 0.0);
  for (;;) {
    if (tid == 0) s_item = atomicAdd(counter, 1);
    __syncthreads();
    const int item = s_item;
    __syncthreads();
    if (item >= nitems) break;
    const int2 it = items[item];
    Prob<R> p = make_prob<R>(ks[it.x], op, first, it.x, nq, nb, Bb, Cb);
    const int tile = it.y / nsplit, chunk = it.y - tile * nsplit;
    int64_t klo = 0, khi = p.K;
    if (nsplit > 1) {
      const int64_t kc = ((p.K + nsplit - 1) / nsplit + BKb - 1) / BKb * BKb;
      klo = min(p.K, (int64_t)chunk * kc);
      khi = min(p.K, klo + kc);
      p.C = ws + ((int64_t)it.x * nsplit + chunk) * p.M * p.N;
      p.ldc = p.M;
      p.alpha = 1;
      p.beta = 0;
    }
    const int64_t tm = (p.M + BM - 1) / BM;
    const int64_t i0 = (int64_t)(tile % tm) * BM, j0 = (int64_t)(tile / tm) * BN;
    R accr[TM][TN], acci[TM][TN];
#pragma unroll
    for (int a = 0; a < TM; ++a)
#pragma unroll
      for (int b = 0; b < TN; ++b) accr[a][b] = acci[a][b] = (R)0;
    C ra[LA], rb[LB];
    auto fetch = [&](int64_t k0) {
#pragma unroll
      for (int l = 0; l < LA; ++l) {
        const int e = l * 256 + tid;
        int i, k;
        if (!CA) { i = e % BM; k = e / BM; } else { k = e % BKb; i = e / BKb; }
        const int64_t gi = i0 + i, gk = k0 + k;
        C v = zero;
        if (gi < p.M && gk < khi) {
          v = CA ? p.A[gk + gi * p.lda] : p.A[gi + gk * p.lda];
          if (CA) v.y = -v.y;
        }
        ra[l] = v;
      }
#pragma unroll
      for (int l = 0; l < LB; ++l) {
        const int e = l * 256 + tid;
        const int k = e % BKb, j = e / BKb;
        const int64_t gj = j0 + j, gk = k0 + k;
        rb[l] = (gj < p.N && gk < khi) ? p.B[gk + gj * p.ldb] : zero;
      }
    };
    auto stash = [&](int buf) {
      C* as = As + buf * BKb * (BM + 1);
      C* bs = Bs + buf * BKb * (BN + 1);
#pragma unroll
      for (int l = 0; l < LA; ++l) {
        const int e = l * 256 + tid;
        int i, k;
        if (!CA) { i = e % BM; k = e / BM; } else { k = e % BKb; i = e / BKb; }
        as[k * (BM + 1) + i] = ra[l];
      }
#pragma unroll
      for (int l = 0; l < LB; ++l) {
        const int e = l * 256 + tid;
        const int k = e % BKb, j = e / BKb;
        bs[k * (BN + 1) + j] = rb[l];
      }
    };
    if (klo < khi) {
      fetch(klo);
      stash(0);
    }
    __syncthreads();
    int buf = 0;
    for (int64_t k0 = klo; k0 < khi; k0 += BKb) {
      const bool more = k0 + BKb < khi;
      if (more) fetch(k0 + BKb);  // in flight while the current slice is multiplied
      const C* as = As + buf * BKb * (BM + 1);
      const C* bs = Bs + buf * BKb * (BN + 1);
#pragma unroll
      for (int k = 0; k < BKb; ++k) {
        C av[TM], bv[TN];
#pragma unroll
        for (int a = 0; a < TM; ++a) av[a] = as[k * (BM + 1) + tx + 16 * a];
#pragma unroll
        for (int b = 0; b < TN; ++b) bv[b] = bs[k * (BN + 1) + ty + 16 * b];
#pragma unroll
        for (int a = 0; a < TM; ++a)
#pragma unroll
          for (int b = 0; b < TN; ++b) {
            accr[a][b] = fma(av[a].x, bv[b].x, accr[a][b]);
            accr[a][b] = fma(-av[a].y, bv[b].y, accr[a][b]);
            acci[a][b] = fma(av[a].x, bv[b].y, acci[a][b]);
            acci[a][b] = fma(av[a].y, bv[b].x, acci[a][b]);
          }
      }
      if (more) stash(buf ^ 1);  // that buffer was last read before the previous barrier
      __syncthreads();
      buf ^= 1;
    }
#pragma unroll
    for (int b = 0; b < TN; ++b) {
      const int64_t gj = j0 + ty + 16 * b;
      if (gj >= p.N) continue;
#pragma unroll
      for (int a = 0; a < TM; ++a) {
        const int64_t gi = i0 + tx + 16 * a;
        if (gi >= p.M) continue;
        C r;
        r.x = p.alpha * accr[a][b];
        r.y = p.alpha * acci[a][b];
        if (p.beta != (R)0) {
          const C c = p.C[gi + gj * p.ldc];
          r.x = fma(p.beta, c.x, r.x);
          r.y = fma(p.beta, c.y, r.y);
        }
        p.C[gi + gj * p.ldc] = r;
      }
    }
  }
}

// C_k = sum over chunks of the split-K slices (per = M x N elements of one problem)
template <typename R>
__global__ void k_bsplit_reduce(int64_t n, int64_t per, int nsplit, const cplx<R>* __restrict__ ws,
                                cplx<R>* __restrict__ C) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t k = i / per, e = i - k * per;
  cplx<R> acc = ws[(k * nsplit) * per + e];
  for (int c = 1; c < nsplit; ++c) {
    const cplx<R> v = ws[(k * nsplit + c) * per + e];
    acc.x += v.x;
    acc.y += v.y;
  }
  C[i] = acc;
}

// tile shapes the autotuner chooses from: (TM, TN) -> BM x BN = 16 TM x 16 TN
constexpr int kNumShapes = 4;
constexpr int kMaxSplit = 8;  // split-K factors tried for P^H Z: 1, 2, 4, 8
constexpr int kShapeTM[kNumShapes] = {4, 2, 4, 8};
constexpr int kShapeTN[kNumShapes] = {4, 4, 2, 4};

template <typename R> size_t bgemm_smem_of(int shape) {
  switch (shape) {
    case 0: return bgemm_smem<R, 4, 4>();
    case 1: return bgemm_smem<R, 2, 4>();
    case 2: return bgemm_smem<R, 4, 2>();
    default: return bgemm_smem<R, 8, 4>();
  }
}

template <typename R, bool CA> const void* bgemm_fn(int shape) {
  switch (shape) {
    case 0: return (const void*)k_bgemm<R, 4, 4, CA>;
    case 1: return (const void*)k_bgemm<R, 2, 4, CA>;
    case 2: return (const void*)k_bgemm<R, 4, 2, CA>;
    default: return (const void*)k_bgemm<R, 8, 4, CA>;
  }
}

}  // namespace
}  // namespace chebfi

using namespace chebfi;

// GEMM classes the autotuner tunes separately
enum { GC_PHY = 0, GC_SMALL = 1, GC_PW = 2, GC_N = 3 };

struct chebfi_batch {
  int device = 0;
  std::string err;
  int64_t launches = 0;
  std::vector<chebfi_ctx*> ks;
  int nk = 0, N = 0;
  int64_t nb = 0, nq = 0;
  bool paw = false;
  std::vector<int64_t> npw, y_off, t_off;
  int64_t ytot = 0, ttot = 0;
  // block tables of the z passes
  DevBuf<int32_t> cb_k, cb_c0;
  int ncb = 0;
  // descriptors (FP64 and FP32 forms) and their host images
  DevBuf<KDesc<double>> d64;
  DevBuf<KDesc<float>> d32;
  std::vector<KDesc<double>> h64;
  std::vector<KDesc<float>> h32;
  // workspaces
  DevBuf<double2> Y64[2], Z64, T64, p64[5], ws64;
  DevBuf<float2> Y32[2], Z32, T32, p32[5], ws32;
  DevBuf<int> counters;
  // autotuned tile shape per (form, GEMM class); -1 = not tuned yet
  int shape[2][GC_N] = {{-1, -1, -1}, {-1, -1, -1}};
  int split[2] = {1, 1};  // split-K factor of the P^H Z class
  double tune_ms[2][GC_N][kNumShapes] = {};
  double split_ms[2][4] = {};
  // work-queue items per (GEMM class, shape)
  std::map<std::pair<int, int>, DevBuf<int2>*> items;
  std::map<std::pair<int, int>, int> nitems;
  int grid_per_sm[2][kNumShapes] = {};
  int nsm = 0;
  // mixed form (form 2): FP32 iterates and FFT, projector products as grouped tensor-core
  // GEMMs with bf16 (hi, lo) operands; problem tables built on first use
  bool tc_built = false;
  SplitBF16Buf zb, sb;                   // bf16 pairs of Z (per k: nb rows of 2 npw_k reals) and of the projection blocks
  std::vector<int64_t> zb_off, zb_ld;    // per k: first element and row stride of its Z pair
  DevBuf<int64_t> d_zb_off, d_zb_ld;
  DevBuf<CUtensorMap> tcmaps;            // [kind][k][A hi, A lo, B hi, B lo]
  std::vector<TcGroupProb> h_tcprobs;    // [variant][k]
  DevBuf<TcGroupProb> tcprobs;
  DevBuf<int2> tcitems[7];
  int ntcitems[7] = {0, 0, 0, 0, 0, 0, 0};
  double tcwork[7] = {0, 0, 0, 0, 0, 0, 0};
  // captured filters: (form, degree) -> graph
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
  std::map<std::pair<int, int>, int64_t> graph_launches;
  cudaStream_t cap = nullptr;
  ~chebfi_batch() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second);
    for (auto& kv : items) delete kv.second;
    if (cap) cudaStreamDestroy(cap);
  }
};

namespace {

template <typename R> struct BatchOps;
template <> struct BatchOps<double> {
  static constexpr int form = 0;
  static DevBuf<KDesc<double>>& desc(chebfi_batch* b) { return b->d64; }
  static std::vector<KDesc<double>>& hdesc(chebfi_batch* b) { return b->h64; }
  static DevBuf<double2>* Y(chebfi_batch* b) { return b->Y64; }
  static DevBuf<double2>& Z(chebfi_batch* b) { return b->Z64; }
  static DevBuf<double2>& T(chebfi_batch* b) { return b->T64; }
  static DevBuf<double2>* p(chebfi_batch* b) { return b->p64; }
  static DevBuf<double2>& ws(chebfi_batch* b) { return b->ws64; }
  static const double* K(chebfi_ctx* c) { return c->d_K.p; }
  static const double2* P(chebfi_ctx* c) { return c->d_P.p; }
  static const double2* G(chebfi_ctx* c) { return c->d_G.p; }
  static const double2* M(chebfi_ctx* c) { return c->d_M.p; }
  static const double* D(chebfi_ctx* c) { return c->d_Dblk.p; }
  static const double* Vs(chebfi_ctx* c) { return c->d_vs.p; }
  static const double2* tw(chebfi_ctx* c) { return c->ax[0].tw64.p; }
};
template <> struct BatchOps<float> {
  static constexpr int form = 1;
  static DevBuf<KDesc<float>>& desc(chebfi_batch* b) { return b->d32; }
  static std::vector<KDesc<float>>& hdesc(chebfi_batch* b) { return b->h32; }
  static DevBuf<float2>* Y(chebfi_batch* b) { return b->Y32; }
  static DevBuf<float2>& Z(chebfi_batch* b) { return b->Z32; }
  static DevBuf<float2>& T(chebfi_batch* b) { return b->T32; }
  static DevBuf<float2>* p(chebfi_batch* b) { return b->p32; }
  static DevBuf<float2>& ws(chebfi_batch* b) { return b->ws32; }
  static const float* K(chebfi_ctx* c) { return c->d_Kf.p; }
  static const float2* P(chebfi_ctx* c) { return c->d_Pf.p; }
  static const float2* G(chebfi_ctx* c) { return c->d_Gf.p; }
  static const float2* M(chebfi_ctx* c) { return c->d_Mf.p; }
  static const float* D(chebfi_ctx* c) { return c->d_Dblkf.p; }
  static const float* Vs(chebfi_ctx* c) { return c->d_vsf.p; }
  static const float2* tw(chebfi_ctx* c) { return c->ax[0].tw32.p; }
};

FastArgs fast_args(const chebfi_ctx* c) {
  const SphereFFT& s = c->sph;
  FastArgs fa;
  fa.ncol = s.ncol;
  fa.nxa = s.nxa;
  fa.pitch = s.pitch;
  fa.zpitch = s.zpitch;
  fa.ncolp = (s.ncol + 15) / 16 * 16;
  fa.ldt = (int64_t)c->grid[2] * fa.ncolp;
  fa.col_start = s.col_start.p;
  fa.pw_line = s.pw_line.p;
  fa.pw_z = s.pw_z.p;
  fa.col_off = s.col_off_nat.p;
  fa.row_off = s.rows_nat.p;
  return fa;
}

// (k, tile[, chunk]) items of a GEMM class for tile shape `shape` and split factor
// `nsplit`, longest problems first
void build_items(chebfi_batch* bt, int gc, int shape, int nsplit) {
  const auto key = std::make_pair(gc, shape * 16 + nsplit);
  if (bt->items.count(key)) return;
  const int64_t BM = 16 * kShapeTM[shape], BN = 16 * kShapeTN[shape];
  std::vector<int> order(bt->nk);
  std::iota(order.begin(), order.end(), 0);
  if (gc == GC_PHY)  // cost of a tile grows with the sphere size (the inner dimension)
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bt->npw[a] > bt->npw[b]; });
  std::vector<int2> v;
  for (int k : order) {
    const int64_t M = gc == GC_PW ? bt->npw[k] : bt->nq;
    const int64_t tiles = ((M + BM - 1) / BM) * ((bt->nb + BN - 1) / BN) * nsplit;
    for (int64_t t = 0; t < tiles; ++t) v.push_back(make_int2(k, (int)t));
  }
  auto* buf = new DevBuf<int2>();
  buf->upload(v.data(), v.size());
  bt->items[key] = buf;
  bt->nitems[key] = (int)v.size();
}

template <typename R, bool CA>
void launch_bgemm(chebfi_batch* bt, int shape, int nsplit, int op, int first, const cplx<R>* Bb, cplx<R>* Cb,
                  int* counter, cudaStream_t st, const char* tag) {
  const int gc = op == OP_PHY ? GC_PHY : (op == OP_PW ? GC_PW : GC_SMALL);
  build_items(bt, gc, shape, nsplit);
  const auto key = std::make_pair(gc, shape * 16 + nsplit);
  const int n = bt->nitems[key];
  const int per_sm = std::max(1, bt->grid_per_sm[BatchOps<R>::form][shape]);
  const unsigned grid = (unsigned)std::max(1, std::min(n, bt->nsm * per_sm));
  const KDesc<R>* d = BatchOps<R>::desc(bt).p;
  const int2* it = bt->items[key]->p;
  const int64_t nq = bt->nq, nb = bt->nb;
  cplx<R>* ws = BatchOps<R>::ws(bt).p;
  switch (shape) {
    case 0: CHEBFI_LAUNCH(tag, st, (k_bgemm<R, 4, 4, CA><<<grid, 256, bgemm_smem<R, 4, 4>(), st>>>(d, op, first, nq, nb, it, n, counter, Bb, Cb, nsplit, ws))); break;
    case 1: CHEBFI_LAUNCH(tag, st, (k_bgemm<R, 2, 4, CA><<<grid, 256, bgemm_smem<R, 2, 4>(), st>>>(d, op, first, nq, nb, it, n, counter, Bb, Cb, nsplit, ws))); break;
    case 2: CHEBFI_LAUNCH(tag, st, (k_bgemm<R, 4, 2, CA><<<grid, 256, bgemm_smem<R, 4, 2>(), st>>>(d, op, first, nq, nb, it, n, counter, Bb, Cb, nsplit, ws))); break;
    default: CHEBFI_LAUNCH(tag, st, (k_bgemm<R, 8, 4, CA><<<grid, 256, bgemm_smem<R, 8, 4>(), st>>>(d, op, first, nq, nb, it, n, counter, Bb, Cb, nsplit, ws))); break;
  }
  if (nsplit > 1) {
    const int64_t per = nq * nb, tot = (int64_t)bt->nk * per;
    CHEBFI_LAUNCH("k_bsplit_reduce", st, (k_bsplit_reduce<R><<<nblk(tot), 256, 0, st>>>(tot, per, nsplit, ws, Cb)));
  }
}

// grouped GEMM of one op with the tuned shape; counter slot `slot`
template <typename R>
void bgemm(chebfi_batch* bt, int op, int first, const cplx<R>* Bb, cplx<R>* Cb, int slot, cudaStream_t st) {
  const int f = BatchOps<R>::form;
  const int gc = op == OP_PHY ? GC_PHY : (op == OP_PW ? GC_PW : GC_SMALL);
  const int shape = bt->shape[f][gc];
  int* counter = bt->counters.p + slot;
  if (op == OP_PHY) launch_bgemm<R, true>(bt, shape, bt->split[f], op, first, Bb, Cb, counter, st, "bgemm_PhY");
  else launch_bgemm<R, false>(bt, shape, 1, op, first, Bb, Cb, counter, st, op == OP_PW ? "bgemm_PW" : "bgemm_small");
}

template <typename R, int N>
void set_fft_smem(chebfi_batch* bt) {
  const SphereFFT& s = bt->ks[0]->sph;
  const size_t zbytes = (size_t)(N + kCBF * s.zpitch) * sizeof(cplx<R>);
  const size_t pbytes = (size_t)(N + N * s.pitch) * sizeof(cplx<R>);
  CHEBFI_CUDA(cudaFuncSetAttribute((const void*)k_bzinv<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zbytes));
  CHEBFI_CUDA(cudaFuncSetAttribute((const void*)k_bzfwd<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)zbytes));
  CHEBFI_CUDA(cudaFuncSetAttribute((const void*)k_bplane<R, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)pbytes));
}

// (K + V_loc) Y for every k-point with the step's Chebyshev epilogue
template <typename R, int N>
void blocal(chebfi_batch* bt, const cplx<R>* cur, cplx<R>* Z, cplx<R>* prev, int first, cudaStream_t st) {
  chebfi_ctx* c0 = bt->ks[0];
  const SphereFFT& s = c0->sph;
  const size_t zbytes = (size_t)(N + kCBF * s.zpitch) * sizeof(cplx<R>);
  const size_t pbytes = (size_t)(N + N * s.pitch) * sizeof(cplx<R>);
  const KDesc<R>* d = BatchOps<R>::desc(bt).p;
  const cplx<R>* tw = BatchOps<R>::tw(c0);
  cplx<R>* T = BatchOps<R>::T(bt).p;
  const dim3 gz((unsigned)bt->ncb, (unsigned)bt->nb);
  CHEBFI_LAUNCH("k_bzinv", st, (k_bzinv<R, N><<<gz, kT, zbytes, st>>>(d, cur, T, tw, bt->cb_k.p, bt->cb_c0.p)));
  CHEBFI_LAUNCH("k_bplane", st, (k_bplane<R, N><<<dim3(N, (unsigned)(bt->nk * bt->nb)), kT, pbytes, st>>>(d, bt->nb, T, BatchOps<R>::Vs(c0), tw)));
  CHEBFI_LAUNCH("k_bzfwd", st, (k_bzfwd<R, N><<<gz, kT, zbytes, st>>>(d, T, tw, bt->cb_k.p, bt->cb_c0.p, cur, Z, prev, first)));
}

template <typename R>
void blocal_n(chebfi_batch* bt, const cplx<R>* cur, cplx<R>* Z, cplx<R>* prev, int first, cudaStream_t st) {
  switch (bt->N) {
    case 24: blocal<R, 24>(bt, cur, Z, prev, first, st); break;
    case 32: blocal<R, 32>(bt, cur, Z, prev, first, st); break;
    case 48: blocal<R, 48>(bt, cur, Z, prev, first, st); break;
    case 64: blocal<R, 64>(bt, cur, Z, prev, first, st); break;
    case 72: blocal<R, 72>(bt, cur, Z, prev, first, st); break;
    default: blocal<R, 96>(bt, cur, Z, prev, first, st); break;
  }
}

template <typename R> void set_fft_smem_n(chebfi_batch* bt) {
  switch (bt->N) {
    case 24: set_fft_smem<R, 24>(bt); break;
    case 32: set_fft_smem<R, 32>(bt); break;
    case 48: set_fft_smem<R, 48>(bt); break;
    case 64: set_fft_smem<R, 64>(bt); break;
    case 72: set_fft_smem<R, 72>(bt); break;
    default: set_fft_smem<R, 96>(bt); break;
  }
}

template <typename R> void ensure_ws(chebfi_batch* bt) {
  const size_t np = (size_t)bt->nk * std::max<int64_t>(bt->nq, 1) * bt->nb;
  BatchOps<R>::Y(bt)[0].alloc((size_t)bt->ytot);
  BatchOps<R>::Y(bt)[1].alloc((size_t)bt->ytot);
  BatchOps<R>::Z(bt).alloc((size_t)bt->ytot);
  BatchOps<R>::T(bt).alloc((size_t)bt->ttot);
  for (int i = 0; i < 5; ++i) BatchOps<R>::p(bt)[i].alloc(np);
  BatchOps<R>::ws(bt).alloc(np * kMaxSplit);
}

// Algorithm 2's filter of degree n for all k-points (the same steps as the single-problem
// filter with projection reuse, Section 5.1); launches on st.  Counter slots: 6 per step + 1.
template <typename R>
void batch_filter_body(chebfi_batch* bt, int degree, cudaStream_t st) {
  using C = cplx<R>;
  const KDesc<R>* d = BatchOps<R>::desc(bt).p;
  C* Yb[2] = {BatchOps<R>::Y(bt)[0].p, BatchOps<R>::Y(bt)[1].p};
  C* Z = BatchOps<R>::Z(bt).p;
  DevBuf<C>* pp = BatchOps<R>::p(bt);
  C *pa = pp[0].p, *pb = pp[1].p, *pz = pp[2].p, *pw = pp[3].p, *pq = pp[4].p;
  const int64_t nq = bt->nq, nb = bt->nb, nk = bt->nk;
  int slot = 0;
  CHEBFI_CUDA(cudaMemsetAsync(bt->counters.p, 0, sizeof(int) * bt->counters.n, st));
  const dim3 gg(nblk(*std::max_element(bt->npw.begin(), bt->npw.end())), (unsigned)(nk * nb));
  CHEBFI_LAUNCH("k_bgather", st, (k_bgather<R><<<gg, 256, 0, st>>>(d, nb, Yb[0])));
  C *cur = Yb[0], *prev = Yb[1], *pcur = pa, *pprev = pb;
  if (nq > 0) bgemm<R>(bt, OP_PHY, 0, cur, pcur, slot++, st);
  for (int k = 0; k < degree; ++k) {
    const int first = k == 0 ? 1 : 0;
    blocal_n<R>(bt, cur, nq > 0 ? Z : nullptr, prev, first, st);
    if (nq > 0) {
      bgemm<R>(bt, OP_PHY, first, Z, pz, slot++, st);                       // P^H Z
      blockdiag_apply<R>(bt->ks[0], BatchOps<R>::D(bt->ks[0]), pcur, nq, pw, nq, nk * nb, st);  // D p
      bgemm<R>(bt, OP_G, first, pw, pz, slot++, st);                        // + G D p
      if (bt->paw) {
        bgemm<R>(bt, OP_M, first, pz, pq, slot++, st);                      // q = M P^H H Y
        axpby<R>(nq, nk * nb, (R)1, pw, nq, (R)-1, pq, nq, pw, nq, st);     // W = D p - q
        bgemm<R>(bt, OP_GNEG, first, pq, pz, slot++, st);                   // P^H S^{-1} H Y
      }
      bgemm<R>(bt, OP_PW, first, pw, prev, slot++, st);                     // Y_{k+1} = T + a P W
      CHEBFI_LAUNCH("k_bcombine", st, (k_bcombine<R><<<nblk(nk * nq * nb), 256, 0, st>>>(d, nq * nb, nk * nq * nb, pz, pcur, pprev, first)));
    }
    std::swap(cur, prev);
    std::swap(pcur, pprev);
  }
  CHEBFI_LAUNCH("k_bscatter", st, (k_bscatter<R><<<gg, 256, 0, st>>>(d, nb, cur)));
  (void)slot;
}

// ---------------------------------------------------------------- mixed form
// problem variants of the mixed step, each one problem per k-point
enum TcVariant : int { TV_PHY0 = 0, TV_PHY = 1, TV_G = 2, TV_M = 3, TV_GNEG = 4, TV_PW0 = 5, TV_PW1 = 6 };
// tensor-map kinds: (A operand, B operand) of the GEMM class
enum TcKind : int { TK_PHY = 0, TK_G = 1, TK_M = 2, TK_PW = 3 };

// Operands, tensor maps, problem tables and work items of the mixed form (first use).
void ensure_tc_batch(chebfi_batch* bt, cudaStream_t st) {
  if (bt->tc_built) return;
  const int nk = bt->nk;
  const int64_t nq = bt->nq, nb = bt->nb;
  CHEBFI_REQUIRE(nq > 0, CHEBFI_ERR_ARG, "the mixed batch needs projectors");
  ensure_ws<float>(bt);
  for (chebfi_ctx* c : bt->ks) ensure_tc_operands(c, st);
  // Z pairs: per k nb rows of 2 npw_k reals, rows 8-element aligned (TMA's 16-byte rule)
  bt->zb_off.resize(nk);
  bt->zb_ld.resize(nk);
  int64_t tot = 0;
  for (int k = 0; k < nk; ++k) {
    bt->zb_ld[k] = (2 * bt->npw[k] + 7) / 8 * 8;
    bt->zb_off[k] = tot;
    tot += bt->zb_ld[k] * nb;
  }
  bt->zb.alloc((size_t)tot);
  bt->zb.ld = 0;
  bt->d_zb_off.upload(bt->zb_off.data(), nk, st);
  bt->d_zb_ld.upload(bt->zb_ld.data(), nk, st);
  bt->sb.ld = (2 * nq + 7) / 8 * 8;
  bt->sb.alloc((size_t)bt->sb.ld * nb * nk);
  // tensor maps [kind][k][4]
  std::vector<CUtensorMap> maps((size_t)4 * nk * 4);
  for (int k = 0; k < nk; ++k) {
    chebfi_ctx* c = bt->ks[k];
    const int64_t np2 = 2 * bt->npw[k];
    const __nv_bfloat16* sbh = bt->sb.hi.p + (int64_t)k * nb * bt->sb.ld;
    const __nv_bfloat16* sbl = bt->sb.lo.p + (int64_t)k * nb * bt->sb.ld;
    CUtensorMap* m = maps.data() + ((size_t)TK_PHY * nk + k) * 4;
    m[0] = tc_map(c->tcA1.hi.p, np2, 2 * nq, c->tcA1.ld);
    m[1] = tc_map(c->tcA1.lo.p, np2, 2 * nq, c->tcA1.ld);
    m[2] = tc_map(bt->zb.hi.p + bt->zb_off[k], np2, nb, bt->zb_ld[k]);
    m[3] = tc_map(bt->zb.lo.p + bt->zb_off[k], np2, nb, bt->zb_ld[k]);
    m = maps.data() + ((size_t)TK_G * nk + k) * 4;
    m[0] = tc_map(c->tcAG.hi.p, 2 * nq, 2 * nq, c->tcAG.ld);
    m[1] = tc_map(c->tcAG.lo.p, 2 * nq, 2 * nq, c->tcAG.ld);
    m[2] = tc_map(sbh, 2 * nq, nb, bt->sb.ld);
    m[3] = tc_map(sbl, 2 * nq, nb, bt->sb.ld);
    m = maps.data() + ((size_t)TK_M * nk + k) * 4;
    if (bt->paw) {
      m[0] = tc_map(c->tcAM.hi.p, 2 * nq, 2 * nq, c->tcAM.ld);
      m[1] = tc_map(c->tcAM.lo.p, 2 * nq, 2 * nq, c->tcAM.ld);
    } else {
      m[0] = m[1] = maps[((size_t)TK_G * nk + k) * 4];
    }
    m[2] = tc_map(sbh, 2 * nq, nb, bt->sb.ld);
    m[3] = tc_map(sbl, 2 * nq, nb, bt->sb.ld);
    m = maps.data() + ((size_t)TK_PW * nk + k) * 4;
    m[0] = tc_map(c->tcA2.hi.p, 2 * nq, np2, c->tcA2.ld);
    m[1] = tc_map(c->tcA2.lo.p, 2 * nq, np2, c->tcA2.ld);
    m[2] = tc_map(sbh, 2 * nq, nb, bt->sb.ld);
    m[3] = tc_map(sbl, 2 * nq, nb, bt->sb.ld);
  }
  bt->tcmaps.upload(maps.data(), maps.size(), st);
  // problems [variant][k]; the PW alphas (1/r_k) are refreshed every call
  float2* pa = bt->p32[0].p;
  float2* pz = bt->p32[2].p;
  float2* pq = bt->p32[4].p;
  bt->h_tcprobs.assign((size_t)7 * nk, TcGroupProb{});
  for (int v = 0; v < 7; ++v) {
    std::vector<std::pair<int64_t, int>> order;  // (work of one tile, k): longest first
    for (int k = 0; k < nk; ++k) {
      TcGroupProb& p = bt->h_tcprobs[(size_t)v * nk + k];
      const int64_t np2 = 2 * bt->npw[k];
      float* pzk = (float*)(pz + (int64_t)k * nq * nb);
      p.N = (int)nb;
      p.alpha = 1.f;
      p.beta = 0.f;
      p.scale_alpha = 0;
      p.C = nullptr;
      p.ldc = 2 * nq;
      p.ldd = 2 * nq;
      if (v == TV_PHY0 || v == TV_PHY) {
        p.M = (int)(2 * nq);
        p.K = (int)np2;
        p.map = TK_PHY * nk + k;
        p.D = (float*)((v == TV_PHY0 ? pa : pz) + (int64_t)k * nq * nb);
      } else if (v == TV_G || v == TV_GNEG || v == TV_M) {
        p.M = (int)(2 * nq);
        p.K = (int)(2 * nq);
        p.map = (v == TV_M ? TK_M : TK_G) * nk + k;
        if (v == TV_M) {
          p.D = (float*)(pq + (int64_t)k * nq * nb);
        } else {
          p.D = pzk;
          p.C = pzk;
          p.beta = 1.f;
          p.alpha = v == TV_GNEG ? -1.f : 1.f;
        }
      } else {
        float2* Yv = bt->Y32[v == TV_PW0 ? 0 : 1].p + bt->y_off[k];
        p.M = (int)np2;
        p.K = (int)(2 * nq);
        p.map = TK_PW * nk + k;
        p.D = (float*)Yv;
        p.C = (const float*)Yv;
        p.ldd = p.ldc = np2;
        p.beta = 1.f;
        p.scale_alpha = 1;
      }
      order.emplace_back((int64_t)p.K, k);
    }
    std::stable_sort(order.begin(), order.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
    std::vector<int2> items;
    double work = 0.0;
    for (const auto& o : order) {
      const TcGroupProb& p = bt->h_tcprobs[(size_t)v * nk + o.second];
      const int tiles = ((p.M + 127) / 128) * ((p.N + 127) / 128);
      for (int t = 0; t < tiles; ++t) items.push_back(make_int2(v * nk + o.second, t));
      work += 2.0 * p.M * p.N * p.K;
    }
    bt->tcitems[v].upload(items.data(), items.size(), st);
    bt->ntcitems[v] = (int)items.size();
    bt->tcwork[v] = work;
  }
  bt->tcprobs.upload(bt->h_tcprobs.data(), bt->h_tcprobs.size(), st);
  CHEBFI_CUDA(cudaStreamSynchronize(st));
  bt->tc_built = true;
}

void tc_group(chebfi_batch* bt, int v, float alpha_mul, cudaStream_t st) {
  static const char* tags[7] = {"tcb_gemm_PhY", "tcb_gemm_PhY", "tcb_gemm_small", "tcb_gemm_small",
                                "tcb_gemm_small", "tcb_gemm_PW", "tcb_gemm_PW"};
  tc_gemm_grouped(bt->tcmaps.p, bt->tcprobs.p, bt->tcitems[v].p, bt->ntcitems[v], alpha_mul, bt->ks[0]->d_status.p, st,
                  tags[v], bt->tcwork[v]);
}

// The mixed form of batch_filter_body: the same steps with the projector products as grouped
// tensor-core GEMMs on bf16 (hi, lo) pairs of the FP32 operands.
void batch_filter_body_mixed(chebfi_batch* bt, int degree, cudaStream_t st) {
  using C = float2;
  const KDesc<float>* d = bt->d32.p;
  C* Yb[2] = {bt->Y32[0].p, bt->Y32[1].p};
  C* Z = bt->Z32.p;
  C *pa = bt->p32[0].p, *pb = bt->p32[1].p, *pz = bt->p32[2].p, *pw = bt->p32[3].p, *pq = bt->p32[4].p;
  const int64_t nq = bt->nq, nb = bt->nb, nk = bt->nk;
  const dim3 gg(nblk(*std::max_element(bt->npw.begin(), bt->npw.end())), (unsigned)(nk * nb));
  CHEBFI_LAUNCH("k_bgather", st, (k_bgather<float><<<gg, 256, 0, st>>>(d, nb, Yb[0])));
  C *cur = Yb[0], *prev = Yb[1], *pcur = pa, *pprev = pb;
  CHEBFI_LAUNCH("k_bsplit_z", st, (k_bsplit_z<float><<<gg, 256, 0, st>>>(d, nb, cur, bt->d_zb_off.p, bt->d_zb_ld.p, bt->zb.hi.p, bt->zb.lo.p)));
  tc_group(bt, TV_PHY0, 1.f, st);  // p_0 = P^H Y_0, into pa
  for (int k = 0; k < degree; ++k) {
    const int first = k == 0 ? 1 : 0;
    blocal_n<float>(bt, cur, Z, prev, first, st);
    CHEBFI_LAUNCH("k_bsplit_z", st, (k_bsplit_z<float><<<gg, 256, 0, st>>>(d, nb, Z, bt->d_zb_off.p, bt->d_zb_ld.p, bt->zb.hi.p, bt->zb.lo.p)));
    tc_group(bt, TV_PHY, 1.f, st);                                                                    // P^H Z
    blockdiag_apply<float>(bt->ks[0], BatchOps<float>::D(bt->ks[0]), pcur, nq, pw, nq, nk * nb, st);  // D p
    split_block(nq, nk * nb, pw, nq, bt->sb, st);
    tc_group(bt, TV_G, 1.f, st);                                                                      // + G D p
    if (bt->paw) {
      split_block(nq, nk * nb, pz, nq, bt->sb, st);
      tc_group(bt, TV_M, 1.f, st);                                                // q = M P^H H Y
      axpby<float>(nq, nk * nb, 1.f, pw, nq, -1.f, pq, nq, pw, nq, st);           // W = D p - q
      split_block(nq, nk * nb, pq, nq, bt->sb, st);
      tc_group(bt, TV_GNEG, 1.f, st);                                             // P^H S^{-1} H Y
    }
    split_block(nq, nk * nb, pw, nq, bt->sb, st);
    tc_group(bt, prev == Yb[0] ? TV_PW0 : TV_PW1, first ? 1.f : 2.f, st);       // Y_{k+1} = T + a P W
    CHEBFI_LAUNCH("k_bcombine", st, (k_bcombine<float><<<nblk(nk * nq * nb), 256, 0, st>>>(d, nq * nb, nk * nq * nb, pz, pcur, pprev, first)));
    std::swap(cur, prev);
    std::swap(pcur, pprev);
  }
  CHEBFI_LAUNCH("k_bscatter", st, (k_bscatter<float><<<gg, 256, 0, st>>>(d, nb, cur)));
}

// Time every tile shape of every GEMM class on the batch's own problems; keep the fastest.
template <typename R>
void autotune(chebfi_batch* bt, cudaStream_t st) {
  const int f = BatchOps<R>::form;
  if (bt->shape[f][0] >= 0) return;
  ensure_ws<R>(bt);
  using C = cplx<R>;
  C* Y = BatchOps<R>::Y(bt)[0].p;
  C* Y2 = BatchOps<R>::Y(bt)[1].p;
  DevBuf<C>* pp = BatchOps<R>::p(bt);
  CHEBFI_CUDA(cudaMemsetAsync(Y, 0, sizeof(C) * bt->ytot, st));
  CHEBFI_CUDA(cudaMemsetAsync(Y2, 0, sizeof(C) * bt->ytot, st));
  for (int i = 0; i < 5; ++i) CHEBFI_CUDA(cudaMemsetAsync(pp[i].p, 0, sizeof(C) * pp[i].n, st));
  for (int s = 0; s < kNumShapes; ++s) {
    const size_t smem = bgemm_smem_of<R>(s);
    for (const void* fn : {bgemm_fn<R, false>(s), bgemm_fn<R, true>(s)})
      CHEBFI_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int nb_per_sm = 0;
    CHEBFI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb_per_sm, bgemm_fn<R, false>(s), 256, smem));
    bt->grid_per_sm[f][s] = std::max(1, nb_per_sm);
  }
  cudaEvent_t a, b;
  CHEBFI_CUDA(cudaEventCreate(&a));
  CHEBFI_CUDA(cudaEventCreate(&b));
  const int ops[GC_N] = {OP_PHY, OP_G, OP_PW};
  for (int gc = 0; gc < GC_N; ++gc) {
    if (bt->nq == 0) {
      bt->shape[f][gc] = 0;
      continue;
    }
    int best = 0;
    for (int s = 0; s < kNumShapes; ++s) {
      bt->shape[f][gc] = s;
      const int op = ops[gc];
      const C* Bb = op == OP_PHY ? Y : pp[0].p;
      C* Cb = op == OP_PW ? Y2 : pp[1].p;
      float best_ms = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        CHEBFI_CUDA(cudaMemsetAsync(bt->counters.p, 0, sizeof(int), st));
        CHEBFI_CUDA(cudaEventRecord(a, st));
        bgemm<R>(bt, op, 0, Bb, Cb, 0, st);
        CHEBFI_CUDA(cudaEventRecord(b, st));
        CHEBFI_CUDA(cudaEventSynchronize(b));
        float ms = 0.f;
        CHEBFI_CUDA(cudaEventElapsedTime(&ms, a, b));
        if (rep > 0) best_ms = std::min(best_ms, ms);
      }
      bt->tune_ms[f][gc][s] = best_ms;
      if (best_ms < bt->tune_ms[f][gc][best]) best = s;
    }
    bt->shape[f][gc] = best;
  }
  // split-K factor of P^H Z: every shape again with each factor, keep the fastest pair
  if (bt->nq > 0) {
    int best_shape = bt->shape[f][GC_PHY], best_split = 1;
    float best_all = (float)bt->tune_ms[f][GC_PHY][best_shape];
    for (int si = 0, sp = 1; sp <= kMaxSplit; sp *= 2, ++si) {
      float best_sp = 1e30f;
      for (int s = 0; s < kNumShapes; ++s) {
        bt->shape[f][GC_PHY] = s;
        bt->split[f] = sp;
        float best_ms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
          CHEBFI_CUDA(cudaMemsetAsync(bt->counters.p, 0, sizeof(int), st));
          CHEBFI_CUDA(cudaEventRecord(a, st));
          bgemm<R>(bt, OP_PHY, 0, Y, pp[1].p, 0, st);
          CHEBFI_CUDA(cudaEventRecord(b, st));
          CHEBFI_CUDA(cudaEventSynchronize(b));
          float ms = 0.f;
          CHEBFI_CUDA(cudaEventElapsedTime(&ms, a, b));
          if (rep > 0) best_ms = std::min(best_ms, ms);
        }
        best_sp = std::min(best_sp, best_ms);
        if (best_ms < best_all) {
          best_all = best_ms;
          best_shape = s;
          best_split = sp;
        }
      }
      bt->split_ms[f][si] = best_sp;
    }
    bt->shape[f][GC_PHY] = best_shape;
    bt->split[f] = best_split;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
}

// mixed: the FP32 form with the projector products on the tensor cores (R = float only)
template <typename R>
void batch_filter(chebfi_batch* bt, void* const* Y, const int64_t* ld, int degree, const double* lo, const double* hi,
                  cudaStream_t st, bool mixed = false) {
  const int f = mixed ? 2 : BatchOps<R>::form;
  if (mixed) ensure_tc_batch(bt, st);
  else autotune<R>(bt, st);
  ensure_ws<R>(bt);
  set_fft_smem_n<R>(bt);
  fk::init_twiddles();
  // per-call descriptor fields
  auto& h = BatchOps<R>::hdesc(bt);
  for (int k = 0; k < bt->nk; ++k) {
    h[k].user = (double2*)Y[k];
    h[k].ld = ld[k];
    h[k].c = (R)(0.5 * (hi[k] + lo[k]));
    h[k].r = (R)(0.5 * (hi[k] - lo[k]));
  }
  // pageable source: the copy is staged before cudaMemcpyAsync returns
  CHEBFI_CUDA(cudaMemcpyAsync(BatchOps<R>::desc(bt).p, h.data(), sizeof(KDesc<R>) * h.size(), cudaMemcpyHostToDevice, st));
  if (mixed) {  // alpha of Y_{k+1} = T + alpha P W is 1/r_k (times 2 after the first step)
    const int nk = bt->nk;
    for (int v = TV_PW0; v <= TV_PW1; ++v)
      for (int k = 0; k < nk; ++k) bt->h_tcprobs[(size_t)v * nk + k].alpha = (float)(1.0 / (double)h[k].r);
    CHEBFI_CUDA(cudaMemcpyAsync(bt->tcprobs.p + (size_t)TV_PW0 * nk, bt->h_tcprobs.data() + (size_t)TV_PW0 * nk,
                                sizeof(TcGroupProb) * 2 * nk, cudaMemcpyHostToDevice, st));
  }
  const auto key = std::make_pair(f, degree);
  auto itg = bt->graphs.find(key);
  if (itg == bt->graphs.end()) {
    // capture on the batch's own stream, with the profiler and the launch counter detached
    Profiler* prof = g_prof;
    int64_t* counter = g_launch_counter;
    int64_t captured = 0;
    g_prof = nullptr;
    g_launch_counter = &captured;
    cudaGraph_t graph = nullptr;
    CHEBFI_CUDA(cudaStreamBeginCapture(bt->cap, cudaStreamCaptureModeThreadLocal));
    try {
      if (mixed) batch_filter_body_mixed(bt, degree, bt->cap);
      else batch_filter_body<R>(bt, degree, bt->cap);
    } catch (...) {
      cudaStreamEndCapture(bt->cap, &graph);
      if (graph) cudaGraphDestroy(graph);
      g_prof = prof;
      g_launch_counter = counter;
      throw;
    }
    CHEBFI_CUDA(cudaStreamEndCapture(bt->cap, &graph));
    g_prof = prof;
    g_launch_counter = counter;
    cudaGraphExec_t exec = nullptr;
    const cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CHEBFI_CUDA(e);
    itg = bt->graphs.emplace(key, exec).first;
    bt->graph_launches[key] = captured;
  }
  CHEBFI_CUDA(cudaGraphLaunch(itg->second, st));
  bt->launches += bt->graph_launches[key];
}

}  // namespace

#define BAPI_BEGIN(bt)                                      \
  if (!(bt)) return CHEBFI_ERR_ARG;                         \
  try {                                                     \
    (bt)->err.clear();                                      \
    CHEBFI_CUDA(cudaSetDevice((bt)->device));

#define BAPI_END(bt)                                        \
  }                                                         \
  catch (const chebfi::Error& e) {                          \
    (bt)->err = e.msg;                                      \
    return e.code;                                          \
  }                                                         \
  catch (const std::exception& e) {                         \
    (bt)->err = e.what();                                   \
    return CHEBFI_ERR_CUDA;                                 \
  }                                                         \
  return CHEBFI_OK;

extern "C" {

int chebfi_batch_create(chebfi_batch** out, chebfi_ctx* const* kctx, int nk, int64_t nb) {
  if (!out) return CHEBFI_ERR_ARG;
  *out = nullptr;
  if (!kctx || nk < 1 || nb < 1) return CHEBFI_ERR_ARG;
  for (int k = 0; k < nk; ++k)
    if (!kctx[k]) return CHEBFI_ERR_ARG;
  auto* bt = new chebfi_batch();
  bt->device = kctx[0]->device;
  try {
    CHEBFI_CUDA(cudaSetDevice(bt->device));
    chebfi_ctx* c0 = kctx[0];
    for (int k = 0; k < nk; ++k) {
      chebfi_ctx* c = kctx[k];
      CHEBFI_REQUIRE(c->has_cell && c->has_sphere && c->has_vloc && c->has_proj, CHEBFI_ERR_STATE,
                     "k-point context " + std::to_string(k) + " is not fully set up");
      CHEBFI_REQUIRE(c->device == c0->device, CHEBFI_ERR_ARG, "k-point contexts on different devices");
      CHEBFI_REQUIRE(c->fast_fft, CHEBFI_ERR_ARG,
                     "batched k-points need a cubic grid of 24, 32, 48, 64, 72 or 96 points per side");
      CHEBFI_REQUIRE(c->grid[0] == c0->grid[0] && c->grid[1] == c0->grid[1] && c->grid[2] == c0->grid[2],
                     CHEBFI_ERR_ARG, "k-point contexts with different grids");
      CHEBFI_REQUIRE(c->nproj == c0->nproj && c->natoms == c0->natoms && c->offs == c0->offs && c->paw == c0->paw,
                     CHEBFI_ERR_ARG, "k-point contexts with different atoms or projector blocks");
      CHEBFI_REQUIRE(c->sph.pitch == c0->sph.pitch && c->sph.zpitch == c0->sph.zpitch, CHEBFI_ERR_ARG,
                     "k-point contexts with different FFT layouts");
    }
    // V_loc, D and Q are shared: compare every context's copies with the first one's
    auto same = [&](const double* a, const double* b, size_t n) {
      if (n == 0 || a == b) return true;
      std::vector<double> ha(n), hb(n);
      CHEBFI_CUDA(cudaMemcpy(ha.data(), a, n * sizeof(double), cudaMemcpyDeviceToHost));
      CHEBFI_CUDA(cudaMemcpy(hb.data(), b, n * sizeof(double), cudaMemcpyDeviceToHost));
      return std::memcmp(ha.data(), hb.data(), n * sizeof(double)) == 0;
    };
    const size_t n3 = (size_t)c0->grid[0] * c0->grid[1] * c0->grid[2];
    for (int k = 1; k < nk; ++k) {
      chebfi_ctx* c = kctx[k];
      CHEBFI_REQUIRE(same(c->d_vs.p, c0->d_vs.p, n3), CHEBFI_ERR_ARG, "k-point contexts with different V_loc");
      CHEBFI_REQUIRE(c0->nproj == 0 || same(c->d_Dblk.p, c0->d_Dblk.p, c0->d_Dblk.n), CHEBFI_ERR_ARG,
                     "k-point contexts with different D");
      CHEBFI_REQUIRE(!c0->paw || c->h_Qblk == c0->h_Qblk, CHEBFI_ERR_ARG, "k-point contexts with different Q");
    }
    bt->ks.assign(kctx, kctx + nk);
    bt->nk = nk;
    bt->nb = nb;
    bt->N = c0->grid[0];
    bt->nq = c0->nproj;
    bt->paw = c0->paw;
    CHEBFI_REQUIRE((int64_t)nk * nb <= 65535, CHEBFI_ERR_ARG, "at most 65535 bands over all k-points");
    bt->npw.resize(nk);
    bt->y_off.resize(nk);
    bt->t_off.resize(nk);
    std::vector<int32_t> cbk, cbc;
    for (int k = 0; k < nk; ++k) {
      chebfi_ctx* c = kctx[k];
      bt->npw[k] = c->npw;
      bt->y_off[k] = bt->ytot;
      bt->ytot += c->npw * nb;
      bt->t_off[k] = bt->ttot;
      bt->ttot += (int64_t)local_workspace_elems(c, nb);
      for (int c0i = 0; c0i < c->sph.ncol; c0i += kCBF) {
        cbk.push_back(k);
        cbc.push_back(c0i);
      }
    }
    bt->ncb = (int)cbk.size();
    CHEBFI_REQUIRE(bt->ncb <= 0x7fffffff, CHEBFI_ERR_ARG, "too many column blocks");
    bt->cb_k.upload(cbk.data(), cbk.size());
    bt->cb_c0.upload(cbc.data(), cbc.size());
    bt->h64.resize(nk);
    bt->h32.resize(nk);
    for (int k = 0; k < nk; ++k) {
      chebfi_ctx* c = kctx[k];
      KDesc<double>& a = bt->h64[k];
      KDesc<float>& b = bt->h32[k];
      a.fa = b.fa = fast_args(c);
      a.K = BatchOps<double>::K(c);
      b.K = BatchOps<float>::K(c);
      a.P = BatchOps<double>::P(c);
      b.P = BatchOps<float>::P(c);
      a.G = BatchOps<double>::G(c);
      b.G = BatchOps<float>::G(c);
      a.M = BatchOps<double>::M(c);
      b.M = BatchOps<float>::M(c);
      a.perm = b.perm = c->d_sorted_to_user.p;
      a.npw = b.npw = c->npw;
      a.y_off = b.y_off = bt->y_off[k];
      a.t_off = b.t_off = bt->t_off[k];
      a.user = b.user = nullptr;
      a.ld = b.ld = c->npw;
      a.c = 0.0;
      a.r = 1.0;
      b.c = 0.f;
      b.r = 1.f;
    }
    bt->d64.upload(bt->h64.data(), nk);
    bt->d32.upload(bt->h32.data(), nk);
    bt->counters.alloc(8 * 1001 + 8);
    int dev = 0;
    CHEBFI_CUDA(cudaGetDevice(&dev));
    CHEBFI_CUDA(cudaDeviceGetAttribute(&bt->nsm, cudaDevAttrMultiProcessorCount, dev));
    CHEBFI_CUDA(cudaStreamCreateWithFlags(&bt->cap, cudaStreamNonBlocking));
    CHEBFI_CUDA(cudaDeviceSynchronize());
  } catch (const chebfi::Error& e) {
    delete bt;
    return e.code;
  }
  *out = bt;
  return CHEBFI_OK;
}

int chebfi_batch_destroy(chebfi_batch* bt) {
  if (!bt) return CHEBFI_ERR_ARG;
  cudaSetDevice(bt->device);
  cudaDeviceSynchronize();
  delete bt;
  return CHEBFI_OK;
}

const char* chebfi_batch_last_error(const chebfi_batch* bt) { return bt ? bt->err.c_str() : "null batch"; }

int64_t chebfi_batch_kernel_launches(const chebfi_batch* bt) { return bt ? bt->launches : -1; }

int chebfi_batch_autotune(chebfi_batch* bt, int prec, int* shapes, double* ms) {
  BAPI_BEGIN(bt)
  CHEBFI_REQUIRE(prec == CHEBFI_F64 || prec == CHEBFI_F32 || prec == CHEBFI_MIXED, CHEBFI_ERR_ARG,
                 "the batch runs the FP64, FP32 or mixed form");
  CHEBFI_REQUIRE(prec != CHEBFI_MIXED || bt->nq > 0, CHEBFI_ERR_ARG, "the mixed batch needs projectors");
  const int f = prec == CHEBFI_F64 ? 0 : 1;
  if (prec == CHEBFI_F64) autotune<double>(bt, 0);
  else autotune<float>(bt, 0);
  CHEBFI_CUDA(cudaDeviceSynchronize());
  for (int gc = 0; gc < GC_N; ++gc) {
    if (shapes) shapes[gc] = bt->shape[f][gc];
    if (ms)
      for (int s = 0; s < kNumShapes; ++s) ms[gc * kNumShapes + s] = bt->tune_ms[f][gc][s];
  }
  if (shapes) shapes[GC_N] = bt->split[f];
  if (ms)
    for (int i = 0; i < 4; ++i) ms[GC_N * kNumShapes + i] = bt->split_ms[f][i];
  BAPI_END(bt)
}

int chebfi_batch_set_tiles(chebfi_batch* bt, int prec, const int* shapes, int split) {
  BAPI_BEGIN(bt)
  CHEBFI_REQUIRE(prec == CHEBFI_F64 || prec == CHEBFI_F32 || prec == CHEBFI_MIXED, CHEBFI_ERR_ARG,
                 "the batch runs the FP64, FP32 or mixed form");
  CHEBFI_REQUIRE(prec != CHEBFI_MIXED || bt->nq > 0, CHEBFI_ERR_ARG, "the mixed batch needs projectors");
  CHEBFI_REQUIRE(shapes, CHEBFI_ERR_ARG, "null shapes");
  for (int gc = 0; gc < GC_N; ++gc)
    CHEBFI_REQUIRE(shapes[gc] >= 0 && shapes[gc] < kNumShapes, CHEBFI_ERR_ARG, "tile shape index out of range");
  CHEBFI_REQUIRE(split == 1 || split == 2 || split == 4 || split == 8, CHEBFI_ERR_ARG, "split-K factor must be 1, 2, 4 or 8");
  const int f = prec == CHEBFI_F64 ? 0 : 1;
  // occupancy and buffers as the autotuner would have set them
  if (prec == CHEBFI_F64) autotune<double>(bt, 0);
  else autotune<float>(bt, 0);
  CHEBFI_CUDA(cudaDeviceSynchronize());
  for (int gc = 0; gc < GC_N; ++gc) bt->shape[f][gc] = shapes[gc];
  bt->split[f] = split;
  // graphs captured with the previous tiles are stale
  for (auto it = bt->graphs.begin(); it != bt->graphs.end();) {
    if (it->first.first == f) {
      cudaGraphExecDestroy(it->second);
      it = bt->graphs.erase(it);
    } else {
      ++it;
    }
  }
  BAPI_END(bt)
}

int chebfi_batch_cheb_filter(chebfi_batch* bt, void* const* Y, const int64_t* ld, int degree, const double* lambda_lo,
                             const double* lambda_hi, int prec, void* stream) {
  BAPI_BEGIN(bt)
  CHEBFI_REQUIRE(Y && ld && lambda_lo && lambda_hi, CHEBFI_ERR_ARG, "null argument");
  CHEBFI_REQUIRE(degree >= 0 && degree <= 1000, CHEBFI_ERR_ARG, "degree out of range");
  CHEBFI_REQUIRE(prec == CHEBFI_F64 || prec == CHEBFI_F32 || prec == CHEBFI_MIXED, CHEBFI_ERR_ARG,
                 "the batch runs the FP64, FP32 or mixed form");
  CHEBFI_REQUIRE(prec != CHEBFI_MIXED || bt->nq > 0, CHEBFI_ERR_ARG, "the mixed batch needs projectors");
  for (int k = 0; k < bt->nk; ++k) {
    CHEBFI_REQUIRE(Y[k] && ld[k] >= bt->npw[k], CHEBFI_ERR_ARG, "bad block of k-point " + std::to_string(k));
    CHEBFI_REQUIRE(std::isfinite(lambda_lo[k]) && std::isfinite(lambda_hi[k]) && lambda_hi[k] > lambda_lo[k],
                   CHEBFI_ERR_ARG, "need finite lambda_lo < lambda_hi at k-point " + std::to_string(k));
  }
  if (degree == 0) return CHEBFI_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (prec == CHEBFI_F64) batch_filter<double>(bt, Y, ld, degree, lambda_lo, lambda_hi, st);
  else batch_filter<float>(bt, Y, ld, degree, lambda_lo, lambda_hi, st, prec == CHEBFI_MIXED);
  BAPI_END(bt)
}

}  // extern "C"
