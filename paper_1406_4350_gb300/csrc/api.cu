// C ABI of libchebfi: context, setup (Section 2.1 operators, Section 5.1 Woodbury core),
// and the orchestration of Algorithm 2 (filter, Rayleigh-Ritz, sweeps) on the device.
//
// Internally every wavefunction block is kept in "column-sorted" plane-wave order (the
// sphere points of one (x, y) FFT column are contiguous, z ascending), which makes the
// FFT passes read contiguous runs; the caller's order is restored at the ABI.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <stdexcept>
#include <vector>
#include <complex>
#include <functional>
#include <type_traits>

#include "internal.cuh"
#include "kernels.cuh"

namespace chebfi {

thread_local int64_t* g_launch_counter = nullptr;
thread_local Profiler* g_prof = nullptr;

cudaEvent_t Profiler::get() {
  if (pool.empty()) {
    cudaEvent_t e;
    CHEBFI_CUDA(cudaEventCreate(&e));
    return e;
  }
  cudaEvent_t e = pool.back();
  pool.pop_back();
  return e;
}

void Profiler::flush() {
  if (pending.empty()) return;
  CHEBFI_CUDA(cudaEventSynchronize(pending.back().b));
  for (const Rec& r : pending) {
    float t = 0.f;
    CHEBFI_CUDA(cudaEventElapsedTime(&t, r.a, r.b));
    size_t i = 0;
    while (i < names.size() && names[i] != r.name) ++i;
    if (i == names.size()) {
      names.push_back(r.name);
      ms.push_back(0.0);
      count.push_back(0);
      work.push_back(0.0);
    }
    ms[i] += t;
    count[i] += 1;
    work[i] += r.work;
    pool.push_back(r.a);
    pool.push_back(r.b);
  }
  pending.clear();
}

Profiler::~Profiler() {
  for (const Rec& r : pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : pool) cudaEventDestroy(e);
}

void prof_begin(const char* name, cudaStream_t st, double work) {
  if (!g_prof || !g_prof->on) return;
  g_prof->cur = name;
  g_prof->cur_work = work;
  g_prof->cur_a = g_prof->get();
  CHEBFI_CUDA(cudaEventRecord(g_prof->cur_a, st));
}

void prof_end(cudaStream_t st) {
  if (!g_prof || !g_prof->on || !g_prof->cur_a) return;
  cudaEvent_t b = g_prof->get();
  CHEBFI_CUDA(cudaEventRecord(b, st));
  g_prof->pending.push_back({g_prof->cur, g_prof->cur_a, b, g_prof->cur_work});
  g_prof->cur_a = nullptr;
  if (g_prof->pending.size() >= 8192) g_prof->flush();
}

void after_launch(const char* name) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error{CHEBFI_ERR_CUDA, std::string("launch of ") + name + ": " + cudaGetErrorString(e)};
  if (g_launch_counter) ++*g_launch_counter;
}

namespace {

__global__ void k_dense_from_blocks(int64_t nproj, const int32_t* atom_of, const int32_t* offs, const int64_t* blk_off,
                                    const double* blk, double2* out) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nproj * nproj) return;
  const int64_t i = idx % nproj, j = idx / nproj;
  const int a = atom_of[i];
  double v = 0.0;
  if (atom_of[j] == a) {
    const int o = offs[a], na = offs[a + 1] - o;
    v = blk[blk_off[a] + (i - o) * na + (j - o)];
  }
  out[idx] = make_double2(v, 0.0);
}

__global__ void k_add_identity(int64_t n, double2* A, int64_t lda) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) A[i + i * lda].x += 1.0;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }

void check_status(chebfi_ctx* ctx, cudaStream_t st, const char* where) {
  int h = 0;
  CHEBFI_CUDA(cudaMemcpyAsync(&h, ctx->d_status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
  CHEBFI_CUDA(cudaStreamSynchronize(st));
  if (h != 0) {
    int zero = 0;
    CHEBFI_CUDA(cudaMemcpy(ctx->d_status.p, &zero, sizeof(int), cudaMemcpyHostToDevice));
    const char* what = h == CHEBFI_ERR_NOT_SPD ? "matrix not positive definite"
                       : h == CHEBFI_ERR_NONFINITE ? "Inf or NaN in the block or matrix"
                       : h == CHEBFI_ERR_NO_CONVERGENCE ? "Jacobi eigensolver did not converge"
                                                         : "device error";
    throw Error{h, std::string(where) + ": " + what};
  }
}

void require_ready(const chebfi_ctx* ctx) {
  CHEBFI_REQUIRE(ctx->has_cell && ctx->has_sphere && ctx->has_vloc && ctx->has_proj, CHEBFI_ERR_STATE,
                 "set_cell, set_sphere, set_vloc and set_projectors must all be called first");
}

void require_block(const chebfi_ctx* ctx, const void* Y, int64_t nb, int64_t ld) {
  CHEBFI_REQUIRE(nb >= 0, CHEBFI_ERR_ARG, "nb must be >= 0");
  CHEBFI_REQUIRE(ld >= ctx->npw, CHEBFI_ERR_ARG, "ld must be >= npw");
  CHEBFI_REQUIRE(nb == 0 || Y != nullptr, CHEBFI_ERR_ARG, "null wavefunction pointer");
}

// ------------------------------------------------------------------ operator pieces (sorted order)
template <typename R> struct Ops;
template <> struct Ops<double> {
  static const double2* P(const chebfi_ctx* c) { return c->d_P.p; }
  static const double2* G(const chebfi_ctx* c) { return c->d_G.p; }
  static const double2* M(const chebfi_ctx* c) { return c->d_M.p; }
  static const double* D(const chebfi_ctx* c) { return c->d_Dblk.p; }
  static DevBuf<double2>* ws(chebfi_ctx* c) { return &c->w.splitk; }
  static DevBuf<double2>& pool(chebfi_ctx* c) { return c->w.gpool; }
  static DevBuf<double2>& T(chebfi_ctx* c) { return c->w.T1; }
  static DevBuf<double2>& pa(chebfi_ctx* c) { return c->w.pz; }
  static DevBuf<double2>& pb(chebfi_ctx* c) { return c->w.pw; }
};
template <> struct Ops<float> {
  static const float2* P(const chebfi_ctx* c) { return c->d_Pf.p; }
  static const float2* G(const chebfi_ctx* c) { return c->d_Gf.p; }
  static const float2* M(const chebfi_ctx* c) { return c->d_Mf.p; }
  static const float* D(const chebfi_ctx* c) { return c->d_Dblkf.p; }
  static DevBuf<float2>* ws(chebfi_ctx* c) { return &c->w.fsplitk; }
  static DevBuf<float2>& pool(chebfi_ctx* c) { return c->w.fgpool; }
  static DevBuf<float2>& T(chebfi_ctx* c) { return c->w.fT1; }
  static DevBuf<float2>& pa(chebfi_ctx* c) { return c->w.fpz; }
  static DevBuf<float2>& pb(chebfi_ctx* c) { return c->w.fpw; }
};

// ------------------------------------------------------------------ FP64 GEMM routing
// FP64 complex GEMMs large enough to amortise the operand preparation run on the tensor
// cores through the modular emulation (ozaki.cu), the others on the CUDA cores; the context
// can force either engine (chebfi_set_fp64_gemm).
bool use_tensor_fp64(const chebfi_ctx* ctx, int64_t M, int64_t N, int64_t K) {
  if (M <= 0 || N <= 0 || K <= 0 || ctx->fp64_gemm == CHEBFI_GEMM_CUDA_CORES) return false;
  if (ctx->fp64_gemm == CHEBFI_GEMM_TENSOR) return true;
  return K >= 64 && 8.0 * (double)M * (double)N * (double)K >= 1e9;
}

// residues of P^H (conj) or P as the A operand, kept while the modulus count is unchanged
const OzOperand& oz_P(chebfi_ctx* ctx, bool conj, cudaStream_t st) {
  OzOperand& o = conj ? ctx->ozPh : ctx->ozP;
  if (o.nmod != ctx->oz_nmod)
    oz_prepare(ctx->d_P.p, ctx->npw, conj ? ctx->nproj : ctx->npw, conj ? ctx->npw : ctx->nproj, conj, conj, true,
               ctx->oz_nmod, o, st);
  return o;
}

// C = alpha op(A) op(B) + beta C in FP64 (the signature of gemm<double> with the context first)
void gemm64(chebfi_ctx* ctx, bool conjA, bool conjB, int64_t M, int64_t N, int64_t K, double alpha, const double2* A,
            int64_t lda, const double2* B, int64_t ldb, double beta, double2* C, int64_t ldc, cudaStream_t st,
            DevBuf<double2>* ws = nullptr, const char* tag = "k_gemm", bool lower = false) {
  if (!use_tensor_fp64(ctx, M, N, K)) {
    gemm<double>(conjA, conjB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, ws, tag, lower);
    return;
  }
  OzWork& z = ctx->oz;
  const OzOperand* a = &z.A;
  const bool is_P = ctx->has_proj && A == ctx->d_P.p && lda == ctx->npw &&
                    (conjA ? (M == ctx->nproj && K == ctx->npw) : (M == ctx->npw && K == ctx->nproj));
  if (is_P) a = &oz_P(ctx, conjA, st);
  else oz_prepare(A, lda, M, K, conjA, conjA, true, ctx->oz_nmod, z.A, st);
  oz_prepare(B, ldb, N, K, !conjB, conjB, false, ctx->oz_nmod, z.B, st);
  oz_gemm(*a, z.B, alpha, beta, C, ldc, lower, z.R, ctx->d_status.p, st, tag);
}

// A = L L^H (A's lower triangle becomes L, its upper triangle zero) and Li = L^{-1}, by
// halving: with A = [A11 .; A21 A22],
//   L11, Li11 from A11;  L21 = A21 Li11^H;  A22 <- A22 - L21 L21^H;  L22, Li22 from A22;
//   Li21 = -Li22 L21 Li11,
// so all but the leaves (n <= 256: the blocked kernels) are FP64-accurate GEMMs on the
// tensor cores.  T: scratch of n^2 / 2 complex values.
void chol_inv(chebfi_ctx* ctx, int64_t n, double2* A, int64_t lda, double2* Li, int64_t ldi, double2* T,
              cudaStream_t st) {
  DevBuf<double2>* ws = &ctx->w.splitk;
  if (n <= 256) {
    cholesky(n, A, lda, ctx->d_status.p, st, ws);
    set_identity(n, Li, ldi, st);
    trsm_lower(n, n, A, lda, Li, ldi, st, ws);
    return;
  }
  const int64_t n1 = (n / 2 + 31) / 32 * 32, n2 = n - n1;
  double2 *A21 = A + n1, *A22 = A + n1 + n1 * lda, *Li11 = Li, *Li21 = Li + n1, *Li22 = Li + n1 + n1 * ldi;
  const size_t z = sizeof(double2);
  chol_inv(ctx, n1, A, lda, Li11, ldi, T, st);
  gemm64(ctx, false, true, n2, n1, n1, 1.0, A21, lda, Li11, ldi, 0.0, T, n2, st, ws, "gemm_chol");
  CHEBFI_CUDA(cudaMemcpy2DAsync(A21, lda * z, T, n2 * z, n2 * z, n1, cudaMemcpyDeviceToDevice, st));
  gemm64(ctx, false, true, n2, n2, n1, -1.0, A21, lda, A21, lda, 1.0, A22, lda, st, ws, "gemm_chol");
  chol_inv(ctx, n2, A22, lda, Li22, ldi, T, st);
  gemm64(ctx, false, false, n2, n1, n1, 1.0, A21, lda, Li11, ldi, 0.0, T, n2, st, ws, "gemm_chol");
  gemm64(ctx, false, false, n2, n1, n2, -1.0, Li22, ldi, T, n2, 0.0, Li21, ldi, st, ws, "gemm_chol");
  CHEBFI_CUDA(cudaMemset2DAsync(A + n1 * lda, lda * z, 0, n1 * z, n2, st));   // upper blocks
  CHEBFI_CUDA(cudaMemset2DAsync(Li + n1 * ldi, ldi * z, 0, n1 * z, n2, st));
}

// the GEMM of the form's precision: FP64 through gemm64, FP32 on the CUDA cores
template <typename R>
void cgemm(chebfi_ctx* ctx, bool conjA, bool conjB, int64_t M, int64_t N, int64_t K, double alpha, const cplx<R>* A,
           int64_t lda, const cplx<R>* B, int64_t ldb, double beta, cplx<R>* C, int64_t ldc, cudaStream_t st,
           DevBuf<cplx<R>>* ws = nullptr, const char* tag = "k_gemm", bool lower = false) {
  if constexpr (std::is_same<R, double>::value) gemm64(ctx, conjA, conjB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, ws, tag, lower);
  else gemm<R>(conjA, conjB, M, N, K, alpha, A, lda, B, ldb, beta, C, ldc, st, ws, tag, lower);
}

// H Y (FP64 or FP32) with the projections p = P^H Y returned; sorted order, ld = npw.
template <typename R>
void apply_H_sorted(chebfi_ctx* ctx, const cplx<R>* Y, cplx<R>* HY, cplx<R>* p, cplx<R>* Dp, cplx<R>* T, int64_t nb,
                    cudaStream_t st, const char* tag = "gemm_H") {
  const int64_t npw = ctx->npw, nq = ctx->nproj;
  LocalEpi<R> ep;
  ep.Y = Y;
  ep.ldy = npw;
  ep.Z = HY;
  ep.ldz = npw;
  local_apply<R>(ctx, Y, npw, nb, T, ep, st);
  if (nq > 0) {
    cgemm<R>(ctx, true, false, nq, nb, npw, 1.0, Ops<R>::P(ctx), npw, Y, npw, 0.0, p, nq, st, Ops<R>::ws(ctx), tag);
    blockdiag_apply<R>(ctx, Ops<R>::D(ctx), p, nq, Dp, nq, nb, st);
    cgemm<R>(ctx, false, false, npw, nb, nq, 1.0, Ops<R>::P(ctx), npw, Dp, nq, 1.0, HY, npw, st, Ops<R>::ws(ctx), tag);
  }
}

// Locking (Section 5.4): bands [m_next, m) have reached their own degree; their iterate, in
// the buffer `cur`, goes to its column of the result buffer, which later steps leave alone.
template <typename R>
void keep_finished(int64_t npw, const cplx<R>* cur, cplx<R>* result, int64_t m_next, int64_t m, cudaStream_t st) {
  if (cur == result || m <= m_next) return;
  CHEBFI_CUDA(cudaMemcpyAsync(result + m_next * npw, cur + m_next * npw, sizeof(cplx<R>) * npw * (m - m_next),
                              cudaMemcpyDeviceToDevice, st));
}

template <typename R> struct FilterBufs {
  cplx<R>*Ya, *Yb, *Z, *T, *pa, *pb, *pz, *pw, *pq;
};

// Algorithm 2's inner loop with the projection-reuse identity of Section 5.1, in place on
// Y (sorted, ld = npw, its buffer is bufs.Ya on entry).  Returns the buffer holding Y_n.
template <typename R>
cplx<R>* filter_sorted(chebfi_ctx* ctx, FilterBufs<R> b, int64_t nb0, int degree, double lo, double hi,
                       cudaStream_t st, const int64_t* active = nullptr, const double2* p0 = nullptr) {
  const int64_t npw = ctx->npw, nq = ctx->nproj;
  const double c = 0.5 * (hi + lo), r = 0.5 * (hi - lo);
  cplx<R>*cur = b.Ya, *prev = b.Yb, *pcur = b.pa, *pprev = b.pb;
  if (nq > 0 && p0) {
    // p_0 = P^H Y_0 handed over by the Rayleigh-Ritz step that produced Y_0
    if constexpr (std::is_same<R, double>::value)
      CHEBFI_CUDA(cudaMemcpyAsync(pcur, p0, sizeof(double2) * nq * nb0, cudaMemcpyDeviceToDevice, st));
    else
      convert(nq, nb0, p0, nq, pcur, nq, st);
  } else if (nq > 0) {
    cgemm<R>(ctx, true, false, nq, active ? active[0] : nb0, npw, 1.0, Ops<R>::P(ctx), npw, cur, npw, 0.0, pcur, nq, st,
            Ops<R>::ws(ctx), "gemm_PhY");
  }
  for (int k = 0; k < degree; ++k) {
    const int64_t nb = active ? active[k] : nb0;  // bands still being filtered (a prefix)
    const double a = (k == 0 ? 1.0 : 2.0) / r;
    const double bp = k == 0 ? 0.0 : 1.0;
    // Z = (K + V_loc) Y_k and T = a (Z - c Y_k) - bp Y_{k-1}, T written over Y_{k-1}
    LocalEpi<R> ep;
    ep.Y = cur;
    ep.ldy = npw;
    ep.Z = nq > 0 ? b.Z : nullptr;
    ep.ldz = npw;
    ep.T = prev;
    ep.Yprev = k == 0 ? nullptr : prev;
    ep.ldt = npw;
    ep.a = (R)a;
    ep.c = (R)c;
    ep.bprev = (R)bp;
    local_apply<R>(ctx, cur, npw, nb, b.T, ep, st);
    if (nq > 0) {
      // P^H H Y_k = P^H Z + G D p_k
      cgemm<R>(ctx, true, false, nq, nb, npw, 1.0, Ops<R>::P(ctx), npw, b.Z, npw, 0.0, b.pz, nq, st, Ops<R>::ws(ctx),
              "gemm_PhY");
      blockdiag_apply<R>(ctx, Ops<R>::D(ctx), pcur, nq, b.pw, nq, nb, st);
      cgemm<R>(ctx, false, false, nq, nb, nq, 1.0, Ops<R>::G(ctx), nq, b.pw, nq, 1.0, b.pz, nq, st, Ops<R>::ws(ctx),
              "gemm_small");
      if (ctx->paw) {
        // q = M P^H H Y_k;  W = D p_k - q;  P^H S^{-1} H Y_k = P^H H Y_k - G q
        cgemm<R>(ctx, false, false, nq, nb, nq, 1.0, Ops<R>::M(ctx), nq, b.pz, nq, 0.0, b.pq, nq, st, Ops<R>::ws(ctx),
                "gemm_small");
        axpby<R>(nq, nb, (R)1, b.pw, nq, (R)-1, b.pq, nq, b.pw, nq, st);
        cgemm<R>(ctx, false, false, nq, nb, nq, -1.0, Ops<R>::G(ctx), nq, b.pq, nq, 1.0, b.pz, nq, st, Ops<R>::ws(ctx),
                "gemm_small");
      }
      // Y_{k+1} = T + a P W
      cgemm<R>(ctx, false, false, npw, nb, nq, a, Ops<R>::P(ctx), npw, b.pw, nq, 1.0, prev, npw, st, Ops<R>::ws(ctx),
              "gemm_PW");
      // p_{k+1} = a (P^H S^{-1} H Y_k - c p_k) - bp p_{k-1}
      cheb_combine<R>(nq, nb, (R)a, b.pz, nq, (R)c, pcur, nq, (R)bp, k == 0 ? nullptr : pprev, nq, pprev, nq, st);
    }
    std::swap(cur, prev);
    std::swap(pcur, pprev);
    if (active) keep_finished<R>(npw, cur, b.Ya, k + 1 < degree ? active[k + 1] : 0, nb, st);
  }
  return active ? b.Ya : cur;
}

// bf16 (hi, lo) operands of the tensor-core GEMMs, built on first use: the real embeddings
// of G and M, of P^H (the P^H Z product) and, with P_too, of P (the batched k-points' P W);
// and the (Re, Im, Re + Im) planes of P for the three-multiplication P W of a single problem.
// P^H Z keeps the real embedding: its two operands are both long streams, and the three
// products of the plane form re-read them from DRAM several times more (measured), which
// costs more than the quarter of the tensor work it saves; P W's W fits in L2.
void ensure_tc(chebfi_ctx* ctx, cudaStream_t st, bool P_too = false) {
  if (ctx->nproj == 0) return;
  const int64_t npw = ctx->npw, nq = ctx->nproj;
  if (!ctx->tc_ready) {
    embed_n(nq, nq, ctx->d_G.p, nq, ctx->tcAG, st);
    if (ctx->paw) embed_n(nq, nq, ctx->d_M.p, nq, ctx->tcAM, st);
    embed_ph(npw, nq, ctx->d_P.p, npw, ctx->tcA1, st);
    ctx->tc_ready = true;
  }
  if (P_too && !ctx->tcP_ready) {
    embed_n(npw, nq, ctx->d_P.p, npw, ctx->tcA2, st);
    ctx->tcP_ready = true;
  }
}

void ensure_tc3(chebfi_ctx* ctx, cudaStream_t st) {
  if (ctx->tc3_ready || ctx->nproj == 0) return;
  embed3_n(ctx->npw, ctx->nproj, ctx->d_P.p, ctx->npw, ctx->tcP3, st);
  ctx->tc3_ready = true;
}

// Mixed form of the filter: FP32 iterates and FFT, projector GEMMs on the tensor cores
// with split bf16 operands.  Same steps as filter_sorted; Y_0 and the result are the FP32
// buffers b.Ya / returned pointer.
float2* filter_mixed(chebfi_ctx* ctx, FilterBufs<float> b, int64_t nb0, int degree, double lo, double hi,
                     cudaStream_t st, const int64_t* active = nullptr, const double2* p0 = nullptr) {
  const int64_t nb = active ? active[0] : nb0;
  const int64_t npw = ctx->npw, nq = ctx->nproj;
  const double c = 0.5 * (hi + lo), r = 0.5 * (hi - lo);
  Work& w = ctx->w;
  int* status = ctx->d_status.p;
  float2 *cur = b.Ya, *prev = b.Yb, *pcur = b.pa, *pprev = b.pb;
  const int64_t ldzb = (2 * npw + 7) / 8 * 8;
  if (nq > 0) {
    ensure_tc(ctx, st);
    ensure_tc3(ctx, st);
    w.Zb.ld = ldzb;
    w.Zb.alloc((size_t)ldzb * nb);
    if (p0) {
      convert(nq, nb, p0, nq, pcur, nq, st);  // FP64 projections from the Rayleigh-Ritz step
    } else {
      split_block(npw, nb, cur, npw, w.Zb, st);
      tc_gemm(ctx->tcA1.view(), w.Zb.view(), 2 * nq, nb, 2 * npw, 1.f, 0.f, nullptr, 0, (float*)pcur, 2 * nq, status,
              st, "tc_gemm_PhY", &ctx->w.tcws);
    }
  }
  for (int k = 0; k < degree; ++k) {
    const int64_t nb = active ? active[k] : nb0;  // bands still being filtered (a prefix)
    const double a = (k == 0 ? 1.0 : 2.0) / r;
    const double bp = k == 0 ? 0.0 : 1.0;
    LocalEpi<float> ep;
    ep.Y = cur;
    ep.ldy = npw;
    if (nq > 0) {
      ep.Zhi = w.Zb.hi.p;
      ep.Zlo = w.Zb.lo.p;
      ep.ldzb = ldzb;
    }
    ep.T = prev;
    ep.Yprev = k == 0 ? nullptr : prev;
    ep.ldt = npw;
    ep.a = (float)a;
    ep.c = (float)c;
    ep.bprev = (float)bp;
    local_apply<float>(ctx, cur, npw, nb, b.T, ep, st);
    if (nq > 0) {
      // P^H H Y_k = P^H Z + G D p_k
      tc_gemm(ctx->tcA1.view(), w.Zb.view(), 2 * nq, nb, 2 * npw, 1.f, 0.f, nullptr, 0, (float*)b.pz, 2 * nq, status,
              st, "tc_gemm_PhY", &ctx->w.tcws);
      blockdiag_apply<float>(ctx, ctx->d_Dblkf.p, pcur, nq, b.pw, nq, nb, st);
      split_block(nq, nb, b.pw, nq, w.Sb, st);
      tc_gemm(ctx->tcAG.view(), w.Sb.view(), 2 * nq, nb, 2 * nq, 1.f, 1.f, (float*)b.pz, 2 * nq, (float*)b.pz, 2 * nq,
              status, st, "tc_gemm_small", &ctx->w.tcws);
      if (ctx->paw) {
        split_block(nq, nb, b.pz, nq, w.Sb, st);
        tc_gemm(ctx->tcAM.view(), w.Sb.view(), 2 * nq, nb, 2 * nq, 1.f, 0.f, nullptr, 0, (float*)b.pq, 2 * nq, status,
                st, "tc_gemm_small", &ctx->w.tcws);
        axpby<float>(nq, nb, 1.f, b.pw, nq, -1.f, b.pq, nq, b.pw, nq, st);
        split_block(nq, nb, b.pq, nq, w.Sb, st);
        tc_gemm(ctx->tcAG.view(), w.Sb.view(), 2 * nq, nb, 2 * nq, -1.f, 1.f, (float*)b.pz, 2 * nq, (float*)b.pz,
                2 * nq, status, st, "tc_gemm_small", &ctx->w.tcws);
      }
      // Y_{k+1} = T + a P W
      split3_block(nq, nb, b.pw, nq, w.W3, st);
      tc_cgemm3(ctx->tcP3, w.W3, false, npw, nb, nq, (float)a, 1.f, prev, npw, prev, npw, status, st, "tc_gemm_PW",
                &ctx->w.tcws);
      cheb_combine<float>(nq, nb, (float)a, b.pz, nq, (float)c, pcur, nq, (float)bp, k == 0 ? nullptr : pprev, nq,
                          pprev, nq, st);
    }
    std::swap(cur, prev);
    std::swap(pcur, pprev);
    if (active) keep_finished<float>(npw, cur, b.Ya, k + 1 < degree ? active[k + 1] : 0, nb, st);
  }
  return active ? b.Ya : cur;
}

void ensure_filter_ws(chebfi_ctx* ctx, int64_t nb, int prec) {
  const size_t ny = (size_t)ctx->npw * nb, np = (size_t)std::max<int64_t>(ctx->nproj, 1) * nb;
  const size_t nt = local_workspace_elems(ctx, nb);
  Work& w = ctx->w;
  w.Ya.alloc(ny);
  if (prec == CHEBFI_F64) {
    w.Yb.alloc(ny);
    w.Z.alloc(ny);
    w.T1.alloc(nt);
    w.pa.alloc(np);
    w.pb.alloc(np);
    w.pz.alloc(np);
    w.pw.alloc(np);
    w.pq.alloc(np);
  } else {
    w.fYa.alloc(ny);
    w.fYb.alloc(ny);
    w.fZ.alloc(ny);
    w.fT1.alloc(nt);
    w.fpa.alloc(np);
    w.fpb.alloc(np);
    w.fpz.alloc(np);
    w.fpw.alloc(np);
    w.fpq.alloc(np);
  }
}

// Filter on the sorted FP64 block ctx->w.Ya (in place).  p0: P^H Y_0 when already known
// (the rotated projections of the Rayleigh-Ritz step that produced Y_0), else null.
void filter_on_Ya(chebfi_ctx* ctx, int64_t nb, int degree, double lo, double hi, int prec, cudaStream_t st,
                  const double2* p0 = nullptr) {
  ensure_filter_ws(ctx, nb, prec);
  Work& w = ctx->w;
  const int64_t npw = ctx->npw;
  w.pc_of = nullptr;  // the filter replaces the block
  if (prec == CHEBFI_F64) {
    FilterBufs<double> b{w.Ya.p, w.Yb.p, w.Z.p, w.T1.p, w.pa.p, w.pb.p, w.pz.p, w.pw.p, w.pq.p};
    double2* out = filter_sorted<double>(ctx, b, nb, degree, lo, hi, st, nullptr, p0);
    if (out != w.Ya.p) CHEBFI_CUDA(cudaMemcpyAsync(w.Ya.p, out, sizeof(double2) * npw * nb, cudaMemcpyDeviceToDevice, st));
  } else {
    convert(npw, nb, w.Ya.p, npw, w.fYa.p, npw, st);
    FilterBufs<float> b{w.fYa.p, w.fYb.p, w.fZ.p, w.fT1.p, w.fpa.p, w.fpb.p, w.fpz.p, w.fpw.p, w.fpq.p};
    float2* out = prec == CHEBFI_MIXED ? filter_mixed(ctx, b, nb, degree, lo, hi, st, nullptr, p0)
                                       : filter_sorted<float>(ctx, b, nb, degree, lo, hi, st, nullptr, p0);
    convert(npw, nb, out, npw, w.Ya.p, npw, st);
  }
}


// Locking (Section 5.4): band j of the sorted FP64 block w.Ya filtered to its own degree
// deg[j].  Bands are reordered by decreasing degree so that the bands still filtered at
// step k form a prefix of the block; each step then runs on that prefix only.
void filter_on_Ya_adaptive(chebfi_ctx* ctx, int64_t nb, const std::vector<int>& deg, double lo, double hi, int prec,
                           cudaStream_t st) {
  const int dmax = nb ? *std::max_element(deg.begin(), deg.end()) : 0;
  if (dmax == 0) return;
  std::vector<int32_t> order(nb);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) { return deg[a] > deg[b]; });
  std::vector<int64_t> active(dmax, 0);
  for (int k = 0; k < dmax; ++k)
    for (int64_t j = 0; j < nb; ++j) active[k] += deg[j] > k ? 1 : 0;
  ensure_filter_ws(ctx, nb, prec);
  Work& w = ctx->w;
  const int64_t npw = ctx->npw;
  w.Yc.alloc((size_t)npw * nb);
  w.order.upload(order.data(), nb, st);
  permute_cols(npw, nb, w.order.p, w.Ya.p, w.Yc.p, false, st);
  if (prec == CHEBFI_F64) {
    FilterBufs<double> b{w.Yc.p, w.Yb.p, w.Z.p, w.T1.p, w.pa.p, w.pb.p, w.pz.p, w.pw.p, w.pq.p};
    filter_sorted<double>(ctx, b, nb, dmax, lo, hi, st, active.data());
  } else {
    convert(npw, nb, w.Yc.p, npw, w.fYa.p, npw, st);
    FilterBufs<float> b{w.fYa.p, w.fYb.p, w.fZ.p, w.fT1.p, w.fpa.p, w.fpb.p, w.fpz.p, w.fpw.p, w.fpq.p};
    if (prec == CHEBFI_MIXED) filter_mixed(ctx, b, nb, dmax, lo, hi, st, active.data());
    else filter_sorted<float>(ctx, b, nb, dmax, lo, hi, st, active.data());
    // only the filtered prefix comes back: locked bands keep their FP64 values untouched
    convert(npw, active[0], w.fYa.p, npw, w.Yc.p, npw, st);
  }
  permute_cols(npw, nb, w.order.p, w.Yc.p, w.Ya.p, true, st);
}

// Section 5.4's degree estimate: the smallest n in 1..max_degree with
// ||r_i|| <= tol |T_n((lambda_i - c)/r)|, max_degree if none, 0 when ||r_i|| <= tol.
void degrees_for_tolerance(const double* ritz, const double* resid, int64_t nb, double lo, double hi, double tol,
                           int max_degree, int* deg) {
  const double c = 0.5 * (hi + lo), r = 0.5 * (hi - lo);
  for (int64_t i = 0; i < nb; ++i) {
    if (resid[i] <= tol) {
      deg[i] = 0;
      continue;
    }
    const double x = (ritz[i] - c) / r;
    double t_prev = 1.0, t = x;  // T_0, T_1 by the recurrence of Section 4.2
    int n_i = max_degree;
    for (int n = 1; n <= max_degree; ++n) {
      if (n > 1) {
        const double t_next = 2.0 * x * t - t_prev;
        t_prev = t;
        t = t_next;
      }
      if (resid[i] <= tol * std::fabs(t)) {
        n_i = n;
        break;
      }
    }
    deg[i] = n_i;
  }
}


// Rayleigh quotients of the sorted FP64 block Y.
void rq_sorted(chebfi_ctx* ctx, const double2* Y, int64_t nb, double* rq, cudaStream_t st) {
  Work& w = ctx->w;
  const int64_t npw = ctx->npw, nq = ctx->nproj;
  const size_t np = (size_t)std::max<int64_t>(nq, 1) * nb;
  w.HY.alloc((size_t)npw * nb);
  w.T1.alloc(local_workspace_elems(ctx, nb));
  w.pa.alloc(np);
  w.pb.alloc(np);
  w.dvec1.alloc(nb);
  w.dvec2.alloc(nb);
  apply_H_sorted<double>(ctx, Y, w.HY.p, w.pa.p, w.pb.p, w.T1.p, nb, st);
  column_dots(npw, nb, Y, npw, w.HY.p, npw, w.dvec1.p, false, st);
  column_dots(npw, nb, Y, npw, Y, npw, w.dvec2.p, false, st);
  if (ctx->paw) {
    blockdiag_apply<double>(ctx, ctx->d_Qblk.p, w.pa.p, nq, w.pb.p, nq, nb, st);
    column_dots(nq, nb, w.pa.p, nq, w.pb.p, nq, w.dvec2.p, true, st);
  }
  divide(nb, w.dvec1.p, w.dvec2.p, rq, st);
}

// Dense Hermitian eigenproblem of the Rayleigh-Ritz step (Algorithm 2; the paper calls
// ELPA): A (n x n, ld n) -> ascending eigenvalues w and orthonormal eigenvectors X (ld n).
// FP64 cyclic Jacobi for small n; from n = 512 up (or when selected) the FP32 Jacobi gives
// approximate vectors, which the iterative refinement of Ogita & Aishima (2018) brings to
// FP64 accuracy with FP64 GEMMs (quadratic convergence, 2-4 steps), or, for a nearly
// diagonal A, the refinement starts from the identity; pairs too close for its formula end
// in a dense FP64 Jacobi of their cluster's block.  A is destroyed.
void eigh_rr(chebfi_ctx* ctx, int64_t n, double2* A, double* w, double2* X, cudaStream_t st) {
  Work& wk = ctx->w;
  int* status = ctx->d_status.p;
  const bool refined = ctx->eig_mode == CHEBFI_EIG_REFINED || (ctx->eig_mode == CHEBFI_EIG_AUTO && n >= 512);
  ctx->eig_iters = 0;
  if (!refined || n < 2) {
    jacobi_eigh(n, A, n, w, X, n, status, st, &wk.small5);
    return;
  }
  check_status(ctx, st, "rayleigh_ritz");  // a non-finite block was flagged before the Gram matrices
  const size_t nn = (size_t)n * n;
  constexpr int kCap = 1 << 16;
  wk.e32a.alloc(nn);
  wk.e32b.alloc(nn);
  wk.e32w.alloc(n);
  wk.eG.alloc(nn);
  wk.eS.alloc(nn);
  wk.eAX.alloc(nn);
  wk.eM.alloc(nn);
  wk.eX.alloc(nn);
  wk.elam.alloc(n);
  wk.estats.alloc(2);
  wk.enp.alloc(1);
  wk.epairs.alloc(kCap);
  DevBuf<double2>* ws = &wk.splitk;
  double2 *Xc = X, *Xn = wk.eX.p;
  bool conv = false;
  int npairs = 0;
  ctx->eig_iters = 0;
  // refinement in FP64 from the vectors in Xc, at most `iters` steps
  auto refine = [&](int iters) {
    for (int it = 0; it < iters && !conv; ++it) {
      gemm64(ctx, true, false, n, n, n, 1.0, Xc, n, Xc, n, 0.0, wk.eG.p, n, st, ws, "gemm_eig", true);
      mirror_lower(n, wk.eG.p, n, st);
      gemm64(ctx, false, false, n, n, n, 1.0, A, n, Xc, n, 0.0, wk.eAX.p, n, st, ws, "gemm_eig");
      gemm64(ctx, true, false, n, n, n, 1.0, Xc, n, wk.eAX.p, n, 0.0, wk.eS.p, n, st, ws, "gemm_eig", true);
      mirror_lower(n, wk.eS.p, n, st);
      oa_step(n, wk.eG.p, wk.eS.p, wk.elam.p, wk.eM.p, wk.estats.p, wk.enp.p, wk.epairs.p, kCap, st);
      unsigned long long hs[2];
      CHEBFI_CUDA(cudaMemcpyAsync(hs, wk.estats.p, sizeof(hs), cudaMemcpyDeviceToHost, st));
      CHEBFI_CUDA(cudaMemcpyAsync(&npairs, wk.enp.p, sizeof(int), cudaMemcpyDeviceToHost, st));
      gemm64(ctx, false, false, n, n, n, 1.0, Xc, n, wk.eM.p, n, 0.0, Xn, n, st, ws, "gemm_eig");
      std::swap(Xc, Xn);
      CHEBFI_CUDA(cudaStreamSynchronize(st));
      double emax;
      std::memcpy(&emax, &hs[1], sizeof(double));
      ++ctx->eig_iters;
      // after an update of size emax the vectors are accurate to O(emax^2): below rounding
      conv = std::isfinite(emax) && emax <= 1e-10;
    }
  };
  // Fast path: when A is already nearly diagonal (the later sweeps of a converging solve,
  // whose Ritz vectors barely turn), the identity is a good enough first approximation.
  // Its refinement step needs no GEMM (G = I, S = A, X = I + E); when that step is small
  // (max |E| <= kFastE) and finds few close pairs, refine from there and skip stage 1.
  constexpr double kFastE = 0.01;
  {
    set_identity(n, wk.eG.p, n, st);
    oa_step(n, wk.eG.p, A, wk.elam.p, X, wk.estats.p, wk.enp.p, wk.epairs.p, kCap, st);
    unsigned long long hs[2];
    CHEBFI_CUDA(cudaMemcpyAsync(hs, wk.estats.p, sizeof(hs), cudaMemcpyDeviceToHost, st));
    CHEBFI_CUDA(cudaMemcpyAsync(&npairs, wk.enp.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CHEBFI_CUDA(cudaStreamSynchronize(st));
    double emax;
    std::memcpy(&emax, &hs[1], sizeof(double));
    if (std::isfinite(emax) && emax <= kFastE && npairs <= n) {
      ctx->eig_iters = 1;
      conv = emax <= 1e-10;
      refine(5);
    }
  }
  if (!conv) {
    // stage 1: FP32 Jacobi on a copy; stage 2: refinement from its vectors
    convert(n, n, A, n, wk.e32a.p, n, st);
    jacobi_eigh_f32(n, wk.e32a.p, n, wk.e32w.p, wk.e32b.p, n, status, st, &wk.small5);
    convert(n, n, wk.e32b.p, n, X, n, st);
    Xc = X;
    Xn = wk.eX.p;
    ctx->eig_iters = 0;
    refine(8);
  }
  if (!conv || npairs > kCap) {
    // not converged (or too many near-equal pairs): the FP64 Jacobi of the original matrix
    // (A is still intact; the refinement only read it)
    ctx->eig_iters = 0;
    jacobi_eigh(n, A, n, w, X, n, status, st, &wk.small5);
    return;
  }
  if (npairs > 0) {
    // clusters: connected components of the listed pairs; each block of X^H A X on a
    // component is diagonalised by FP64 Jacobi and its columns rotated
    std::vector<int2> hp(npairs);
    CHEBFI_CUDA(cudaMemcpyAsync(hp.data(), wk.epairs.p, sizeof(int2) * npairs, cudaMemcpyDeviceToHost, st));
    gemm64(ctx, false, false, n, n, n, 1.0, A, n, Xc, n, 0.0, wk.eAX.p, n, st, ws, "gemm_eig");
    gemm64(ctx, true, false, n, n, n, 1.0, Xc, n, wk.eAX.p, n, 0.0, wk.eS.p, n, st, ws, "gemm_eig");
    CHEBFI_CUDA(cudaStreamSynchronize(st));
    std::vector<int> parent(n);
    std::iota(parent.begin(), parent.end(), 0);
    std::function<int(int)> find = [&](int v) { return parent[v] == v ? v : parent[v] = find(parent[v]); };
    for (const int2& pr : hp) parent[find(pr.x)] = find(pr.y);
    std::map<int, std::vector<int>> comp;
    for (const int2& pr : hp) {
      comp[find(pr.x)];
    }
    for (int v = 0; v < (int)n; ++v)
      if (comp.count(find(v))) comp[find(v)].push_back(v);
    for (auto& kv : comp) {
      const std::vector<int>& idx = kv.second;
      const int k = (int)idx.size();
      wk.eidx.upload(idx.data(), k, st);
      wk.esub.alloc((size_t)k * k);
      wk.eZ.alloc((size_t)k * k);
      wk.esw.alloc(k);
      wk.eC1.alloc((size_t)n * k);
      wk.eC2.alloc((size_t)n * k);
      gather_sub(k, wk.eidx.p, wk.eS.p, n, wk.esub.p, st);
      hermitize(k, wk.esub.p, k, st);
      jacobi_eigh(k, wk.esub.p, k, wk.esw.p, wk.eZ.p, k, status, st, &wk.small5);
      gather_cols(n, k, wk.eidx.p, Xc, n, wk.eC1.p, n, st);
      gemm<double>(false, false, n, k, k, 1.0, wk.eC1.p, n, wk.eZ.p, k, 0.0, wk.eC2.p, n, st, ws, "gemm_eig");
      scatter_cols(n, k, wk.eidx.p, Xc, n, wk.eC2.p, n, st);
      scatter_vals(k, wk.eidx.p, wk.esw.p, wk.elam.p, st);
      CHEBFI_CUDA(cudaStreamSynchronize(st));  // the index list is reused by the next cluster
    }
  }
  if (Xc == X) {
    CHEBFI_CUDA(cudaMemcpyAsync(wk.eX.p, X, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, st));
    Xc = wk.eX.p;
  }
  sort_eigpairs(n, wk.elam.p, Xc, w, X, st);
}

// Rayleigh-Ritz (Algorithm 2, last three steps) on the sorted FP64 block w.Ya.
void rr_on_Ya(chebfi_ctx* ctx, int64_t nb, double* evals, double* resid, cudaStream_t st) {
  Work& w = ctx->w;
  const int64_t npw = ctx->npw, nq = ctx->nproj;
  const size_t ny = (size_t)npw * nb, np = (size_t)std::max<int64_t>(nq, 1) * nb, ns = (size_t)nb * nb;
  w.HY.alloc(ny);
  w.tmp.alloc(ny);
  w.T1.alloc(local_workspace_elems(ctx, nb));
  w.pa.alloc(np);
  w.pb.alloc(np);
  w.pc.alloc(np);
  w.small1.alloc(ns);
  w.small2.alloc(ns);
  w.small3.alloc(ns);
  w.small4.alloc(ns);
  w.dvec1.alloc(nb);
  double2* Y = w.Ya.p;
  DevBuf<double2>* ws = &w.splitk;
  scan_nonfinite(npw, nb, Y, npw, ctx->d_status.p, st);  // first flag wins: reported before any NOT_SPD
  // H Y and p = P^H Y
  apply_H_sorted<double>(ctx, Y, w.HY.p, w.pa.p, w.pb.p, w.T1.p, nb, st, "gemm_rr");
  double2 *Hs = w.small1.p, *Ss = w.small2.p, *Li = w.small3.p, *X = w.small4.p;
  // H_Psi and S_Psi are Hermitian: only their lower triangles are computed, then mirrored
  gemm64(ctx, true, false, nb, nb, npw, 1.0, Y, npw, w.HY.p, npw, 0.0, Hs, nb, st, ws, "gemm_rr", true);
  gemm64(ctx, true, false, nb, nb, npw, 1.0, Y, npw, Y, npw, 0.0, Ss, nb, st, ws, "gemm_rr", true);
  if (ctx->paw) {
    blockdiag_apply<double>(ctx, ctx->d_Qblk.p, w.pa.p, nq, w.pb.p, nq, nb, st);
    gemm64(ctx, true, false, nb, nb, nq, 1.0, w.pa.p, nq, w.pb.p, nq, 1.0, Ss, nb, st, ws, "gemm_rr", true);
  }
  mirror_lower(nb, Hs, nb, st);
  mirror_lower(nb, Ss, nb, st);
  // columns scaled to unit S-norm: S~ = s S s, H~ = s H s with s = diag(S)^{-1/2}
  diag_of(nb, Ss, nb, w.dvec1.p, st);
  scale_sym(nb, Hs, nb, w.dvec1.p, st);
  scale_sym(nb, Ss, nb, w.dvec1.p, st);
  // S~ = L L^H, C = L^{-1} H~ L^{-H}
  chol_inv(ctx, nb, Ss, nb, Li, nb, X, st);
  gemm64(ctx, false, false, nb, nb, nb, 1.0, Li, nb, Hs, nb, 0.0, X, nb, st, ws, "gemm_rr");
  gemm64(ctx, false, true, nb, nb, nb, 1.0, X, nb, Li, nb, 0.0, Hs, nb, st, ws, "gemm_rr");
  hermitize(nb, Hs, nb, st);
  // C = Z Lambda Z^H
  eigh_rr(ctx, nb, Hs, evals, X, st);
  check_status(ctx, st, "rayleigh_ritz");
  // rotation R = s L^{-H} Z; Y <- Y R, HY <- HY R, p <- p R
  gemm64(ctx, true, false, nb, nb, nb, 1.0, Li, nb, X, nb, 0.0, Ss, nb, st, ws, "gemm_rr");
  scale_rows(nb, nb, Ss, nb, w.dvec1.p, st);
  gemm64(ctx, false, false, npw, nb, nb, 1.0, Y, npw, Ss, nb, 0.0, w.tmp.p, npw, st, ws, "gemm_rr");
  std::swap(w.Ya.p, w.tmp.p);  // buffers have equal capacity
  std::swap(w.Ya.n, w.tmp.n);
  Y = w.Ya.p;
  // p_new = P^H Y_new = p R: the residuals' S Y_new, and p_0 of the next filter in a solve
  if (nq > 0) gemm64(ctx, false, false, nq, nb, nb, 1.0, w.pa.p, nq, Ss, nb, 0.0, w.pc.p, nq, st, ws, "gemm_rr");
  w.pc_of = nq > 0 ? Y : nullptr;
  if (resid) {
    gemm64(ctx, false, false, npw, nb, nb, 1.0, w.HY.p, npw, Ss, nb, 0.0, w.tmp.p, npw, st, ws, "gemm_rr");  // H Y_new
    double2* SY = w.HY.p;  // reuse
    CHEBFI_CUDA(cudaMemcpyAsync(SY, Y, sizeof(double2) * ny, cudaMemcpyDeviceToDevice, st));
    if (ctx->paw) {
      blockdiag_apply<double>(ctx, ctx->d_Qblk.p, w.pc.p, nq, w.pb.p, nq, nb, st);
      gemm64(ctx, false, false, npw, nb, nq, 1.0, ctx->d_P.p, npw, w.pb.p, nq, 1.0, SY, npw, st, ws, "gemm_rr");
    }
    residual_norms(npw, nb, w.tmp.p, npw, SY, npw, evals, resid, st);
  }
}

// S-orthonormalisation by Cholesky-QR on the sorted FP64 block w.Ya.
void ortho_on_Ya(chebfi_ctx* ctx, int64_t nb, cudaStream_t st) {
  Work& w = ctx->w;
  const int64_t npw = ctx->npw, nq = ctx->nproj;
  const size_t np = (size_t)std::max<int64_t>(nq, 1) * nb, ns = (size_t)nb * nb;
  w.tmp.alloc((size_t)npw * nb);
  w.pa.alloc(np);
  w.pb.alloc(np);
  w.small2.alloc(ns);
  w.small3.alloc(ns);
  w.small4.alloc(ns);
  DevBuf<double2>* ws = &w.splitk;
  double2 *Ss = w.small2.p, *Li = w.small3.p, *Y = w.Ya.p;
  scan_nonfinite(npw, nb, Y, npw, ctx->d_status.p, st);
  gemm64(ctx, true, false, nb, nb, npw, 1.0, Y, npw, Y, npw, 0.0, Ss, nb, st, ws);
  if (ctx->paw) {
    gemm64(ctx, true, false, nq, nb, npw, 1.0, ctx->d_P.p, npw, Y, npw, 0.0, w.pa.p, nq, st, ws);
    blockdiag_apply<double>(ctx, ctx->d_Qblk.p, w.pa.p, nq, w.pb.p, nq, nb, st);
    gemm64(ctx, true, false, nb, nb, nq, 1.0, w.pa.p, nq, w.pb.p, nq, 1.0, Ss, nb, st, ws);
  }
  hermitize(nb, Ss, nb, st);
  chol_inv(ctx, nb, Ss, nb, Li, nb, w.small4.p, st);
  check_status(ctx, st, "orthonormalise");
  gemm64(ctx, false, true, npw, nb, nb, 1.0, Y, npw, Li, nb, 0.0, w.tmp.p, npw, st, ws);
  std::swap(w.Ya.p, w.tmp.p);
  std::swap(w.Ya.n, w.tmp.n);
}

void gather_to_Ya(chebfi_ctx* ctx, const void* Y, int64_t nb, int64_t ld, cudaStream_t st) {
  ctx->w.pc_of = nullptr;  // new contents: no projections known for them
  ctx->w.Ya.alloc((size_t)ctx->npw * nb);
  gather_rows(ctx->npw, nb, ctx->d_sorted_to_user.p, (const double2*)Y, ld, ctx->w.Ya.p, ctx->npw, st);
}
void scatter_from(chebfi_ctx* ctx, const double2* src, void* Y, int64_t nb, int64_t ld, cudaStream_t st) {
  scatter_rows(ctx->npw, nb, ctx->d_sorted_to_user.p, src, ctx->npw, (double2*)Y, ld, st);
}

// Algorithm 2's filter in place on a caller's device block (caller's row order, leading
// dimension ld), stream-ordered on st.
void filter_device_block(chebfi_ctx* ctx, void* Y, int64_t nb, int64_t ld, int degree, double lo, double hi,
                         int prec, cudaStream_t st, const double2* p0 = nullptr) {
  if (prec == CHEBFI_F64) {
    gather_to_Ya(ctx, Y, nb, ld, st);
    filter_on_Ya(ctx, nb, degree, lo, hi, prec, st, p0);
    scatter_from(ctx, ctx->w.Ya.p, Y, nb, ld, st);
    return;
  }
  // FP32 iterates straight from and to the caller's FP64 block (reorder and convert in one pass)
  ensure_filter_ws(ctx, nb, prec);
  Work& w = ctx->w;
  const int64_t npw = ctx->npw;
  gather_rows(npw, nb, ctx->d_sorted_to_user.p, (const double2*)Y, ld, w.fYa.p, npw, st);
  FilterBufs<float> b{w.fYa.p, w.fYb.p, w.fZ.p, w.fT1.p, w.fpa.p, w.fpb.p, w.fpz.p, w.fpw.p, w.fpq.p};
  float2* out = prec == CHEBFI_MIXED ? filter_mixed(ctx, b, nb, degree, lo, hi, st, nullptr, p0)
                                     : filter_sorted<float>(ctx, b, nb, degree, lo, hi, st, nullptr, p0);
  scatter_rows(npw, nb, ctx->d_sorted_to_user.p, out, npw, (double2*)Y, ld, st);
}


double cheb_T_abs(int n, double x) {  // |T_n(x)| for |x| >= 1 by its cosh form, else <= 1
  const double ax = std::fabs(x);
  if (ax <= 1.0) return 1.0;
  return std::cosh(n * std::acosh(ax));
}

double host_max(chebfi_ctx* ctx, const double* d, int64_t n, cudaStream_t st, bool minimum = false) {
  std::vector<double> h(n);
  CHEBFI_CUDA(cudaMemcpyAsync(h.data(), d, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  CHEBFI_CUDA(cudaStreamSynchronize(st));
  double m = minimum ? INFINITY : -INFINITY;
  for (double v : h) {
    if (std::isnan(v)) return v;  // a NaN must not hide behind the comparisons
    m = minimum ? std::min(m, v) : std::max(m, v);
  }
  return m;
}

double rigorous_bound(chebfi_ctx* ctx) {
  if (ctx->bound_rigorous >= 0.0) return ctx->bound_rigorous;
  const int64_t nq = ctx->nproj;
  double num = ctx->kmax + ctx->vmax;
  double smin = 1.0;
  if (nq > 0) {
    cudaStream_t st = 0;
    DevBuf<double2> Dd, T, A, V;
    DevBuf<double> w;
    Dd.alloc(nq * nq);
    T.alloc(nq * nq);
    A.alloc(nq * nq);
    V.alloc(nq * nq);
    w.alloc(nq);
    DevBuf<double2>* ws = &ctx->w.splitk;
    // eigenvalues of L^H X L, G = P^H P = L L^H, for X = D and X = Q
    for (int which = 0; which < (ctx->paw ? 2 : 1); ++which) {
      CHEBFI_LAUNCH("k_dense_from_blocks", 0, k_dense_from_blocks<<<nblk(nq * nq), 256>>>(nq, ctx->d_atom_of.p, ctx->d_offs.p, ctx->d_blk_off.p,
                                                  which == 0 ? ctx->d_Dblk.p : ctx->d_Qblk.p, Dd.p));
      gemm64(ctx, false, false, nq, nq, nq, 1.0, Dd.p, nq, ctx->d_L.p, nq, 0.0, T.p, nq, st, ws);
      gemm64(ctx, true, false, nq, nq, nq, 1.0, ctx->d_L.p, nq, T.p, nq, 0.0, A.p, nq, st, ws);
      hermitize(nq, A.p, nq, st);
      eigh_rr(ctx, nq, A.p, w.p, V.p, st);
      check_status(ctx, st, "upper_bound");
      if (which == 0) num += std::max(0.0, host_max(ctx, w.p, nq, st));
      else smin = 1.0 + std::min(0.0, host_max(ctx, w.p, nq, st, true));
    }
  }
  ctx->bound_rigorous = std::max(0.0, num) / smin;
  ctx->smin = smin;
  return ctx->bound_rigorous;
}


// ---------------------------------------------------------------- Woodbury by refinement
// Section 5.1 solves the reduced system A q = P^H x, A = D_S^{-1} + P^H P, by iterative
// refinement preconditioned with the atom-diagonal blocks B of A:
//   q <- q + B^{-1} (P^H x - A q),  starting from q = 0,
// then S^{-1} x = x - P q.  A and B^{-1} are formed on first use.

// In-place Gauss-Jordan inverse with partial pivoting of an n x n column-major matrix;
// false if a pivot is zero or tiny relative to the largest entry.
template <typename T> bool gj_inverse(int n, std::vector<T>& a) {
  std::vector<int> perm(n);
  std::iota(perm.begin(), perm.end(), 0);
  double amax = 0.0;
  for (const T& v : a) amax = std::max(amax, (double)std::abs(v));
  if (amax == 0.0) return false;
  for (int k = 0; k < n; ++k) {
    int piv = k;
    for (int i = k + 1; i < n; ++i)
      if (std::abs(a[i + k * n]) > std::abs(a[piv + k * n])) piv = i;
    if (std::abs(a[piv + k * n]) <= 1e-14 * amax) return false;
    if (piv != k) {
      for (int j = 0; j < n; ++j) std::swap(a[k + j * n], a[piv + j * n]);
      std::swap(perm[k], perm[piv]);
    }
    const T inv = T(1) / a[k + k * n];
    a[k + k * n] = T(1);
    for (int j = 0; j < n; ++j) a[k + j * n] *= inv;
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const T f = a[i + k * n];
      if (f == T(0)) continue;
      a[i + k * n] = T(0);
      for (int j = 0; j < n; ++j) a[i + j * n] -= f * a[k + j * n];
    }
  }
  // undo the row interchanges as column interchanges of the inverse
  std::vector<T> out(a.size());
  for (int j = 0; j < n; ++j)
    for (int i = 0; i < n; ++i) out[i + perm[j] * n] = a[i + j * n];
  a.swap(out);
  return true;
}

void ensure_refine(chebfi_ctx* ctx, cudaStream_t st) {
  if (ctx->refine_ready) return;
  const int64_t nq = ctx->nproj;
  const int natoms = ctx->natoms;
  std::vector<double> dinv(ctx->h_Qblk.size());
  std::vector<int64_t> cblk(natoms);
  int64_t off = 0, coff = 0;
  for (int a = 0; a < natoms; ++a) {
    const int o = ctx->offs[a], na = ctx->offs[a + 1] - o;
    std::vector<double> blk(ctx->h_Qblk.begin() + off, ctx->h_Qblk.begin() + off + (int64_t)na * na);
    CHEBFI_REQUIRE(gj_inverse(na, blk), CHEBFI_ERR_ARG,
                   "the D_S (Q) block of atom " + std::to_string(a) +
                       " is singular: the refinement needs D_S^{-1}; use chebfi_apply_Sinv");
    // Q blocks are symmetric, so the row-major packing of the inverse equals its column-major one
    std::copy(blk.begin(), blk.end(), dinv.begin() + off);
    cblk[a] = coff;
    off += (int64_t)na * na;
    coff += (int64_t)na * na;
  }
  DevBuf<double> dd;
  dd.upload(dinv.data(), dinv.size(), st);
  ctx->d_Aref.alloc((size_t)nq * nq);
  CHEBFI_LAUNCH("k_dense_from_blocks", st, k_dense_from_blocks<<<nblk(nq * nq), 256, 0, st>>>(nq, ctx->d_atom_of.p, ctx->d_offs.p, ctx->d_blk_off.p, dd.p, ctx->d_Aref.p));
  axpby<double>(nq, nq, 1.0, ctx->d_G.p, nq, 1.0, ctx->d_Aref.p, nq, ctx->d_Aref.p, nq, st);
  // B^{-1}: inverses of the atom-diagonal blocks of A = D_S^{-1} + G
  std::vector<std::complex<double>> binv((size_t)coff);
  for (int a = 0; a < natoms; ++a) {
    const int o = ctx->offs[a], na = ctx->offs[a + 1] - o;
    std::vector<std::complex<double>> blk((size_t)na * na);
    CHEBFI_CUDA(cudaMemcpy2DAsync(blk.data(), sizeof(double2) * na, ctx->d_Aref.p + o + (int64_t)o * nq,
                                  sizeof(double2) * nq, sizeof(double2) * na, na, cudaMemcpyDeviceToHost, st));
    CHEBFI_CUDA(cudaStreamSynchronize(st));
    CHEBFI_REQUIRE(gj_inverse(na, blk), CHEBFI_ERR_ARG,
                   "the diagonal block of D_S^{-1} + P^H P of atom " + std::to_string(a) + " is singular");
    std::copy(blk.begin(), blk.end(), binv.begin() + cblk[a]);
  }
  ctx->d_Binv.upload(reinterpret_cast<const double2*>(binv.data()), binv.size(), st);
  ctx->d_cblk_off.upload(cblk.data(), cblk.size(), st);
  CHEBFI_CUDA(cudaStreamSynchronize(st));
  ctx->refine_ready = true;
}

// ---------------------------------------------------------------- filter backward
// The filter of Algorithm 2 is Y_{k+1} = a_k (A - c) Y_k - b_k Y_{k-1} with A = S^{-1} H,
// a_0 = 1/r, a_k = 2/r, b_0 = 0, b_k = 1.  For a real loss L with G_n = dL/dY_n (PyTorch's
// convention), the adjoint iterates L_k = dL/dY_k obey the same recurrence run backwards with
// the adjoint operator A^H = H S^{-1} (H and S Hermitian):
//   L_k = a_k (H S^{-1} L_{k+1} - c L_{k+1}) - L_{k+2},      L_{n+1} = 0,
// and gY_0 = L_0.  Only the term a_k S^{-1} (dH) Y_k of dY_{k+1} depends on V_loc and D, so
// their gradients are sums over k of the H-gradient of the pair (Y_k, a_k S^{-1} L_{k+1}),
// the quantity chebfi_apply_H_backward computes for one pair.
//
// The iterates Y_k are needed in reverse order.  They are recomputed from checkpoints: a
// first forward pass keeps (Y_{j-1}, Y_j) at j = 0, s, 2s, ...; each segment [j, j + s) is
// then recomputed from its checkpoint when the backward sweep reaches it.  Memory is
// 2 ceil(n/s) + s + 4 blocks (s = ceil(sqrt n) by default) instead of n + 4; the extra work
// is at most n forward steps.

// S^{-1} X (Section 5.1, Woodbury with the precomputed core M) into out; X itself when S = I.
template <typename R>
const cplx<R>* sinv_sorted(chebfi_ctx* ctx, const cplx<R>* X, cplx<R>* out, cplx<R>* pa, cplx<R>* pb, int64_t nb,
                           cudaStream_t st) {
  const int64_t npw = ctx->npw, nq = ctx->nproj;
  if (!ctx->paw) return X;
  CHEBFI_CUDA(cudaMemcpyAsync(out, X, sizeof(cplx<R>) * npw * nb, cudaMemcpyDeviceToDevice, st));
  cgemm<R>(ctx, true, false, nq, nb, npw, 1.0, Ops<R>::P(ctx), npw, X, npw, 0.0, pa, nq, st, Ops<R>::ws(ctx), "gemm_grad");
  cgemm<R>(ctx, false, false, nq, nb, nq, 1.0, Ops<R>::M(ctx), nq, pa, nq, 0.0, pb, nq, st, Ops<R>::ws(ctx), "gemm_grad");
  cgemm<R>(ctx, false, false, npw, nb, nq, -1.0, Ops<R>::P(ctx), npw, pb, nq, 1.0, out, npw, st, Ops<R>::ws(ctx),
          "gemm_grad");
  return out;
}

template <typename R> struct StepBufs {
  cplx<R>*HX, *U, *T, *pa, *pb;
};

// out = a (B X - c X) - bp Xprev with B = S^{-1} H (forward) or B = H S^{-1} (adjoint).
// out may alias Xprev, not X.  Returns S^{-1} X in the adjoint case (the gradient partner).
template <typename R>
const cplx<R>* cheb_step(chebfi_ctx* ctx, bool adjoint, const cplx<R>* X, const cplx<R>* Xprev, cplx<R>* out, double a,
                         double c, double bp, StepBufs<R> b, int64_t nb, cudaStream_t st) {
  const int64_t npw = ctx->npw;
  const cplx<R>* u;
  const cplx<R>* sx = nullptr;
  if (!adjoint) {
    apply_H_sorted<R>(ctx, X, b.HX, b.pa, b.pb, b.T, nb, st, "gemm_grad");
    u = sinv_sorted<R>(ctx, b.HX, b.U, b.pa, b.pb, nb, st);
  } else {
    sx = sinv_sorted<R>(ctx, X, b.U, b.pa, b.pb, nb, st);
    apply_H_sorted<R>(ctx, sx, b.HX, b.pa, b.pb, b.T, nb, st, "gemm_grad");
    u = b.HX;
  }
  cheb_combine<R>(npw, nb, (R)a, u, npw, (R)c, X, npw, (R)(Xprev ? bp : 0.0), Xprev, npw, out, npw, st);
  return sx;
}

// gV += scale * dRe<G, H Y>/dV_loc and gD += scale * dRe<G, H Y>/dD for a sorted pair, in the
// pair's precision (the sums over bands and grid points are accumulated in FP64).
template <typename R> struct GradBufs;
template <> struct GradBufs<double> {
  static DevBuf<double2>& q(chebfi_ctx* c) { return c->w.pc; }
  static DevBuf<double2>& p(chebfi_ctx* c) { return c->w.pt; }
  static DevBuf<double2>& T(chebfi_ctx* c) { return c->w.T2; }
  static DevBuf<double2>& Rg(chebfi_ctx* c) { return c->w.tmp; }
  static DevBuf<double2>& Gg(chebfi_ctx* c) { return c->w.tmp2; }
};
template <> struct GradBufs<float> {
  static DevBuf<float2>& q(chebfi_ctx* c) { return c->w.fpq; }
  static DevBuf<float2>& p(chebfi_ctx* c) { return c->w.fpt; }
  static DevBuf<float2>& T(chebfi_ctx* c) { return c->w.fgT; }
  static DevBuf<float2>& Rg(chebfi_ctx* c) { return c->w.fgR; }
  static DevBuf<float2>& Gg(chebfi_ctx* c) { return c->w.fgG; }
};

template <typename R>
void accumulate_pair(chebfi_ctx* ctx, const cplx<R>* Y, const cplx<R>* G, double scale, int64_t nb, double* gV,
                     double* gD, cudaStream_t st) {
  const int64_t npw = ctx->npw, nq = ctx->nproj;
  if (gD && nq > 0) {
    DevBuf<cplx<R>>& q = GradBufs<R>::q(ctx);
    DevBuf<cplx<R>>& pp = GradBufs<R>::p(ctx);
    q.alloc((size_t)nq * nb);
    pp.alloc((size_t)nq * nb);
    cgemm<R>(ctx, true, false, nq, nb, npw, 1.0, Ops<R>::P(ctx), npw, G, npw, 0.0, q.p, nq, st, Ops<R>::ws(ctx), "gemm_grad");
    cgemm<R>(ctx, true, false, nq, nb, npw, 1.0, Ops<R>::P(ctx), npw, Y, npw, 0.0, pp.p, nq, st, Ops<R>::ws(ctx), "gemm_grad");
    block_outer_grad(ctx, q.p, pp.p, nq, nb, gD, st, scale, true);
  }
  if (gV)
    vloc_gradient<R>(ctx, Y, G, nb, gV, st, GradBufs<R>::T(ctx), GradBufs<R>::Rg(ctx), GradBufs<R>::Gg(ctx), scale,
                     true);
}

void to_f64(const chebfi_ctx* ctx, const float2* x, double2* y, int64_t nb, cudaStream_t st) {
  convert(ctx->npw, nb, x, ctx->npw, y, ctx->npw, st);
}
template <typename R> void from_f64(const chebfi_ctx* ctx, const double2* x, cplx<R>* y, int64_t nb, cudaStream_t st) {
  if constexpr (sizeof(R) == 8) {
    CHEBFI_CUDA(cudaMemcpyAsync(y, x, sizeof(double2) * ctx->npw * nb, cudaMemcpyDeviceToDevice, st));
  } else {
    convert(ctx->npw, nb, x, ctx->npw, y, ctx->npw, st);
  }
}

// Backward of the degree-n filter on sorted FP64 blocks: Y_0 in w.Ya, G_n in w.Yb; gY_0 is
// left in w.Ya.  gV and gD (if not null) must be zeroed by the caller; they are accumulated.
template <typename R>
void filter_backward(chebfi_ctx* ctx, int64_t nb, int n, double lo, double hi, int s, double* gV, double* gD,
                     cudaStream_t st) {
  using C = cplx<R>;
  Work& w = ctx->w;
  const int64_t npw = ctx->npw;
  const size_t blk = (size_t)npw * nb, np = (size_t)std::max<int64_t>(ctx->nproj, 1) * nb;
  const double c = 0.5 * (hi + lo), r = 0.5 * (hi - lo);
  const int nseg = (n + s - 1) / s, sl = std::max(s, 2);
  const int nslots = 2 * nseg + sl + 4;
  DevBuf<C>& pool = Ops<R>::pool(ctx);
  pool.alloc(blk * nslots);
  Ops<R>::T(ctx).alloc(local_workspace_elems(ctx, nb));
  Ops<R>::pa(ctx).alloc(np);
  Ops<R>::pb(ctx).alloc(np);
  auto slot = [&](int i) { return pool.p + blk * i; };
  auto ck = [&](int seg, int which) { return slot(2 * seg + which); };  // which 0: Y_{j-1}, 1: Y_j
  C* segb = slot(2 * nseg);
  C* lam1 = slot(2 * nseg + sl);
  C* lam2 = slot(2 * nseg + sl + 1);
  StepBufs<R> sb{slot(2 * nseg + sl + 2), slot(2 * nseg + sl + 3), Ops<R>::T(ctx).p, Ops<R>::pa(ctx).p,
                 Ops<R>::pb(ctx).p};
  auto alpha = [&](int k) { return (k == 0 ? 1.0 : 2.0) / r; };
  const size_t bytes = sizeof(C) * blk;
  from_f64<R>(ctx, w.Ya.p, ck(0, 1), nb, st);
  from_f64<R>(ctx, w.Yb.p, lam1, nb, st);
  // forward pass: Y_1 .. Y_{n-1} in two rolling buffers, checkpoints at multiples of s
  {
    C* yk = segb;
    C* ykm1 = nullptr;
    CHEBFI_CUDA(cudaMemcpyAsync(yk, ck(0, 1), bytes, cudaMemcpyDeviceToDevice, st));
    for (int k = 0; k + 1 < n; ++k) {
      C* out = ykm1 ? ykm1 : segb + blk;  // Y_{k+1} over Y_{k-1}
      cheb_step<R>(ctx, false, yk, ykm1, out, alpha(k), c, 1.0, sb, nb, st);
      ykm1 = yk;
      yk = out;
      const int j = k + 1;
      if (j % s == 0) {
        CHEBFI_CUDA(cudaMemcpyAsync(ck(j / s, 0), ykm1, bytes, cudaMemcpyDeviceToDevice, st));
        CHEBFI_CUDA(cudaMemcpyAsync(ck(j / s, 1), yk, bytes, cudaMemcpyDeviceToDevice, st));
      }
    }
  }
  // backward sweep, segment by segment
  bool have2 = false;
  for (int seg = nseg - 1; seg >= 0; --seg) {
    const int j = seg * s, e = std::min(j + s, n);
    CHEBFI_CUDA(cudaMemcpyAsync(segb, ck(seg, 1), bytes, cudaMemcpyDeviceToDevice, st));
    for (int m = 1; m < e - j; ++m) {
      const int k = j + m - 1;  // Y_{k+1} from Y_k and Y_{k-1}
      const C* ykm1 = m >= 2 ? segb + blk * (m - 2) : (j > 0 ? ck(seg, 0) : nullptr);
      cheb_step<R>(ctx, false, segb + blk * (m - 1), ykm1, segb + blk * m, alpha(k), c, 1.0, sb, nb, st);
    }
    for (int k = e - 1; k >= j; --k) {
      const double a = alpha(k);
      // L_k = a (H S^{-1} L_{k+1} - c L_{k+1}) - L_{k+2}, written over L_{k+2}
      const C* u = cheb_step<R>(ctx, true, lam1, have2 ? lam2 : nullptr, lam2, a, c, 1.0, sb, nb, st);
      const C* yk = segb + blk * (k - j);
      if (gV || gD) accumulate_pair<R>(ctx, yk, u, a, nb, gV, gD, st);
      std::swap(lam1, lam2);
      have2 = true;
    }
  }
  if constexpr (sizeof(R) == 8) {
    CHEBFI_CUDA(cudaMemcpyAsync(w.Ya.p, lam1, bytes, cudaMemcpyDeviceToDevice, st));
  } else {
    to_f64(ctx, lam1, w.Ya.p, nb, st);
  }
}

}  // namespace

void ensure_tc_operands(chebfi_ctx* ctx, cudaStream_t st) { ensure_tc(ctx, st, true); }

}  // namespace chebfi

using namespace chebfi;

#define API_BEGIN(ctx)                                      \
  if (!(ctx)) return CHEBFI_ERR_ARG;                        \
  try {                                                     \
    (ctx)->err.clear();                                     \
    g_launch_counter = &(ctx)->launches;                    \
    g_prof = &(ctx)->prof;                                  \
    CHEBFI_CUDA(cudaSetDevice((ctx)->device));

#define API_END(ctx)                                        \
  }                                                         \
  catch (const chebfi::Error& e) {                          \
    (ctx)->err = e.msg;                                     \
    return e.code;                                          \
  }                                                         \
  catch (const std::exception& e) {                         \
    (ctx)->err = e.what();                                  \
    return CHEBFI_ERR_CUDA;                                 \
  }                                                         \
  return CHEBFI_OK;

extern "C" {

int chebfi_create(chebfi_ctx** out, int device) {
  if (!out) return CHEBFI_ERR_ARG;
  *out = nullptr;
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return CHEBFI_ERR_ARG;
  chebfi_ctx* ctx = new chebfi_ctx();
  ctx->device = device;
  try {
    CHEBFI_CUDA(cudaSetDevice(device));
    ctx->d_status.alloc(1);
    CHEBFI_CUDA(cudaMemset(ctx->d_status.p, 0, sizeof(int)));
  } catch (const Error&) {
    delete ctx;
    return CHEBFI_ERR_CUDA;
  }
  *out = ctx;
  return CHEBFI_OK;
}

int chebfi_destroy(chebfi_ctx* ctx) {
  if (!ctx) return CHEBFI_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  delete ctx;
  return CHEBFI_OK;
}

const char* chebfi_last_error(const chebfi_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int64_t chebfi_kernel_launches(const chebfi_ctx* ctx) { return ctx ? ctx->launches : 0; }

int chebfi_set_cell(chebfi_ctx* ctx, const double* lattice, const int* grid, const double* kpt) {
  API_BEGIN(ctx)
  CHEBFI_REQUIRE(lattice && grid && kpt, CHEBFI_ERR_ARG, "null argument");
  CHEBFI_REQUIRE(!ctx->has_sphere, CHEBFI_ERR_STATE, "set_cell after set_sphere");
  for (int i = 0; i < 3; ++i) ctx->ax[i].build(grid[i]);
  std::memcpy(ctx->lattice, lattice, sizeof(ctx->lattice));
  std::memcpy(ctx->kpt, kpt, sizeof(ctx->kpt));
  for (int i = 0; i < 3; ++i) ctx->grid[i] = grid[i];
  // reciprocal rows b_j with a_i . b_j = 2 pi delta_ij: B = 2 pi (A^{-1})^T
  const double* a = lattice;
  const double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
                     a[2] * (a[3] * a[7] - a[4] * a[6]);
  CHEBFI_REQUIRE(std::fabs(det) > 1e-12, CHEBFI_ERR_ARG, "singular lattice");
  double inv[9];  // inverse of A (row-major)
  inv[0] = (a[4] * a[8] - a[5] * a[7]) / det;
  inv[1] = (a[2] * a[7] - a[1] * a[8]) / det;
  inv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
  inv[3] = (a[5] * a[6] - a[3] * a[8]) / det;
  inv[4] = (a[0] * a[8] - a[2] * a[6]) / det;
  inv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
  inv[6] = (a[3] * a[7] - a[4] * a[6]) / det;
  inv[7] = (a[1] * a[6] - a[0] * a[7]) / det;
  inv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
  for (int j = 0; j < 3; ++j)
    for (int c = 0; c < 3; ++c) ctx->recip[j * 3 + c] = 2.0 * M_PI * inv[c * 3 + j];
  ctx->has_cell = true;
  API_END(ctx)
}

int chebfi_set_sphere(chebfi_ctx* ctx, int64_t npw, const int32_t* miller) {
  API_BEGIN(ctx)
  CHEBFI_REQUIRE(ctx->has_cell, CHEBFI_ERR_STATE, "set_cell must precede set_sphere");
  CHEBFI_REQUIRE(!ctx->has_sphere, CHEBFI_ERR_STATE, "the sphere is already set");
  CHEBFI_REQUIRE(npw >= 1 && npw < (int64_t)1 << 31 && miller, CHEBFI_ERR_ARG, "bad npw or null miller");
  const int n1 = ctx->grid[0], n2 = ctx->grid[1], n3 = ctx->grid[2];
  std::vector<int64_t> key(npw);
  std::vector<int> zz(npw);
  for (int64_t i = 0; i < npw; ++i) {
    const int m[3] = {miller[3 * i], miller[3 * i + 1], miller[3 * i + 2]};
    for (int d = 0; d < 3; ++d)
      CHEBFI_REQUIRE(2 * std::abs(m[d]) < ctx->grid[d], CHEBFI_ERR_ARG,
                     "Miller index outside (-N/2, N/2) at plane wave " + std::to_string(i));
    const int x = (m[0] % n1 + n1) % n1, y = (m[1] % n2 + n2) % n2, z = (m[2] % n3 + n3) % n3;
    key[i] = (int64_t)x * n2 + y;
    zz[i] = z;
  }
  std::vector<int32_t> order(npw);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int32_t a, int32_t b) {
    return key[a] != key[b] ? key[a] < key[b] : zz[a] < zz[b];
  });
  for (int64_t j = 1; j < npw; ++j)
    CHEBFI_REQUIRE(!(key[order[j]] == key[order[j - 1]] && zz[order[j]] == zz[order[j - 1]]), CHEBFI_ERR_ARG,
                   "duplicate plane wave in the sphere");
  SphereFFT& s = ctx->sph;
  s.n1 = n1;
  s.n2 = n2;
  s.n3 = n3;
  s.pitch = n2 % 2 ? n2 : n2 + 1;
  s.zpitch = n3 % 2 ? n3 : n3 + 1;
  std::vector<int32_t> col_start, pw_line(npw), pw_zrev(npw), col_off, pw_znat(npw), col_nat;
  std::vector<char> xact(n1, 0);
  const std::vector<int>&rx = ctx->ax[0].rev, &ry = ctx->ax[1].rev, &rz = ctx->ax[2].rev;
  for (int64_t j = 0; j < npw; ++j) {
    const int32_t u = order[j];
    if (j == 0 || key[u] != key[order[j - 1]]) {
      col_start.push_back((int32_t)j);
      const int x = (int)(key[u] / n2), y = (int)(key[u] % n2);
      col_off.push_back(rx[x] * s.pitch + ry[y]);
      col_nat.push_back(((x + n1 / 2) % n1) * s.pitch + y);
      xact[x] = 1;
    }
    pw_line[j] = (int32_t)col_start.size() - 1;
    pw_zrev[j] = rz[zz[u]];
    pw_znat[j] = zz[u];
  }
  s.ncol = (int)col_start.size();
  col_start.push_back((int32_t)npw);
  // The compile-time-length kernels keep plane row x in slot (x + n1/2) mod n1: the rows
  // holding sphere columns (signed x in [-m, m]) then sit in consecutive slots, so the y
  // passes over them, one row per thread, meet no bank conflicts at the wrap of x.  A cyclic
  // relabelling of x only multiplies the real-space values of the x transform by a phase,
  // which the transform back removes; V_loc is indexed by the transform's own positions.
  std::vector<int32_t> rows, rows_nat;
  for (int x = 0; x < n1; ++x)
    if (xact[x]) rows.push_back(rx[x] * s.pitch);
  for (int r = 0; r < n1; ++r) {
    const int x = (r - n1 / 2 + n1) % n1;
    if (xact[x]) rows_nat.push_back(r * s.pitch);
  }
  s.nxa = (int)rows.size();
  // for the pruned plane pass: the slot range [act_lo, act_lo + nact) covering the active
  // rows, and which column sits at (row act_lo + a, natural y)
  {
    s.act_lo = rows_nat.front() / s.pitch;
    s.nact = rows_nat.back() / s.pitch - s.act_lo + 1;
    std::vector<int32_t> row_col((size_t)s.nact * n2, -1);
    for (int c = 0; c < s.ncol; ++c) {
      const int slot = col_nat[c] / s.pitch, y = col_nat[c] % s.pitch;
      row_col[(size_t)(slot - s.act_lo) * n2 + y] = c;
    }
    s.row_col.upload(row_col.data(), row_col.size());
  }
  s.col_start.upload(col_start.data(), col_start.size());
  s.pw_line.upload(pw_line.data(), npw);
  s.pw_zrev.upload(pw_zrev.data(), npw);
  s.col_off.upload(col_off.data(), col_off.size());
  s.rows_act.upload(rows.data(), rows.size());
  s.pw_z.upload(pw_znat.data(), npw);
  s.col_off_nat.upload(col_nat.data(), col_nat.size());
  s.rows_nat.upload(rows_nat.data(), rows_nat.size());
  ctx->sorted_to_user = order;
  ctx->d_sorted_to_user.upload(order.data(), npw);
  // kinetic diagonal |k + G|^2 / 2 (Section 2.1), sorted order
  std::vector<double> K(npw);
  std::vector<float> Kf(npw);
  double kmax = 0.0;
  for (int64_t j = 0; j < npw; ++j) {
    const int32_t u = order[j];
    double g[3];
    for (int c = 0; c < 3; ++c)
      g[c] = ctx->kpt[c] + miller[3 * u] * ctx->recip[c] + miller[3 * u + 1] * ctx->recip[3 + c] +
             miller[3 * u + 2] * ctx->recip[6 + c];
    K[j] = 0.5 * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    Kf[j] = (float)K[j];
    kmax = std::max(kmax, K[j]);
  }
  ctx->d_K.upload(K.data(), npw);
  ctx->d_Kf.upload(Kf.data(), npw);
  ctx->kmax = kmax;
  ctx->npw = npw;
  CHEBFI_CUDA(cudaDeviceSynchronize());
  ctx->has_sphere = true;
  API_END(ctx)
}

int chebfi_set_vloc(chebfi_ctx* ctx, const double* vloc, int on_device) {
  API_BEGIN(ctx)
  CHEBFI_REQUIRE(ctx->has_cell, CHEBFI_ERR_STATE, "set_cell must precede set_vloc");
  CHEBFI_REQUIRE(vloc, CHEBFI_ERR_ARG, "null vloc");
  const int n1 = ctx->grid[0], n2 = ctx->grid[1], n3 = ctx->grid[2];
  const size_t n = (size_t)n1 * n2 * n3;
  std::vector<double> h(n);
  if (on_device) CHEBFI_CUDA(cudaMemcpy(h.data(), vloc, n * sizeof(double), cudaMemcpyDeviceToHost));
  else std::memcpy(h.data(), vloc, n * sizeof(double));
  std::vector<double> t(n);
  std::vector<float> tf(n);
  double vmax = -INFINITY;
  for (int x = 0; x < n1; ++x)
    for (int y = 0; y < n2; ++y)
      for (int z = 0; z < n3; ++z) {
        const double v = h[((size_t)x * n2 + y) * n3 + z];
        CHEBFI_REQUIRE(std::isfinite(v), CHEBFI_ERR_NONFINITE, "V_loc is not finite");
        t[((size_t)z * n1 + x) * n2 + y] = v;
        tf[((size_t)z * n1 + x) * n2 + y] = (float)v;
        vmax = std::max(vmax, v);
      }
  ctx->d_vt.upload(t.data(), n);
  ctx->d_vtf.upload(tf.data(), n);
  ctx->fast_fft = fast_fft_supported(n1, n2, n3);
  if (ctx->fast_fft) {
    // position (z', x', y') of the two-pass kernels holds real-space point
    // (split_index(x'), split_index(y'), split_index(z'))
    std::vector<double> vs(n);
    std::vector<float> vsf(n);
    for (int pz = 0; pz < n3; ++pz)
      for (int px = 0; px < n1; ++px)
        for (int py = 0; py < n2; ++py) {
          const int x = split_index(n1, px), y = split_index(n2, py), z = split_index(n3, pz);
          const double v = h[((size_t)x * n2 + y) * n3 + z];
          vs[((size_t)pz * n1 + px) * n2 + py] = v;
          vsf[((size_t)pz * n1 + px) * n2 + py] = (float)v;
        }
    std::vector<float2> vsdf(n);
    for (size_t i = 0; i < (size_t)n; ++i) {
      const float h = (float)vs[i];
      vsdf[i] = make_float2(h, (float)(vs[i] - (double)h));
    }
    ctx->d_vs.upload(vs.data(), n);
    ctx->d_vsf.upload(vsf.data(), n);
    ctx->d_vsdf.upload(vsdf.data(), n);
  }
  CHEBFI_CUDA(cudaDeviceSynchronize());
  ctx->vmax = vmax;
  ctx->has_vloc = true;
  ctx->bound_rigorous = -1.0;
  API_END(ctx)
}

int chebfi_set_projectors(chebfi_ctx* ctx, int64_t nproj, const void* P, int64_t ldP, int P_on_device, int natoms,
                          const int32_t* proj_offsets, const double* D, const double* Q) {
  API_BEGIN(ctx)
  CHEBFI_REQUIRE(ctx->has_sphere, CHEBFI_ERR_STATE, "set_sphere must precede set_projectors");
  CHEBFI_REQUIRE(nproj >= 0 && natoms >= 0, CHEBFI_ERR_ARG, "negative size");
  const int64_t npw = ctx->npw;
  cudaStream_t st = 0;
  ctx->nproj = nproj;
  ctx->natoms = natoms;
  ctx->paw = false;
  ctx->bound_rigorous = -1.0;
  ctx->has_proj = false;
  ctx->ozPh.nmod = ctx->ozP.nmod = 0;  // residues of the previous P are stale
  ctx->tc_ready = ctx->tcP_ready = ctx->tc3_ready = false;  // and so are its bf16 embeddings
  if (nproj == 0) {
    ctx->has_proj = true;
    return CHEBFI_OK;
  }
  CHEBFI_REQUIRE(P && proj_offsets && D && ldP >= npw && natoms >= 1, CHEBFI_ERR_ARG, "bad projector arguments");
  std::vector<int32_t> offs(proj_offsets, proj_offsets + natoms + 1);
  CHEBFI_REQUIRE(offs[0] == 0 && offs[natoms] == nproj, CHEBFI_ERR_ARG, "proj_offsets must run from 0 to nproj");
  std::vector<int32_t> atom_of(nproj);
  std::vector<int64_t> blk_off(natoms);
  int64_t nblkv = 0;
  for (int a = 0; a < natoms; ++a) {
    const int na = offs[a + 1] - offs[a];
    CHEBFI_REQUIRE(na >= 1 && na <= 64, CHEBFI_ERR_ARG, "projector block sizes must be 1..64");
    blk_off[a] = nblkv;
    nblkv += (int64_t)na * na;
    for (int i = offs[a]; i < offs[a + 1]; ++i) atom_of[i] = a;
  }
  for (int64_t i = 0; i < nblkv; ++i) {
    CHEBFI_REQUIRE(std::isfinite(D[i]), CHEBFI_ERR_NONFINITE, "D is not finite");
    CHEBFI_REQUIRE(!Q || std::isfinite(Q[i]), CHEBFI_ERR_NONFINITE, "Q is not finite");
  }
  ctx->offs = offs;
  ctx->d_offs.upload(offs.data(), offs.size());
  ctx->d_atom_of.upload(atom_of.data(), nproj);
  ctx->d_blk_off.upload(blk_off.data(), natoms);
  ctx->d_Dblk.upload(D, nblkv);
  std::vector<float> Df(D, D + nblkv);
  ctx->d_Dblkf.upload(Df.data(), nblkv);
  ctx->refine_ready = false;
  ctx->h_Qblk.clear();
  if (Q) {
    ctx->d_Qblk.upload(Q, nblkv);
    ctx->h_Qblk.assign(Q, Q + nblkv);
    ctx->paw = true;
  }
  // P in sorted row order
  ctx->d_P.alloc((size_t)npw * nproj);
  if (P_on_device) {
    gather_rows(npw, nproj, ctx->d_sorted_to_user.p, (const double2*)P, ldP, ctx->d_P.p, npw, st);
  } else {
    std::vector<double2> h((size_t)npw * nproj);
    const double2* src = (const double2*)P;
    for (int64_t i = 0; i < nproj; ++i)
      for (int64_t j = 0; j < npw; ++j) h[i * npw + j] = src[i * ldP + ctx->sorted_to_user[j]];
    CHEBFI_CUDA(cudaMemcpy(ctx->d_P.p, h.data(), h.size() * sizeof(double2), cudaMemcpyHostToDevice));
  }
  scan_nonfinite(npw, nproj, ctx->d_P.p, npw, ctx->d_status.p, st);
  check_status(ctx, st, "set_projectors (P)");
  DevBuf<double2>* ws = &ctx->w.splitk;
  // G = P^H P (Section 5.1, precomputed once)
  ctx->d_G.alloc((size_t)nproj * nproj);
  gemm64(ctx, true, false, nproj, nproj, npw, 1.0, ctx->d_P.p, npw, ctx->d_P.p, npw, 0.0, ctx->d_G.p, nproj, st, ws);
  hermitize(nproj, ctx->d_G.p, nproj, st);
  // L = chol(G): used by the Woodbury core and the rigorous bound
  ctx->d_L.alloc((size_t)nproj * nproj);
  CHEBFI_CUDA(cudaMemcpyAsync(ctx->d_L.p, ctx->d_G.p, sizeof(double2) * nproj * nproj, cudaMemcpyDeviceToDevice, st));
  cholesky(nproj, ctx->d_L.p, nproj, ctx->d_status.p, st, ws);
  check_status(ctx, st, "set_projectors (P^H P, projectors linearly dependent?)");
  if (ctx->paw) {
    // M = Q (I + G Q)^{-1} = (Q L) B^{-1} L^{-1} with B = I + L^H Q L = R R^H
    DevBuf<double2> Qd, T, B, Li, Ri, X;
    const size_t nn = (size_t)nproj * nproj;
    Qd.alloc(nn);
    T.alloc(nn);
    B.alloc(nn);
    Li.alloc(nn);
    Ri.alloc(nn);
    X.alloc(nn);
    CHEBFI_LAUNCH("k_dense_from_blocks", st, k_dense_from_blocks<<<nblk(nproj * nproj), 256, 0, st>>>(nproj, ctx->d_atom_of.p, ctx->d_offs.p, ctx->d_blk_off.p,
                                                             ctx->d_Qblk.p, Qd.p));
    gemm64(ctx, false, false, nproj, nproj, nproj, 1.0, Qd.p, nproj, ctx->d_L.p, nproj, 0.0, T.p, nproj, st, ws);
    gemm64(ctx, true, false, nproj, nproj, nproj, 1.0, ctx->d_L.p, nproj, T.p, nproj, 0.0, B.p, nproj, st, ws);
    CHEBFI_LAUNCH("k_add_identity", st, k_add_identity<<<nblk(nproj), 256, 0, st>>>(nproj, B.p, nproj));
    hermitize(nproj, B.p, nproj, st);
    cholesky(nproj, B.p, nproj, ctx->d_status.p, st, ws);
    check_status(ctx, st, "set_projectors (S = I + P Q P^H is not positive definite)");
    set_identity(nproj, Li.p, nproj, st);
    trsm_lower(nproj, nproj, ctx->d_L.p, nproj, Li.p, nproj, st, ws);
    set_identity(nproj, Ri.p, nproj, st);
    trsm_lower(nproj, nproj, B.p, nproj, Ri.p, nproj, st, ws);
    // M = T R^{-H} R^{-1} L^{-1}
    gemm64(ctx, false, true, nproj, nproj, nproj, 1.0, T.p, nproj, Ri.p, nproj, 0.0, X.p, nproj, st, ws);
    gemm64(ctx, false, false, nproj, nproj, nproj, 1.0, X.p, nproj, Ri.p, nproj, 0.0, B.p, nproj, st, ws);
    ctx->d_M.alloc(nn);
    gemm64(ctx, false, false, nproj, nproj, nproj, 1.0, B.p, nproj, Li.p, nproj, 0.0, ctx->d_M.p, nproj, st, ws);
    hermitize(nproj, ctx->d_M.p, nproj, st);
    ctx->d_Mf.alloc(nn);
    convert(nproj, nproj, ctx->d_M.p, nproj, ctx->d_Mf.p, nproj, st);
  }
  ctx->d_Pf.alloc((size_t)npw * nproj);
  convert(npw, nproj, ctx->d_P.p, npw, ctx->d_Pf.p, npw, st);
  ctx->d_Gf.alloc((size_t)nproj * nproj);
  convert(nproj, nproj, ctx->d_G.p, nproj, ctx->d_Gf.p, nproj, st);
  CHEBFI_CUDA(cudaStreamSynchronize(st));
  ctx->has_proj = true;
  API_END(ctx)
}

int chebfi_upper_bound(chebfi_ctx* ctx, int mode, double* lambda_hi) {
  API_BEGIN(ctx)
  require_ready(ctx);
  CHEBFI_REQUIRE(lambda_hi, CHEBFI_ERR_ARG, "null output");
  if (mode == CHEBFI_BOUND_PAPER) *lambda_hi = ctx->kmax;
  else if (mode == CHEBFI_BOUND_RIGOROUS) *lambda_hi = rigorous_bound(ctx);
  else throw Error{CHEBFI_ERR_ARG, "unknown bound mode"};
  API_END(ctx)
}

int chebfi_overlap_lower_bound(chebfi_ctx* ctx, double* smin) {
  API_BEGIN(ctx)
  require_ready(ctx);
  CHEBFI_REQUIRE(smin, CHEBFI_ERR_ARG, "null output");
  rigorous_bound(ctx);
  *smin = ctx->smin;
  API_END(ctx)
}

int chebfi_apply_H(chebfi_ctx* ctx, const void* Y, void* HY, int64_t nb, int64_t ld, int prec, void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  require_block(ctx, Y, nb, ld);
  CHEBFI_REQUIRE(nb == 0 || HY, CHEBFI_ERR_ARG, "null HY");
  CHEBFI_REQUIRE(prec >= 0 && prec <= 2, CHEBFI_ERR_ARG, "bad precision");
  if (nb == 0) return CHEBFI_OK;
  cudaStream_t st = S(stream);
  Work& w = ctx->w;
  const int64_t npw = ctx->npw;
  const size_t np = (size_t)std::max<int64_t>(ctx->nproj, 1) * nb;
  gather_to_Ya(ctx, Y, nb, ld, st);
  w.HY.alloc((size_t)npw * nb);
  if (prec == CHEBFI_F64) {
    w.T1.alloc(local_workspace_elems(ctx, nb));
    w.pa.alloc(np);
    w.pb.alloc(np);
    apply_H_sorted<double>(ctx, w.Ya.p, w.HY.p, w.pa.p, w.pb.p, w.T1.p, nb, st);
  } else {
    w.fYa.alloc((size_t)npw * nb);
    w.fZ.alloc((size_t)npw * nb);
    w.fT1.alloc(local_workspace_elems(ctx, nb));
    w.fpa.alloc(np);
    w.fpb.alloc(np);
    convert(npw, nb, w.Ya.p, npw, w.fYa.p, npw, st);
    if (prec == CHEBFI_MIXED && ctx->nproj > 0) {
      // local part in FP32, projector products on the tensor cores
      const int64_t nq = ctx->nproj;
      ensure_tc(ctx, st);
      ensure_tc3(ctx, st);
      LocalEpi<float> ep;
      ep.Y = w.fYa.p;
      ep.ldy = npw;
      ep.Z = w.fZ.p;
      ep.ldz = npw;
      local_apply<float>(ctx, w.fYa.p, npw, nb, w.fT1.p, ep, st);
      w.Zb.ld = (2 * npw + 7) / 8 * 8;
      w.Zb.alloc((size_t)w.Zb.ld * nb);
      split_block(npw, nb, w.fYa.p, npw, w.Zb, st);
      tc_gemm(ctx->tcA1.view(), w.Zb.view(), 2 * nq, nb, 2 * npw, 1.f, 0.f, nullptr, 0, (float*)w.fpa.p, 2 * nq,
              ctx->d_status.p, st, "tc_gemm_PhY", &ctx->w.tcws);
      blockdiag_apply<float>(ctx, ctx->d_Dblkf.p, w.fpa.p, nq, w.fpb.p, nq, nb, st);
      split3_block(nq, nb, w.fpb.p, nq, w.W3, st);
      tc_cgemm3(ctx->tcP3, w.W3, false, npw, nb, nq, 1.f, 1.f, w.fZ.p, npw, w.fZ.p, npw, ctx->d_status.p, st,
                "tc_gemm_PW", &ctx->w.tcws);
    } else {
      apply_H_sorted<float>(ctx, w.fYa.p, w.fZ.p, w.fpa.p, w.fpb.p, w.fT1.p, nb, st);
    }
    convert(npw, nb, w.fZ.p, npw, w.HY.p, npw, st);
  }
  scatter_from(ctx, w.HY.p, HY, nb, ld, st);
  API_END(ctx)
}

int chebfi_apply_S(chebfi_ctx* ctx, const void* Y, void* SY, int64_t nb, int64_t ld, void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  require_block(ctx, Y, nb, ld);
  CHEBFI_REQUIRE(nb == 0 || SY, CHEBFI_ERR_ARG, "null SY");
  if (nb == 0) return CHEBFI_OK;
  cudaStream_t st = S(stream);
  Work& w = ctx->w;
  const int64_t npw = ctx->npw, nq = ctx->nproj;
  gather_to_Ya(ctx, Y, nb, ld, st);
  if (ctx->paw) {
    const size_t np = (size_t)nq * nb;
    w.pa.alloc(np);
    w.pb.alloc(np);
    gemm64(ctx, true, false, nq, nb, npw, 1.0, ctx->d_P.p, npw, w.Ya.p, npw, 0.0, w.pa.p, nq, st, &w.splitk);
    blockdiag_apply<double>(ctx, ctx->d_Qblk.p, w.pa.p, nq, w.pb.p, nq, nb, st);
    gemm64(ctx, false, false, npw, nb, nq, 1.0, ctx->d_P.p, npw, w.pb.p, nq, 1.0, w.Ya.p, npw, st, &w.splitk);
  }
  scatter_from(ctx, w.Ya.p, SY, nb, ld, st);
  API_END(ctx)
}

int chebfi_apply_Sinv(chebfi_ctx* ctx, const void* X, void* out, int64_t nb, int64_t ld, void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  require_block(ctx, X, nb, ld);
  CHEBFI_REQUIRE(nb == 0 || out, CHEBFI_ERR_ARG, "null out");
  if (nb == 0) return CHEBFI_OK;
  cudaStream_t st = S(stream);
  Work& w = ctx->w;
  const int64_t npw = ctx->npw, nq = ctx->nproj;
  gather_to_Ya(ctx, X, nb, ld, st);
  if (ctx->paw) {
    // S^{-1} x = x - P M P^H x (Section 5.1)
    const size_t np = (size_t)nq * nb;
    w.pa.alloc(np);
    w.pb.alloc(np);
    gemm64(ctx, true, false, nq, nb, npw, 1.0, ctx->d_P.p, npw, w.Ya.p, npw, 0.0, w.pa.p, nq, st, &w.splitk);
    gemm64(ctx, false, false, nq, nb, nq, 1.0, ctx->d_M.p, nq, w.pa.p, nq, 0.0, w.pb.p, nq, st, &w.splitk);
    gemm64(ctx, false, false, npw, nb, nq, -1.0, ctx->d_P.p, npw, w.pb.p, nq, 1.0, w.Ya.p, npw, st, &w.splitk);
  }
  scatter_from(ctx, w.Ya.p, out, nb, ld, st);
  API_END(ctx)
}

int chebfi_cheb_filter(chebfi_ctx* ctx, void* Y, int64_t nb, int64_t ld, int degree, double lambda_lo,
                       double lambda_hi, int prec, void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  require_block(ctx, Y, nb, ld);
  CHEBFI_REQUIRE(degree >= 0 && degree <= 1000, CHEBFI_ERR_ARG, "degree out of range");
  CHEBFI_REQUIRE(std::isfinite(lambda_lo) && std::isfinite(lambda_hi) && lambda_hi > lambda_lo, CHEBFI_ERR_ARG,
                 "need finite lambda_lo < lambda_hi");
  CHEBFI_REQUIRE(prec >= 0 && prec <= 2, CHEBFI_ERR_ARG, "bad precision");
  if (nb == 0 || degree == 0) return CHEBFI_OK;
  filter_device_block(ctx, Y, nb, ld, degree, lambda_lo, lambda_hi, prec, S(stream));
  API_END(ctx)
}

int chebfi_cheb_filter_proj(chebfi_ctx* ctx, void* Y, const void* proj, int64_t ldp, int64_t nb, int64_t ld,
                            int degree, double lambda_lo, double lambda_hi, int prec, void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  require_block(ctx, Y, nb, ld);
  CHEBFI_REQUIRE(degree >= 0 && degree <= 1000, CHEBFI_ERR_ARG, "degree out of range");
  CHEBFI_REQUIRE(std::isfinite(lambda_lo) && std::isfinite(lambda_hi) && lambda_hi > lambda_lo, CHEBFI_ERR_ARG,
                 "need finite lambda_lo < lambda_hi");
  CHEBFI_REQUIRE(prec >= 0 && prec <= 2, CHEBFI_ERR_ARG, "bad precision");
  const int64_t nq = ctx->nproj;
  CHEBFI_REQUIRE(!proj || nq == 0 || ldp >= nq, CHEBFI_ERR_ARG, "projection leading dimension below nproj");
  if (nb == 0 || degree == 0) return CHEBFI_OK;
  cudaStream_t st = S(stream);
  const double2* p0 = nq > 0 ? (const double2*)proj : nullptr;
  if (p0 && ldp != nq) {  // the filter reads p_0 with leading dimension nproj
    ctx->w.p0.alloc((size_t)nq * nb);
    CHEBFI_CUDA(cudaMemcpy2DAsync(ctx->w.p0.p, sizeof(double2) * nq, p0, sizeof(double2) * ldp, sizeof(double2) * nq,
                                  nb, cudaMemcpyDeviceToDevice, st));
    p0 = ctx->w.p0.p;
  }
  filter_device_block(ctx, Y, nb, ld, degree, lambda_lo, lambda_hi, prec, st, p0);
  API_END(ctx)
}

int chebfi_cheb_filter_adaptive(chebfi_ctx* ctx, void* Y, int64_t nb, int64_t ld, const int32_t* degrees,
                                double lambda_lo, double lambda_hi, int prec, void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  require_block(ctx, Y, nb, ld);
  CHEBFI_REQUIRE(nb == 0 || degrees, CHEBFI_ERR_ARG, "null degrees");
  CHEBFI_REQUIRE(std::isfinite(lambda_lo) && std::isfinite(lambda_hi) && lambda_hi > lambda_lo, CHEBFI_ERR_ARG,
                 "need finite lambda_lo < lambda_hi");
  CHEBFI_REQUIRE(prec >= 0 && prec <= 2, CHEBFI_ERR_ARG, "bad precision");
  std::vector<int> deg(nb);
  for (int64_t j = 0; j < nb; ++j) {
    CHEBFI_REQUIRE(degrees[j] >= 0 && degrees[j] <= 1000, CHEBFI_ERR_ARG, "degree out of range");
    deg[j] = degrees[j];
  }
  if (nb == 0 || *std::max_element(deg.begin(), deg.end()) == 0) return CHEBFI_OK;
  cudaStream_t st = S(stream);
  gather_to_Ya(ctx, Y, nb, ld, st);
  filter_on_Ya_adaptive(ctx, nb, deg, lambda_lo, lambda_hi, prec, st);
  scatter_from(ctx, ctx->w.Ya.p, Y, nb, ld, st);
  API_END(ctx)
}

int chebfi_adaptive_degrees(const double* ritz, const double* resid, int64_t nb, double lambda_lo, double lambda_hi,
                            double tol, int max_degree, int32_t* degrees) {
  if (nb < 0 || (nb > 0 && (!ritz || !resid || !degrees)) || !(tol > 0.0) || max_degree < 1 ||
      !(lambda_hi > lambda_lo) || !std::isfinite(lambda_lo) || !std::isfinite(lambda_hi))
    return CHEBFI_ERR_ARG;
  std::vector<int> d(nb);
  degrees_for_tolerance(ritz, resid, nb, lambda_lo, lambda_hi, tol, max_degree, d.data());
  for (int64_t i = 0; i < nb; ++i) degrees[i] = d[i];
  return CHEBFI_OK;
}

int chebfi_solve_stats(const chebfi_ctx* ctx, int* sweeps_done, int64_t* band_applies) {
  if (!ctx) return CHEBFI_ERR_ARG;
  if (sweeps_done) *sweeps_done = ctx->last_sweeps;
  if (band_applies) *band_applies = ctx->last_applies;
  return CHEBFI_OK;
}

// chebfi_cheb_filter_host[_proj]: proj (host, nproj x nb, leading dimension ldp) or null
static int filter_host(chebfi_ctx* ctx, void* Y, const void* proj, int64_t ldp, int64_t nb, int64_t ld, int degree,
                double lambda_lo, double lambda_hi, int prec, int nchunks, void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  CHEBFI_REQUIRE(nb >= 0 && (nb == 0 || Y) && ld >= ctx->npw, CHEBFI_ERR_ARG, "bad host block");
  CHEBFI_REQUIRE(degree >= 0 && degree <= 1000, CHEBFI_ERR_ARG, "degree out of range");
  CHEBFI_REQUIRE(std::isfinite(lambda_lo) && std::isfinite(lambda_hi) && lambda_hi > lambda_lo, CHEBFI_ERR_ARG,
                 "need finite lambda_lo < lambda_hi");
  CHEBFI_REQUIRE(prec >= 0 && prec <= 2, CHEBFI_ERR_ARG, "bad precision");
  CHEBFI_REQUIRE(nchunks >= 0, CHEBFI_ERR_ARG, "negative chunk count");
  const int64_t nq = ctx->nproj;
  CHEBFI_REQUIRE(!proj || nq == 0 || ldp >= nq, CHEBFI_ERR_ARG, "projection leading dimension below nproj");
  if (nb == 0 || degree == 0) return CHEBFI_OK;
  cudaStream_t st = S(stream);
  const int64_t npw = ctx->npw;
  const bool with_p = proj && nq > 0;
  // bands are filtered independently, so the block is processed in band chunks: chunk c is
  // copied in while chunk c-1 is filtered and chunk c-2 is copied out (two staging buffers).
  // Only the first chunk's copy in and the last chunk's copy out overlap no filter, so the
  // automatic split from 2048 bands up makes those two chunks half as wide as the three
  // between them; below that, or with nchunks given, the chunks are equal.
  std::vector<int64_t> start;
  if (nchunks == 0 && nb >= 2048) {
    const int64_t half = (nb + 7) / 8;
    start = {0, half, 3 * half, 5 * half, 7 * half, nb};
  } else {
    int nc = nchunks > 0 ? nchunks : (nb >= 1024 ? 2 : 1);
    nc = (int)std::min<int64_t>(nc, nb);
    const int64_t per = (nb + nc - 1) / nc;
    for (int64_t b0 = 0; b0 < nb; b0 += per) start.push_back(b0);
    start.push_back(nb);
  }
  const int nc = (int)start.size() - 1;
  int64_t per = 0;
  for (int c = 0; c < nc; ++c) per = std::max<int64_t>(per, start[c + 1] - start[c]);
  if (!ctx->copy_in) {
    CHEBFI_CUDA(cudaStreamCreateWithFlags(&ctx->copy_in, cudaStreamNonBlocking));
    CHEBFI_CUDA(cudaStreamCreateWithFlags(&ctx->copy_out, cudaStreamNonBlocking));
    for (int i = 0; i < 2; ++i) {
      CHEBFI_CUDA(cudaEventCreateWithFlags(&ctx->ev_in[i], cudaEventDisableTiming));
      CHEBFI_CUDA(cudaEventCreateWithFlags(&ctx->ev_filt[i], cudaEventDisableTiming));
      CHEBFI_CUDA(cudaEventCreateWithFlags(&ctx->ev_out[i], cudaEventDisableTiming));
    }
  }
  const int nbuf = nc > 1 ? 2 : 1;
  for (int i = 0; i < nbuf; ++i) {
    ctx->stage[i].alloc((size_t)npw * per);
    if (with_p) ctx->stage_p[i].alloc((size_t)nq * per);
  }
  // the copies start after whatever the caller queued on st before this call
  CHEBFI_CUDA(cudaEventRecord(ctx->ev_filt[0], st));
  CHEBFI_CUDA(cudaStreamWaitEvent(ctx->copy_in, ctx->ev_filt[0], 0));
  bool used[2] = {false, false};
  char* host = static_cast<char*>(Y);
  const char* hproj = static_cast<const char*>(proj);
  for (int c = 0; c < nc; ++c) {
    const int64_t b0 = start[c], nbc = start[c + 1] - b0;
    if (nbc <= 0) continue;
    const int k = c % nbuf;
    double2* dev = ctx->stage[k].p;
    // chunk c-2 copied out and filtered (its projections read)
    if (used[k]) CHEBFI_CUDA(cudaStreamWaitEvent(ctx->copy_in, ctx->ev_out[k], 0));
    CHEBFI_CUDA(cudaMemcpy2DAsync(dev, sizeof(double2) * npw, host + sizeof(double2) * b0 * ld, sizeof(double2) * ld,
                                  sizeof(double2) * npw, nbc, cudaMemcpyHostToDevice, ctx->copy_in));
    if (with_p)
      CHEBFI_CUDA(cudaMemcpy2DAsync(ctx->stage_p[k].p, sizeof(double2) * nq, hproj + sizeof(double2) * b0 * ldp,
                                    sizeof(double2) * ldp, sizeof(double2) * nq, nbc, cudaMemcpyHostToDevice,
                                    ctx->copy_in));
    CHEBFI_CUDA(cudaEventRecord(ctx->ev_in[k], ctx->copy_in));
    CHEBFI_CUDA(cudaStreamWaitEvent(st, ctx->ev_in[k], 0));
    filter_device_block(ctx, dev, nbc, npw, degree, lambda_lo, lambda_hi, prec, st,
                        with_p ? ctx->stage_p[k].p : nullptr);
    CHEBFI_CUDA(cudaEventRecord(ctx->ev_filt[k], st));
    CHEBFI_CUDA(cudaStreamWaitEvent(ctx->copy_out, ctx->ev_filt[k], 0));
    CHEBFI_CUDA(cudaMemcpy2DAsync(host + sizeof(double2) * b0 * ld, sizeof(double2) * ld, dev, sizeof(double2) * npw,
                                  sizeof(double2) * npw, nbc, cudaMemcpyDeviceToHost, ctx->copy_out));
    CHEBFI_CUDA(cudaEventRecord(ctx->ev_out[k], ctx->copy_out));
    used[k] = true;
  }
  // completion on st covers the last copies out
  for (int k = 0; k < nbuf; ++k)
    if (used[k]) CHEBFI_CUDA(cudaStreamWaitEvent(st, ctx->ev_out[k], 0));
  API_END(ctx)
}

int chebfi_cheb_filter_host(chebfi_ctx* ctx, void* Y, int64_t nb, int64_t ld, int degree, double lambda_lo,
                            double lambda_hi, int prec, int nchunks, void* stream) {
  return filter_host(ctx, Y, nullptr, 0, nb, ld, degree, lambda_lo, lambda_hi, prec, nchunks, stream);
}

int chebfi_cheb_filter_host_proj(chebfi_ctx* ctx, void* Y, const void* proj, int64_t ldp, int64_t nb, int64_t ld,
                                 int degree, double lambda_lo, double lambda_hi, int prec, int nchunks,
                                 void* stream) {
  return filter_host(ctx, Y, proj, ldp, nb, ld, degree, lambda_lo, lambda_hi, prec, nchunks, stream);
}

int chebfi_orthonormalise(chebfi_ctx* ctx, void* Y, int64_t nb, int64_t ld, void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  require_block(ctx, Y, nb, ld);
  if (nb == 0) return CHEBFI_OK;
  cudaStream_t st = S(stream);
  gather_to_Ya(ctx, Y, nb, ld, st);
  ctx->w.tmp.alloc(ctx->w.Ya.n);
  ortho_on_Ya(ctx, nb, st);
  scatter_from(ctx, ctx->w.Ya.p, Y, nb, ld, st);
  CHEBFI_CUDA(cudaStreamSynchronize(st));
  API_END(ctx)
}

int chebfi_rayleigh_ritz(chebfi_ctx* ctx, void* Y, double* evals, double* resid, int64_t nb, int64_t ld,
                         void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  require_block(ctx, Y, nb, ld);
  CHEBFI_REQUIRE(nb == 0 || evals, CHEBFI_ERR_ARG, "null evals");
  if (nb == 0) return CHEBFI_OK;
  cudaStream_t st = S(stream);
  gather_to_Ya(ctx, Y, nb, ld, st);
  ctx->w.tmp.alloc(ctx->w.Ya.n);
  rr_on_Ya(ctx, nb, evals, resid, st);
  scatter_from(ctx, ctx->w.Ya.p, Y, nb, ld, st);
  CHEBFI_CUDA(cudaStreamSynchronize(st));
  API_END(ctx)
}

int chebfi_rayleigh_ritz_proj(chebfi_ctx* ctx, void* Y, double* evals, double* resid, void* proj, int64_t ldp,
                              int64_t nb, int64_t ld, void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  require_block(ctx, Y, nb, ld);
  CHEBFI_REQUIRE(nb == 0 || evals, CHEBFI_ERR_ARG, "null evals");
  const int64_t nq = ctx->nproj;
  CHEBFI_REQUIRE(!proj || nq == 0 || ldp >= nq, CHEBFI_ERR_ARG, "projection leading dimension below nproj");
  if (nb == 0) return CHEBFI_OK;
  cudaStream_t st = S(stream);
  gather_to_Ya(ctx, Y, nb, ld, st);
  ctx->w.tmp.alloc(ctx->w.Ya.n);
  rr_on_Ya(ctx, nb, evals, resid, st);
  scatter_from(ctx, ctx->w.Ya.p, Y, nb, ld, st);
  if (proj && nq > 0)  // P^H Y of the rotated block, formed by the rotation for S Y
    CHEBFI_CUDA(cudaMemcpy2DAsync(proj, sizeof(double2) * ldp, ctx->w.pc.p, sizeof(double2) * nq,
                                  sizeof(double2) * nq, nb, cudaMemcpyDeviceToDevice, st));
  CHEBFI_CUDA(cudaStreamSynchronize(st));
  API_END(ctx)
}

int chebfi_rayleigh_quotients(chebfi_ctx* ctx, const void* Y, double* rq, int64_t nb, int64_t ld, void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  require_block(ctx, Y, nb, ld);
  CHEBFI_REQUIRE(nb == 0 || rq, CHEBFI_ERR_ARG, "null rq");
  if (nb == 0) return CHEBFI_OK;
  cudaStream_t st = S(stream);
  gather_to_Ya(ctx, Y, nb, ld, st);
  rq_sorted(ctx, ctx->w.Ya.p, nb, rq, st);
  API_END(ctx)
}

int chebfi_solve(chebfi_ctx* ctx, void* Y, double* evals, double* resid, int64_t nb, int64_t ld,
                 const chebfi_params* params, void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  require_block(ctx, Y, nb, ld);
  CHEBFI_REQUIRE(params && evals, CHEBFI_ERR_ARG, "null params or evals");
  CHEBFI_REQUIRE(params->degree >= 1 && params->sweeps >= 1, CHEBFI_ERR_ARG, "degree and sweeps must be >= 1");
  CHEBFI_REQUIRE(params->prec >= 0 && params->prec <= 2, CHEBFI_ERR_ARG, "bad precision");
  if (nb == 0) return CHEBFI_OK;
  cudaStream_t st = S(stream);
  double hi = params->lambda_hi;
  if (!(hi > 0.0)) {
    if (params->bound_mode == CHEBFI_BOUND_PAPER) hi = ctx->kmax;
    else if (params->bound_mode == CHEBFI_BOUND_RIGOROUS) hi = rigorous_bound(ctx);
    else throw Error{CHEBFI_ERR_ARG, "unknown bound mode"};
  }
  // precision in which the filtered vectors are held (FP32 for both FP32 and mixed forms;
  // the mixed form's tensor-core products perturb each application, not the storage)
  const double eps = params->prec == CHEBFI_F64 ? 2.220446049250313e-16 : 1.1920928955078125e-07;
  gather_to_Ya(ctx, Y, nb, ld, st);
  ctx->w.tmp.alloc(ctx->w.Ya.n);
  // the first sweep's lambda_- comes from Rayleigh quotients; later sweeps reuse the Ritz
  // values of the previous one (the Rayleigh quotients of Ritz vectors)
  ctx->w.dvec3.alloc(nb);
  rq_sorted(ctx, ctx->w.Ya.p, nb, ctx->w.dvec3.p, st);
  double lo = host_max(ctx, ctx->w.dvec3.p, nb, st);
  double l1 = host_max(ctx, ctx->w.dvec3.p, nb, st, true);
  CHEBFI_REQUIRE(std::isfinite(lo) && std::isfinite(l1), CHEBFI_ERR_NONFINITE,
                 "solve: Inf or NaN in the Rayleigh quotients of the starting block");
  // locking (Section 5.4): after a full-degree sweep, each band gets the degree its residual
  // estimate needs for params->tol; converged bands are not filtered
  const bool lock = params->lock != 0;
  CHEBFI_REQUIRE(!lock || params->tol > 0.0, CHEBFI_ERR_ARG, "locking needs tol > 0");
  std::vector<int> deg(nb, params->degree);
  double* res = resid;
  if (lock && !res) {
    ctx->w.dvec2.alloc(nb);
    res = ctx->w.dvec2.p;
  }
  int dmax = params->degree;
  int sweeps_done = 0;
  int64_t applies = 0;
  for (int s = 0; s < params->sweeps && dmax > 0; ++s) {
    CHEBFI_REQUIRE(hi > lo, CHEBFI_ERR_ARG, "upper bound below the largest Rayleigh quotient");
    const double c = 0.5 * (hi + lo), r = 0.5 * (hi - lo);
    if (cheb_T_abs(dmax, (l1 - c) / r) >= 1.0 / (100.0 * eps))
      throw Error{CHEBFI_ERR_FILTER_OVERFLOW, "T_n((lambda_1 - c)/r) exceeds 1/(100 eps) of the filter precision"};
    if (lock && s > 0) {
      filter_on_Ya_adaptive(ctx, nb, deg, lo, hi, params->prec, st);
    } else {
      // after the first sweep the previous Rayleigh-Ritz step holds P^H Y (FP64): the
      // filter starts from it instead of forming it again
      const double2* p0 = (s > 0 && ctx->w.pc_of == ctx->w.Ya.p) ? ctx->w.pc.p : nullptr;
      filter_on_Ya(ctx, nb, params->degree, lo, hi, params->prec, st, p0);
    }
    for (int64_t j = 0; j < nb; ++j) applies += (lock && s > 0) ? deg[j] : params->degree;
    sweeps_done = s + 1;
    ctx->w.tmp.alloc(ctx->w.Ya.n);
    rr_on_Ya(ctx, nb, evals, res, st);
    lo = host_max(ctx, evals, nb, st);
    l1 = host_max(ctx, evals, nb, st, true);
    CHEBFI_REQUIRE(std::isfinite(lo) && std::isfinite(l1), CHEBFI_ERR_NONFINITE,
                   "solve: Inf or NaN in the Ritz values of sweep " + std::to_string(s + 1));
    if (lock) {
      std::vector<double> he(nb), hr(nb);
      CHEBFI_CUDA(cudaMemcpyAsync(he.data(), evals, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
      CHEBFI_CUDA(cudaMemcpyAsync(hr.data(), res, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
      CHEBFI_CUDA(cudaStreamSynchronize(st));
      degrees_for_tolerance(he.data(), hr.data(), nb, lo, hi, params->tol, params->degree, deg.data());
      dmax = *std::max_element(deg.begin(), deg.end());
    }
  }
  ctx->last_sweeps = sweeps_done;
  ctx->last_applies = applies;
  scatter_from(ctx, ctx->w.Ya.p, Y, nb, ld, st);
  CHEBFI_CUDA(cudaStreamSynchronize(st));
  API_END(ctx)
}

int chebfi_profile_enable(chebfi_ctx* ctx, int enable) {
  API_BEGIN(ctx)
  ctx->prof.flush();
  if (enable) {
    ctx->prof.names.clear();
    ctx->prof.ms.clear();
    ctx->prof.count.clear();
    ctx->prof.work.clear();
  }
  ctx->prof.on = enable != 0;
  API_END(ctx)
}

int chebfi_profile_count(chebfi_ctx* ctx) {
  if (!ctx) return CHEBFI_ERR_ARG;
  try {
    CHEBFI_CUDA(cudaSetDevice(ctx->device));
    ctx->prof.flush();
  } catch (const Error& e) {
    ctx->err = e.msg;
    return e.code;
  }
  return (int)ctx->prof.names.size();
}

int chebfi_profile_entry(chebfi_ctx* ctx, int i, char* name, int name_len, double* ms, int64_t* launches,
                         double* work) {
  API_BEGIN(ctx)
  ctx->prof.flush();
  CHEBFI_REQUIRE(i >= 0 && i < (int)ctx->prof.names.size(), CHEBFI_ERR_ARG, "profile entry out of range");
  if (name && name_len > 0) {
    std::strncpy(name, ctx->prof.names[i].c_str(), name_len - 1);
    name[name_len - 1] = 0;
  }
  if (ms) *ms = ctx->prof.ms[i];
  if (launches) *launches = ctx->prof.count[i];
  if (work) *work = ctx->prof.work[i];
  API_END(ctx)
}

int chebfi_set_D(chebfi_ctx* ctx, const double* D, int on_device) {
  API_BEGIN(ctx)
  CHEBFI_REQUIRE(ctx->has_proj && ctx->nproj > 0, CHEBFI_ERR_STATE, "set_projectors (with projectors) first");
  CHEBFI_REQUIRE(D, CHEBFI_ERR_ARG, "null D");
  int64_t nblkv = 0;
  for (int a = 0; a < ctx->natoms; ++a) {
    const int64_t na = ctx->offs[a + 1] - ctx->offs[a];
    nblkv += na * na;
  }
  std::vector<double> h(nblkv);
  if (on_device) CHEBFI_CUDA(cudaMemcpy(h.data(), D, sizeof(double) * nblkv, cudaMemcpyDeviceToHost));
  else std::memcpy(h.data(), D, sizeof(double) * nblkv);
  for (double v : h) CHEBFI_REQUIRE(std::isfinite(v), CHEBFI_ERR_NONFINITE, "D is not finite");
  ctx->d_Dblk.upload(h.data(), nblkv);
  std::vector<float> hf(h.begin(), h.end());
  ctx->d_Dblkf.upload(hf.data(), nblkv);
  CHEBFI_CUDA(cudaDeviceSynchronize());
  ctx->bound_rigorous = -1.0;
  API_END(ctx)
}

int chebfi_apply_H_backward(chebfi_ctx* ctx, const void* Y, const void* G, void* gY, double* gV, double* gD, int64_t nb,
                            int64_t ld, void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  require_block(ctx, Y, nb, ld);
  CHEBFI_REQUIRE(nb == 0 || G, CHEBFI_ERR_ARG, "null G");
  cudaStream_t st = S(stream);
  Work& w = ctx->w;
  const int64_t npw = ctx->npw, nq = ctx->nproj;
  if (nb == 0) {
    if (gV) CHEBFI_CUDA(cudaMemsetAsync(gV, 0, sizeof(double) * ctx->grid[0] * ctx->grid[1] * ctx->grid[2], st));
    return CHEBFI_OK;
  }
  // sorted copies: Y -> Ya, G -> Yb
  w.Ya.alloc((size_t)npw * nb);
  w.Yb.alloc((size_t)npw * nb);
  gather_rows(npw, nb, ctx->d_sorted_to_user.p, (const double2*)Y, ld, w.Ya.p, npw, st);
  gather_rows(npw, nb, ctx->d_sorted_to_user.p, (const double2*)G, ld, w.Yb.p, npw, st);
  if (gY) {  // H is Hermitian: the gradient with respect to Y is H G
    const size_t np = (size_t)std::max<int64_t>(nq, 1) * nb;
    w.HY.alloc((size_t)npw * nb);
    w.T1.alloc(local_workspace_elems(ctx, nb));
    w.pa.alloc(np);
    w.pb.alloc(np);
    apply_H_sorted<double>(ctx, w.Yb.p, w.HY.p, w.pa.p, w.pb.p, w.T1.p, nb, st, "gemm_H");
    scatter_from(ctx, w.HY.p, gY, nb, ld, st);
  }
  if (gD && nq > 0) {  // gD_ij = sum_n Re(conj((P^H G)_in) (P^H Y)_jn) on the atom blocks
    w.pa.alloc((size_t)nq * nb);
    w.pc.alloc((size_t)nq * nb);
    gemm64(ctx, true, false, nq, nb, npw, 1.0, ctx->d_P.p, npw, w.Yb.p, npw, 0.0, w.pa.p, nq, st, &w.splitk, "gemm_H");
    gemm64(ctx, true, false, nq, nb, npw, 1.0, ctx->d_P.p, npw, w.Ya.p, npw, 0.0, w.pc.p, nq, st, &w.splitk, "gemm_H");
    block_outer_grad(ctx, w.pa.p, w.pc.p, nq, nb, gD, st);
  }
  if (gV) vloc_gradient<double>(ctx, w.Ya.p, w.Yb.p, nb, gV, st, w.T2, w.tmp, w.tmp2);
  API_END(ctx)
}

int chebfi_apply_Sinv_refined(chebfi_ctx* ctx, const void* X, void* out, int64_t nb, int64_t ld, double tol,
                              int maxit, int* iterations, void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  require_block(ctx, X, nb, ld);
  CHEBFI_REQUIRE(nb == 0 || out, CHEBFI_ERR_ARG, "null out");
  CHEBFI_REQUIRE(tol > 0.0 && std::isfinite(tol) && maxit >= 0, CHEBFI_ERR_ARG, "need tol > 0 and maxit >= 0");
  if (iterations) *iterations = 0;
  if (nb == 0) return CHEBFI_OK;
  cudaStream_t st = S(stream);
  Work& w = ctx->w;
  const int64_t npw = ctx->npw, nq = ctx->nproj;
  gather_to_Ya(ctx, X, nb, ld, st);
  int it = 0;
  bool converged = true;
  if (ctx->paw) {
    ensure_refine(ctx, st);
    const size_t np = (size_t)nq * nb;
    w.pa.alloc(np);  // b = P^H x
    w.pb.alloc(np);  // q
    w.pc.alloc(np);  // r
    w.pt.alloc(np);  // B^{-1} r
    w.dvec1.alloc(nb);
    w.dvec2.alloc(nb);
    gemm64(ctx, true, false, nq, nb, npw, 1.0, ctx->d_P.p, npw, w.Ya.p, npw, 0.0, w.pa.p, nq, st, &w.splitk, "gemm_refine");
    column_dots(nq, nb, w.pa.p, nq, w.pa.p, nq, w.dvec1.p, false, st);
    std::vector<double> bn(nb), rn(nb);
    CHEBFI_CUDA(cudaMemcpyAsync(bn.data(), w.dvec1.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
    CHEBFI_CUDA(cudaMemsetAsync(w.pb.p, 0, sizeof(double2) * np, st));
    for (it = 0; it <= maxit; ++it) {
      // r = b - A q
      CHEBFI_CUDA(cudaMemcpyAsync(w.pc.p, w.pa.p, sizeof(double2) * np, cudaMemcpyDeviceToDevice, st));
      if (it > 0)
        gemm64(ctx, false, false, nq, nb, nq, -1.0, ctx->d_Aref.p, nq, w.pb.p, nq, 1.0, w.pc.p, nq, st, &w.splitk,
                     "gemm_refine");
      column_dots(nq, nb, w.pc.p, nq, w.pc.p, nq, w.dvec2.p, false, st);
      CHEBFI_CUDA(cudaMemcpyAsync(rn.data(), w.dvec2.p, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
      CHEBFI_CUDA(cudaStreamSynchronize(st));
      converged = true;
      for (int64_t b = 0; b < nb; ++b)
        if (!(std::sqrt(std::max(rn[b], 0.0)) <= tol * std::sqrt(std::max(bn[b], 0.0)))) converged = false;
      if (converged || it == maxit) break;
      // q <- q + B^{-1} r
      blockdiag_apply_c(ctx, ctx->d_Binv.p, ctx->d_cblk_off.p, w.pc.p, nq, w.pt.p, nq, nb, st);
      axpby<double>(nq, nb, 1.0, w.pt.p, nq, 1.0, w.pb.p, nq, w.pb.p, nq, st);
    }
    // S^{-1} x = x - P q
    gemm64(ctx, false, false, npw, nb, nq, -1.0, ctx->d_P.p, npw, w.pb.p, nq, 1.0, w.Ya.p, npw, st, &w.splitk,
                 "gemm_refine");
  }
  scatter_from(ctx, w.Ya.p, out, nb, ld, st);
  CHEBFI_CUDA(cudaStreamSynchronize(st));
  if (iterations) *iterations = it;
  CHEBFI_REQUIRE(converged, CHEBFI_ERR_NO_CONVERGENCE,
                 "iterative refinement did not reach the tolerance in " + std::to_string(maxit) + " iterations");
  API_END(ctx)
}

int chebfi_cheb_filter_backward(chebfi_ctx* ctx, const void* Y0, const void* gYn, void* gY0, double* gV, double* gD,
                                int64_t nb, int64_t ld, int degree, double lambda_lo, double lambda_hi, int prec,
                                int checkpoint_every, void* stream) {
  API_BEGIN(ctx)
  require_ready(ctx);
  require_block(ctx, Y0, nb, ld);
  CHEBFI_REQUIRE(nb == 0 || gYn, CHEBFI_ERR_ARG, "null gYn");
  CHEBFI_REQUIRE(degree >= 0 && degree <= 1000, CHEBFI_ERR_ARG, "degree out of range");
  CHEBFI_REQUIRE(std::isfinite(lambda_lo) && std::isfinite(lambda_hi) && lambda_hi > lambda_lo, CHEBFI_ERR_ARG,
                 "need finite lambda_lo < lambda_hi");
  CHEBFI_REQUIRE(prec == CHEBFI_F64 || prec == CHEBFI_F32, CHEBFI_ERR_ARG,
                 "the filter backward runs in the FP64 or the FP32 form");
  CHEBFI_REQUIRE(checkpoint_every >= 0, CHEBFI_ERR_ARG, "negative checkpoint interval");
  cudaStream_t st = S(stream);
  Work& w = ctx->w;
  const int64_t npw = ctx->npw;
  int64_t nblkv = 0;
  for (int a = 0; a < ctx->natoms; ++a) {
    const int64_t na = ctx->offs[a + 1] - ctx->offs[a];
    nblkv += na * na;
  }
  if (gV) CHEBFI_CUDA(cudaMemsetAsync(gV, 0, sizeof(double) * ctx->grid[0] * ctx->grid[1] * ctx->grid[2], st));
  if (gD && nblkv > 0) CHEBFI_CUDA(cudaMemsetAsync(gD, 0, sizeof(double) * nblkv, st));
  if (nb == 0) return CHEBFI_OK;
  w.Ya.alloc((size_t)npw * nb);
  w.Yb.alloc((size_t)npw * nb);
  gather_rows(npw, nb, ctx->d_sorted_to_user.p, (const double2*)Y0, ld, w.Ya.p, npw, st);
  gather_rows(npw, nb, ctx->d_sorted_to_user.p, (const double2*)gYn, ld, w.Yb.p, npw, st);
  if (degree == 0) {  // the filter is the identity
    if (gY0) scatter_from(ctx, w.Yb.p, gY0, nb, ld, st);
    return CHEBFI_OK;
  }
  int s = checkpoint_every;
  if (s == 0) s = (int)std::ceil(std::sqrt((double)degree));
  s = std::max(1, std::min(s, degree));
  if (prec == CHEBFI_F64) filter_backward<double>(ctx, nb, degree, lambda_lo, lambda_hi, s, gV, gD, st);
  else filter_backward<float>(ctx, nb, degree, lambda_lo, lambda_hi, s, gV, gD, st);
  if (gY0) scatter_from(ctx, w.Ya.p, gY0, nb, ld, st);
  API_END(ctx)
}

int chebfi_set_fp64_gemm(chebfi_ctx* ctx, int engine, int nmod, int* precision_bits) {
  API_BEGIN(ctx)
  CHEBFI_REQUIRE(engine >= CHEBFI_GEMM_AUTO && engine <= CHEBFI_GEMM_TENSOR, CHEBFI_ERR_ARG, "unknown GEMM engine");
  CHEBFI_REQUIRE(nmod == 0 || (nmod >= kOzMinMod && nmod <= kOzMaxMod), CHEBFI_ERR_ARG,
                 "modulus count must be 0 or 8..15");
  ctx->fp64_gemm = engine;
  if (nmod) ctx->oz_nmod = nmod;
  if (precision_bits) *precision_bits = oz_precision_bits(ctx->oz_nmod);
  API_END(ctx)
}

int chebfi_set_eigensolver(chebfi_ctx* ctx, int mode) {
  API_BEGIN(ctx)
  CHEBFI_REQUIRE(mode >= CHEBFI_EIG_AUTO && mode <= CHEBFI_EIG_REFINED, CHEBFI_ERR_ARG, "unknown eigensolver");
  ctx->eig_mode = mode;
  API_END(ctx)
}

int chebfi_eigensolver_steps(const chebfi_ctx* ctx) { return ctx ? ctx->eig_iters : CHEBFI_ERR_ARG; }

int chebfi_gemm_fp64(chebfi_ctx* ctx, int conjA, int conjB, int64_t m, int64_t n, int64_t k, double alpha,
                     const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C, int64_t ldc,
                     void* stream) {
  API_BEGIN(ctx)
  CHEBFI_REQUIRE(m >= 0 && n >= 0 && k >= 0, CHEBFI_ERR_ARG, "negative size");
  if (m == 0 || n == 0) return CHEBFI_OK;
  CHEBFI_REQUIRE(C && ldc >= m, CHEBFI_ERR_ARG, "C must be non-null with ldc >= m");
  CHEBFI_REQUIRE(k == 0 || (A && B), CHEBFI_ERR_ARG, "null A or B");
  CHEBFI_REQUIRE(lda >= (conjA ? k : m) && lda >= 1 && ldb >= (conjB ? n : k) && ldb >= 1, CHEBFI_ERR_ARG,
                 "leading dimension too small");
  cudaStream_t st = S(stream);
  if (k == 0) {
    // C = beta C: an empty product through the CUDA-core path (it applies beta)
    gemm<double>(false, false, m, n, 0, alpha, nullptr, m, nullptr, 1, beta, (double2*)C, ldc, st);
    return CHEBFI_OK;
  }
  gemm64(ctx, conjA != 0, conjB != 0, m, n, k, alpha, (const double2*)A, lda, (const double2*)B, ldb, beta,
         (double2*)C, ldc, st, &ctx->w.splitk, "gemm_fp64");
  API_END(ctx)
}

int chebfi_set_fft64(chebfi_ctx* ctx, int mode) {
  API_BEGIN(ctx)
  CHEBFI_REQUIRE(mode == CHEBFI_FFT64_NATIVE || mode == CHEBFI_FFT64_DOUBLE_FLOAT, CHEBFI_ERR_ARG,
                 "fft64 mode must be CHEBFI_FFT64_NATIVE or CHEBFI_FFT64_DOUBLE_FLOAT");
  ctx->fft64 = mode;
  API_END(ctx)
}

int chebfi_gemm_mixed(chebfi_ctx* ctx, int conjA, int64_t m, int64_t n, int64_t k, float alpha, const void* A,
                      int64_t lda, const void* B, int64_t ldb, float beta, void* C, int64_t ldc, void* stream) {
  API_BEGIN(ctx)
  CHEBFI_REQUIRE(m >= 0 && n >= 0 && k >= 1, CHEBFI_ERR_ARG, "need m, n >= 0 and k >= 1");
  if (m == 0 || n == 0) return CHEBFI_OK;
  CHEBFI_REQUIRE(A && B && C, CHEBFI_ERR_ARG, "null A, B or C");
  CHEBFI_REQUIRE(lda >= (conjA ? k : m) && ldb >= k && ldc >= m, CHEBFI_ERR_ARG, "leading dimension too small");
  cudaStream_t st = S(stream);
  Work& w = ctx->w;
  if (conjA) embed3f(true, k, m, (const float2*)A, lda, w.gA3, st);
  else embed3f(false, m, k, (const float2*)A, lda, w.gA3, st);
  split3_block(k, n, (const float2*)B, ldb, w.gB3, st);
  tc_cgemm3(w.gA3, w.gB3, conjA != 0, m, n, k, alpha, beta, (const float2*)C, ldc, (float2*)C, ldc, ctx->d_status.p,
            st, "gemm_mixed", &w.tcws);
  API_END(ctx)
}

int chebfi_sync_status(chebfi_ctx* ctx) {
  API_BEGIN(ctx)
  CHEBFI_CUDA(cudaDeviceSynchronize());
  check_status(ctx, 0, "device");
  API_END(ctx)
}

}  // extern "C"
