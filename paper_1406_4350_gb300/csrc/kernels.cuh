// Launchers of the device kernels (one translation unit each: fft.cu, gemm.cu,
// blas.cu, dense.cu).  All matrices are column-major; complex values interleaved.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.cuh"

namespace chebfi {

// ---------------------------------------------------------------- local operator (fft.cu)
// Epilogue of the (K + V_loc) pass for sphere point j of band b:
//   Z = K_j Y_j + (V_loc Y)_j                      -> Z[b*ldz + j]     (if Z)
//   T = a (Z - c Y_j) - bprev Yprev[b*ldt + j]     -> T[b*ldt + j]     (if T; may alias Yprev)
//   (hi, lo) bf16 pair of Z, 2 reals per point           -> Zhi/Zlo[b*ldzb + 2j + {0,1}] (if Zhi)
template <typename R> struct LocalEpi {
  const cplx<R>* Y = nullptr;
  int64_t ldy = 0;
  cplx<R>* Z = nullptr;
  int64_t ldz = 0;
  // bf16 (hi, lo) pair of Z: interleaved (re, im) at Zhi + b * ldzb + 2 j (zplane = 0), or the
  // planes (re, im, re + im) of the three-multiplication product at Zhi + q * zplane + b * ldzb + j
  __nv_bfloat16* Zhi = nullptr;
  __nv_bfloat16* Zlo = nullptr;
  int64_t ldzb = 0, zplane = 0;
  cplx<R>* T = nullptr;
  const cplx<R>* Yprev = nullptr;
  int64_t ldt = 0;
  R a = 0, c = 0, bprev = 0, inv_n3 = 0;
};
#ifdef __CUDACC__
// element j of band b of Z into the epilogue's bf16 planes
template <typename R>
__device__ __forceinline__ void epi_split_z(const LocalEpi<R>& ep, int64_t b, int64_t j, float zr, float zi) {
  if (ep.zplane == 0) {
    const int64_t o = b * ep.ldzb + 2 * j;
    const __nv_bfloat16 hr = __float2bfloat16_rn(zr), hi_ = __float2bfloat16_rn(zi);
    ep.Zhi[o] = hr;
    ep.Zhi[o + 1] = hi_;
    ep.Zlo[o] = __float2bfloat16_rn(zr - __bfloat162float(hr));
    ep.Zlo[o + 1] = __float2bfloat16_rn(zi - __bfloat162float(hi_));
    return;
  }
  const int64_t o = b * ep.ldzb + j;
  const float zs = zr + zi;
  const __nv_bfloat16 hr = __float2bfloat16_rn(zr), hi_ = __float2bfloat16_rn(zi), hs = __float2bfloat16_rn(zs);
  ep.Zhi[o] = hr;
  ep.Zhi[o + ep.zplane] = hi_;
  ep.Zhi[o + 2 * ep.zplane] = hs;
  ep.Zlo[o] = __float2bfloat16_rn(zr - __bfloat162float(hr));
  ep.Zlo[o + ep.zplane] = __float2bfloat16_rn(zi - __bfloat162float(hi_));
  ep.Zlo[o + 2 * ep.zplane] = __float2bfloat16_rn(zs - __bfloat162float(hs));
}
#endif
size_t local_workspace_elems(const chebfi_ctx* ctx, int64_t nb);
// Derivative of (V_loc psi) with respect to V_loc for a real loss whose gradient at the
// output is g: gV(x, y, z) = (1/N^3) sum_b Re(conj(g_b(r)) psi_b(r)) with psi_b, g_b the
// real-space values of sorted-order sphere blocks Ys, Gs (ld = npw).  FP64.
template <typename R>
void vloc_gradient(chebfi_ctx* ctx, const cplx<R>* Ys, const cplx<R>* Gs, int64_t nb, double* gV, cudaStream_t st,
                   DevBuf<cplx<R>>& T, DevBuf<cplx<R>>& Rb, DevBuf<cplx<R>>& Gb, double scale = 1.0,
                   bool accumulate = false);
// gD[entry (i, j) of atom block a] = scale * sum_b Re(conj(q_ib) p_jb)  (+= if accumulate)
template <typename C>
void block_outer_grad(const chebfi_ctx* ctx, const C* q, const C* p, int64_t ldp, int64_t nb, double* gD,
                      cudaStream_t st, double scale = 1.0, bool accumulate = false);
// the two-pass FFT kernels cover cubic grids of a few compiled sizes; split_index(n, p) is
// the natural index held at position p of their split order
bool fast_fft_supported(int n1, int n2, int n3);
int split_index(int n, int p);
template <typename R>
void local_apply(chebfi_ctx* ctx, const cplx<R>* Y, int64_t ldy, int64_t nb, cplx<R>* T, LocalEpi<R> ep,
                 cudaStream_t st);

// ---------------------------------------------------------------- complex GEMM (gemm.cu)
// C = alpha op(A) op(B) + beta C, op = identity or conjugate transpose; real alpha, beta.
// M x N result, inner dimension K.  ws: optional split-K workspace (nullptr = no split).
// tag: the name the launch is timed under when profiling is on.  lower: square result,
// only tiles touching the lower triangle are computed (the rest of C is left undefined).
template <typename R>
void gemm(bool conjA, bool conjB, int64_t M, int64_t N, int64_t K, double alpha, const cplx<R>* A,
          int64_t lda, const cplx<R>* B, int64_t ldb, double beta, cplx<R>* C, int64_t ldc, cudaStream_t st,
          DevBuf<cplx<R>>* ws = nullptr, const char* tag = "k_gemm", bool lower = false);

// ---------------------------------------------------------------- tensor cores (gemm_tc.cu)
// D (M x N, FP32 column-major) = alpha A B + beta C with A (M x K) and B (K x N) K-major
// bf16 pairs; tcgen05 tensor cores with FP32 accumulation.  C may equal D.
void tc_gemm(const SplitBF16& A, const SplitBF16& B, int64_t M, int64_t N, int64_t K, float alpha, float beta,
             const float* C, int64_t ldc, float* D, int64_t ldd, int* status, cudaStream_t st, const char* tag,
             DevBuf<float>* ws = nullptr);
// Grouped form: items (problem, output tile of 128 x 128) over problems whose tensor maps
// and sizes sit in device tables; CTA b takes items b, b + grid, ...  work: the algorithmic
// flops of all items, for the profiler.
void tc_gemm_grouped(const CUtensorMap* maps, const TcGroupProb* probs, const int2* items, int nitems, float alpha_mul,
                     int* status, cudaStream_t st, const char* tag, double work);
// the bf16 (hi, lo) real embeddings of P^H, P, G and M of a context, built on first use
void ensure_tc_operands(chebfi_ctx* ctx, cudaStream_t st);
// bf16 tensor map of a K-major operand (k reals per row, `rows` rows, row stride ld) with the
// boxes of the tensor-core GEMMs
CUtensorMap tc_map(const __nv_bfloat16* base, int64_t k, int64_t rows, int64_t ld);
// Real embeddings (bf16 pairs) of complex operators applied to interleaved complex data:
// embed_ph: the (2 nq) x (2 npw) matrix of x -> P^H x;  embed_n: the (2m) x (2k) matrix of x -> A x.
void embed_ph(int64_t npw, int64_t nq, const double2* P, int64_t ldp, SplitBF16Buf& out, cudaStream_t st);
void embed_n(int64_t m, int64_t k, const double2* A, int64_t lda, SplitBF16Buf& out, cudaStream_t st);
// complex FP32 block (m x nb) -> K-major bf16 pair with 2m reals per column
void split_block(int64_t m, int64_t nb, const float2* x, int64_t ldx, SplitBF16Buf& out, cudaStream_t st);
// The three planes of the three-multiplication products: of P (Re, Im, Re + Im; rows =
// plane waves, K = projectors) and of a complex FP32 block (re, im, re + im; rows = its
// columns).
void embed3_n(int64_t npw, int64_t nq, const double2* P, int64_t ldp, SplitBF16x3& out, cudaStream_t st);
void split3_block(int64_t m, int64_t nb, const float2* x, int64_t ldx, SplitBF16x3& out, cudaStream_t st);
// the planes of a complex FP32 matrix A (rows x cols): of A^H (conj) or of A
void embed3f(bool conj, int64_t rows, int64_t cols, const float2* A, int64_t lda, SplitBF16x3& out, cudaStream_t st);
// Complex D = alpha op(A) B + beta C (M x N, column-major, interleaved FP32; C may be D) by
// three real tensor-core products of the planes (Gauss's form); conjA: op(A) = A^H with A's
// planes (Re, Im, Re - Im) of A^T, else op(A) = A with planes (Re, Im, Re + Im) of A (embed3f,
// embed3_n).  K-split partial sums in ws.
void tc_cgemm3(const SplitBF16x3& A, const SplitBF16x3& B, bool conjA, int64_t M, int64_t N, int64_t K, float alpha,
               float beta, const float2* C, int64_t ldc, float2* D, int64_t ldd, int* status, cudaStream_t st,
               const char* tag, DevBuf<float>* ws);

// ---------------------------------------------------------------- FP64-accurate GEMM on tensor cores (ozaki.cu)
// Residues of op(X) (nrows x K complex; row r is column r of X when rows_are_columns, else
// row r of X; conjugated if conj) for the modular GEMM; doubled: the A operand's two real
// rows per complex row.  The scale makes every row's 2-norm 2^(E-1)..2^E, E = oz_precision_bits.
void oz_prepare(const double2* X, int64_t ldx, int64_t nrows, int64_t K, bool rows_are_columns, bool conj,
                bool doubled, int nmod, OzOperand& out, cudaStream_t st);
// C = alpha op(A) op(B) + beta C (complex, M = A.crows, N = B.crows; lower: only the complex
// lower triangle of a square C is written) from prepared operands; R: residue workspace.
void oz_gemm(const OzOperand& A, const OzOperand& B, double alpha, double beta, double2* C, int64_t ldc, bool lower,
             DevBuf<signed char>& R, int* status, cudaStream_t st, const char* tag);
int oz_precision_bits(int nmod);

// ---------------------------------------------------------------- small kernels (blas.cu)
// out = Dbd p: block-diagonal real D (packed row-major per-atom blocks) times complex p.
template <typename R>
void blockdiag_apply(const chebfi_ctx* ctx, const R* Dblk, const cplx<R>* p, int64_t ldp, cplx<R>* out,
                     int64_t ldo, int64_t nb, cudaStream_t st);
// out = Bbd p with complex per-atom blocks (column-major, block a at cblk_off[a])
void blockdiag_apply_c(const chebfi_ctx* ctx, const double2* Bblk, const int64_t* cblk_off, const double2* p,
                       int64_t ldp, double2* out, int64_t ldo, int64_t nb, cudaStream_t st);
// out = a (u - c x) - b y   (elementwise on an m x nb block; y may be null, out may alias y)
template <typename R>
void cheb_combine(int64_t m, int64_t nb, R a, const cplx<R>* u, int64_t ldu, R c, const cplx<R>* x,
                  int64_t ldx, R b, const cplx<R>* y, int64_t ldy, cplx<R>* out, int64_t ldo, cudaStream_t st);
// out = alpha x + beta y (y may be null)
template <typename R>
void axpby(int64_t m, int64_t nb, R alpha, const cplx<R>* x, int64_t ldx, R beta, const cplx<R>* y, int64_t ldy,
           cplx<R>* out, int64_t ldo, cudaStream_t st);
// column permutation of an m x nb block: dst[:, j] = src[:, order[j]] (inverse: dst[:, order[j]] = src[:, j])
void permute_cols(int64_t m, int64_t nb, const int32_t* order, const double2* src, double2* dst, bool inverse,
                  cudaStream_t st);
// copy with precision conversion
void convert(int64_t m, int64_t nb, const double2* x, int64_t ldx, float2* y, int64_t ldy, cudaStream_t st);
void convert(int64_t m, int64_t nb, const float2* x, int64_t ldx, double2* y, int64_t ldy, cudaStream_t st);
// sorted <-> caller order: dst[:, b] = src[perm[:], b]  or  dst[perm[:], b] = src[:, b]
void gather_rows(int64_t m, int64_t nb, const int32_t* perm, const double2* src, int64_t lds, double2* dst,
                 int64_t ldd, cudaStream_t st);
void scatter_rows(int64_t m, int64_t nb, const int32_t* perm, const double2* src, int64_t lds, double2* dst,
                  int64_t ldd, cudaStream_t st);
// the same with the conversion to / from FP32 fused in
void gather_rows(int64_t m, int64_t nb, const int32_t* perm, const double2* src, int64_t lds, float2* dst, int64_t ldd,
                 cudaStream_t st);
void scatter_rows(int64_t m, int64_t nb, const int32_t* perm, const float2* src, int64_t lds, double2* dst, int64_t ldd,
                  cudaStream_t st);
// out[b] = Re sum_j conj(x_jb) y_jb  (+= if accumulate)
void column_dots(int64_t m, int64_t nb, const double2* x, int64_t ldx, const double2* y, int64_t ldy,
                 double* out, bool accumulate, cudaStream_t st);
// out[b] = || h_b - w_b s_b ||_2
void residual_norms(int64_t m, int64_t nb, const double2* h, int64_t ldh, const double2* s, int64_t lds,
                    const double* w, double* out, cudaStream_t st);
// *status = CHEBFI_ERR_NONFINITE (unless already set) if the m x nb block holds Inf or NaN
void scan_nonfinite(int64_t m, int64_t nb, const double2* x, int64_t ldx, int* status, cudaStream_t st);
// out[b] = num[b] / den[b]
void divide(int64_t n, const double* num, const double* den, double* out, cudaStream_t st);
// identity matrix n x n
void set_identity(int64_t n, double2* A, int64_t lda, cudaStream_t st);
// A[i, j] = s_i A[i, j] s_j with s_i = 1/sqrt(Re d_i)  (d = diagonal of S taken before)
void diag_of(int64_t n, const double2* A, int64_t lda, double* d, cudaStream_t st);
void scale_sym(int64_t n, double2* A, int64_t lda, const double* d, cudaStream_t st);
// rows of X scaled by 1/sqrt(d): X[i, j] /= sqrt(d_i)
void scale_rows(int64_t n, int64_t m, double2* X, int64_t ldx, const double* d, cudaStream_t st);
// A <- (A + A^H) / 2
void hermitize(int64_t n, double2* A, int64_t lda, cudaStream_t st);
// upper triangle <- conjugate of the lower triangle, diagonal made real
void mirror_lower(int64_t n, double2* A, int64_t lda, cudaStream_t st);
// max over an array (device scalar out)
void reduce_max(int64_t n, const double* x, double* out, cudaStream_t st);
// y = D x for a real matrix D (n x n) applied to complex block x: used for Q p
// zero-fill
template <typename T> void zero(T* p, size_t count, cudaStream_t st) {
  CHEBFI_CUDA(cudaMemsetAsync(p, 0, count * sizeof(T), st));
}

// ---------------------------------------------------------------- dense FP64 (dense.cu)
// In-place Cholesky A = L L^H of a Hermitian positive definite n x n matrix (lower
// triangle referenced and overwritten, upper set to zero).  On a non-positive pivot the
// device flag *status gets CHEBFI_ERR_NOT_SPD (first failure wins) and the pivot is
// replaced by 1 so the computation stays finite.
void cholesky(int64_t n, double2* A, int64_t lda, int* status, cudaStream_t st, DevBuf<double2>* ws);
// B <- L^{-1} B for lower-triangular L (n x n) and B (n x m).
void trsm_lower(int64_t n, int64_t m, const double2* L, int64_t ldl, double2* B, int64_t ldb, cudaStream_t st,
                DevBuf<double2>* ws);
// Eigenvalues (ascending, w[n]) and eigenvectors (V, n x n) of a Hermitian n x n matrix A
// (destroyed).  Cyclic Jacobi with round-robin pairs; sets *status to
// CHEBFI_ERR_NO_CONVERGENCE on the sweep limit.  Synchronises the stream (sweep test).
void jacobi_eigh(int64_t n, double2* A, int64_t lda, double* w, double2* V, int64_t ldv, int* status,
                 cudaStream_t st, DevBuf<double2>* ws);
// The same in FP32, stopping at the FP32 rounding level (first stage of the refined solver;
// never reports a sweep limit).  ws holds its rotations, pair list and a copy of V.
void jacobi_eigh_f32(int64_t n, float2* A, int64_t lda, float* w, float2* V, int64_t ldv, int* status,
                     cudaStream_t st, DevBuf<double2>* ws);
// One Ogita-Aishima refinement step (n x n, lda = n): from G = X^H X and S = X^H A X, the
// approximate eigenvalues lam and M = I + E with X (I + E) the refined vectors; stats[0] =
// max |lam| bits, stats[1] = max |E| bits (doubles as ordered integers); pairs whose gap is
// too small for the formula are listed (i < j, at most cap) and only orthogonalised.
void oa_step(int64_t n, const double2* G, const double2* S, double* lam, double2* M, unsigned long long* stats,
             int* npairs, int2* pairs, int cap, cudaStream_t st);
// (w, X) sorted ascending in w (stable): wout, Xout (n x n, ld n)
void sort_eigpairs(int64_t n, const double* win, const double2* Xin, double* wout, double2* Xout, cudaStream_t st);
// index-list gathers: sub = A[idx, idx] (k x k); Y = X[:, idx]; X[:, idx] = Y; dst[idx] = src
void gather_sub(int k, const int* idx, const double2* A, int64_t lda, double2* sub, cudaStream_t st);
void gather_cols(int64_t m, int k, const int* idx, const double2* X, int64_t ldx, double2* Y, int64_t ldy,
                 cudaStream_t st);
void scatter_cols(int64_t m, int k, const int* idx, double2* X, int64_t ldx, const double2* Y, int64_t ldy,
                  cudaStream_t st);
void scatter_vals(int k, const int* idx, const double* src, double* dst, cudaStream_t st);

}  // namespace chebfi
