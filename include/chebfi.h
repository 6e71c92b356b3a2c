/*
 * chebfi.h -- C ABI of the GB300 (sm_103a) Chebyshev-filtered subspace iteration for the
 * plane-wave Kohn-Sham eigenproblem H psi = lambda S psi (Levitt & Torrent, arXiv:1406.4350,
 * Eq. (KS) of Section 2.1; Algorithm 2 of Section 4.2; Section 5.1 for S^{-1}).
 *
 * Operators (Section 2.1):
 *   H = K + V_loc + P D P^H       K diagonal |k+G|^2/2, V_loc multiplication in real space
 *   S = I + P Q P^H               Q = 0 (NULL) is the norm-conserving case S = I
 * with P the N_pw x N_proj projector matrix and D, Q block-diagonal (one symmetric
 * n_a x n_a block per atom).  The paper writes D_V for D and D_S for Q.
 *
 * Conventions shared by every entry point
 *  - Complex numbers are interleaved (re, im) pairs of double (complex128).
 *  - Wavefunction blocks are column-major: band n occupies Y + 2*n*ld doubles, its
 *    N_pw coefficients in the caller's plane-wave order (the order given to
 *    chebfi_set_sphere).  ld >= N_pw.
 *  - Pointers named Y, HY, X, out, evals, resid are DEVICE pointers owned by the caller;
 *    the library never frees them.  Setup data (lattice, Miller indices, V_loc, P, D, Q)
 *    is COPIED at the call; the caller may free its copy afterwards.
 *  - Work is enqueued on the given CUDA stream (cudaStream_t passed as void*, NULL =
 *    legacy default stream) and runs asynchronously, except where a function says it
 *    synchronises.  The context is not thread-safe: one host thread at a time.  Its
 *    workspaces are shared by all its calls, so calls on one context must be ordered on
 *    the device too (one stream, or synchronised between streams).
 *  - Return value 0 = success; negative = error, with a message from chebfi_last_error.
 *    Argument and state errors are detected before any work is enqueued.  Errors found
 *    on the device (a Gram matrix that is not positive definite, a Jacobi sweep limit)
 *    are reported by the functions documented to synchronise, and by chebfi_sync_status.
 */
#ifndef CHEBFI_H
#define CHEBFI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chebfi_ctx chebfi_ctx;

/* Arithmetic of the filter (Algorithm 2's inner loop).  Rayleigh-Ritz, Cholesky-QR,
 * Rayleigh quotients and residuals always run in FP64. */
typedef enum {
  CHEBFI_F64 = 0,   /* FP64 FFT and FP64 GEMMs */
  CHEBFI_F32 = 1,   /* FP32 FFT and FP32 GEMMs on the CUDA cores */
  CHEBFI_MIXED = 2  /* FP32 FFT; projector GEMMs on tcgen05 tensor cores with split
                       bf16 (hi + lo) operands and FP32 accumulation */
} chebfi_prec;

/* Upper end lambda_+ of the filtered interval (Section 5.3, "Choice of the polynomial"). */
typedef enum {
  CHEBFI_BOUND_PAPER = 0,    /* E_cut: the largest |k+G|^2/2 of the sphere (not a proven bound) */
  CHEBFI_BOUND_RIGOROUS = 1  /* max(0, max K + max V + l_max(L^H D L)) / (1 + min(0, l_min(L^H Q L)))
                                with P^H P = L L^H: a proven upper bound of the pencil */
} chebfi_bound_mode;

enum {
  CHEBFI_OK = 0,
  CHEBFI_ERR_ARG = -1,            /* a null pointer, a size out of range, a bad enum */
  CHEBFI_ERR_STATE = -2,          /* a setter called out of order, or a missing setter */
  CHEBFI_ERR_CUDA = -3,           /* a CUDA runtime call failed (message names it) */
  CHEBFI_ERR_NOT_SPD = -4,        /* Cholesky met a non-positive pivot (Gram or S) */
  CHEBFI_ERR_NO_CONVERGENCE = -5, /* the Jacobi eigensolver hit its sweep limit */
  CHEBFI_ERR_FILTER_OVERFLOW = -6,/* T_degree((lambda_1-c)/r) too large for the precision */
  CHEBFI_ERR_NOMEM = -7,          /* device allocation failed */
  CHEBFI_ERR_NONFINITE = -8       /* Inf or NaN in an input or in a block entering Rayleigh-Ritz */
};

typedef struct {
  int degree;          /* Chebyshev degree n (number of S^{-1}H applications), >= 1 */
  int sweeps;          /* repetitions of Algorithm 2, >= 1 */
  int prec;            /* chebfi_prec of the filter */
  int bound_mode;      /* chebfi_bound_mode, used when lambda_hi <= lambda_lo estimate */
  double lambda_hi;    /* > 0: fixed lambda_+; <= 0: take it from bound_mode */
  double tol;          /* locking tolerance on ||H y - lambda S y|| (used when lock != 0) */
  int lock;            /* 1: locking with per-band degrees after the first sweep (Section 5.4) */
} chebfi_params;

/* Create a context on CUDA device `device` (made current on the calling thread).
 * *out receives the handle; destroy it with chebfi_destroy. */
int chebfi_create(chebfi_ctx** out, int device);
int chebfi_destroy(chebfi_ctx* ctx);
/* Message of the last error on this context (empty string if none); valid until the next call. */
const char* chebfi_last_error(const chebfi_ctx* ctx);

/* Section 2.1: the cell.  lattice: host, 9 doubles, rows a1, a2, a3 in bohr.
 * grid: host, FFT sizes N1, N2, N3, each a product of 2, 3 and 5 and at most 256.
 * kpt: host, 3 doubles, Bloch vector k in Cartesian 1/bohr.  Must precede set_sphere. */
int chebfi_set_cell(chebfi_ctx* ctx, const double* lattice, const int* grid, const double* kpt);

/* Section 2.1: the plane-wave sphere.  miller: host, npw x 3 int32 (row-major), the integer
 * coordinates m of G = m1 b1 + m2 b2 + m3 b3 with |m_i| < N_i/2; the row order is the
 * order of the wavefunction coefficients at this ABI.  Duplicates are an error. */
int chebfi_set_sphere(chebfi_ctx* ctx, int64_t npw, const int32_t* miller);

/* Section 2.1: the local potential V_loc(r) on the grid, N1*N2*N3 doubles, index
 * (i1*N2 + i2)*N3 + i3 (third index fastest).  on_device: 1 if vloc is a device pointer. */
int chebfi_set_vloc(chebfi_ctx* ctx, const double* vloc, int on_device);

/* Section 2.1: projectors and their coefficients.
 *  P: complex128 column-major npw x nproj with leading dimension ldP >= npw, host or
 *     device (P_on_device); rows in the sphere order of set_sphere.
 *  proj_offsets: host, natoms+1 int32, atom a owns projector columns
 *     [proj_offsets[a], proj_offsets[a+1]); proj_offsets[0] = 0, proj_offsets[natoms] = nproj,
 *     block sizes 1..64.
 *  D: host, the per-atom symmetric blocks of D_V concatenated, each n_a x n_a row-major.
 *  Q: host, same layout for D_S; NULL for S = I (norm-conserving).
 * Precomputes G = P^H P and the Woodbury core M = Q (I + G Q)^{-1} (Section 5.1) on the
 * device.  Synchronises; returns CHEBFI_ERR_NOT_SPD if S is not positive definite. */
int chebfi_set_projectors(chebfi_ctx* ctx, int64_t nproj, const void* P, int64_t ldP,
                          int P_on_device, int natoms, const int32_t* proj_offsets,
                          const double* D, const double* Q);

/* Section 5.3: lambda_+ for the filter.  Synchronises. */
int chebfi_upper_bound(chebfi_ctx* ctx, int mode, double* lambda_hi);
/* A proven lower bound of the smallest eigenvalue of S: 1 + min(0, l_min(L^H Q L)) with
 * P^H P = L L^H (1 for S = I).  With it a Ritz pair (theta, y), y S-normalised, certifies
 * an eigenvalue of the pencil within ||H y - theta S y||_2 / sqrt(smin) of theta (the
 * residual in the S^{-1} norm bounds the distance).  Synchronises. */
int chebfi_overlap_lower_bound(chebfi_ctx* ctx, double* smin);

/* Algorithm 1: HY = H Y for nb bands.  prec selects FP64 or FP32 arithmetic (MIXED acts
 * as F32 here).  Y and HY must not overlap. */
int chebfi_apply_H(chebfi_ctx* ctx, const void* Y, void* HY, int64_t nb, int64_t ld,
                   int prec, void* stream);
/* Replace the nonlocal coefficients D_V (Section 2.1) without rebuilding the projector
 * data: D in the packed per-atom block layout of chebfi_set_projectors, host or device.
 * G = P^H P and the Woodbury core do not depend on D.  Synchronises. */
int chebfi_set_D(chebfi_ctx* ctx, const double* D, int on_device);

/* Reverse-mode derivative of Algorithm 1's HY = H Y (FP64) for a real loss L, given
 * G = the gradient of L at HY in the convention dL = Re sum conj(G) dHY (PyTorch's):
 *   gY = H G                                               (H is Hermitian)
 *   gV(r) = (1/(N1 N2 N3)) Re sum_n conj(g_n(r)) psi_n(r)  (g_n, psi_n: real-space values of
 *           the columns of G and Y; gV laid out like V_loc in chebfi_set_vloc)
 *   gD    = Re sum_n conj((P^H G)_in) (P^H Y)_jn on the per-atom blocks (packed like D).
 * Any of gY (device, like Y), gV (device, N1*N2*N3 doubles), gD (device, packed) may be
 * NULL to skip it.  With Y = G = an S-normalised eigenvector, gV is the Hellmann-Feynman
 * derivative d lambda / d V_loc(r). */
int chebfi_apply_H_backward(chebfi_ctx* ctx, const void* Y, const void* G, void* gY, double* gV, double* gD,
                            int64_t nb, int64_t ld, void* stream);

/* Backward of chebfi_cheb_filter (Algorithm 2's inner loop) for a real loss L of its output
 * Y_n, given gYn = dL/dY_n in PyTorch's convention (dL = Re sum conj(gYn) dY_n).  The adjoint
 * recurrence L_k = a_k (H S^{-1} L_{k+1} - c L_{k+1}) - L_{k+2} (a_0 = 1/r, a_k = 2/r,
 * L_n = gYn, L_{n+1} = 0) gives gY0 = L_0; V_loc and D enter only through H, so
 *   gV(r) = sum_k a_k (1/N^3) Re sum_b conj(u_kb(r)) y_kb(r),   u_k = S^{-1} L_{k+1},
 *   gD_ij = sum_k a_k Re sum_b conj((P^H u_k)_ib) (P^H Y_k)_jb   (atom blocks),
 * for the same c, r, lambda_lo, lambda_hi and degree as the forward call.  The iterates Y_k
 * are recomputed from checkpoints (Y_{j-1}, Y_j) kept every checkpoint_every steps
 * (0: ceil(sqrt(degree))), so device memory is O(degree / s + s) blocks of npw x nb.
 * Y0, gYn: device complex128 blocks like chebfi_apply_H's Y (same nb, ld).  gY0 (like Y0),
 * gV (N1*N2*N3 doubles, z fastest) and gD (packed like D) are device outputs, each NULL to
 * skip; gV and gD are overwritten.  prec: CHEBFI_F64, or CHEBFI_F32 (iterates and operators
 * in FP32, gradient sums in FP64); CHEBFI_MIXED is rejected with CHEBFI_ERR_ARG.  The V_loc
 * and D of the context are the point of differentiation. */
int chebfi_cheb_filter_backward(chebfi_ctx* ctx, const void* Y0, const void* gYn, void* gY0, double* gV,
                                double* gD, int64_t nb, int64_t ld, int degree, double lambda_lo,
                                double lambda_hi, int prec, int checkpoint_every, void* stream);

/* Algorithm 1: SY = S Y = Y + P Q P^H Y (FP64). */
int chebfi_apply_S(chebfi_ctx* ctx, const void* Y, void* SY, int64_t nb, int64_t ld, void* stream);
/* Section 5.1 (Woodbury): out = S^{-1} X = X - P M P^H X (FP64). */
int chebfi_apply_Sinv(chebfi_ctx* ctx, const void* X, void* out, int64_t nb, int64_t ld, void* stream);

/* Section 5.1's own solve of the Woodbury reduced system (FP64): out = S^{-1} X = X - P q with
 * A q = P^H X, A = D_S^{-1} + P^H P, found by iterative refinement q <- q + B^{-1}(P^H X - A q)
 * from q = 0, B = the atom-diagonal blocks of A.  It stops when every column has
 * ||P^H x - A q|| <= tol ||P^H x||, or after maxit updates; *iterations (nullable) receives the
 * number of updates.  Needs every D_S block invertible (CHEBFI_ERR_ARG otherwise; the direct
 * chebfi_apply_Sinv has no such limit).  Returns CHEBFI_ERR_NO_CONVERGENCE, with out written,
 * when the tolerance is not met.  A and B^{-1} are formed on the first call.  S = I: out = X.
 * Synchronises. */
int chebfi_apply_Sinv_refined(chebfi_ctx* ctx, const void* X, void* out, int64_t nb, int64_t ld, double tol,
                              int maxit, int* iterations, void* stream);

/* Algorithm 2's inner loop, in place on Y: psi^1 = (S^{-1}H psi^0 - c psi^0)/r,
 * psi^i = 2/r (S^{-1}H psi^{i-1} - c psi^{i-1}) - psi^{i-2}, i = 2..degree, with
 * c = (lambda_hi + lambda_lo)/2, r = (lambda_hi - lambda_lo)/2 and the projection-reuse
 * identity of Section 5.1.  Requires lambda_hi > lambda_lo. */
int chebfi_cheb_filter(chebfi_ctx* ctx, void* Y, int64_t nb, int64_t ld, int degree,
                       double lambda_lo, double lambda_hi, int prec, void* stream);

/* chebfi_cheb_filter with p_0 = P^H Y given: proj (device, complex128, nproj x nb
 * column-major, leading dimension ldp >= nproj) as chebfi_rayleigh_ritz_proj returns it for
 * this Y.  Algorithm 2's filter starts from the block that Rayleigh-Ritz has just rotated,
 * whose projections that step forms anyway, so the filter's first P^H Y product is saved.
 * The caller vouches that proj belongs to Y (not checked: a stale proj gives a wrong filter).
 * proj NULL, or no projectors: exactly chebfi_cheb_filter. */
int chebfi_cheb_filter_proj(chebfi_ctx* ctx, void* Y, const void* proj, int64_t ldp, int64_t nb, int64_t ld,
                            int degree, double lambda_lo, double lambda_hi, int prec, void* stream);

/* Locking (Section 5.4), in place on Y: band j filtered to its own degree degrees[j] (host
 * array of nb ints in 0..1000; 0 leaves the band as it is) on [lambda_lo, lambda_hi], i.e.
 * chebfi_cheb_filter applied band by band.  Bands are reordered internally by decreasing
 * degree so each Chebyshev step runs on the still-active prefix of the block. */
int chebfi_cheb_filter_adaptive(chebfi_ctx* ctx, void* Y, int64_t nb, int64_t ld, const int32_t* degrees,
                                double lambda_lo, double lambda_hi, int prec, void* stream);

/* Section 5.4's a-priori degree (host arrays, no context): the residual of band i after one
 * filter of degree n and Rayleigh-Ritz is estimated as resid[i] / |T_n((ritz[i] - c)/r)|,
 * c, r from [lambda_lo, lambda_hi]; degrees[i] = the smallest n in 1..max_degree with the
 * estimate <= tol (T_n by the three-term recurrence), max_degree if none, 0 if
 * resid[i] <= tol.  The paper prints lambda_1 in T_n's argument; each band's own Ritz
 * value is used so that each band gets its own degree. */
int chebfi_adaptive_degrees(const double* ritz, const double* resid, int64_t nb, double lambda_lo,
                            double lambda_hi, double tol, int max_degree, int32_t* degrees);

/* Sweeps performed by the last chebfi_solve on ctx and the band-H-applications of its
 * filters (sum over sweeps of the bands' degrees). */
int chebfi_solve_stats(const chebfi_ctx* ctx, int* sweeps_done, int64_t* band_applies);

/* chebfi_cheb_filter on a block in HOST memory (complex128, npw x nb column-major, leading
 * dimension ld, caller's row order; page-locked memory for full copy bandwidth), in place.
 * Bands are filtered independently, so the block goes through the GPU in nchunks equal band
 * chunks (0: from 2048 bands up five chunks of nb/8, nb/4, nb/4, nb/4 and the rest, so that
 * the two copies that overlap no filter are short; 2 from 1024; else 1): the copy in of chunk
 * c, the filter of chunk c-1 and the copy out of chunk c-2 overlap (two device staging
 * buffers, two copy streams).
 * Stream-ordered on `stream`: the host block is final once `stream` completes.  The host
 * block must not be touched until then. */
int chebfi_cheb_filter_host(chebfi_ctx* ctx, void* Y, int64_t nb, int64_t ld, int degree, double lambda_lo,
                            double lambda_hi, int prec, int nchunks, void* stream);

/* chebfi_cheb_filter_host with p_0 = P^H Y given in HOST memory (complex128, nproj x nb
 * column-major, leading dimension ldp >= nproj; page-locked for full copy bandwidth), as
 * chebfi_cheb_filter_proj takes it on the device: each band chunk's projections are copied in
 * with the chunk.  proj NULL, or no projectors: exactly chebfi_cheb_filter_host. */
int chebfi_cheb_filter_host_proj(chebfi_ctx* ctx, void* Y, const void* proj, int64_t ldp, int64_t nb, int64_t ld,
                                 int degree, double lambda_lo, double lambda_hi, int prec, int nchunks,
                                 void* stream);

/* S-orthonormalisation by Cholesky-QR (FP64): G_Y = Y^H S Y = L L^H, Y <- Y L^{-H}.
 * Synchronises; CHEBFI_ERR_NOT_SPD if G_Y is not positive definite. */
int chebfi_orthonormalise(chebfi_ctx* ctx, void* Y, int64_t nb, int64_t ld, void* stream);

/* Algorithm 2's last three steps (FP64): columns scaled to unit S-norm, H_Psi = Y^H H Y,
 * S_Psi = Y^H S Y, H_Psi X = S_Psi X Lambda (Cholesky reduction + Jacobi), Y <- Y X.
 * evals: device, nb doubles, ascending.  resid: device, nb doubles ||H y - lambda S y||_2,
 * or NULL.  Synchronises.  A block holding Inf or NaN is reported as CHEBFI_ERR_NONFINITE. */
int chebfi_rayleigh_ritz(chebfi_ctx* ctx, void* Y, double* evals, double* resid, int64_t nb,
                         int64_t ld, void* stream);

/* chebfi_rayleigh_ritz that also writes proj = P^H Y of the rotated block (device,
 * complex128, nproj x nb column-major, leading dimension ldp >= nproj; FP64, the product
 * p R of the step's own projections and rotation), for chebfi_cheb_filter_proj.  proj NULL
 * or no projectors: proj is not written.  Synchronises. */
int chebfi_rayleigh_ritz_proj(chebfi_ctx* ctx, void* Y, double* evals, double* resid, void* proj, int64_t ldp,
                              int64_t nb, int64_t ld, void* stream);

/* Generalized Rayleigh quotients y^H H y / y^H S y of every band (FP64), device nb doubles
 * (Algorithm 2's first step). */
int chebfi_rayleigh_quotients(chebfi_ctx* ctx, const void* Y, double* rq, int64_t nb, int64_t ld,
                              void* stream);

/* Algorithm 2 repeated params->sweeps times on Y (in place): lambda_- = max Rayleigh
 * quotient, lambda_+ from params, filter, Rayleigh-Ritz.  evals/resid as in
 * chebfi_rayleigh_ritz.  With params->lock (Section 5.4), the first sweep uses
 * params->degree for every band and each later sweep gives band i the degree
 * chebfi_adaptive_degrees predicts for params->tol from its Ritz value and residual (at
 * most params->degree; 0 = locked, not filtered, still in the Rayleigh-Ritz space); the
 * solve stops early when every band is locked.  Synchronises.  Every sweep checks the block
 * entering Rayleigh-Ritz and the Ritz values for Inf / NaN (CHEBFI_ERR_NONFINITE). */
int chebfi_solve(chebfi_ctx* ctx, void* Y, double* evals, double* resid, int64_t nb, int64_t ld,
                 const chebfi_params* params, void* stream);

/* Allocation-free variant of chebfi_apply_H (FP64): HY = H Y with the same arguments and
 * result, for callers that cannot allocate device memory where they make the call -- host
 * callbacks or latency-critical sections that must not take the CUDA allocator's lock,
 * frameworks that own every byte of device memory through their own pool, and processes
 * that have already reserved all of it.  The paper has no counterpart; this is a
 * deployment convenience of this library.
 *  - It calls no cudaMalloc / cudaFree and no allocating routine.  Its scratch is one
 *    file-scope device array of 32 MiB inside the library; every GPU that loads the library
 *    holds that array until the process exits.  (The context's own buffers were allocated
 *    earlier, by the setters.)
 *  - Bands are processed in chunks that fit the array.  A problem whose single band needs
 *    more than 32 MiB of scratch (FFT column buffer N3 x columns, plus 2 npw + 2 nproj, in
 *    complex doubles) is rejected with CHEBFI_ERR_ARG and a message naming the sizes.
 *  - The first call on each device does one-time set-up with that device current: it looks
 *    up the array's device address (cudaGetSymbolAddress) and uploads the FFT twiddle tables
 *    to constant memory (a synchronous copy).  Make that first call before any stream
 *    capture.
 *  - All calls share the one array, which keeps the previous call's contents (nothing in it
 *    needs to start at zero); calls that overlap on the GPU (other streams, other contexts
 *    on the same device, other host threads) race on it. */
int chebfi_apply_H_noalloc(chebfi_ctx* ctx, const void* Y, void* HY, int64_t nb, int64_t ld, void* stream);

/* Engines of the FP64 complex GEMMs behind every FP64 step (Rayleigh-Ritz and Cholesky-QR
 * of Algorithm 2, the FP64 filter's projector products P^H psi and P W of Section 5.1, the
 * setup products G = P^H P and the Woodbury core).  GB300 issues FP64 FMAs at about 2 per
 * clock per SM, so large products go to the bf16 tensor cores through an FP64-accurate
 * modular emulation (the integer-modular "Ozaki scheme II"): every row of op(A) and column of
 * op(B) is scaled by a power of two to a 2-norm in [2^(E-1), 2^E) and rounded to integers,
 * one tensor-core GEMM per modulus computes the product of their residues exactly, and the
 * Chinese remainder theorem recovers the integer product.  The result's error is about
 * 2^-E ||row of op(A)|| ||column of op(B)|| per entry, E = 53 with the default 14 moduli:
 * no larger than an FP64 dot product's.  The paper (FP64 BLAS on CPUs) has no counterpart. */
enum {
  CHEBFI_GEMM_AUTO = 0,        /* tensor cores when K >= 64 and 8 M N K >= 1e9, else CUDA cores */
  CHEBFI_GEMM_CUDA_CORES = 1,  /* FP64 FMA on the CUDA cores only */
  CHEBFI_GEMM_TENSOR = 2       /* the modular emulation for every product */
};
/* Select the engine (a CHEBFI_GEMM_* value) and the modulus count of the emulation (8..15;
 * 0 keeps the current one, initially 14; fewer moduli run faster with a smaller E: 8 -> 30,
 * 10 -> 38, 12 -> 45, 14 -> 53, 15 -> 57).  *precision_bits (nullable) receives E.  The
 * emulation keeps residues of P (about 2 x nmod x 4 N_pw N_proj bytes) once used. */
int chebfi_set_fp64_gemm(chebfi_ctx* ctx, int engine, int nmod, int* precision_bits);

/* Complex FP64 GEMM through the context's engine selection: C = alpha op(A) op(B) + beta C,
 * C m x n, inner dimension k; op(A) = A (m x k, lda >= m) or A^H (A k x m, lda >= k) when
 * conjA; op(B) = B (k x n, ldb >= k) or B^H (B n x k, ldb >= n) when conjB.  A, B, C: device,
 * complex128 column-major; C must not overlap A or B.  Needs no cell or projectors. */
int chebfi_gemm_fp64(chebfi_ctx* ctx, int conjA, int conjB, int64_t m, int64_t n, int64_t k, double alpha,
                     const void* A, int64_t lda, const void* B, int64_t ldb, double beta, void* C, int64_t ldc,
                     void* stream);

/* Arithmetic of the FFT passes of the FP64 path (the FP64 form's filter, apply_H and the
 * H application of Rayleigh-Ritz in every form) on the compile-time grids (cubic 24, 32, 48,
 * 64, 72, 96):
 *  CHEBFI_FFT64_DOUBLE_FLOAT (initial): double-float arithmetic on the FP32 units -- each
 *    value the unevaluated sum of two floats (48-bit significand, float's exponent range),
 *    the error-free TwoSum / Fast2Sum / FMA-TwoProd transformations of Knuth and Dekker; a
 *    transform keeps about 2^-44 of its line's norm; GB300's FP64 units run at ~1/64 of the
 *    FP32 rate, so this is several times faster;
 *  CHEBFI_FFT64_NATIVE: FP64 arithmetic on the FP64 units.
 * Blocks, V_loc and the results stay FP64 in memory either way.  Other grids use FP64. */
enum { CHEBFI_FFT64_NATIVE = 0, CHEBFI_FFT64_DOUBLE_FLOAT = 1 };
int chebfi_set_fft64(chebfi_ctx* ctx, int mode);

/* Complex GEMM of the mixed form's projector products (Section 5.1: P^H psi and P W) on the
 * tensor cores: C = alpha op(A) B + beta C, C m x n, inner dimension k >= 1; op(A) = A (m x k,
 * lda >= m) or A^H (A k x m, lda >= k) when conjA; B k x n (ldb >= k).  A, B, C: device,
 * complex64 (interleaved FP32) column-major; C must not overlap A or B.  The operands are
 * split into bf16 pairs (x = hi + lo, about 16 significant bits) and the product is formed by
 * three real products of the planes (Re, Im, Re -+ Im) x (Re, Im, Re + Im) -- Gauss's form,
 * three quarters of the real products of a real embedding -- each with the three bf16 terms
 * hi hi + hi lo + lo hi, FP32 accumulation in the tensor memory in chunks of 512 along k.
 * Needs no cell or projectors. */
int chebfi_gemm_mixed(chebfi_ctx* ctx, int conjA, int64_t m, int64_t n, int64_t k, float alpha, const void* A,
                      int64_t lda, const void* B, int64_t ldb, float beta, void* C, int64_t ldc, void* stream);

/* Dense Hermitian eigensolver of the Rayleigh-Ritz step (Algorithm 2; ELPA in the paper):
 *  CHEBFI_EIG_JACOBI: FP64 cyclic Jacobi (rounds of n/2 disjoint rotations).
 *  CHEBFI_EIG_REFINED: FP32 cyclic Jacobi for approximate eigenvectors, then the iterative
 *    refinement of Ogita & Aishima (2018) in FP64 GEMMs -- from G = X^H X and S = X^H A X,
 *    lambda_i = S_ii / G_ii, E_ij = (S_ij - lambda_j G_ij) / (lambda_j - lambda_i),
 *    E_ii = (1 - G_ii) / 2, X <- X (I + E) -- until max |E| <= 1e-10; pairs too close
 *    for the formula are only orthogonalised and their cluster's block of X^H A X is then
 *    diagonalised by FP64 Jacobi.  A nearly diagonal A (a converging solve's later sweeps)
 *    skips the FP32 Jacobi: the refinement starts from the identity when its first step (G =
 *    I, S = A, no GEMM) has max |E| <= 0.01.  Falls back to CHEBFI_EIG_JACOBI if it does not
 *    converge.
 *  CHEBFI_EIG_AUTO (initial): REFINED from 512 bands up, JACOBI below. */
enum { CHEBFI_EIG_AUTO = 0, CHEBFI_EIG_JACOBI = 1, CHEBFI_EIG_REFINED = 2 };
int chebfi_set_eigensolver(chebfi_ctx* ctx, int mode);
/* Refinement steps taken by the last dense eigensolve on ctx (0: FP64 Jacobi ran). */
int chebfi_eigensolver_steps(const chebfi_ctx* ctx);

/* Self-test of the bounded device waits (a library diagnostic; the paper has no counterpart).
 * Every spin of the library's kernels -- the grid barrier of the cooperative Jacobi sweep,
 * the mbarrier waits of the tensor-core pipelines -- gives up after a time limit, records
 * CHEBFI_ERR_CUDA on the device and lets the kernel end.  which = 0 runs the grid barrier
 * with one block that never arrives, which = 1 an mbarrier wait for an arrival nobody makes,
 * each with a limit of limit_ms (0 < limit_ms <= 2000).  *recorded (nullable) receives the
 * code the waiting threads recorded (CHEBFI_ERR_CUDA when the wait ran out), *elapsed_ms
 * (nullable) the kernel's duration.  Uses its own status word, not the context's.
 * Synchronises. */
int chebfi_selftest_bounded_wait(chebfi_ctx* ctx, int which, double limit_ms, int* recorded, double* elapsed_ms);

/* FMA rate of the device's CUDA cores (a library diagnostic): eight independent FMA chains
 * per thread on every SM, timed with CUDA events after one warm-up run.  prec: CHEBFI_F64 or
 * CHEBFI_F32.  *tflops receives 2 x FMAs / time in TFLOP/s, *ms the timed run.  About 0.2 s
 * of device time.  Synchronises. */
int chebfi_probe_fma_rate(chebfi_ctx* ctx, int prec, double* tflops, double* ms);

/* Synchronise the context's work and return the first device-detected error, if any. */
int chebfi_sync_status(chebfi_ctx* ctx);

/* Number of kernels the library has launched on this context (monotonic counter). */
int64_t chebfi_kernel_launches(const chebfi_ctx* ctx);

/* Per-kernel timing for measurement: while enabled, every kernel launch of this context is
 * bracketed by CUDA events recorded on its own stream, and the elapsed times are summed per
 * kernel name.  enable = 1 clears previous totals; 0 stops recording (totals kept). */
int chebfi_profile_enable(chebfi_ctx* ctx, int enable);
/* Number of distinct kernel names with totals (synchronises); negative on error. */
int chebfi_profile_count(chebfi_ctx* ctx);
/* Entry i (0 <= i < count): kernel name (NUL-terminated, at most name_len bytes including
 * the NUL), total milliseconds, number of launches, and the summed algorithmic work of
 * those launches (flops for GEMMs, 8 M N K complex or 2 M N K real; bytes read + written
 * for the FFT passes).  Any output pointer may be NULL. */
int chebfi_profile_entry(chebfi_ctx* ctx, int i, char* name, int name_len, double* ms, int64_t* launches,
                         double* work);

/* ---------------------------------------------------------------- batched k-points
 * Section 2.1: sampling the Brillouin zone gives one eigenproblem per Bloch vector k; they
 * share the cell, grid, V_loc and atoms (D, Q) and differ in the G-sphere, the kinetic
 * diagonal and P_k.  A batch runs Algorithm 2's filter for all of them at once: every stage
 * is one grouped launch over all k-points (the projector GEMMs are persistent kernels that
 * take (k, tile) items from a device work queue), and the whole degree-n filter is captured
 * in a CUDA graph on first use and replayed afterwards.  Tile shapes of the grouped GEMMs are
 * chosen by timing every candidate on the batch (chebfi_batch_autotune; run implicitly by
 * the first filter call of each form). */
typedef struct chebfi_batch chebfi_batch;

/* kctx: nk fully set-up contexts (set_cell/sphere/vloc/projectors) on one device, with the
 * same cubic grid of a compiled size (24, 32, 48, 64, 72 or 96), the same V_loc, atoms, D and
 * Q (checked; CHEBFI_ERR_ARG otherwise), any k and sphere.  nb bands per k-point,
 * nk * nb <= 65535.  The batch keeps the pointers: the contexts must outlive it and stay
 * unchanged.  Synchronises.  *out is NULL on error. */
int chebfi_batch_create(chebfi_batch** out, chebfi_ctx* const* kctx, int nk, int64_t nb);
int chebfi_batch_destroy(chebfi_batch* batch);
const char* chebfi_batch_last_error(const chebfi_batch* batch);
/* Kernels launched by the batch so far (each graph replay counts its kernel nodes). */
int64_t chebfi_batch_kernel_launches(const chebfi_batch* batch);
/* Time the candidate tile shapes (16TM x 16TN with (TM, TN) = (4,4), (2,4), (4,2), (8,4)) of
 * the three grouped GEMM classes (0: P_k^H Z_k, 1: G_k / M_k products, 2: P_k W_k) in form
 * prec (CHEBFI_F64 or CHEBFI_F32), and for class 0 also the split-K factors 1, 2, 4, 8 of its
 * long inner dimension (chunks summed by a deterministic second pass); keep the fastest.
 * shapes (4 ints, nullable) receives the chosen shape index per class and the split factor;
 * ms (16 doubles, nullable) the times per (class, shape) with split 1, then the best time per
 * split factor.  Overwrites the batch's workspaces; a no-op after the first call for a form.
 * Synchronises. */
int chebfi_batch_autotune(chebfi_batch* batch, int prec, int* shapes, double* ms);
/* Override the autotuner: tile shape index per GEMM class (3 ints, 0..3) and the split-K
 * factor of P_k^H Z_k (1, 2, 4 or 8) for form prec; graphs captured with other tiles are
 * dropped and recaptured on the next call.  Synchronises. */
int chebfi_batch_set_tiles(chebfi_batch* batch, int prec, const int* shapes, int split);
/* In place on Y[k] (device, complex128, npw_k x nb column-major, leading dimension ld[k],
 * caller's plane-wave order) for k = 0..nk-1: Algorithm 2's filter of the given degree on
 * [lambda_lo[k], lambda_hi[k]] (host arrays of nk doubles), exactly as chebfi_cheb_filter
 * computes it per k-point, in the FP64, FP32 or mixed form (CHEBFI_MIXED: FP32 iterates and
 * FFT, the projector products as grouped tcgen05 GEMMs over all k-points on bf16 (hi, lo)
 * pairs; needs projectors).  Stream-ordered on `stream`; the first call of a (form, degree)
 * pair tunes (FP64/FP32) or builds the tensor-core operands (mixed) and captures, later calls
 * replay the graph.  The
 * batch's workspaces and per-call descriptor table are shared by its calls: calls on one
 * batch must be ordered (one stream, or synchronised between streams). */
int chebfi_batch_cheb_filter(chebfi_batch* batch, void* const* Y, const int64_t* ld, int degree,
                             const double* lambda_lo, const double* lambda_hi, int prec, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CHEBFI_H */
