// Dense FP64 linear algebra on the device for the Rayleigh-Ritz step of Algorithm 2 and
// the Woodbury core of Section 5.1: blocked Cholesky, triangular solve, and a cyclic
// Jacobi eigensolver for complex Hermitian matrices.
//
// Jacobi: each rotation removes one off-diagonal entry a_pq = |a_pq| e^{i phi} of the
// 2 x 2 block [[a_pp, a_pq], [conj(a_pq), a_qq]]: U = diag(1, e^{-i phi}) [[c, s], [-s, c]]
// with zeta = (a_qq - a_pp) / (2 |a_pq|), t = sign(zeta) / (|zeta| + sqrt(1 + zeta^2)),
// c = 1/sqrt(1 + t^2), s = t c (the symmetric Schur step of Golub & Van Loan, Section 8.5),
// applied as A <- U^H A U, V <- V U.  One step applies n/2 disjoint rotations chosen by the
// circle method (player 0 fixed, the others rotate), one sweep is n-1 steps.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.cuh"
#include "kernels.cuh"
#include "grid_barrier.cuh"

namespace chebfi {
namespace {

constexpr int NB = 32;

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

__device__ __forceinline__ void flag_error(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Unblocked Cholesky of one nb x nb diagonal block (nb <= NB) in shared memory.
__global__ void k_chol_diag(double2* A, int64_t lda, int nb, int* status) {
  __shared__ double2 a[NB][NB + 1];
  const int tid = threadIdx.x;
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e % nb, j = e / nb;
    a[i][j] = A[i + j * lda];
  }
  __syncthreads();
  for (int j = 0; j < nb; ++j) {
    __shared__ double piv;
    if (tid == 0) {
      double d = a[j][j].x;
      if (!(d > 0.0)) {  // also catches NaN
        flag_error(status, CHEBFI_ERR_NOT_SPD);
        d = 1.0;
      }
      piv = sqrt(d);
      a[j][j] = make_double2(piv, 0.0);
    }
    __syncthreads();
    for (int i = j + 1 + tid; i < nb; i += blockDim.x) {
      a[i][j].x /= piv;
      a[i][j].y /= piv;
    }
    __syncthreads();
    // trailing update of the lower triangle: a[i][k] -= L[i][j] conj(L[k][j]) for i >= k > j
    const int m = nb - j - 1;
    for (int e = tid; e < m * m; e += blockDim.x) {
      const int i = j + 1 + e % m, k = j + 1 + e / m;
      if (i >= k) {
        const double2 li = a[i][j], lk = a[k][j];
        a[i][k].x -= li.x * lk.x + li.y * lk.y;
        a[i][k].y -= li.y * lk.x - li.x * lk.y;
      }
    }
    __syncthreads();
  }
  for (int e = tid; e < nb * nb; e += blockDim.x) {
    const int i = e % nb, j = e / nb;
    A[i + j * lda] = i >= j ? a[i][j] : make_double2(0.0, 0.0);
  }
}

// Panel: rows of B (m x nb) <- B L^{-H}, L = nb x nb lower (diagonal real).
__global__ void k_trsm_right_lh(const double2* __restrict__ L, int64_t ldl, double2* B, int64_t ldb, int64_t m, int nb) {
  __shared__ double2 l[NB][NB + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e % nb, j = e / nb;
    l[i][j] = L[i + j * ldl];
  }
  __syncthreads();
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= m) return;
  double2 x[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < nb) x[j] = B[r + j * ldb];
#pragma unroll
  for (int j = 0; j < NB; ++j) {
    if (j < nb) {
      double2 s = x[j];
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        if (k < j) {  // s -= x_k conj(L[j][k])
          const double2 lj = l[j][k];
          s.x -= x[k].x * lj.x + x[k].y * lj.y;
          s.y -= x[k].y * lj.x - x[k].x * lj.y;
        }
      }
      const double d = l[j][j].x;
      x[j] = make_double2(s.x / d, s.y / d);
    }
  }
#pragma unroll
  for (int j = 0; j < NB; ++j)
    if (j < nb) B[r + j * ldb] = x[j];
}

// Columns of B (nb x m) <- L^{-1} B, L = nb x nb lower.
__global__ void k_trsm_left_l(const double2* __restrict__ L, int64_t ldl, double2* B, int64_t ldb, int64_t m, int nb) {
  __shared__ double2 l[NB][NB + 1];
  for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
    const int i = e % nb, j = e / nb;
    l[i][j] = L[i + j * ldl];
  }
  __syncthreads();
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m) return;
  double2 x[NB];
  double2* b = B + c * ldb;
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < nb) x[i] = b[i];
#pragma unroll
  for (int i = 0; i < NB; ++i) {
    if (i < nb) {
      double2 s = x[i];
#pragma unroll
      for (int k = 0; k < NB; ++k) {
        if (k < i) {  // s -= L[i][k] x_k
          const double2 li = l[i][k];
          s.x -= li.x * x[k].x - li.y * x[k].y;
          s.y -= li.x * x[k].y + li.y * x[k].x;
        }
      }
      const double d = l[i][i].x;
      x[i] = make_double2(s.x / d, s.y / d);
    }
  }
#pragma unroll
  for (int i = 0; i < NB; ++i)
    if (i < nb) b[i] = x[i];
}

__global__ void k_zero_upper(int64_t n, double2* A, int64_t lda) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx % n, j = idx / n;
  if (i < j) A[i + j * lda] = make_double2(0.0, 0.0);
}

// ------------------------------------------------------------------ Jacobi
// Templated on the real type: FP64 for the eigensolver itself, FP32 for the first stage of
// the refined eigensolver (whose vectors are then refined to FP64 accuracy).
template <typename R> struct JacEps;
template <> struct JacEps<double> {
  static constexpr double v = 1.1102230246251565e-16, tiny = 1e-300;
};
template <> struct JacEps<float> {
  static constexpr float v = 5.9604645e-8f, tiny = 1e-37f;
};

__device__ __forceinline__ int64_t rr_player(int64_t pos, int64_t round, int64_t n) {
  return pos == 0 ? 0 : 1 + (pos - 1 + round) % (n - 1);
}

template <typename R> struct RotT {
  R c, s;
  cplx<R> ph;  // e^{i phi}
};

__device__ __forceinline__ double hyp(double a, double b) { return hypot(a, b); }
__device__ __forceinline__ float hyp(float a, float b) { return hypotf(a, b); }

// rotation parameters of pair t of the given round (p < q; q = -1 for the padding player)
template <typename R>
__device__ __forceinline__ void jac_params_item(int64_t t, int64_t n0, int64_t n, int64_t round,
                                                const cplx<R>* __restrict__ A, int64_t lda, RotT<R>* __restrict__ rot,
                                                int* __restrict__ pairs) {
  int64_t p = rr_player(t, round, n), q = rr_player(n - 1 - t, round, n);
  if (p > q) {
    const int64_t tmp = p;
    p = q;
    q = tmp;
  }
  RotT<R> r;
  r.c = (R)1;
  r.s = (R)0;
  r.ph = cmake<cplx<R>>(1.0, 0.0);
  if (q < n0) {
    const cplx<R> h = A[p + q * lda];
    const R g = hyp(h.x, h.y);
    const R app = A[p + p * lda].x, aqq = A[q + q * lda].x;
    if (g > JacEps<R>::tiny && g > JacEps<R>::v * sqrt(fabs(app * aqq))) {
      const R zeta = (aqq - app) / ((R)2 * g);
      const R t_ = (zeta >= (R)0 ? (R)1 : (R)-1) / (fabs(zeta) + hyp((R)1, zeta));
      r.c = (R)1 / sqrt((R)1 + t_ * t_);
      r.s = t_ * r.c;
      r.ph = cmake<cplx<R>>(h.x / g, h.y / g);
    }
  } else {
    q = -1;
  }
  rot[t] = r;
  pairs[2 * t] = (int)p;
  pairs[2 * t + 1] = (int)q;
}

template <typename R>
__global__ void k_jac_params(int64_t n0, int64_t n, int64_t round, const cplx<R>* __restrict__ A, int64_t lda,
                             RotT<R>* __restrict__ rot, int* __restrict__ pairs) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n / 2) jac_params_item<R>(t, n0, n, round, A, lda, rot, pairs);
}

// [a, b] <- [c a - s e^{i phi} b, s a + c e^{i phi} b] (rows, U^H from the left) and
// [a, b] <- [c a - s e^{-i phi} b, s a + c e^{-i phi} b] (columns, U from the right)
template <typename C, typename R>
__device__ __forceinline__ void rot2(C& a, C& b, R c, R s, C ph) {
  C na, nb;
  na.x = c * a.x - s * (ph.x * b.x - ph.y * b.y);
  na.y = c * a.y - s * (ph.x * b.y + ph.y * b.x);
  nb.x = s * a.x + c * (ph.x * b.x - ph.y * b.y);
  nb.y = s * a.y + c * (ph.x * b.y + ph.y * b.x);
  a = na;
  b = nb;
}

// items of one round: h x h blocks of A, n rows x h column pairs of V
__host__ __device__ inline int64_t jac_items(int64_t h, int64_t n) { return h * h + n * h; }

// One round of rotations in one pass: item (t1, t2) maps the 2 x 2 block of A on rows
// {p1, q1} and columns {p2, q2} to U1^H A U2 (the pairs are disjoint, so every element of A
// belongs to exactly one block); the remaining items apply V <- V U2 on columns {p2, q2}.
template <typename R>
__device__ __forceinline__ void jac_apply_item(int64_t idx, int64_t h, int64_t n, cplx<R>* A, int64_t lda,
                                               cplx<R>* V, int64_t ldv, const RotT<R>* __restrict__ rot,
                                               const int* __restrict__ pairs) {
  using C = cplx<R>;
  const int64_t nblk_a = h * h;
  if (idx < nblk_a) {
    const int64_t t1 = idx % h, t2 = idx / h;
    const int q1 = pairs[2 * t1 + 1], q2 = pairs[2 * t2 + 1];
    const int p1 = pairs[2 * t1], p2 = pairs[2 * t2];
    const RotT<R> r1 = rot[t1], r2 = rot[t2];
    const bool act1 = q1 >= 0 && r1.s != (R)0, act2 = q2 >= 0 && r2.s != (R)0;
    if (!act1 && !act2) return;
    const C cph2 = conjg(r2.ph);
    // the padding player (q < 0) owns no row or column of A: 1 x 2 or 2 x 1 blocks
    if (q1 < 0 || q2 < 0) {
      if (q1 < 0 && q2 < 0) return;
      if (q1 < 0) {  // row p1 alone, columns {p2, q2} rotate by U2
        C a = A[p1 + (int64_t)p2 * lda], b = A[p1 + (int64_t)q2 * lda];
        rot2(a, b, r2.c, r2.s, cph2);
        A[p1 + (int64_t)p2 * lda] = a;
        A[p1 + (int64_t)q2 * lda] = b;
      } else {  // column p2 alone, rows {p1, q1} rotate by U1^H
        C a = A[p1 + (int64_t)p2 * lda], b = A[q1 + (int64_t)p2 * lda];
        rot2(a, b, r1.c, r1.s, r1.ph);
        A[p1 + (int64_t)p2 * lda] = a;
        A[q1 + (int64_t)p2 * lda] = b;
      }
      return;
    }
    C m00 = A[p1 + (int64_t)p2 * lda], m10 = A[q1 + (int64_t)p2 * lda];
    C m01 = A[p1 + (int64_t)q2 * lda], m11 = A[q1 + (int64_t)q2 * lda];
    if (act1) {  // rows: [m0*; m1*] <- U1^H [m0*; m1*]
      rot2(m00, m10, r1.c, r1.s, r1.ph);
      rot2(m01, m11, r1.c, r1.s, r1.ph);
    }
    if (act2) {  // columns: [m*0, m*1] <- [m*0, m*1] U2
      rot2(m00, m01, r2.c, r2.s, cph2);
      rot2(m10, m11, r2.c, r2.s, cph2);
    }
    A[p1 + (int64_t)p2 * lda] = m00;
    A[q1 + (int64_t)p2 * lda] = m10;
    A[p1 + (int64_t)q2 * lda] = m01;
    A[q1 + (int64_t)q2 * lda] = m11;
    return;
  }
  const int64_t vidx = idx - nblk_a;
  if (vidx >= n * h) return;
  const int64_t i = vidx % n, t = vidx / n;
  const int q = pairs[2 * t + 1];
  if (q < 0) return;
  const RotT<R> r = rot[t];
  if (r.s == (R)0) return;
  const int p = pairs[2 * t];
  C ap = V[i + (int64_t)p * ldv], aq = V[i + (int64_t)q * ldv];
  rot2(ap, aq, r.c, r.s, conjg(r.ph));
  V[i + (int64_t)p * ldv] = ap;
  V[i + (int64_t)q * ldv] = aq;
}

template <typename R>
__global__ void k_jac_apply(int64_t h, int64_t n, cplx<R>* A, int64_t lda, cplx<R>* V, int64_t ldv,
                            const RotT<R>* __restrict__ rot, const int* __restrict__ pairs) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  jac_apply_item<R>(idx, h, n, A, lda, V, ldv, rot, pairs);
}

// All n-1 rounds of one Jacobi sweep in one cooperative launch: per round, the rotation
// parameters of the n/2 pairs, a grid barrier, the one-pass update of A and V, a barrier.
template <typename R>
__global__ void k_jac_sweep(int64_t n0, int64_t n, cplx<R>* A, int64_t lda, cplx<R>* V, int64_t ldv, RotT<R>* rot,
                            int* pairs, unsigned* bar, int* status) {
  const int64_t h = n / 2;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t round = 0; round < n - 1; ++round) {
    for (int64_t t = tid; t < h; t += nthreads) jac_params_item<R>(t, n0, n, round, A, lda, rot, pairs);
    grid_barrier(bar, bar + 1, gridDim.x, status);
    for (int64_t i = tid; i < jac_items(h, n0); i += nthreads) jac_apply_item<R>(i, h, n0, A, lda, V, ldv, rot, pairs);
    grid_barrier(bar, bar + 1, gridDim.x, status);
  }
}

// Per-block partial sums of |off-diagonal|^2 and |A|^2 (FP64), then one block adds the
// partials in block order: deterministic.
template <typename R>
__global__ void k_offnorm_part(int64_t n, const cplx<R>* A, int64_t lda, double* part) {
  __shared__ double r0[256], r1[256];
  double s0 = 0, s1 = 0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n * n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e % n, j = e / n;
    const cplx<R> a = A[i + j * lda];
    const double v = (double)a.x * a.x + (double)a.y * a.y;
    s1 += v;
    if (i != j) s0 += v;
  }
  r0[threadIdx.x] = s0;
  r1[threadIdx.x] = s1;
  __syncthreads();
  for (int hh = blockDim.x / 2; hh > 0; hh >>= 1) {
    if ((int)threadIdx.x < hh) {
      r0[threadIdx.x] += r0[threadIdx.x + hh];
      r1[threadIdx.x] += r1[threadIdx.x + hh];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = r0[0];
    part[2 * blockIdx.x + 1] = r1[0];
  }
}

__global__ void k_offnorm_sum(int nparts, const double* part, double* out) {
  if (threadIdx.x == 0) {
    double s0 = 0, s1 = 0;
    for (int b = 0; b < nparts; ++b) {
      s0 += part[2 * b];
      s1 += part[2 * b + 1];
    }
    out[0] = s0;
    out[1] = s1;
  }
}

// Sort eigenpairs ascending (stable): rank by counting, then permute w and the columns of V.
template <typename R>
__global__ void k_eig_sort(int64_t n, const cplx<R>* __restrict__ A, int64_t lda, const cplx<R>* __restrict__ Vin,
                           int64_t ldvi, R* __restrict__ w, cplx<R>* __restrict__ Vout, int64_t ldvo) {
  const int64_t i = blockIdx.x;
  __shared__ int64_t rank;
  const R wi = A[i + i * lda].x;
  if (threadIdx.x == 0) rank = 0;
  __syncthreads();
  int64_t cnt = 0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const R wj = A[j + j * lda].x;
    if (wj < wi || (wj == wi && j < i)) ++cnt;
  }
  atomicAdd((unsigned long long*)&rank, (unsigned long long)cnt);
  __syncthreads();
  const int64_t r = rank;
  if (threadIdx.x == 0) w[r] = wi;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) Vout[k + r * ldvo] = Vin[k + i * ldvi];
}

template <typename C> __global__ void k_identity_t(int64_t n, C* A, int64_t lda) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx % n, j = idx / n;
  A[i + j * lda] = cmake<C>(i == j ? 1.0 : 0.0, 0.0);
}
template <typename R> void set_identity_t(int64_t n, cplx<R>* A, int64_t lda, cudaStream_t st) {
  CHEBFI_LAUNCH("k_identity", st, k_identity_t<cplx<R>><<<nblk(n * n), 256, 0, st>>>(n, A, lda));
}

template <typename R>
void jacobi_eigh_t(int64_t n0, cplx<R>* A, int64_t lda, R* w, cplx<R>* V, int64_t ldv, int* status, cudaStream_t st,
                   DevBuf<double2>* ws, double tol_conv, double tol_stall, bool report) {
  using C = cplx<R>;
  if (n0 <= 0) return;
  const int64_t n = n0 + (n0 & 1);  // a padding player never paired for real
  // workspace (in double2 units): rotations, pair list, norm partials, barrier, a copy of V
  constexpr int kParts = 256;
  const size_t rot_c = (size_t)(n / 2) * sizeof(RotT<R>) / sizeof(double2) + 1;
  const size_t pair_c = (size_t)n * sizeof(int) / sizeof(double2) + 1;
  const size_t part_c = kParts + 2;
  const size_t vtmp = ((size_t)n0 * n0 * sizeof(C) + sizeof(double2) - 1) / sizeof(double2);
  ws->alloc(rot_c + pair_c + part_c + 1 + vtmp);
  RotT<R>* rot = reinterpret_cast<RotT<R>*>(ws->p);
  int* pairs = reinterpret_cast<int*>(ws->p + rot_c);
  double* part = reinterpret_cast<double*>(ws->p + rot_c + pair_c);
  double* nrm = part + 2 * kParts;
  unsigned* bar = reinterpret_cast<unsigned*>(ws->p + rot_c + pair_c + part_c);
  C* Vtmp = reinterpret_cast<C*>(ws->p + rot_c + pair_c + part_c + 1);
  if (n0 == 1) {
    set_identity_t<R>(1, Vtmp, 1, st);
    CHEBFI_LAUNCH("k_eig_sort", st, k_eig_sort<R><<<1, 32, 0, st>>>(1, A, lda, Vtmp, 1, w, V, ldv));
    return;
  }
  CHEBFI_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
  // one cooperative launch per sweep when the device allows it (all blocks resident)
  int dev = 0, coop = 0, sms = 0, per_sm = 0;
  CHEBFI_CUDA(cudaGetDevice(&dev));
  CHEBFI_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  CHEBFI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CHEBFI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jac_sweep<R>, 256, 0));
  const int coop_blocks = sms * std::min(per_sm, 8);
  set_identity_t<R>(n0, Vtmp, n0, st);
  const int max_sweeps = 40;
  const unsigned parts = (unsigned)std::min<int64_t>(kParts, std::max<int64_t>(1, n0 * n0 / 4096));
  double prev_off = INFINITY;
  bool done = false;
  for (int sweep = 0; sweep <= max_sweeps && !done; ++sweep) {
    CHEBFI_LAUNCH("k_offnorm", st, k_offnorm_part<R><<<parts, 256, 0, st>>>(n0, A, lda, part));
    CHEBFI_LAUNCH("k_offnorm", st, k_offnorm_sum<<<1, 32, 0, st>>>((int)parts, part, nrm));
    double hn[2];
    CHEBFI_CUDA(cudaMemcpyAsync(hn, nrm, sizeof(hn), cudaMemcpyDeviceToHost, st));
    CHEBFI_CUDA(cudaStreamSynchronize(st));
    const double off = std::sqrt(hn[0]), tot = std::sqrt(hn[1]);
    if (!std::isfinite(tot)) {  // Inf or NaN in the matrix: no sweep can help
      int code = CHEBFI_ERR_NONFINITE;
      CHEBFI_CUDA(cudaMemcpyAsync(status, &code, sizeof(int), cudaMemcpyHostToDevice, st));
      CHEBFI_CUDA(cudaStreamSynchronize(st));
      report = false;
      break;
    }
    // converged: off-diagonal at the rounding level, or no longer decreasing near it
    if (off <= tol_conv * tot || off == 0.0 || (sweep > 2 && off > 0.5 * prev_off && off <= tol_stall * tot)) {
      done = true;
      break;
    }
    if (sweep == max_sweeps) break;
    prev_off = off;
    if (coop && coop_blocks > 0) {
      int64_t n0a = n0, na = n, ldaa = lda, ldva = n0;
      C* Aa = A;
      C* Va = Vtmp;
      void* args[] = {&n0a, &na, &Aa, &ldaa, &Va, &ldva, &rot, &pairs, &bar, &status};
      // work: per round every entry of A gets two rotations and every entry of V one, about
      // 11 real flops per complex entry per rotation: 33 n^3 per sweep
      CHEBFI_LAUNCH_W("k_jac_sweep", st, 33.0 * (double)n0 * (double)n0 * (double)n0,
                      CHEBFI_CUDA(cudaLaunchCooperativeKernel((const void*)k_jac_sweep<R>, dim3(coop_blocks),
                                                              dim3(256), args, 0, st)));
    } else {
      for (int64_t round = 0; round < n - 1; ++round) {
        CHEBFI_LAUNCH("k_jac_params", st,
                      k_jac_params<R><<<nblk(n / 2), 256, 0, st>>>(n0, n, round, A, lda, rot, pairs));
        const int64_t h = n / 2;
        CHEBFI_LAUNCH("k_jac_apply", st,
                      k_jac_apply<R><<<nblk(jac_items(h, n0)), 256, 0, st>>>(h, n0, A, lda, Vtmp, n0, rot, pairs));
      }
    }
  }
  if (!done && report) {
    int code = CHEBFI_ERR_NO_CONVERGENCE;
    // record on the device flag as well so chebfi_sync_status sees it
    CHEBFI_CUDA(cudaMemcpyAsync(status, &code, sizeof(int), cudaMemcpyHostToDevice, st));
    CHEBFI_CUDA(cudaStreamSynchronize(st));
  }
  CHEBFI_LAUNCH("k_eig_sort", st, k_eig_sort<R><<<(unsigned)n0, 128, 0, st>>>(n0, A, lda, Vtmp, n0, w, V, ldv));
}


// ------------------------------------------------------------------ refinement of eigenvectors
// One step of the iterative refinement of Ogita & Aishima (2018) for a Hermitian A and
// approximate eigenvectors X, from G = X^H X (= I - R) and S = X^H A X:
//   lambda_i = S_ii / G_ii,
//   E_ij = (S_ij - lambda_j G_ij) / (lambda_j - lambda_i)   (i != j; = (s_ij + lambda_j r_ij)/(...)),
//   E_ii = (1 - G_ii) / 2,
// and X <- X (I + E).  A pair whose gap is not large against its numerator (|gap| <=
// 4 |num|, or below 1e-13 |A|) is treated as a cluster: E_ij = -G_ij / 2 only restores
// orthogonality, and the pair is listed for a final dense solve of the cluster.
__global__ void k_oa_lambda(int64_t n, const double2* __restrict__ G, int64_t ldg, const double2* __restrict__ S,
                            int64_t lds, double* __restrict__ lam, unsigned long long* __restrict__ amax) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double l = S[i + i * lds].x / G[i + i * ldg].x;
  lam[i] = l;
  atomicMax(amax, (unsigned long long)__double_as_longlong(fabs(l)));
}

__global__ void k_oa_update(int64_t n, const double2* __restrict__ G, int64_t ldg, const double2* __restrict__ S,
                            int64_t lds, const double* __restrict__ lam, const unsigned long long* __restrict__ amax,
                            double2* __restrict__ M, int64_t ldm, unsigned long long* __restrict__ emax,
                            int* __restrict__ npairs, int2* __restrict__ pairs, int cap) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool in = idx < n * n;
  const int64_t i = in ? idx % n : 0, j = in ? idx / n : 0;
  const double2 g = in ? G[i + j * ldg] : make_double2(1.0, 0.0);
  double2 e;
  double mag = 0.0;
  if (!in) {
    e = make_double2(0.0, 0.0);
  } else if (i == j) {
    e = make_double2(0.5 * (1.0 - g.x), 0.0);
    mag = fabs(e.x);
  } else {
    const double2 s = S[i + j * lds];
    const double lj = lam[j], gap = lj - lam[i];
    const double2 num = make_double2(s.x - lj * g.x, s.y - lj * g.y);
    const double anum = hypot(num.x, num.y);
    const double tiny = 1e-13 * __longlong_as_double((long long)*amax);
    if (fabs(gap) > 4.0 * anum && fabs(gap) > tiny) {
      e = make_double2(num.x / gap, num.y / gap);
    } else {
      e = make_double2(-0.5 * g.x, -0.5 * g.y);
      if (i < j) {
        const int k = atomicAdd(npairs, 1);
        if (k < cap) pairs[k] = make_int2((int)i, (int)j);
      }
    }
    mag = hypot(e.x, e.y);
  }
  // max |E| over the warp first (the bits of non-negative doubles order like their values,
  // a NaN above all), then one atomic per warp: one per element serialises on the word
  unsigned long long bits = (unsigned long long)__double_as_longlong(mag);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, bits, o);
    bits = other > bits ? other : bits;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(emax, bits);
  if (in) M[i + j * ldm] = make_double2((i == j ? 1.0 : 0.0) + e.x, e.y);
}

// ascending order of w (stable), columns of X permuted alike
__global__ void k_sort_pairs(int64_t n, const double* __restrict__ win, const double2* __restrict__ Xin, int64_t ldi,
                             double* __restrict__ wout, double2* __restrict__ Xout, int64_t ldo) {
  const int64_t i = blockIdx.x;
  __shared__ unsigned long long rank;
  const double wi = win[i];
  if (threadIdx.x == 0) rank = 0;
  __syncthreads();
  unsigned long long cnt = 0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double wj = win[j];
    if (wj < wi || (wj == wi && j < i)) ++cnt;
  }
  atomicAdd(&rank, cnt);
  __syncthreads();
  const int64_t r = (int64_t)rank;
  if (threadIdx.x == 0) wout[r] = wi;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) Xout[k + r * ldo] = Xin[k + i * ldi];
}

// sub[a, b] = A[idx[a], idx[b]] (k x k); cols: sub[:, b] = X[:, idx[b]] or the reverse
__global__ void k_gather_sub(int k, const int* __restrict__ idx, const double2* __restrict__ A, int64_t lda,
                             double2* __restrict__ sub) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= k * k) return;
  const int a = e % k, b = e / k;
  sub[e] = A[idx[a] + (int64_t)idx[b] * lda];
}
__global__ void k_cols(int64_t m, int k, const int* __restrict__ idx, double2* X, int64_t ldx, double2* Y,
                       int64_t ldy, int to_y) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= m * k) return;
  const int64_t r = e % m;
  const int b = (int)(e / m);
  if (to_y) Y[r + b * ldy] = X[r + idx[b] * ldx];
  else X[r + idx[b] * ldx] = Y[r + b * ldy];
}
__global__ void k_scatter_vals(int k, const int* __restrict__ idx, const double* __restrict__ src, double* dst) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < k) dst[idx[b]] = src[b];
}

// ------------------------------------------------------------------ blocked Jacobi (FP32)
// The two-sided cyclic Jacobi method on blocks: the n columns form n / 32 blocks, paired by
// the round-robin tournament (n / 32 - 1 rounds per sweep, n / 64 disjoint pairs per round).
// For a pair (I, J) the 64 x 64 subproblem A[IJ, IJ] is diagonalised in shared memory by the
// scalar method (same rotations as above) giving a unitary W, then A <- W^H A W on rows and
// columns I u J and V <- V W: each round is one pass over A and V as small dense products
// instead of 63 passes of scalar rotations, which the scalar method spends in grid barriers
// and load latency.
namespace bj {
constexpr int B = 32, S2 = 64, PS = S2 + 1;  // block, subproblem, shared pitch

__device__ __forceinline__ int player(int pos, int round, int m) {
  return pos == 0 ? 0 : 1 + (pos - 1 + round) % (m - 1);
}
__device__ __forceinline__ void blocks_of(int pair, int round, int nbk, int& I, int& J) {
  I = player(pair, round, nbk);
  J = player(nbk - 1 - pair, round, nbk);
  if (I > J) {
    const int t = I;
    I = J;
    J = t;
  }
}
__device__ __forceinline__ int gidx(int l, int I, int J) { return l < B ? I * B + l : J * B + (l - B); }

// One CTA of 1024 threads per pair: gather the subproblem, diagonalise it (up to `sweeps`
// cyclic sweeps, or until its off-diagonal part is below tol of its norm), write the
// rotation W (64 x 64, column-major) to Wout[pair].
__global__ void __launch_bounds__(1024) k_bj_solve(const float2* __restrict__ A, int64_t lda, int nbk, int round,
                                                  float2* __restrict__ Wout, int sweeps, float tol) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* S = reinterpret_cast<float2*>(smem);  // S[i + PS j] = element (i, j)
  float2* W = S + S2 * PS;
  RotT<float>* rot = reinterpret_cast<RotT<float>*>(W + S2 * PS);
  int* pq = reinterpret_cast<int*>(rot + S2 / 2);
  __shared__ float red[2][1024];
  int I, J;
  blocks_of(blockIdx.x, round, nbk, I, J);
  const int tid = threadIdx.x;
  for (int e = tid; e < S2 * S2; e += blockDim.x) {
    const int i = e % S2, j = e / S2;
    S[i + PS * j] = A[gidx(i, I, J) + (int64_t)gidx(j, I, J) * lda];
    W[i + PS * j] = make_float2(i == j ? 1.f : 0.f, 0.f);
  }
  __syncthreads();
  for (int sw = 0; sw < sweeps; ++sw) {
    float o = 0.f, t = 0.f;
    for (int e = tid; e < S2 * S2; e += blockDim.x) {
      const int i = e % S2, j = e / S2;
      const float2 v = S[i + PS * j];
      const float m = v.x * v.x + v.y * v.y;
      t += m;
      if (i != j) o += m;
    }
    red[0][tid] = o;
    red[1][tid] = t;
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
      if (tid < h) {
        red[0][tid] += red[0][tid + h];
        red[1][tid] += red[1][tid + h];
      }
      __syncthreads();
    }
    const bool done = red[0][0] <= tol * tol * red[1][0];
    __syncthreads();
    if (done) break;
    for (int r = 0; r < S2 - 1; ++r) {
      if (tid < S2 / 2) {
        int p = player(tid, r, S2), q = player(S2 - 1 - tid, r, S2);
        if (p > q) {
          const int x = p;
          p = q;
          q = x;
        }
        RotT<float> rr;
        rr.c = 1.f;
        rr.s = 0.f;
        rr.ph = make_float2(1.f, 0.f);
        const float2 h = S[p + PS * q];
        const float g = hypotf(h.x, h.y);
        const float app = S[p + PS * p].x, aqq = S[q + PS * q].x;
        if (g > JacEps<float>::tiny && g > JacEps<float>::v * sqrtf(fabsf(app * aqq))) {
          const float zeta = (aqq - app) / (2.f * g);
          const float tt = (zeta >= 0.f ? 1.f : -1.f) / (fabsf(zeta) + hypotf(1.f, zeta));
          rr.c = 1.f / sqrtf(1.f + tt * tt);
          rr.s = tt * rr.c;
          rr.ph = make_float2(h.x / g, h.y / g);
        }
        rot[tid] = rr;
        pq[2 * tid] = p;
        pq[2 * tid + 1] = q;
      }
      __syncthreads();
      // 2 x 2 blocks of S: U1^H S U2
      for (int it = tid; it < (S2 / 2) * (S2 / 2); it += blockDim.x) {
        const int t1 = it % (S2 / 2), t2 = it / (S2 / 2);
        const RotT<float> r1 = rot[t1], r2 = rot[t2];
        if (r1.s == 0.f && r2.s == 0.f) continue;
        const int p1 = pq[2 * t1], q1 = pq[2 * t1 + 1], p2 = pq[2 * t2], q2 = pq[2 * t2 + 1];
        float2 m00 = S[p1 + PS * p2], m10 = S[q1 + PS * p2], m01 = S[p1 + PS * q2], m11 = S[q1 + PS * q2];
        if (r1.s != 0.f) {
          rot2(m00, m10, r1.c, r1.s, r1.ph);
          rot2(m01, m11, r1.c, r1.s, r1.ph);
        }
        if (r2.s != 0.f) {
          const float2 c2 = conjg(r2.ph);
          rot2(m00, m01, r2.c, r2.s, c2);
          rot2(m10, m11, r2.c, r2.s, c2);
        }
        S[p1 + PS * p2] = m00;
        S[q1 + PS * p2] = m10;
        S[p1 + PS * q2] = m01;
        S[q1 + PS * q2] = m11;
      }
      // W <- W U on columns {p, q}
      for (int it = tid; it < S2 * (S2 / 2); it += blockDim.x) {
        const int i = it % S2, tt = it / S2;
        const RotT<float> rr = rot[tt];
        if (rr.s == 0.f) continue;
        const int p = pq[2 * tt], q = pq[2 * tt + 1];
        float2 a = W[i + PS * p], b = W[i + PS * q];
        rot2(a, b, rr.c, rr.s, conjg(rr.ph));
        W[i + PS * p] = a;
        W[i + PS * q] = b;
      }
      __syncthreads();
    }
  }
  float2* wo = Wout + (int64_t)blockIdx.x * S2 * S2;
  for (int e = tid; e < S2 * S2; e += blockDim.x) wo[e] = W[(e % S2) + PS * (e / S2)];
}

// columns I u J of M (A or V; blockIdx.z) times W: a CTA takes 64 rows, in place
__global__ void __launch_bounds__(256) k_bj_cols(float2* A, int64_t lda, float2* V, int64_t ldv, int nbk, int round,
                                                 const float2* __restrict__ Win, int64_t nrows) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* W = reinterpret_cast<float2*>(smem);  // W[l + PS c]
  float2* X = W + S2 * PS;                       // X[row + PS l]
  int I, J;
  blocks_of(blockIdx.y, round, nbk, I, J);
  float2* M = blockIdx.z == 0 ? A : V;
  const int64_t ld = blockIdx.z == 0 ? lda : ldv;
  const int64_t r0 = (int64_t)blockIdx.x * S2;
  const float2* w = Win + (int64_t)blockIdx.y * S2 * S2;
  const int tid = threadIdx.x;
  for (int e = tid; e < S2 * S2; e += blockDim.x) {
    const int a = e % S2, b = e / S2;
    W[a + PS * b] = w[e];
    const int64_t r = r0 + a;
    X[a + PS * b] = r < nrows ? M[r + (int64_t)gidx(b, I, J) * ld] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  // thread: rows ri + 16 k (k < 4), columns ci + 16 m (m < 4)
  const int ri = tid % 16, ci = tid / 16;
  float2 acc[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[k][m] = make_float2(0.f, 0.f);
  for (int l = 0; l < S2; ++l) {
    float2 x[4], y[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) x[k] = X[ri + 16 * k + PS * l];
#pragma unroll
    for (int m = 0; m < 4; ++m) y[m] = W[l + PS * (ci + 16 * m)];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        acc[k][m].x = fmaf(x[k].x, y[m].x, fmaf(-x[k].y, y[m].y, acc[k][m].x));
        acc[k][m].y = fmaf(x[k].x, y[m].y, fmaf(x[k].y, y[m].x, acc[k][m].y));
      }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int64_t r = r0 + ri + 16 * k;
    if (r >= nrows) continue;
#pragma unroll
    for (int m = 0; m < 4; ++m) M[r + (int64_t)gidx(ci + 16 * m, I, J) * ld] = acc[k][m];
  }
}

// rows I u J of A: W^H times them; a CTA takes 64 columns, in place
__global__ void __launch_bounds__(256) k_bj_rows(float2* A, int64_t lda, int nbk, int round,
                                                 const float2* __restrict__ Win, int64_t ncols) {
  extern __shared__ __align__(16) unsigned char smem[];
  float2* W = reinterpret_cast<float2*>(smem);  // W[l + PS c]
  float2* Z = W + S2 * PS;                       // Z[l + PS col]
  int I, J;
  blocks_of(blockIdx.y, round, nbk, I, J);
  const int64_t c0 = (int64_t)blockIdx.x * S2;
  const float2* w = Win + (int64_t)blockIdx.y * S2 * S2;
  const int tid = threadIdx.x;
  for (int e = tid; e < S2 * S2; e += blockDim.x) {
    const int a = e % S2, b = e / S2;
    W[a + PS * b] = w[e];
    const int64_t c = c0 + b;
    Z[a + PS * b] = c < ncols ? A[gidx(a, I, J) + c * lda] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  // thread: output rows li + 16 k, columns cj + 16 m; out(l, col) = sum_k conj(W(k, l)) Z(k, col)
  const int li = tid % 16, cj = tid / 16;
  float2 acc[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[k][m] = make_float2(0.f, 0.f);
  for (int q = 0; q < S2; ++q) {
    float2 wv[4], z[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) wv[k] = W[q + PS * (li + 16 * k)];
#pragma unroll
    for (int m = 0; m < 4; ++m) z[m] = Z[q + PS * (cj + 16 * m)];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int m = 0; m < 4; ++m) {  // conj(wv) z
        acc[k][m].x = fmaf(wv[k].x, z[m].x, fmaf(wv[k].y, z[m].y, acc[k][m].x));
        acc[k][m].y = fmaf(wv[k].x, z[m].y, fmaf(-wv[k].y, z[m].x, acc[k][m].y));
      }
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int64_t c = c0 + cj + 16 * m;
    if (c >= ncols) continue;
#pragma unroll
    for (int k = 0; k < 4; ++k) A[gidx(li + 16 * k, I, J) + c * lda] = acc[k][m];
  }
}

// zero-padded copy with pad values on the extra diagonal entries
__global__ void k_bj_pad(int64_t n0, int64_t np, const float2* __restrict__ A, int64_t lda, float2* __restrict__ Ap,
                         float pad) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= np * np) return;
  const int64_t i = e % np, j = e / np;
  Ap[e] = (i < n0 && j < n0) ? A[i + j * lda] : make_float2(i == j ? pad : 0.f, 0.f);
}
}  // namespace bj

// The blocked FP32 Jacobi (bj:: kernels) on A (n0 x n0, destroyed): ascending w and V
// (ld ldv).  The matrix is padded to a multiple of 64 with decoupled diagonal entries above
// every eigenvalue (2 ||A||_F + 1), which no rotation touches and the sort puts last.
bool block_jacobi_f32(int64_t n0, float2* A, int64_t lda, float* w, float2* V, int64_t ldv, cudaStream_t st,
                      DevBuf<double2>* ws, double tol_conv, double tol_stall) {
  if (n0 < 128) return false;
  const int64_t np = (n0 + bj::S2 - 1) / bj::S2 * bj::S2;
  const int nbk = (int)(np / bj::B), npairs = nbk / 2;
  constexpr int kParts = 256;
  // workspace in float2 slots: Ap, Vp, Vs (np^2 each), W (npairs x 64^2), wp (np / 2 + 1),
  // norm partials and sums (2 kParts + 2 doubles)
  const size_t nn = (size_t)np * np, nw = (size_t)npairs * bj::S2 * bj::S2;
  const size_t total = 3 * nn + nw + np / 2 + 1 + 2 * kParts + 2;
  ws->alloc(total / 2 + 1);
  float2* Ap = reinterpret_cast<float2*>(ws->p);
  float2* Vp = Ap + nn;
  float2* Vs = Vp + nn;
  float2* Wb = Vs + nn;
  float* wp = reinterpret_cast<float*>(Wb + nw);
  double* part = reinterpret_cast<double*>(Wb + nw + np / 2 + 1);
  double* nrm = part + 2 * kParts;
  auto norms = [&](const float2* M, int64_t n, int64_t ld, double& off, double& tot) {
    const unsigned parts = (unsigned)std::min<int64_t>(kParts, std::max<int64_t>(1, n * n / 4096));
    CHEBFI_LAUNCH("k_offnorm", st, k_offnorm_part<float><<<parts, 256, 0, st>>>(n, M, ld, part));
    CHEBFI_LAUNCH("k_offnorm", st, k_offnorm_sum<<<1, 32, 0, st>>>((int)parts, part, nrm));
    double hn[2];
    CHEBFI_CUDA(cudaMemcpyAsync(hn, nrm, sizeof(hn), cudaMemcpyDeviceToHost, st));
    CHEBFI_CUDA(cudaStreamSynchronize(st));
    off = std::sqrt(hn[0]);
    tot = std::sqrt(hn[1]);
  };
  double off = 0.0, tot = 0.0, tot_p = 0.0;
  norms(A, n0, lda, off, tot);  // ||A||_F: the sweeps keep it (unitary similarity), so it is the scale
  if (!std::isfinite(tot)) return false;  // the scalar path reports it
  CHEBFI_LAUNCH("k_bj_pad", st, bj::k_bj_pad<<<nblk((int64_t)nn), 256, 0, st>>>(n0, np, A, lda, Ap, (float)(2.0 * tot + 1.0)));
  set_identity_t<float>(np, Vp, np, st);
  const size_t s_solve = (size_t)2 * bj::S2 * bj::PS * sizeof(float2) + bj::S2 / 2 * sizeof(RotT<float>) + bj::S2 * sizeof(int);
  const size_t s_mul = (size_t)2 * bj::S2 * bj::PS * sizeof(float2);
  CHEBFI_CUDA(cudaFuncSetAttribute(bj::k_bj_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_solve));
  CHEBFI_CUDA(cudaFuncSetAttribute(bj::k_bj_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_mul));
  CHEBFI_CUDA(cudaFuncSetAttribute(bj::k_bj_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s_mul));
  const unsigned tiles = (unsigned)(np / bj::S2);
  double prev_off = INFINITY;
  for (int sweep = 0; sweep <= 40; ++sweep) {
    norms(Ap, np, np, off, tot_p);  // the pads add nothing off the diagonal
    if (!std::isfinite(tot_p)) break;
    if (off <= tol_conv * tot || off == 0.0 || (sweep > 2 && off > 0.5 * prev_off && off <= tol_stall * tot)) break;
    if (sweep == 40) break;
    prev_off = off;
    // rounds of the block tournament; work: the subproblems' rotations and the two products
    for (int round = 0; round < nbk - 1; ++round) {
      CHEBFI_LAUNCH("k_bj_solve", st, bj::k_bj_solve<<<npairs, 1024, s_solve, st>>>(Ap, np, nbk, round, Wb, 1, 1e-7f));
      CHEBFI_LAUNCH_W("k_bj_update", st, 3.0 * 8.0 * (double)np * bj::S2 * bj::S2 * npairs,
                      bj::k_bj_cols<<<dim3(tiles, npairs, 2), 256, s_mul, st>>>(Ap, np, Vp, np, nbk, round, Wb, np));
      CHEBFI_LAUNCH("k_bj_update", st, bj::k_bj_rows<<<dim3(tiles, npairs), 256, s_mul, st>>>(Ap, np, nbk, round, Wb, np));
    }
  }
  CHEBFI_LAUNCH("k_eig_sort", st, k_eig_sort<float><<<(unsigned)np, 128, 0, st>>>(np, Ap, np, Vp, np, wp, Vs, np));
  CHEBFI_CUDA(cudaMemcpyAsync(w, wp, sizeof(float) * n0, cudaMemcpyDeviceToDevice, st));
  CHEBFI_CUDA(cudaMemcpy2DAsync(V, ldv * sizeof(float2), Vs, np * sizeof(float2), n0 * sizeof(float2), n0,
                                cudaMemcpyDeviceToDevice, st));
  return true;
}

}  // namespace

void oa_step(int64_t n, const double2* G, const double2* S, double* lam, double2* M, unsigned long long* stats,
             int* npairs, int2* pairs, int cap, cudaStream_t st) {
  CHEBFI_CUDA(cudaMemsetAsync(stats, 0, 2 * sizeof(unsigned long long), st));
  CHEBFI_CUDA(cudaMemsetAsync(npairs, 0, sizeof(int), st));
  CHEBFI_LAUNCH("k_oa_lambda", st, k_oa_lambda<<<nblk(n), 256, 0, st>>>(n, G, n, S, n, lam, stats));
  CHEBFI_LAUNCH("k_oa_update", st,
                k_oa_update<<<nblk(n * n), 256, 0, st>>>(n, G, n, S, n, lam, stats, M, n, stats + 1, npairs, pairs, cap));
}

void sort_eigpairs(int64_t n, const double* win, const double2* Xin, double* wout, double2* Xout, cudaStream_t st) {
  CHEBFI_LAUNCH("k_sort_pairs", st, k_sort_pairs<<<(unsigned)n, 128, 0, st>>>(n, win, Xin, n, wout, Xout, n));
}

void gather_sub(int k, const int* idx, const double2* A, int64_t lda, double2* sub, cudaStream_t st) {
  CHEBFI_LAUNCH("k_gather_sub", st, k_gather_sub<<<nblk((int64_t)k * k), 256, 0, st>>>(k, idx, A, lda, sub));
}
void gather_cols(int64_t m, int k, const int* idx, const double2* X, int64_t ldx, double2* Y, int64_t ldy,
                 cudaStream_t st) {
  CHEBFI_LAUNCH("k_cols", st, k_cols<<<nblk(m * k), 256, 0, st>>>(m, k, idx, const_cast<double2*>(X), ldx, Y, ldy, 1));
}
void scatter_cols(int64_t m, int k, const int* idx, double2* X, int64_t ldx, const double2* Y, int64_t ldy,
                  cudaStream_t st) {
  CHEBFI_LAUNCH("k_cols", st, k_cols<<<nblk(m * k), 256, 0, st>>>(m, k, idx, X, ldx, const_cast<double2*>(Y), ldy, 0));
}
void scatter_vals(int k, const int* idx, const double* src, double* dst, cudaStream_t st) {
  CHEBFI_LAUNCH("k_scatter_vals", st, k_scatter_vals<<<nblk(k), 256, 0, st>>>(k, idx, src, dst));
}

void cholesky(int64_t n, double2* A, int64_t lda, int* status, cudaStream_t st, DevBuf<double2>* ws) {
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int nb = (int)std::min<int64_t>(NB, n - k0);
    CHEBFI_LAUNCH("k_chol_diag", st, k_chol_diag<<<1, 256, 0, st>>>(A + k0 + k0 * lda, lda, nb, status));
    const int64_t m2 = n - k0 - nb;
    if (m2 > 0) {
      double2* L21 = A + (k0 + nb) + k0 * lda;
      CHEBFI_LAUNCH("k_trsm_right_lh", st, k_trsm_right_lh<<<nblk(m2, 128), 128, 0, st>>>(A + k0 + k0 * lda, lda, L21, lda, m2, nb));
      gemm<double>(false, true, m2, m2, nb, -1.0, L21, lda, L21, lda, 1.0, A + (k0 + nb) + (k0 + nb) * lda, lda, st,
                   ws);
    }
  }
  CHEBFI_LAUNCH("k_zero_upper", st, k_zero_upper<<<nblk(n * n), 256, 0, st>>>(n, A, lda));
}

void trsm_lower(int64_t n, int64_t m, const double2* L, int64_t ldl, double2* B, int64_t ldb, cudaStream_t st,
                DevBuf<double2>* ws) {
  for (int64_t k0 = 0; k0 < n; k0 += NB) {
    const int nb = (int)std::min<int64_t>(NB, n - k0);
    CHEBFI_LAUNCH("k_trsm_left_l", st, k_trsm_left_l<<<nblk(m, 128), 128, 0, st>>>(L + k0 + k0 * ldl, ldl, B + k0, ldb, m, nb));
    const int64_t m2 = n - k0 - nb;
    if (m2 > 0)
      gemm<double>(false, false, m2, m, nb, -1.0, L + (k0 + nb) + k0 * ldl, ldl, B + k0, ldb, 1.0, B + k0 + nb, ldb, st,
                   ws);
  }
}

void jacobi_eigh(int64_t n0, double2* A, int64_t lda, double* w, double2* V, int64_t ldv, int* status, cudaStream_t st,
                 DevBuf<double2>* ws) {
  jacobi_eigh_t<double>(n0, A, lda, w, V, ldv, status, st, ws, 1e-15, 1e-12, true);
}

void jacobi_eigh_f32(int64_t n0, float2* A, int64_t lda, float* w, float2* V, int64_t ldv, int* status,
                     cudaStream_t st, DevBuf<double2>* ws) {
  // a first stage only: stop at the FP32 rounding level and never report a sweep limit; the
  // blocked method from 128 bands up
  if (block_jacobi_f32(n0, A, lda, w, V, ldv, st, ws, 4e-7, 1e-5)) return;
  jacobi_eigh_t<float>(n0, A, lda, w, V, ldv, status, st, ws, 4e-7, 1e-5, false);
}

}  // namespace chebfi
