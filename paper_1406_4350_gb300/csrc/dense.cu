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
__device__ __forceinline__ int64_t rr_player(int64_t pos, int64_t round, int64_t n) {
  return pos == 0 ? 0 : 1 + (pos - 1 + round) % (n - 1);
}

struct Rot {
  double c, s;
  double2 ph;  // e^{i phi}
};

__global__ void k_jac_params(int64_t n0, int64_t n, int64_t round, const double2* __restrict__ A, int64_t lda,
                             Rot* __restrict__ rot, int* __restrict__ pairs) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n / 2) return;
  int64_t p = rr_player(t, round, n), q = rr_player(n - 1 - t, round, n);
  if (p > q) { const int64_t tmp = p; p = q; q = tmp; }
  Rot r;
  r.c = 1.0;
  r.s = 0.0;
  r.ph = make_double2(1.0, 0.0);
  if (q < n0) {  // skip pairs with the padding player
    const double2 h = A[p + q * lda];
    const double g = hypot(h.x, h.y);
    const double app = A[p + p * lda].x, aqq = A[q + q * lda].x;
    if (g > 1e-300 && g > 1.1102230246251565e-16 * sqrt(fabs(app * aqq))) {
      const double zeta = (aqq - app) / (2.0 * g);
      const double t_ = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
      r.c = 1.0 / sqrt(1.0 + t_ * t_);
      r.s = t_ * r.c;
      r.ph = make_double2(h.x / g, h.y / g);
    }
  } else {
    q = -1;
  }
  rot[t] = r;
  pairs[2 * t] = (int)p;
  pairs[2 * t + 1] = (int)q;
}

// One round of rotations in one pass: thread (t1, t2) maps the 2 x 2 block of A on rows
// {p1, q1} and columns {p2, q2} to U1^H A U2 (the pairs are disjoint, so every element of A
// belongs to exactly one block); the remaining threads apply V <- V U2 on columns {p2, q2}.
__device__ __forceinline__ void jac_apply_item(int64_t idx, int64_t h, int64_t n, double2* A, int64_t lda, double2* V,
                                               int64_t ldv, const Rot* __restrict__ rot, const int* __restrict__ pairs) {
  const int64_t nblk_a = h * h;
  if (idx < nblk_a) {
    const int64_t t1 = idx % h, t2 = idx / h;
    const int q1 = pairs[2 * t1 + 1], q2 = pairs[2 * t2 + 1];
    const int p1 = pairs[2 * t1], p2 = pairs[2 * t2];
    const Rot r1 = rot[t1], r2 = rot[t2];
    const bool act1 = q1 >= 0 && r1.s != 0.0, act2 = q2 >= 0 && r2.s != 0.0;
    if (!act1 && !act2) return;
    // the padding player (q < 0) never owns a row or column of A
    if (q1 < 0 || q2 < 0) {
      // a real pair against the padding: only the real pair's own rotation applies on its
      // side of the blocks it shares with other pairs; handled as a 1 x 2 or 2 x 1 block
      if (q1 < 0 && q2 < 0) return;
      if (q1 < 0) {  // row p1 alone, columns {p2, q2} rotate by U2
        double2 a = A[p1 + (int64_t)p2 * lda], b = A[p1 + (int64_t)q2 * lda];
        const double2 sc = make_double2(r2.s * r2.ph.x, -r2.s * r2.ph.y), cc = make_double2(r2.c * r2.ph.x, -r2.c * r2.ph.y);
        double2 na, nb;
        na.x = r2.c * a.x - (b.x * sc.x - b.y * sc.y);
        na.y = r2.c * a.y - (b.x * sc.y + b.y * sc.x);
        nb.x = r2.s * a.x + (b.x * cc.x - b.y * cc.y);
        nb.y = r2.s * a.y + (b.x * cc.y + b.y * cc.x);
        A[p1 + (int64_t)p2 * lda] = na;
        A[p1 + (int64_t)q2 * lda] = nb;
      } else {  // column p2 alone, rows {p1, q1} rotate by U1^H
        double2 a = A[p1 + (int64_t)p2 * lda], b = A[q1 + (int64_t)p2 * lda];
        const double2 sph = make_double2(r1.s * r1.ph.x, r1.s * r1.ph.y), cph = make_double2(r1.c * r1.ph.x, r1.c * r1.ph.y);
        double2 na, nb;
        na.x = r1.c * a.x - (sph.x * b.x - sph.y * b.y);
        na.y = r1.c * a.y - (sph.x * b.y + sph.y * b.x);
        nb.x = r1.s * a.x + (cph.x * b.x - cph.y * b.y);
        nb.y = r1.s * a.y + (cph.x * b.y + cph.y * b.x);
        A[p1 + (int64_t)p2 * lda] = na;
        A[q1 + (int64_t)p2 * lda] = nb;
      }
      return;
    }
    double2 m00 = A[p1 + (int64_t)p2 * lda], m10 = A[q1 + (int64_t)p2 * lda];
    double2 m01 = A[p1 + (int64_t)q2 * lda], m11 = A[q1 + (int64_t)q2 * lda];
    if (act1) {  // rows: [m0*; m1*] <- U1^H [m0*; m1*]
      const double2 sph = make_double2(r1.s * r1.ph.x, r1.s * r1.ph.y), cph = make_double2(r1.c * r1.ph.x, r1.c * r1.ph.y);
      double2 a0, a1;
      a0.x = r1.c * m00.x - (sph.x * m10.x - sph.y * m10.y);
      a0.y = r1.c * m00.y - (sph.x * m10.y + sph.y * m10.x);
      a1.x = r1.s * m00.x + (cph.x * m10.x - cph.y * m10.y);
      a1.y = r1.s * m00.y + (cph.x * m10.y + cph.y * m10.x);
      m00 = a0;
      m10 = a1;
      a0.x = r1.c * m01.x - (sph.x * m11.x - sph.y * m11.y);
      a0.y = r1.c * m01.y - (sph.x * m11.y + sph.y * m11.x);
      a1.x = r1.s * m01.x + (cph.x * m11.x - cph.y * m11.y);
      a1.y = r1.s * m01.y + (cph.x * m11.y + cph.y * m11.x);
      m01 = a0;
      m11 = a1;
    }
    if (act2) {  // columns: [m*0, m*1] <- [m*0, m*1] U2
      const double2 sc = make_double2(r2.s * r2.ph.x, -r2.s * r2.ph.y), cc = make_double2(r2.c * r2.ph.x, -r2.c * r2.ph.y);
      double2 b0, b1;
      b0.x = r2.c * m00.x - (m01.x * sc.x - m01.y * sc.y);
      b0.y = r2.c * m00.y - (m01.x * sc.y + m01.y * sc.x);
      b1.x = r2.s * m00.x + (m01.x * cc.x - m01.y * cc.y);
      b1.y = r2.s * m00.y + (m01.x * cc.y + m01.y * cc.x);
      m00 = b0;
      m01 = b1;
      b0.x = r2.c * m10.x - (m11.x * sc.x - m11.y * sc.y);
      b0.y = r2.c * m10.y - (m11.x * sc.y + m11.y * sc.x);
      b1.x = r2.s * m10.x + (m11.x * cc.x - m11.y * cc.y);
      b1.y = r2.s * m10.y + (m11.x * cc.y + m11.y * cc.x);
      m10 = b0;
      m11 = b1;
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
  const Rot r = rot[t];
  if (r.s == 0.0) return;
  const int p = pairs[2 * t];
  const double2 ap = V[i + (int64_t)p * ldv], aq = V[i + (int64_t)q * ldv];
  const double2 sc = make_double2(r.s * r.ph.x, -r.s * r.ph.y), cc = make_double2(r.c * r.ph.x, -r.c * r.ph.y);
  double2 np, nq;
  np.x = r.c * ap.x - (aq.x * sc.x - aq.y * sc.y);
  np.y = r.c * ap.y - (aq.x * sc.y + aq.y * sc.x);
  nq.x = r.s * ap.x + (aq.x * cc.x - aq.y * cc.y);
  nq.y = r.s * ap.y + (aq.x * cc.y + aq.y * cc.x);
  V[i + (int64_t)p * ldv] = np;
  V[i + (int64_t)q * ldv] = nq;
}

__global__ void k_jac_apply(int64_t h, int64_t n, double2* A, int64_t lda, double2* V, int64_t ldv,
                            const Rot* __restrict__ rot, const int* __restrict__ pairs) {
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  jac_apply_item(idx, h, n, A, lda, V, ldv, rot, pairs);
}

// Grid-wide barrier for a cooperative launch (all blocks resident).  The wait is bounded:
// after ~1 s it records CHEBFI_ERR_CUDA and lets the block go on.
__device__ __forceinline__ void grid_barrier(unsigned* count, unsigned* gen, unsigned nblocks, int* status) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned g = atomicAdd(gen, 0u);
    __threadfence();
    if (atomicAdd(count, 1u) == nblocks - 1) {
      atomicExch(count, 0u);
      __threadfence();
      atomicAdd(gen, 1u);
    } else {
      unsigned long long t0, t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
      while (atomicAdd(gen, 0u) == g) {
        __nanosleep(32);
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
        if (t - t0 > 1000000000ull) {
          flag_error(status, CHEBFI_ERR_CUDA);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
}

// All n-1 rounds of one Jacobi sweep in one cooperative launch: per round, the rotation
// parameters of the n/2 pairs, a grid barrier, the one-pass update of A and V, a barrier.
__global__ void k_jac_sweep(int64_t n0, int64_t n, double2* A, int64_t lda, double2* V, int64_t ldv, Rot* rot,
                            int* pairs, unsigned* bar, int* status) {
  const int64_t h = n / 2;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int64_t round = 0; round < n - 1; ++round) {
    // parameters (same arithmetic as k_jac_params)
    for (int64_t t = tid; t < h; t += nthreads) {
      int64_t p = rr_player(t, round, n), q = rr_player(n - 1 - t, round, n);
      if (p > q) {
        const int64_t tmp = p;
        p = q;
        q = tmp;
      }
      Rot r;
      r.c = 1.0;
      r.s = 0.0;
      r.ph = make_double2(1.0, 0.0);
      if (q < n0) {
        const double2 hh = A[p + q * lda];
        const double g = hypot(hh.x, hh.y);
        const double app = A[p + p * lda].x, aqq = A[q + q * lda].x;
        if (g > 1e-300 && g > 1.1102230246251565e-16 * sqrt(fabs(app * aqq))) {
          const double zeta = (aqq - app) / (2.0 * g);
          const double t_ = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + hypot(1.0, zeta));
          r.c = 1.0 / sqrt(1.0 + t_ * t_);
          r.s = t_ * r.c;
          r.ph = make_double2(hh.x / g, hh.y / g);
        }
      } else {
        q = -1;
      }
      rot[t] = r;
      pairs[2 * t] = (int)p;
      pairs[2 * t + 1] = (int)q;
    }
    grid_barrier(bar, bar + 1, gridDim.x, status);
    for (int64_t i = tid; i < h * h + n0 * h; i += nthreads) jac_apply_item(i, h, n0, A, lda, V, ldv, rot, pairs);
    grid_barrier(bar, bar + 1, gridDim.x, status);
  }
}

// out[0] = sum of |off-diagonal|^2, out[1] = total |A|^2 (single block, fixed order).
__global__ void k_offnorm(int64_t n, const double2* A, int64_t lda, double* out) {
  __shared__ double r0[256], r1[256];
  double s0 = 0, s1 = 0;
  for (int64_t e = threadIdx.x; e < n * n; e += blockDim.x) {
    const int64_t i = e % n, j = e / n;
    const double2 a = A[i + j * lda];
    const double v = a.x * a.x + a.y * a.y;
    s1 += v;
    if (i != j) s0 += v;
  }
  r0[threadIdx.x] = s0;
  r1[threadIdx.x] = s1;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if ((int)threadIdx.x < h) {
      r0[threadIdx.x] += r0[threadIdx.x + h];
      r1[threadIdx.x] += r1[threadIdx.x + h];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    out[0] = r0[0];
    out[1] = r1[0];
  }
}

// Sort eigenpairs ascending (stable): rank by counting, then permute w and the columns of V.
__global__ void k_eig_sort(int64_t n, const double2* __restrict__ A, int64_t lda, const double2* __restrict__ Vin,
                           int64_t ldvi, double* __restrict__ w, double2* __restrict__ Vout, int64_t ldvo) {
  const int64_t i = blockIdx.x;
  __shared__ int64_t rank;
  const double wi = A[i + i * lda].x;
  if (threadIdx.x == 0) rank = 0;
  __syncthreads();
  int64_t cnt = 0;
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    const double wj = A[j + j * lda].x;
    if (wj < wi || (wj == wi && j < i)) ++cnt;
  }
  atomicAdd((unsigned long long*)&rank, (unsigned long long)cnt);
  __syncthreads();
  const int64_t r = rank;
  if (threadIdx.x == 0) w[r] = wi;
  for (int64_t k = threadIdx.x; k < n; k += blockDim.x) Vout[k + r * ldvo] = Vin[k + i * ldvi];
}

}  // namespace

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
  if (n0 <= 0) return;
  if (n0 == 1) {
    set_identity(1, V, ldv, st);
    diag_of(1, A, lda, w, st);
    return;
  }
  const int64_t n = n0 + (n0 & 1);  // a padding player never paired for real
  // workspace: rotations, pair list, norms, and a copy of V for the final sort
  const size_t rot_c = (size_t)(n / 2) * sizeof(Rot) / sizeof(double2) + 1;
  const size_t pair_c = (size_t)n * sizeof(int) / sizeof(double2) + 1;
  const size_t vtmp = (size_t)n0 * n0;
  ws->alloc(rot_c + pair_c + 3 + vtmp);
  Rot* rot = reinterpret_cast<Rot*>(ws->p);
  int* pairs = reinterpret_cast<int*>(ws->p + rot_c);
  double* nrm = reinterpret_cast<double*>(ws->p + rot_c + pair_c);
  unsigned* bar = reinterpret_cast<unsigned*>(ws->p + rot_c + pair_c + 2);
  double2* Vtmp = ws->p + rot_c + pair_c + 3;
  CHEBFI_CUDA(cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st));
  // one cooperative launch per sweep when the device allows it (all blocks resident)
  int dev = 0, coop = 0, sms = 0, per_sm = 0;
  CHEBFI_CUDA(cudaGetDevice(&dev));
  CHEBFI_CUDA(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
  CHEBFI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CHEBFI_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jac_sweep, 256, 0));
  const int coop_blocks = std::min(sms * std::min(per_sm, 4), 1024);
  set_identity(n0, Vtmp, n0, st);
  const int max_sweeps = 40;
  double prev_off = INFINITY;
  bool done = false;
  for (int sweep = 0; sweep <= max_sweeps && !done; ++sweep) {
    CHEBFI_LAUNCH("k_offnorm", st, k_offnorm<<<1, 256, 0, st>>>(n0, A, lda, nrm));
    double h[2];
    CHEBFI_CUDA(cudaMemcpyAsync(h, nrm, sizeof(h), cudaMemcpyDeviceToHost, st));
    CHEBFI_CUDA(cudaStreamSynchronize(st));
    const double off = std::sqrt(h[0]), tot = std::sqrt(h[1]);
    // converged: off-diagonal at the rounding level, or no longer decreasing
    if (off <= 1e-15 * tot || off == 0.0 || (sweep > 2 && off > 0.5 * prev_off && off <= 1e-12 * tot)) {
      done = true;
      break;
    }
    if (sweep == max_sweeps) break;
    prev_off = off;
    if (coop && coop_blocks > 0) {
      int64_t n0a = n0, na = n, ldaa = lda, ldva = n0;
      double2* Aa = A;
      double2* Va = Vtmp;
      void* args[] = {&n0a, &na, &Aa, &ldaa, &Va, &ldva, &rot, &pairs, &bar, &status};
      CHEBFI_LAUNCH("k_jac_sweep", st,
                    CHEBFI_CUDA(cudaLaunchCooperativeKernel((const void*)k_jac_sweep, dim3(coop_blocks), dim3(256), args,
                                                            0, st)));
    } else {
      for (int64_t round = 0; round < n - 1; ++round) {
        CHEBFI_LAUNCH("k_jac_params", st, k_jac_params<<<nblk(n / 2), 256, 0, st>>>(n0, n, round, A, lda, rot, pairs));
        const int64_t h = n / 2;
        CHEBFI_LAUNCH("k_jac_apply", st,
                      k_jac_apply<<<nblk(h * h + n0 * h), 256, 0, st>>>(h, n0, A, lda, Vtmp, n0, rot, pairs));
      }
    }
  }
  if (!done) {
    int code = CHEBFI_ERR_NO_CONVERGENCE;
    // record on the device flag as well so chebfi_sync_status sees it
    CHEBFI_CUDA(cudaMemcpyAsync(status, &code, sizeof(int), cudaMemcpyHostToDevice, st));
    CHEBFI_CUDA(cudaStreamSynchronize(st));
  }
  CHEBFI_LAUNCH("k_eig_sort", st, k_eig_sort<<<(unsigned)n0, 128, 0, st>>>(n0, A, lda, Vtmp, n0, w, V, ldv));
}

}  // namespace chebfi
