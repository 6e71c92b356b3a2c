// Internal declarations shared by the translation units of libchebfi.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/chebfi.h"

namespace chebfi {

// ----------------------------------------------------------------------------- complex
template <typename R> struct cplx_t;
template <> struct cplx_t<double> { using type = double2; };
template <> struct cplx_t<float> { using type = float2; };
template <typename R> using cplx = typename cplx_t<R>::type;

template <typename C> __host__ __device__ __forceinline__ C cmake(double re, double im) {
  C z; z.x = (decltype(z.x))re; z.y = (decltype(z.y))im; return z;
}
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator*(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
// On the device a complex sum or difference is one packed FP32x2 instruction (sm_100 and up);
// the difference as b (-1) + a, exact in the product and rounded once like a subtraction.
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __fadd2_rn(a, b);
#else
  return make_float2(a.x + b.x, a.y + b.y);
#endif
}
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
#else
  return make_float2(a.x - b.x, a.y - b.y);
#endif
}
__host__ __device__ __forceinline__ float2 operator*(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ double2 conjg(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 conjg(float2 a) { return make_float2(a.x, -a.y); }

// ----------------------------------------------------------------------------- errors
struct Error {
  int code;
  std::string msg;
};

#define CHEBFI_CUDA(call)                                                                  \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      throw ::chebfi::Error{CHEBFI_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

#define CHEBFI_REQUIRE(cond, code, text)                                                   \
  do {                                                                                     \
    if (!(cond)) throw ::chebfi::Error{(code), (text)};                                    \
  } while (0)

// Checked kernel launch: counts the launch and turns a launch error into an exception.
void after_launch(const char* name);
// (per host thread: each thread driving its own context counts into that context)
extern thread_local int64_t* g_launch_counter;

// Optional per-kernel timing: CUDA events recorded on the launching stream around every
// launch while a context has profiling switched on (chebfi_profile_enable).
struct Profiler;
extern thread_local Profiler* g_prof;
// work: the launch's algorithmic flops (GEMMs) or bytes (FFT passes), summed per name.
void prof_begin(const char* name, cudaStream_t st, double work = 0.0);
void prof_end(cudaStream_t st);

#define CHEBFI_LAUNCH_W(name, st, work, ...) \
  do {                                       \
    ::chebfi::prof_begin(name, st, work);    \
    __VA_ARGS__;                             \
    ::chebfi::after_launch(name);            \
    ::chebfi::prof_end(st);                  \
  } while (0)
#define CHEBFI_LAUNCH(name, st, ...) CHEBFI_LAUNCH_W(name, st, 0.0, __VA_ARGS__)

// ----------------------------------------------------------------------------- device buffers
template <typename T> struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void alloc(size_t count) {  // discards contents
    if (count <= n && p) return;
    release();
    if (count == 0) return;
    cudaError_t e = cudaMalloc((void**)&p, count * sizeof(T));
    if (e != cudaSuccess) {
      p = nullptr;
      throw Error{CHEBFI_ERR_NOMEM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) +
                                        " bytes: " + cudaGetErrorString(e)};
    }
    n = count;
  }
  void upload(const T* host, size_t count, cudaStream_t s = 0) {
    alloc(count);
    if (count) CHEBFI_CUDA(cudaMemcpyAsync(p, host, count * sizeof(T), cudaMemcpyHostToDevice, s));
  }
};

// bf16 pair (hi, lo) of a K-major real matrix: row r (of the M or N dimension) starts at
// r * ld elements; x ~= hi + lo carries about 16 significant bits.
struct SplitBF16 {
  const __nv_bfloat16* hi = nullptr;
  const __nv_bfloat16* lo = nullptr;
  int64_t ld = 0;
};
struct SplitBF16Buf {
  DevBuf<__nv_bfloat16> hi, lo;
  int64_t ld = 0;
  void alloc(size_t count) {
    hi.alloc(count);
    lo.alloc(count);
  }
  SplitBF16 view() const { return SplitBF16{hi.p, lo.p, ld}; }
};

// Three bf16 (hi, lo) K-major planes of one complex operand for the three-multiplication
// complex GEMM (gemm_tc.cu): plane q of row r starts at q * plane + r * ld elements.
struct SplitBF16x3 {
  DevBuf<__nv_bfloat16> hi, lo;
  int64_t ld = 0, plane = 0;
  void alloc(int64_t rows, int64_t k) {
    ld = (k + 7) / 8 * 8;
    plane = ld * rows;
    hi.alloc((size_t)(3 * plane));
    lo.alloc((size_t)(3 * plane));
  }
  SplitBF16 view(int q) const { return SplitBF16{hi.p + q * plane, lo.p + q * plane, ld}; }
};

// One problem of a grouped tensor-core GEMM (gemm_tc.cu): D = alpha' A B + beta C with FP32
// column-major C / D, A and B given by the four bf16 tensor maps maps[4 map .. 4 map + 3]
// (A hi, A lo, B hi, B lo; boxes of 128 rows); alpha' = alpha, times the launch's alpha_mul
// when scale_alpha is set.
struct TcGroupProb {
  int M, N, K, map;
  float alpha, beta;
  int scale_alpha, pad;
  float* D;
  int64_t ldd;
  const float* C;
  int64_t ldc;
};

// Residues of a real-embedded complex operand for the modular tensor-core GEMM (ozaki.cu):
// one K-major bf16 matrix per modulus, res[mod * mstride + row * ld + k], and per complex
// row the power of two s applied before rounding to integers.
constexpr int kOzMinMod = 8, kOzMaxMod = 15;
constexpr int kOzBadShift = -0x40000000;  // shift of a row holding Inf or NaN
struct OzOperand {
  DevBuf<__nv_bfloat16> res;
  DevBuf<int32_t> shift;
  int64_t crows = 0;   // complex rows
  int64_t rows = 0;    // real rows (2 crows for the doubled A operand)
  int64_t kreal = 0;   // reals per row (2 K)
  int64_t ld = 0, mstride = 0;
  int nmod = 0;
};
struct OzWork {
  OzOperand A, B;
  DevBuf<signed char> R;  // residue matrices of the product
};

// ----------------------------------------------------------------------------- FFT plan
constexpr int kMaxStages = 12;
constexpr int kMaxN = 256;

template <typename R> struct FFTPlan {
  int n = 0;
  int nst = 0;
  int radix[kMaxStages] = {0};  // DIT stage order r_1 .. r_k
  const cplx<R>* tw = nullptr;  // tw[k] = exp(-2 pi i k / n)
};

struct FFTAxis {
  int n = 0;
  std::vector<int> radices;
  std::vector<int> rev;  // digit-reversed position of index i
  DevBuf<double2> tw64;
  DevBuf<float2> tw32;
  void build(int n_);
  template <typename R> FFTPlan<R> plan() const;
};

// Geometry of the pruned 3-pass FFT (sphere -> z lines -> planes -> z lines -> sphere).
struct SphereFFT {
  int n1 = 0, n2 = 0, n3 = 0;
  int ncol = 0;      // number of (x, y) columns holding sphere points
  int nxa = 0;       // number of x indices holding any column
  int pitch = 0;     // row pitch of a plane in shared memory (complex elements)
  int zpitch = 0;    // pitch of a z line in shared memory
  DevBuf<int32_t> col_start;   // ncol+1, sphere points of column c: [col_start[c], col_start[c+1])
  DevBuf<int32_t> pw_line;     // sorted sphere point -> column index
  DevBuf<int32_t> pw_zrev;     // sorted sphere point -> digit-reversed z position
  DevBuf<int32_t> col_off;     // column -> offset rev(x)*pitch + rev(y) in the plane
  DevBuf<int32_t> rows_act;    // active rows rev(x) of the plane (nxa)
  // natural-index maps of the compile-time-length path
  DevBuf<int32_t> pw_z;        // sorted sphere point -> z
  DevBuf<int32_t> col_off_nat; // column -> slot(x) * pitch + y, slot(x) = (x + n1/2) mod n1
  DevBuf<int32_t> rows_nat;    // slot(x) * pitch of the active rows, consecutive slots
  // the pruned plane pass works on the slot range [act_lo, act_lo + nact) that covers every
  // active row (for a sphere the active rows are that range)
  int act_lo = 0, nact = 0;
  DevBuf<int32_t> row_col;     // row act_lo + a, natural y -> column index, or -1 (nact x n2)
};

// Workspace grown on demand (never shrinks while the context lives).
struct Work {
  DevBuf<double2> Ya, Yb, Yc, Z, HY, T1, T2, tmp, tmp2;   // FP64 (npw x nb or grid)
  DevBuf<float2> fYa, fYb, fZ, fT1, fT2, ftmp;            // FP32 filter iterates
  DevBuf<double2> pa, pb, pc, pz, pw, pq, pt;             // nproj x nb projections (FP64)
  const double2* pc_of = nullptr;  // the block whose P^H Y is held in pc (set by Rayleigh-Ritz)
  DevBuf<double2> p0;              // a caller's P^H Y_0 repacked to leading dimension nproj
  DevBuf<float2> fpa, fpb, fpz, fpw, fpq, fpt;            // FP32 projections
  DevBuf<double2> small1, small2, small3, small4, small5;  // nb x nb
  // refined eigensolver: FP32 first stage, FP64 refinement matrices, stats, cluster pairs
  DevBuf<float2> e32a, e32b;
  DevBuf<float> e32w;
  DevBuf<double2> eG, eS, eAX, eM, eX, esub, eZ, eC1, eC2;
  DevBuf<double> elam, esw;
  DevBuf<unsigned long long> estats;
  DevBuf<int> enp, eidx;
  DevBuf<int2> epairs;
  DevBuf<double> dvec1, dvec2, dvec3;
  DevBuf<double2> splitk;
  DevBuf<float2> fsplitk;
  SplitBF16Buf Zb, Sb;  // bf16 pairs of Z (or Y) and of the projection-space operands
  SplitBF16x3 W3;       // (re, im, re + im) planes of W for the three-multiplication P W
  SplitBF16x3 gA3, gB3; // operand planes of chebfi_gemm_mixed
  DevBuf<float> tcws;   // K-split partial sums of the tensor-core GEMMs
  DevBuf<double2> gpool;          // filter backward: checkpoints, segment, adjoint iterates
  DevBuf<float2> fgT, fgR, fgG;   // FP32 backward: column buffer and real-space grids of the V gradient
  DevBuf<int32_t> order;          // band order of the locking filter
  DevBuf<float2> fgpool;
};

}  // namespace chebfi

namespace chebfi {
struct Profiler {
  bool on = false;
  struct Rec {
    const char* name;
    cudaEvent_t a, b;
    double work;
  };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  const char* cur = nullptr;
  cudaEvent_t cur_a = nullptr;
  double cur_work = 0.0;
  std::vector<std::string> names;
  std::vector<double> ms;
  std::vector<int64_t> count;
  std::vector<double> work;
  cudaEvent_t get();
  void flush();  // synchronises, folds pending records into the totals
  ~Profiler();
};
}  // namespace chebfi

struct chebfi_ctx {
  int device = 0;
  chebfi::Profiler prof;
  std::string err;
  int64_t launches = 0;

  bool has_cell = false, has_sphere = false, has_vloc = false, has_proj = false;
  double lattice[9] = {0}, recip[9] = {0}, kpt[3] = {0};
  int grid[3] = {0, 0, 0};
  chebfi::FFTAxis ax[3];

  int64_t npw = 0;
  std::vector<int32_t> sorted_to_user;  // host copy
  chebfi::DevBuf<int32_t> d_sorted_to_user;
  chebfi::SphereFFT sph;
  chebfi::DevBuf<double> d_K;
  chebfi::DevBuf<float> d_Kf;
  double kmax = 0.0;

  chebfi::DevBuf<double> d_vt;   // V_loc, plane-major [z][x][y]
  chebfi::DevBuf<float> d_vtf;
  bool fast_fft = false;         // cubic grid of a compiled size: two-pass FFT kernels
  chebfi::DevBuf<double> d_vs;   // V_loc in split order [z'][x'][y'] for those kernels
  chebfi::DevBuf<float> d_vsf;
  chebfi::DevBuf<float2> d_vsdf;               // the same table as double-float pairs (h, l)
  int fft64 = CHEBFI_FFT64_DOUBLE_FLOAT;       // arithmetic of the FP64 path's transforms
  double vmax = 0.0;

  int64_t nproj = 0;
  int natoms = 0;
  bool paw = false;
  std::vector<int32_t> offs;
  std::vector<double> h_Qblk;                 // host copy of the D_S (Q) blocks
  bool refine_ready = false;                  // A and B^{-1} of the iterative Woodbury solve
  chebfi::DevBuf<double2> d_Aref, d_Binv;     // A = D_S^{-1} + P^H P (dense), packed B^{-1} blocks
  chebfi::DevBuf<int64_t> d_cblk_off;         // atom -> offset of its complex block in d_Binv
  chebfi::DevBuf<int32_t> d_offs;
  chebfi::DevBuf<int32_t> d_atom_of;          // projector -> atom
  chebfi::DevBuf<double> d_Dblk, d_Qblk;      // packed blocks (row-major per atom)
  chebfi::DevBuf<int64_t> d_blk_off;          // atom -> offset of its block
  chebfi::DevBuf<double2> d_P, d_G, d_M, d_L; // P sorted rows (npw x nproj), G = P^H P, Woodbury M, chol(G)
  chebfi::DevBuf<float2> d_Pf, d_Gf, d_Mf;
  chebfi::DevBuf<float> d_Dblkf;
  chebfi::DevBuf<int> d_status;               // device error flag
  // mixed form: bf16 (hi, lo) real embeddings of P^H, P, G and M, built on first use
  bool tc_ready = false, tcP_ready = false;
  chebfi::SplitBF16Buf tcA1, tcA2, tcAG, tcAM;
  // (Re, Im, Re + Im) planes of P for the three-multiplication P W
  chebfi::SplitBF16x3 tcP3;
  bool tc3_ready = false;
  chebfi::Work w;
  // FP64 complex GEMMs: engine choice (chebfi_set_fp64_gemm), modulus count of the
  // tensor-core emulation, its workspace, and the residues of P^H and P (built on first use)
  int fp64_gemm = CHEBFI_GEMM_AUTO;
  int eig_mode = CHEBFI_EIG_AUTO;  // dense eigensolver of Rayleigh-Ritz (chebfi_set_eigensolver)
  int eig_iters = 0;               // refinement steps of its last call (0: FP64 Jacobi ran)
  int oz_nmod = 14;
  chebfi::OzWork oz;
  chebfi::OzOperand ozPh, ozP;
  double bound_rigorous = -1.0;
  double smin = 1.0;  // lower bound of lambda_min(S), set with bound_rigorous
  // host-block filter: staging buffers, copy streams and their events (created on first use)
  chebfi::DevBuf<double2> stage[2];
  chebfi::DevBuf<double2> stage_p[2];  // the host filter's projection chunks
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_filt[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  ~chebfi_ctx() {
    for (int i = 0; i < 2; ++i) {
      if (ev_in[i]) cudaEventDestroy(ev_in[i]);
      if (ev_filt[i]) cudaEventDestroy(ev_filt[i]);
      if (ev_out[i]) cudaEventDestroy(ev_out[i]);
    }
    if (copy_in) cudaStreamDestroy(copy_in);
    if (copy_out) cudaStreamDestroy(copy_out);
  }
  int last_sweeps = 0;            // sweeps performed by the last chebfi_solve
  int64_t last_applies = 0;       // band-H-applications of its filters
};
