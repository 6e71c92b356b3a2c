// Diagnostics of the library on the device it runs on.
//
// Bounded waits: the grid barrier of the cooperative Jacobi sweep and the mbarrier waits of
// the tensor-core pipelines.  Each test waits for something that nothing will ever provide
// (a barrier one block never reaches, an mbarrier arrival nobody makes), so the wait must
// run out after its limit, record CHEBFI_ERR_CUDA on the device and let the kernel finish;
// the context stays usable.
//
// FMA rate: eight independent FMA chains per thread over the whole device, timed with CUDA
// events -- the measured FP64 and FP32 peaks the roofline fractions of the CUDA-core kernels
// (Jacobi, the SIMT GEMMs, the FFT passes) are taken against.
#include "grid_barrier.cuh"
#include "internal.cuh"
#include "tc_ptx.cuh"

namespace chebfi {
namespace {

// block 0 returns at once; the others meet at the grid barrier and give up after limit_ns
__global__ void k_wait_barrier(unsigned* bar, int* status, unsigned long long limit_ns) {
  if (blockIdx.x == 0) return;
  grid_barrier(bar, bar + 1, gridDim.x, status, limit_ns);
}

// an mbarrier expecting one arrival that never comes
__global__ void k_wait_mbarrier(int* status, unsigned long long limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    tc::mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !tc::mbar_wait_ns(&bar, 0, limit_ns)) atomicCAS(status, 0, CHEBFI_ERR_CUDA);
}

// 8 chains x 16 unrolled FMAs per iteration; the sum is stored so nothing is dead code
template <typename R> __global__ void k_fma_rate(R* out, int iters) {
  R a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = (R)(threadIdx.x + c) * (R)1e-3;
  const R b = (R)0.9999999, d = (R)1e-7;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int c = 0; c < 8; ++c) a[c] = fma(a[c], b, d);
    }
  }
  R s = 0;
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace chebfi

using namespace chebfi;

extern "C" int chebfi_probe_fma_rate(chebfi_ctx* ctx, int prec, double* tflops, double* ms_out) {
  if (!ctx) return CHEBFI_ERR_ARG;
  try {
    ctx->err.clear();
    CHEBFI_REQUIRE(prec == CHEBFI_F64 || prec == CHEBFI_F32, CHEBFI_ERR_ARG, "prec: CHEBFI_F64 or CHEBFI_F32");
    CHEBFI_CUDA(cudaSetDevice(ctx->device));
    int sms = 0;
    CHEBFI_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
    const int threads = 256, blocks = sms * 8;
    // about 0.2 s of work at each form's rate on this part
    const int iters = prec == CHEBFI_F64 ? 2000 : 100000;
    DevBuf<double> out;
    out.alloc((size_t)blocks * threads);
    cudaEvent_t a, b;
    CHEBFI_CUDA(cudaEventCreate(&a));
    CHEBFI_CUDA(cudaEventCreate(&b));
    float ms = 0.f;
    for (int rep = 0; rep < 2; ++rep) {  // the first run warms up clocks and caches
      CHEBFI_CUDA(cudaEventRecord(a, 0));
      if (prec == CHEBFI_F64) k_fma_rate<double><<<blocks, threads>>>(out.p, iters);
      else k_fma_rate<float><<<blocks, threads>>>(reinterpret_cast<float*>(out.p), iters);
      CHEBFI_CUDA(cudaGetLastError());
      CHEBFI_CUDA(cudaEventRecord(b, 0));
      CHEBFI_CUDA(cudaEventSynchronize(b));
      CHEBFI_CUDA(cudaEventElapsedTime(&ms, a, b));
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    ctx->launches += 2;
    const double flops = 2.0 * 8 * 16 * (double)iters * blocks * threads;
    if (tflops) *tflops = flops / (ms * 1e-3) / 1e12;
    if (ms_out) *ms_out = ms;
  } catch (const Error& e) {
    ctx->err = e.msg;
    return e.code;
  }
  return CHEBFI_OK;
}

extern "C" int chebfi_selftest_bounded_wait(chebfi_ctx* ctx, int which, double limit_ms, int* recorded,
                                            double* elapsed_ms) {
  if (!ctx) return CHEBFI_ERR_ARG;
  try {
    ctx->err.clear();
    CHEBFI_REQUIRE(which == 0 || which == 1, CHEBFI_ERR_ARG, "which: 0 grid barrier, 1 mbarrier");
    CHEBFI_REQUIRE(limit_ms > 0.0 && limit_ms <= 2000.0, CHEBFI_ERR_ARG, "limit must be in (0, 2000] ms");
    CHEBFI_CUDA(cudaSetDevice(ctx->device));
    DevBuf<unsigned> buf;  // barrier counter, generation, status word
    buf.alloc(3);
    CHEBFI_CUDA(cudaMemset(buf.p, 0, 3 * sizeof(unsigned)));
    int* status = reinterpret_cast<int*>(buf.p + 2);
    const unsigned long long limit_ns = (unsigned long long)(limit_ms * 1e6);
    cudaEvent_t a, b;
    CHEBFI_CUDA(cudaEventCreate(&a));
    CHEBFI_CUDA(cudaEventCreate(&b));
    CHEBFI_CUDA(cudaEventRecord(a, 0));
    if (which == 0) k_wait_barrier<<<4, 64>>>(buf.p, status, limit_ns);
    else k_wait_mbarrier<<<1, 32>>>(status, limit_ns);
    CHEBFI_CUDA(cudaGetLastError());
    CHEBFI_CUDA(cudaEventRecord(b, 0));
    CHEBFI_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    CHEBFI_CUDA(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    int h = 0;
    CHEBFI_CUDA(cudaMemcpy(&h, status, sizeof(int), cudaMemcpyDeviceToHost));
    if (recorded) *recorded = h;
    if (elapsed_ms) *elapsed_ms = ms;
    ctx->launches += 1;
  } catch (const Error& e) {
    ctx->err = e.msg;
    return e.code;
  }
  return CHEBFI_OK;
}
