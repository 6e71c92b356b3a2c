// Allocation-free application of H, for callers that cannot allocate device memory at
// the point of use: code inside a host callback or a latency-critical section that must
// not take the CUDA allocator's lock, frameworks that hand out every byte of device memory
// through their own pool and forbid outside allocations, and processes that have already
// reserved all of it.
//
// Everything this entry point needs beyond its inputs and outputs lives in one
// file-scope __device__ array of fixed size.  The context must have been set up before
// (its setters allocate); this call itself allocates nothing.
#include <map>
#include <mutex>

#include "internal.cuh"
#include "kernels.cuh"

namespace chebfi {
namespace {

// 32 MiB (2^21 complex doubles).  Every GPU that loads the library holds this array
// until the process exits.
constexpr size_t kScratchElems = (size_t)1 << 21;
__device__ __align__(256) double2 g_apply_h_scratch[kScratchElems];

// In host code the name g_apply_h_scratch is only a host-side stand-in; the device
// address is looked up once per device, with that device current.
std::mutex g_scratch_mu;
std::map<int, double2*> g_scratch_addr;

double2* scratch_for(int device) {
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  auto it = g_scratch_addr.find(device);
  if (it != g_scratch_addr.end()) return it->second;
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_apply_h_scratch);
  CHEBFI_REQUIRE(e == cudaSuccess && p != nullptr, CHEBFI_ERR_CUDA,
                 std::string("cudaGetSymbolAddress of the static scratch: ") + cudaGetErrorString(e));
  g_scratch_addr[device] = static_cast<double2*>(p);
  return static_cast<double2*>(p);
}

}  // namespace
}  // namespace chebfi

using namespace chebfi;

extern "C" int chebfi_apply_H_noalloc(chebfi_ctx* ctx, const void* Y, void* HY, int64_t nb, int64_t ld,
                                      void* stream) {
  if (!ctx) return CHEBFI_ERR_ARG;
  try {
    ctx->err.clear();
    g_launch_counter = &ctx->launches;
    g_prof = &ctx->prof;
    CHEBFI_CUDA(cudaSetDevice(ctx->device));
    CHEBFI_REQUIRE(ctx->has_cell && ctx->has_sphere && ctx->has_vloc && ctx->has_proj, CHEBFI_ERR_STATE,
                   "set_cell, set_sphere, set_vloc and set_projectors must all be called first");
    CHEBFI_REQUIRE(nb >= 0 && ld >= ctx->npw, CHEBFI_ERR_ARG, "need nb >= 0 and ld >= npw");
    CHEBFI_REQUIRE(nb == 0 || (Y && HY), CHEBFI_ERR_ARG, "null Y or HY");
    if (nb == 0) return CHEBFI_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    const int64_t npw = ctx->npw, nq = ctx->nproj;
    // per band: FFT column buffer, Y and HY in sorted order, projections and D p
    const size_t col = local_workspace_elems(ctx, 1);
    const size_t per_band = col + 2 * (size_t)npw + 2 * (size_t)nq;
    CHEBFI_REQUIRE(per_band <= kScratchElems, CHEBFI_ERR_ARG,
                   "one band needs " + std::to_string(per_band * sizeof(double2)) +
                       " bytes of scratch, more than the 32 MiB static array of chebfi_apply_H_noalloc");
    double2* s = scratch_for(ctx->device);
    const int64_t chunk = (int64_t)(kScratchElems / per_band);
    for (int64_t b0 = 0; b0 < nb; b0 += chunk) {
      const int64_t n = std::min(chunk, nb - b0);
      double2* T = s;
      double2* Ys = T + col * n;
      double2* Hs = Ys + npw * n;
      double2* p = Hs + npw * n;
      double2* Dp = p + nq * n;
      // every scratch region is fully written before it is read, so nothing is cleared
      gather_rows(npw, n, ctx->d_sorted_to_user.p, (const double2*)Y + b0 * ld, ld, Ys, npw, st);
      LocalEpi<double> ep;
      ep.Y = Ys;
      ep.ldy = npw;
      ep.Z = Hs;
      ep.ldz = npw;
      local_apply<double>(ctx, Ys, npw, n, T, ep, st);
      if (nq > 0) {
        gemm<double>(true, false, nq, n, npw, 1.0, ctx->d_P.p, npw, Ys, npw, 0.0, p, nq, st, nullptr, "gemm_H");
        blockdiag_apply<double>(ctx, ctx->d_Dblk.p, p, nq, Dp, nq, n, st);
        gemm<double>(false, false, npw, n, nq, 1.0, ctx->d_P.p, npw, Dp, nq, 1.0, Hs, npw, st, nullptr, "gemm_H");
      }
      scatter_rows(npw, n, ctx->d_sorted_to_user.p, Hs, npw, (double2*)HY + b0 * ld, ld, st);
    }
  } catch (const Error& e) {
    ctx->err = e.msg;
    return e.code;
  } catch (const std::exception& e) {
    ctx->err = e.what();
    return CHEBFI_ERR_CUDA;
  }
  return CHEBFI_OK;
}
