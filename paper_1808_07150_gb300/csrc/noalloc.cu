// Subset backprojection that allocates no device memory.
//
// Some callers cannot let a library call cudaMalloc: runtimes whose device memory is owned by
// their own pool or arena with a hard budget, and latency-critical loops where cudaMalloc /
// cudaFree would synchronise the device.  spdhg_backproject keeps its gathered sinogram in a
// buffer the context allocates on first use; this variant keeps that scratch in a fixed
// file-scope device array instead, so the call itself allocates nothing.
#include "internal.cuh"

using namespace spdhg;

namespace {

// Scratch for the subset-local sinogram mult * y: room for 2^21 bins (8 MiB).  Every device that
// loads the library holds this array until the process exits.
constexpr int64_t kNoallocScratchFloats = int64_t(1) << 21;
static __device__ __align__(256) float g_noalloc_scratch[kNoallocScratchFloats];

// Device address of the scratch array on the current device (host code only sees a stand-in
// symbol).  Looked up on every call, with the context's device current: the lookup is cheap, and
// an address cached across calls would go stale if the device's primary context were reset.
cudaError_t scratch_address(float** out) {
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<float*>(p);
  return cudaSuccess;
}

}  // namespace

extern "C" int spdhg_backproject_noalloc(spdhg_ctx* ctx, const float* y, float* x, int subset, void* stream) {
  if (!ctx || !x || !y) return SPDHG_ERR_ARG;
  if (subset < 0 || subset >= ctx->geom.n_subsets) {
    ctx->err = "spdhg_backproject_noalloc: subset must be in [0, n_subsets)";
    return SPDHG_ERR_ARG;
  }
  const int64_t bins = (int64_t)subset_views(ctx->dg, subset) * ctx->dg.R * ctx->dg.P;
  if (bins > kNoallocScratchFloats) {
    ctx->err = "spdhg_backproject_noalloc: the subset has " + std::to_string(bins) +
               " bins, more than the fixed scratch of " + std::to_string(kNoallocScratchFloats) + " floats";
    return SPDHG_ERR_ARG;
  }
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess && dev != ctx->device) {
    ctx->err = "spdhg_backproject_noalloc: current CUDA device differs from the context's device";
    return SPDHG_ERR_STATE;
  }
  float* scratch = nullptr;
  if (e == cudaSuccess) e = scratch_address(&scratch);
  if (e != cudaSuccess) {
    ctx->err = std::string("spdhg_backproject_noalloc: ") + cudaGetErrorString(e);
    return SPDHG_ERR_CUDA;
  }
  cudaStream_t s = (cudaStream_t)stream;
  // every scratch entry the backprojection reads is written by the gather first
  e = launch_gather_subset(ctx->dg, subset, y, ctx->has_mult ? ctx->mult : nullptr, scratch, s);
  if (e == cudaSuccess) {
    BwdArgs a{};
    a.w = scratch;
    a.out = x;
    e = launch_backward(ctx->dg, subset, BWD_OUT, a, s);
  }
  if (e != cudaSuccess) {
    ctx->err = std::string("spdhg_backproject_noalloc: ") + cudaGetErrorString(e);
    return SPDHG_ERR_CUDA;
  }
  return SPDHG_OK;
}
