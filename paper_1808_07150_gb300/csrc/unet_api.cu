// C ABI of the learned warm start (include/unet.h): the tensor-core GEMM entry point.
#include <cuda_bf16.h>

#include "../../include/unet.h"
#include "igemm.cuh"

using namespace spdhg;

extern "C" int unet_gemm(const uint16_t* a, const uint16_t* b, float* d, int M, int N, int K, int flags,
                         void* stream) {
  if (!a || !b || !d || M <= 0 || N < 16 || N > 256 || (N & 15) || K <= 0 || (K & 7)) return UNET_ERR_ARG;
  const bool a_mn = flags & UNET_GEMM_A_MN, b_mn = flags & UNET_GEMM_B_MN;
  if ((a_mn && (M & 7)) || (!a_mn && (K & 7))) return UNET_ERR_ARG;
  ig::GemmArgs g{};
  g.M = M;
  g.N = N;
  g.K = K;
  g.a = reinterpret_cast<const __nv_bfloat16*>(a);
  g.a_stride = a_mn ? M : K;
  g.b = reinterpret_cast<const __nv_bfloat16*>(b);
  g.b_stride = b_mn ? N : K;
  g.outf = d;
  dim3 grid((M + 127) / 128, 1, 1);
  cudaError_t e = ig::launch(a_mn ? ig::A_GEMM_MN : ig::A_GEMM_K, b_mn ? ig::B_GEMM_MN : ig::B_GEMM_K, ig::E_F32, g,
                             grid, (cudaStream_t)stream);
  return e == cudaSuccess ? UNET_OK : UNET_ERR_CUDA;
}

extern "C" int unet_device_error(void* stream) {
  const int e = ig::read_error((cudaStream_t)stream);
  return e < 0 ? UNET_ERR_CUDA : (e ? UNET_ERR_TIMEOUT : UNET_OK);
}
