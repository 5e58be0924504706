// Implicit-GEMM tensor-core kernel (igemm.cu): modes and arguments.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace spdhg {
namespace ig {

// A operand (rows of D, reduction k)
enum AMode {
  A_GEMM_K = 0,    // A[m][k] at a + m * a_stride + k                         (K-major)
  A_GEMM_MN = 1,   // A[m][k] at a + k * a_stride + m                         (MN-major)
  A_CONV3 = 2,     // rows = voxels v of (ny, nx, nz); k = tap * a_c + c: in[v + tap - 1][c]
  A_ROWS = 3,      // rows = voxels v; k = c: in[v][c]
  A_CHILD8 = 4,    // rows = coarse voxels p; k = o * a_c + c: in[child(p, o)][c] on the 2x grid
  A_WG_CONV3 = 5,  // rows = tap * a_c + c, k = voxel v: in[v + tap - 1][c]   (MN-major)
  A_WG_TCONV = 6,  // rows = c, k = coarse voxel p: in[p][c]                  (MN-major)
};
// B operand (columns of D, reduction k)
enum BMode {
  B_GEMM_K = 0,    // B[n][k] at b + z * b_zstride + n * b_stride + k        (K-major)
  B_GEMM_MN = 1,   // B[n][k] at b + k * b_stride + n                         (MN-major)
  B_WG_ROWS = 2,   // n = c, k = voxel v: g[v][c]                             (MN-major)
  B_WG_CHILD = 3,  // n = c, k = coarse voxel p: g[child(p, z)][c]            (MN-major)
};
// epilogue
enum EMode {
  E_BF16 = 0,      // out[row][off + n] = bf16(mask ? relu?(D + bias) : 0)
  E_F32 = 1,       // outf[row * N + n] = relu?(D + bias), masked
  E_PART = 2,      // outf[((z * splits + split) * M + m) * N + n] = partial D over a k range
};

struct GemmArgs {
  int M, N, K;                 // D is M x N, reduction length K (multiple of 8; N multiple of 16)
  const __nv_bfloat16* a; int a_stride, a_off, a_c;
  const __nv_bfloat16* b; int b_stride, b_off; long long b_zstride;
  int ny, nx, nz;              // voxel grid of the A rows (the coarse grid in child modes)
  const float* bias;
  int relu;
  __nv_bfloat16* out; int out_stride, out_off;
  float* outf;
  const __nv_bfloat16* mask; int mask_stride, mask_off;  // zero where mask <= 0 (ReLU gradient)
  int mask_from;               // columns below this one are not masked
  int out_child;               // rows go to child(row, blockIdx.z) on the 2x grid
  int k_per_split;             // E_PART: reduction elements per blockIdx.y (multiple of 64)
};

cudaError_t launch(int am, int bm, int em, const GemmArgs& g, dim3 grid, cudaStream_t s);
// 3x3x3 convolution (A_CONV3 operands, B = weights [N][27 a_c]) from a staged input halo with the
// taps as shifted shared-memory descriptors; cudaErrorNotSupported when the shape does not fit
// (a_c in {16, 32}, N <= 64, nx % 16 == 0, nz % 8 == 0), in which case launch() serves it
cudaError_t launch_conv3_halo(int em, const GemmArgs& g, cudaStream_t s);
// first failure code recorded by any launch (0: none); synchronises s
int read_error(cudaStream_t s);

}  // namespace ig
}  // namespace spdhg
