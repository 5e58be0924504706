// Implicit-GEMM tensor-core kernel (tcgen05, BF16 x BF16 -> FP32 in TMEM) behind every
// convolution of the learned warm start (3x3x3 convolution, 2x2x2 transposed convolution, their
// data and weight gradients) and a plain GEMM used to check the operand layouts.
//
// One CTA computes a 128 x N tile of D = A B^T (N = output channels, 16..256, a multiple of 16).
// The reduction runs in chunks of 64 elements through a two-stage shared-memory ring: all 128
// threads stage the chunk's A (128 x 64) and B (N x 64) tiles with 16-byte cp.async copies
// (zero-filled outside the volume, so padding costs no branch in the MMA), one thread issues four
// tcgen05.mma (K = 16 each) and commits them to the stage's mbarrier, and the ring slot is reused
// once that mbarrier reports the MMAs that read it complete.  The epilogue reads the accumulator
// from TMEM (tcgen05.ld, one row per thread) and applies bias, ReLU and a ReLU-gradient mask.
//
// Operands are gathered from channels-last BF16 tensors (element (v, c) at p[v * stride + off + c]):
//   K-major operands hold 8 consecutive reduction elements per 16-byte chunk (channels of one
//   voxel); MN-major operands hold 8 consecutive rows/columns at one reduction index (again the
//   channels of one voxel), which is what the weight gradients need (reduction over voxels).
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>

#include "igemm.cuh"
#include "umma.cuh"

namespace spdhg {
namespace ig {

constexpr int BM = 128;     // rows per CTA tile
constexpr int BK = 64;      // reduction elements per stage
constexpr int STAGES = 2;
constexpr int THREADS = 128;
constexpr long long WAIT_CYCLES = 4000000000ll;  // ~2 s at 2 GHz: a lost completion ends the kernel

__device__ int g_error;     // first failure code of any launch (0 = none)

struct Vox {
  int y, x, z;
};
__device__ __forceinline__ Vox decomp(int v, int nx, int nz) {
  Vox r;
  r.z = v % nz;
  const int t = v / nz;
  r.x = t % nx;
  r.y = t / nx;
  return r;
}

// ---- operand chunk addressing: returns the source pointer and whether the chunk exists ----

// A, K-major: chunk (row r, k-block kb) = A[r][8 kb .. 8 kb + 7]
template <int AM>
__device__ __forceinline__ const __nv_bfloat16* a_chunk_k(const GemmArgs& g, int r, int kb, bool& ok) {
  ok = false;
  if (r >= g.M || kb * 8 >= g.K) return g.a;
  if (AM == A_GEMM_K) {
    ok = true;
    return g.a + (size_t)r * g.a_stride + kb * 8;
  } else if (AM == A_ROWS) {
    ok = true;
    return g.a + (size_t)r * g.a_stride + g.a_off + kb * 8;
  } else if (AM == A_CONV3) {
    const int c8 = g.a_c >> 3;
    const int tap = kb / c8, cg = kb - tap * c8;
    const Vox p = decomp(r, g.nx, g.nz);
    const int yy = p.y + tap / 9 - 1, xx = p.x + (tap / 3) % 3 - 1, zz = p.z + tap % 3 - 1;
    if (yy < 0 || yy >= g.ny || xx < 0 || xx >= g.nx || zz < 0 || zz >= g.nz) return g.a;
    ok = true;
    return g.a + ((size_t)(yy * g.nx + xx) * g.nz + zz) * g.a_stride + g.a_off + cg * 8;
  } else {  // A_CHILD8: child o of coarse voxel r on the grid (2 ny, 2 nx, 2 nz)
    const int c8 = g.a_c >> 3;
    const int o = kb / c8, cg = kb - o * c8;
    const Vox p = decomp(r, g.nx, g.nz);
    const int fy = 2 * p.y + (o >> 2), fx = 2 * p.x + ((o >> 1) & 1), fz = 2 * p.z + (o & 1);
    ok = true;
    return g.a + ((size_t)(fy * 2 * g.nx + fx) * (2 * g.nz) + fz) * g.a_stride + g.a_off + cg * 8;
  }
}

// A, MN-major: chunk (reduction index k, row block mb) = A[8 mb .. 8 mb + 7][k]
template <int AM>
__device__ __forceinline__ const __nv_bfloat16* a_chunk_mn(const GemmArgs& g, int k, int mb, int kend, bool& ok) {
  ok = false;
  const int m0 = mb * 8;
  if (m0 >= g.M || k >= kend) return g.a;
  if (AM == A_GEMM_MN) {
    ok = true;
    return g.a + (size_t)k * g.a_stride + m0;
  } else if (AM == A_WG_CONV3) {  // rows (tap, c), reduction over voxels v = k
    const int tap = m0 / g.a_c, c0 = m0 - tap * g.a_c;
    const Vox p = decomp(k, g.nx, g.nz);
    const int yy = p.y + tap / 9 - 1, xx = p.x + (tap / 3) % 3 - 1, zz = p.z + tap % 3 - 1;
    if (yy < 0 || yy >= g.ny || xx < 0 || xx >= g.nx || zz < 0 || zz >= g.nz) return g.a;
    ok = true;
    return g.a + ((size_t)(yy * g.nx + xx) * g.nz + zz) * g.a_stride + g.a_off + c0;
  } else {  // A_WG_TCONV: rows c, reduction over coarse voxels p = k
    ok = true;
    return g.a + (size_t)k * g.a_stride + g.a_off + m0;
  }
}

// B, K-major: chunk (column n, k-block kb) = B[n][8 kb ..]; per-z weight slices at b_zstride
template <int BMODE>
__device__ __forceinline__ const __nv_bfloat16* b_chunk_k(const GemmArgs& g, int n, int kb, bool& ok) {
  ok = n < g.N && kb * 8 < g.K;
  if (!ok) return g.b;
  return g.b + (size_t)blockIdx.z * g.b_zstride + (size_t)n * g.b_stride + kb * 8;
}

// B, MN-major: chunk (reduction index k, column block nb) = B[8 nb .. 8 nb + 7][k]
template <int BMODE>
__device__ __forceinline__ const __nv_bfloat16* b_chunk_mn(const GemmArgs& g, int k, int nb, int kend, bool& ok) {
  ok = false;
  const int n0 = nb * 8;
  if (n0 >= g.N || k >= kend) return g.b;
  if (BMODE == B_GEMM_MN) {
    ok = true;
    return g.b + (size_t)k * g.b_stride + n0;
  } else if (BMODE == B_WG_ROWS) {
    ok = true;
    return g.b + (size_t)k * g.b_stride + g.b_off + n0;
  } else {  // B_WG_CHILD: gradient at child o = blockIdx.z of coarse voxel k
    const int o = blockIdx.z;
    const Vox p = decomp(k, g.nx, g.nz);
    const int fy = 2 * p.y + (o >> 2), fx = 2 * p.x + ((o >> 1) & 1), fz = 2 * p.z + (o & 1);
    ok = true;
    return g.b + ((size_t)(fy * 2 * g.nx + fx) * (2 * g.nz) + fz) * g.b_stride + g.b_off + n0;
  }
}

__device__ __forceinline__ void set_error(int code) { atomicCAS(&g_error, 0, code); }

template <int AM, int BMODE, int EM>
__global__ void __launch_bounds__(THREADS) k_igemm(GemmArgs g) {
  constexpr bool A_MN = (AM == A_GEMM_MN || AM == A_WG_CONV3 || AM == A_WG_TCONV);
  constexpr bool B_MN = (BMODE == B_GEMM_MN || BMODE == B_WG_ROWS || BMODE == B_WG_CHILD);
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ uint64_t mbar[STAGES];
  __shared__ uint32_t tmem_slot;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int NP = (g.N + 15) & ~15;                     // columns of the MMA (multiple of 16)
  const uint32_t a_bytes = BM * BK * 2, b_bytes = (uint32_t)NP * BK * 2;
  const uint32_t sbase = umma::smem_u32(smem);
  const int row0 = blockIdx.x * BM;
  // reduction range of this CTA (split over blockIdx.y for partial sums)
  const int kbeg = (EM == E_PART) ? blockIdx.y * g.k_per_split : 0;
  const int kend = (EM == E_PART) ? min(g.K, kbeg + g.k_per_split) : g.K;
  const int ktiles = kend > kbeg ? (kend - kbeg + BK - 1) / BK : 0;
  uint32_t ncols = 32;
  while ((int)ncols < NP) ncols <<= 1;

  if (warp == 0) umma::tmem_alloc(&tmem_slot, ncols);
  if (tid == 0) {
    for (int s = 0; s < STAGES; ++s) umma::mbar_init(&mbar[s], 1);
    umma::fence_mbar_init();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tmem = tmem_slot;

  // no-swizzle core-matrix layouts (8 rows x 16 bytes per core matrix):
  //   K-major tile:  core (row block rb, k block kb) at (rb * 8 + kb) * 128   -> LBO 128, SBO 1024
  //   MN-major tile: core (k block kb, row block rb) at (kb * R/8 + rb) * 128 -> LBO R*16, SBO 128
  const uint32_t a_lbo = A_MN ? (uint32_t)BM * 16 : 128u, a_sbo = A_MN ? 128u : 1024u;
  const uint32_t b_lbo = B_MN ? (uint32_t)NP * 16 : 128u, b_sbo = B_MN ? 128u : 1024u;
  const uint32_t a_kstep = A_MN ? 2u * BM * 16 : 256u;  // bytes between K = 16 slices
  const uint32_t b_kstep = B_MN ? 2u * NP * 16 : 256u;
  const uint32_t idesc = umma::idesc_bf16(BM, NP, A_MN, B_MN);

  bool failed = false;
  for (int kt = 0; kt < ktiles; ++kt) {
    const int s = kt % STAGES;
    if (kt >= STAGES) {
      const bool ok = umma::mbar_wait(&mbar[s], ((kt / STAGES) - 1) & 1, WAIT_CYCLES);
      if (__syncthreads_or(!ok)) {  // the whole block leaves together
        failed = true;
        break;
      }
    }
    const uint32_t sa = sbase + s * (a_bytes + b_bytes), sb = sa + a_bytes;
    const int k0 = kbeg + kt * BK;
    // stage A: 1024 chunks
    for (int idx = tid; idx < BM * 8; idx += THREADS) {
      bool ok;
      const __nv_bfloat16* src;
      uint32_t dst;
      if (!A_MN) {
        const int i = idx & (BM - 1), j = idx >> 7;  // row, k block
        src = a_chunk_k<AM>(g, row0 + i, (k0 >> 3) + j, ok);
        if (k0 + j * 8 >= kend) ok = false;
        dst = sa + ((i >> 3) * 8 + j) * 128 + (i & 7) * 16;
      } else {
        const int kk = idx & (BK - 1), rb = idx >> 6;  // reduction index, row block
        src = a_chunk_mn<AM>(g, k0 + kk, (row0 >> 3) + rb, kend, ok);
        dst = sa + ((kk >> 3) * (BM / 8) + rb) * 128 + (kk & 7) * 16;
      }
      umma::cp16(dst, src, ok ? 16u : 0u);
    }
    // stage B: NP * 8 chunks
    for (int idx = tid; idx < NP * 8; idx += THREADS) {
      bool ok;
      const __nv_bfloat16* src;
      uint32_t dst;
      if (!B_MN) {
        const int i = idx % NP, j = idx / NP;
        src = b_chunk_k<BMODE>(g, i, (k0 >> 3) + j, ok);
        if (k0 + j * 8 >= kend) ok = false;
        dst = sb + ((i >> 3) * 8 + j) * 128 + (i & 7) * 16;
      } else {
        const int kk = idx & (BK - 1), nb = idx >> 6;
        src = b_chunk_mn<BMODE>(g, k0 + kk, nb, kend, ok);
        dst = sb + ((kk >> 3) * (NP / 8) + nb) * 128 + (kk & 7) * 16;
      }
      umma::cp16(dst, src, ok ? 16u : 0u);
    }
    umma::cp_commit_wait_all();
    umma::fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      umma::fence_after_sync();
#pragma unroll
      for (int kk = 0; kk < BK / 16; ++kk) {
        const uint64_t ad = umma::smem_desc(sa + kk * a_kstep, a_lbo, a_sbo);
        const uint64_t bd = umma::smem_desc(sb + kk * b_kstep, b_lbo, b_sbo);
        umma::mma_bf16(tmem, ad, bd, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
      }
      umma::commit(&mbar[s]);
    }
  }
  // every MMA of the tile completes before the last commit's mbarrier phase
  if (!failed && ktiles > 0) {
    const int last = ktiles - 1;
    const bool ok = umma::mbar_wait(&mbar[last % STAGES], (last / STAGES) & 1, WAIT_CYCLES);
    failed = __syncthreads_or(!ok);
  }
  if (failed) {
    set_error(1);
    // give MMAs that may still be in flight a bounded chance to finish before TMEM is released
    const long long t0 = clock64();
    while (clock64() - t0 < 2000000ll) {
    }
  }
  umma::fence_after_sync();

  // ---- epilogue: warp w holds rows 32 w .. 32 w + 31 (TMEM lanes), one row per thread ----
  const int r = row0 + warp * 32 + lane;
  const bool row_ok = r < g.M && !failed;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  for (int n0 = 0; n0 < NP; n0 += 8) {
    float v[8];
    if (ktiles > 0) {
      umma::tmem_ld8(trow + n0, v);
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = 0.f;
    }
    if (!row_ok || n0 >= g.N) continue;
    if (EM == E_PART) {
      float* dst = g.outf + ((size_t)blockIdx.z * gridDim.y + blockIdx.y) * (size_t)g.M * g.N + (size_t)r * g.N + n0;
#pragma unroll
      for (int j = 0; j < 8; ++j) dst[j] = v[j];
      continue;
    }
    int orow = r;
    if (g.out_child) {  // transposed convolution: row r of the coarse grid -> child blockIdx.z
      const Vox p = decomp(r, g.nx, g.nz);
      const int o = blockIdx.z;
      orow = ((2 * p.y + (o >> 2)) * 2 * g.nx + 2 * p.x + ((o >> 1) & 1)) * (2 * g.nz) + 2 * p.z + (o & 1);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (g.bias) v[j] += g.bias[n0 + j];
      if (g.relu) v[j] = fmaxf(v[j], 0.f);
    }
    if (g.mask) {
      const __nv_bfloat16* mk = g.mask + (size_t)orow * g.mask_stride + g.mask_off + n0;
#pragma unroll
      for (int j = 0; j < 8; ++j)
        if (n0 + j >= g.mask_from && !(__bfloat162float(mk[j]) > 0.f)) v[j] = 0.f;
    }
    if (EM == E_F32) {
      float* dst = g.outf + (size_t)orow * g.N + n0;
#pragma unroll
      for (int j = 0; j < 8; ++j) dst[j] = v[j];
    } else {
      __align__(16) __nv_bfloat162 h[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
      *reinterpret_cast<uint4*>(g.out + (size_t)orow * g.out_stride + g.out_off + n0) = *reinterpret_cast<uint4*>(h);
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tmem, ncols);
}

template <int AM, int BMODE, int EM>
static cudaError_t launch_t(const GemmArgs& g, dim3 grid, cudaStream_t s) {
  const int NP = (g.N + 15) & ~15;
  const size_t smem = (size_t)STAGES * (BM * BK * 2 + (size_t)NP * BK * 2) + 1024;
  auto kern = k_igemm<AM, BMODE, EM>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, THREADS, smem, s>>>(g);
  return cudaGetLastError();
}

cudaError_t launch(int am, int bm, int em, const GemmArgs& g, dim3 grid, cudaStream_t s) {
  // K-major operands move 8 reduction elements per chunk, MN-major ones 8 rows per chunk
  const bool a_k = am == A_GEMM_K || am == A_CONV3 || am == A_ROWS || am == A_CHILD8;
  const bool b_k = bm == B_GEMM_K;
  if (g.N < 16 || g.N > 256 || (g.N & 15) || g.M <= 0 || g.K <= 0) return cudaErrorInvalidValue;
  if ((a_k || b_k) && (g.K & 7)) return cudaErrorInvalidValue;
  if (!a_k && (g.M & 7)) return cudaErrorInvalidValue;
#define IG_CASE(A, B, E) \
  if (am == A && bm == B && em == E) return launch_t<A, B, E>(g, grid, s);
  IG_CASE(A_GEMM_K, B_GEMM_K, E_F32)
  IG_CASE(A_GEMM_K, B_GEMM_MN, E_F32)
  IG_CASE(A_GEMM_MN, B_GEMM_K, E_F32)
  IG_CASE(A_GEMM_MN, B_GEMM_MN, E_F32)
  IG_CASE(A_CONV3, B_GEMM_K, E_BF16)
  IG_CASE(A_CONV3, B_GEMM_K, E_F32)
  IG_CASE(A_ROWS, B_GEMM_K, E_BF16)
  IG_CASE(A_ROWS, B_GEMM_K, E_F32)
  IG_CASE(A_CHILD8, B_GEMM_K, E_BF16)
  IG_CASE(A_CHILD8, B_GEMM_K, E_F32)
  IG_CASE(A_WG_CONV3, B_WG_ROWS, E_PART)
  IG_CASE(A_WG_TCONV, B_WG_CHILD, E_PART)
#undef IG_CASE
  return cudaErrorInvalidValue;
}

int read_error(cudaStream_t s) {
  int h = 0;
  if (cudaMemcpyFromSymbolAsync(&h, g_error, sizeof(int), 0, cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
  if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
  return h;
}

}  // namespace ig
}  // namespace spdhg
