// The learned warm start: a 3-D U-Net trained and evaluated with the library's own kernels.
//
// Network (levels L, channels c_0 .. c_{L-1}): encoder level l = conv3 + ReLU, conv3 + ReLU
// (2x2x2 max-pooling before every level but the first); decoder level l = L-2 .. 0: 2x2x2
// transposed convolution of the level below, concatenated with the encoder output of level l
// ([up, skip]), conv3 + ReLU, conv3 + ReLU; a 1x1x1 head and a residual connection:
// pred = x_n + sum_c w_c h_c + b.  Input x_n = x / s with s the mean of the early iterate; the
// warm start is x0 = s * pred.
//
// Storage: BF16 channels-last activations (element (v, c) at p[v * stride + off + c]); the
// encoder output of level l < L-1 is written straight into the right half of the decoder's
// concatenation buffer, the transposed convolution into its left half.  Every convolution
// (forward, data gradient, weight gradient) runs on the tensor cores (igemm.cu); weights are
// FP32 masters with BF16 copies in the layouts the GEMM operands need (forward [co][tap][ci],
// flipped for the data gradient [ci][tap][co]).  Weight gradients are reduced deterministically
// (partial sums per reduction split, then a fixed-order sum).
#include <cuda_bf16.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include <string>
#include <vector>

#include "../../include/unet.h"
#include "igemm.cuh"

using namespace spdhg;
typedef __nv_bfloat16 bf16;

namespace {

constexpr int kMaxLevels = 5;
constexpr int kColsumBlocks = 1024;  // blocks of the column sums (bias gradients)

// ------------------------------------------------------------------------------------------
// small kernels
// ------------------------------------------------------------------------------------------

__global__ void k_prep_input(const float* __restrict__ x, const float* __restrict__ inv_s_p, bf16* __restrict__ in0,
                             float* __restrict__ xn, int64_t V) {
  const float inv_s = *inv_s_p;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    const float a = x[v] * inv_s;
    const bf16 h = __float2bfloat16_rn(a);
    xn[v] = __bfloat162float(h);  // the residual uses the same rounded input the network sees
    __align__(16) bf16 row[8];
    row[0] = h;
#pragma unroll
    for (int c = 1; c < 8; ++c) row[c] = __float2bfloat16_rn(0.f);
    *reinterpret_cast<uint4*>(in0 + v * 8) = *reinterpret_cast<uint4*>(row);
  }
}

// 2x2x2 max-pooling of src (fine grid 2ny x 2nx x 2nz) into dst (ny, nx, nz); arg = child index of
// the first maximum (child order (ty, tx, tz))
__global__ void k_pool_fwd(const bf16* __restrict__ src, int s_stride, int s_off, bf16* __restrict__ dst, int d_stride,
                           uint8_t* __restrict__ arg, int C, int ny, int nx, int nz) {
  const int64_t n = (int64_t)ny * nx * nz * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t v = i / C;
    const int z = (int)(v % nz), x = (int)((v / nz) % nx), y = (int)(v / ((int64_t)nz * nx));
    float best = -INFINITY;
    int bi = 0;
    for (int o = 0; o < 8; ++o) {
      const int64_t f = ((int64_t)(2 * y + (o >> 2)) * 2 * nx + 2 * x + ((o >> 1) & 1)) * (2 * nz) + 2 * z + (o & 1);
      const float a = __bfloat162float(src[f * s_stride + s_off + c]);
      if (a > best) {
        best = a;
        bi = o;
      }
    }
    dst[v * d_stride + c] = __float2bfloat16_rn(best);
    arg[i] = (uint8_t)bi;
  }
}

// g_fine[child arg] += g_coarse where the fine value is positive (ReLU gradient of the encoder
// output that was pooled)
__global__ void k_pool_bwd_add(const bf16* __restrict__ gc, int gc_stride, const uint8_t* __restrict__ arg,
                               const bf16* __restrict__ act, int a_stride, int a_off, bf16* __restrict__ gf, int gf_stride,
                               int gf_off, int C, int ny, int nx, int nz) {
  const int64_t n = (int64_t)ny * nx * nz * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t v = i / C;
    const int z = (int)(v % nz), x = (int)((v / nz) % nx), y = (int)(v / ((int64_t)nz * nx));
    const int o = arg[i];
    const int64_t f = ((int64_t)(2 * y + (o >> 2)) * 2 * nx + 2 * x + ((o >> 1) & 1)) * (2 * nz) + 2 * z + (o & 1);
    if (__bfloat162float(act[f * a_stride + a_off + c]) > 0.f) {
      bf16* d = gf + f * gf_stride + gf_off + c;
      *d = __float2bfloat16_rn(__bfloat162float(*d) + __bfloat162float(gc[v * gc_stride + c]));
    }
  }
}

// pred = xn + sum_c w_c h_c + b
__global__ void k_head_fwd(const bf16* __restrict__ h, int C, const float* __restrict__ w, const float* __restrict__ b,
                           const float* __restrict__ xn, float* __restrict__ pred, int64_t V) {
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    float a = xn[v] + b[0];
    for (int c = 0; c < C; ++c) a = fmaf(w[c], __bfloat162float(h[v * C + c]), a);
    pred[v] = a;
  }
}

// gpred = 2 (pred - t / s) / V and per-block partial sums of the squared error (FP64)
__global__ void k_mse(const float* __restrict__ pred, const float* __restrict__ t, const float* __restrict__ inv_s_p,
                      float* __restrict__ gpred, int64_t V, double* __restrict__ part) {
  __shared__ double red[256];
  const float inv_s = *inv_s_p;
  double acc = 0.0;
  const float k = 2.f / (float)V;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) {
    const float d = pred[v] - t[v] * inv_s;
    gpred[v] = k * d;
    acc += (double)d * d;
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// gradient of the pre-activation of the last decoder conv: w_c gpred (h_c > 0)
__global__ void k_head_bwd(const float* __restrict__ gpred, const bf16* __restrict__ h, int C, const float* __restrict__ w,
                           bf16* __restrict__ gh, int64_t V) {
  const int64_t n = V * C;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(i % C);
    const int64_t v = i / C;
    gh[i] = __float2bfloat16_rn(__bfloat162float(h[i]) > 0.f ? w[c] * gpred[v] : 0.f);
  }
}

// column sums of a V x C view (FP32 or BF16 source), C <= 256: per-block partials [block][C]
template <class T>
__global__ void k_colsum_part(const T* __restrict__ src, int stride, int off, int C, int64_t V, const float* __restrict__ wv,
                              float* __restrict__ part) {
  // thread layout: C columns x (blockDim / C) row lanes
  const int lanes = blockDim.x / C;
  const int c = threadIdx.x % C, lane = threadIdx.x / C;
  float acc = 0.f;
  if (lane < lanes) {
    for (int64_t v = (int64_t)blockIdx.x * lanes + lane; v < V; v += (int64_t)gridDim.x * lanes) {
      float a;
      if constexpr (sizeof(T) == 4) a = (float)src[v * stride + off + c];
      else a = __bfloat162float(src[v * stride + off + c]);
      if (wv) a *= wv[v];
      acc += a;
    }
  }
  extern __shared__ float red[];
  red[threadIdx.x] = lane < lanes ? acc : 0.f;
  __syncthreads();
  if (threadIdx.x < C) {
    float s = 0.f;
    for (int l = 0; l < lanes; ++l) s += red[l * C + c];
    part[(size_t)blockIdx.x * C + c] = s;
  }
}

// out[c] (+)= sum_b part[b][c]
// one block per column c, 256 threads: strided partial sums, then a fixed-order tree
__global__ void k_sum_parts(const float* __restrict__ part, int nb, int C, float* __restrict__ out, int accumulate) {
  __shared__ float red[256];
  const int c = blockIdx.x;
  float s = 0.f;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) s += part[(size_t)b * C + c];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[c] = accumulate ? out[c] + red[0] : red[0];
}

// conv3 weight gradient: part[split][tap * cin + ci][co] -> g[co][tap][ci] (+)=
__global__ void k_wg_conv3(const float* __restrict__ part, int splits, int cin, int cout, float* __restrict__ g,
                           int accumulate) {
  const int n = 27 * cin * cout;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int co = i % cout, m = i / cout;  // m = tap * cin + ci
    float s = 0.f;
    for (int k = 0; k < splits; ++k) s += part[((size_t)k * 27 * cin + m) * cout + co];
    const int tap = m / cin, ci = m % cin;
    float* d = g + ((size_t)co * 27 + tap) * cin + ci;
    *d = accumulate ? *d + s : s;
  }
}

// tconv weight gradient: part[o][split][ci][co] -> g[o][co][ci] (+)=
__global__ void k_wg_tconv(const float* __restrict__ part, int splits, int cin, int cout, float* __restrict__ g,
                           int accumulate) {
  const int n = 8 * cin * cout;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int co = i % cout, ci = (i / cout) % cin, o = i / (cout * cin);
    float s = 0.f;
    for (int k = 0; k < splits; ++k) s += part[(((size_t)o * splits + k) * cin + ci) * cout + co];
    float* d = g + ((size_t)o * cout + co) * cin + ci;
    *d = accumulate ? *d + s : s;
  }
}

// BF16 weight copies: conv3 forward [co][tap][ci] and flipped data-gradient [ci][tap][co]
__global__ void k_bf16_conv3(const float* __restrict__ w, int cin, int cout, bf16* __restrict__ wf, bf16* __restrict__ wb) {
  const int n = cout * 27 * cin;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int ci = i % cin, tap = (i / cin) % 27, co = i / (27 * cin);
    const bf16 h = __float2bfloat16_rn(w[i]);
    wf[i] = h;
    wb[((size_t)ci * 27 + (26 - tap)) * cout + co] = h;
  }
}

// BF16 weight copies: tconv forward [o][co][ci] and data-gradient [ci][o][co]
__global__ void k_bf16_tconv(const float* __restrict__ w, int cin, int cout, bf16* __restrict__ wf, bf16* __restrict__ wb) {
  const int n = 8 * cout * cin;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int ci = i % cin, co = (i / cin) % cout, o = i / (cin * cout);
    const bf16 h = __float2bfloat16_rn(w[i]);
    wf[i] = h;
    wb[((size_t)ci * 8 + o) * cout + co] = h;
  }
}

// Adam (Kingma & Ba) on FP32 masters with the gradient averaged over `count` samples
__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float bc1, float bc2, float inv_count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i] * inv_count;
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  }
}

// out = a / inv_s (the warm start in image units)
__global__ void k_unscale(const float* __restrict__ a, const float* __restrict__ inv_s_p, float* __restrict__ out,
                          int64_t n) {
  const float s = 1.f / *inv_s_p;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a[i] * s;
}

// inv_s = 1 / scale, or 1 / mean(x) when scale <= 0: per-block FP64 partial sums in a fixed
// order, then one block adds the partials in a fixed order
constexpr int kMeanBlocks = 256;
__global__ void k_sum_part(const float* __restrict__ x, int64_t V, double* __restrict__ part) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < V; v += (int64_t)gridDim.x * blockDim.x) acc += x[v];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void k_inv_scale(const double* __restrict__ part, int nparts, int64_t V, float scale, float* __restrict__ inv_s) {
  __shared__ double red[256];
  if (scale > 0.f) {
    if (threadIdx.x == 0) *inv_s = 1.f / scale;
    return;
  }
  double acc = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double m = red[0] / (double)V;
    *inv_s = m > 1e-30 ? (float)(1.0 / m) : 1.f;
  }
}

int blocks_for(int64_t n, int t = 256) {
  int64_t b = (n + t - 1) / t;
  if (b > 152 * 16) b = 152 * 16;
  return (int)(b < 1 ? 1 : b);
}

}  // namespace

// ------------------------------------------------------------------------------------------
// the network object
// ------------------------------------------------------------------------------------------

struct Param {
  int kind;          // 0 conv3, 1 tconv, 2 head
  int cin, cout;     // cin of conv3 padded to a multiple of 8 on the device
  int cin_true;
  size_t n;          // FP32 weights (device layout)
  size_t off_w, off_b;   // offsets into the FP32 master array
  bf16* wf = nullptr;    // BF16 forward copy
  bf16* wb = nullptr;    // BF16 data-gradient copy
};

struct unet_net {
  int L = 0;
  int ch[kMaxLevels] = {0};
  int ny[kMaxLevels], nx[kMaxLevels], nz[kMaxLevels];
  int64_t V[kMaxLevels];
  std::vector<Param> P;    // order: enc{l}a, enc{l}b (l = 0..L-1), then per decoder level l = L-2..0: up, dec a, dec b; head
  size_t n_master = 0;
  float *w = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;  // FP32 masters, grads, Adam moments
  int64_t adam_t = 0;
  int grad_count = 0;
  // activations
  bf16* in0 = nullptr;                  // [V0][8]
  float *xn = nullptr, *pred = nullptr, *gpred = nullptr;
  bf16* ea[kMaxLevels] = {};             // encoder conv a outputs [V_l][c_l]
  bf16* cat[kMaxLevels] = {};            // [V_l][2 c_l] (l < L-1): [up, skip]
  bf16* bottom = nullptr;                // encoder output of the bottom level [V][c]
  bf16* pool[kMaxLevels] = {};           // pooled input of level l >= 1 [V_l][c_{l-1}]
  uint8_t* arg[kMaxLevels] = {};
  bf16* da[kMaxLevels] = {};             // decoder conv a outputs [V_l][c_l]
  bf16* db[kMaxLevels] = {};             // decoder conv b outputs [V_l][c_l]
  // gradients (BF16): two scratch buffers and the [up, skip] gradient of every decoder level
  // (its skip half is consumed by the encoder pass)
  bf16 *gA = nullptr, *gB = nullptr;
  bf16* gcat[kMaxLevels] = {};
  float* part = nullptr;
  size_t part_cap = 0;
  double* lpart = nullptr;
  float* cpart = nullptr;                // column-sum partials
  float* inv_s = nullptr;                // device: 1 / scale of the last forward
  std::string err;
};

namespace {

int fail(unet_net* n, int code, const std::string& msg) {
  if (n) n->err = msg;
  return code;
}

#define UCK(call)                                                                               \
  do {                                                                                          \
    cudaError_t e_ = (call);                                                                    \
    if (e_ != cudaSuccess)                                                                      \
      return fail(net, e_ == cudaErrorMemoryAllocation ? UNET_ERR_OOM : UNET_ERR_CUDA,         \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                          \
  } while (0)

template <class T>
cudaError_t zalloc(T** p, size_t n) {
  cudaError_t e = cudaMalloc((void**)p, n * sizeof(T) + 16);
  if (e == cudaSuccess) e = cudaMemset(*p, 0, n * sizeof(T) + 16);
  return e;
}

// index helpers into P
int pi_enc(int l, int k) { return 2 * l + k; }
int pi_up(const unet_net* n, int l) { return 2 * n->L + 3 * (n->L - 2 - l); }
int pi_dec(const unet_net* n, int l, int k) { return pi_up(n, l) + 1 + k; }
int pi_head(const unet_net* n) { return (int)n->P.size() - 1; }

struct View {
  const bf16* p;
  int stride, off, c;
};

// 3x3x3 convolution pass: the halo kernel where the shape allows it, else the gather kernel
int conv3_launch(unet_net* net, const ig::GemmArgs& a, cudaStream_t s) {
  cudaError_t e = ig::launch_conv3_halo(ig::E_BF16, a, s);
  if (e == cudaErrorNotSupported)  // returned before any CUDA call: the shape does not fit
    e = ig::launch(ig::A_CONV3, ig::B_GEMM_K, ig::E_BF16, a, dim3((a.M + 127) / 128), s);
  UCK(e);
  return UNET_OK;
}

int conv3_fwd(unet_net* net, int l, const Param& pr, View x, bf16* out, int o_stride, int o_off, cudaStream_t s) {
  ig::GemmArgs a{};
  a.M = (int)net->V[l];
  a.N = pr.cout;
  a.K = 27 * pr.cin;
  a.a = x.p; a.a_stride = x.stride; a.a_off = x.off; a.a_c = pr.cin;
  a.b = pr.wf; a.b_stride = 27 * pr.cin;
  a.ny = net->ny[l]; a.nx = net->nx[l]; a.nz = net->nz[l];
  a.bias = net->w + pr.off_b;
  a.relu = 1;
  a.out = out; a.out_stride = o_stride; a.out_off = o_off;
  return conv3_launch(net, a, s);
}

// dX = conv3^T(G) masked by (mask > 0) on columns >= mask_from
int conv3_bwd_data(unet_net* net, int l, const Param& pr, View gv, bf16* out, int o_stride, int o_off, View mask,
                   int mask_from, cudaStream_t s) {
  ig::GemmArgs a{};
  a.M = (int)net->V[l];
  a.N = pr.cin;
  a.K = 27 * pr.cout;
  a.a = gv.p; a.a_stride = gv.stride; a.a_off = gv.off; a.a_c = pr.cout;
  a.b = pr.wb; a.b_stride = 27 * pr.cout;
  a.ny = net->ny[l]; a.nx = net->nx[l]; a.nz = net->nz[l];
  a.out = out; a.out_stride = o_stride; a.out_off = o_off;
  a.mask = mask.p; a.mask_stride = mask.stride; a.mask_off = mask.off; a.mask_from = mask_from;
  return conv3_launch(net, a, s);
}

int ensure_part(unet_net* net, size_t n) {
  if (n <= net->part_cap) return UNET_OK;
  if (net->part) cudaFree(net->part);
  net->part = nullptr;
  net->part_cap = 0;
  UCK(cudaMalloc(&net->part, n * sizeof(float)));
  net->part_cap = n;
  return UNET_OK;
}

int split_count(int64_t K, int tiles) {
  int64_t want = (2 * 152 + tiles - 1) / tiles;
  int64_t maxs = (K + 255) / 256;  // at least 256 reduction elements per split
  if (want > maxs) want = maxs;
  return (int)(want < 1 ? 1 : want);
}

// column sums of a gradient view into out (+)= (deterministic)
int colsum(unet_net* net, View gv, int64_t V, float* out, int accumulate, cudaStream_t s) {
  const int C = gv.c;
  const int threads = C >= 256 ? 256 : (256 / C) * C;
  const int nb = kColsumBlocks;
  k_colsum_part<bf16><<<nb, threads, threads * sizeof(float), s>>>(gv.p, gv.stride, gv.off, C, V, nullptr, net->cpart);
  k_sum_parts<<<C, 256, 0, s>>>(net->cpart, nb, C, out, accumulate);
  UCK(cudaGetLastError());
  return UNET_OK;
}

int conv3_wgrad(unet_net* net, int l, const Param& pr, View x, View gv, int accumulate, cudaStream_t s) {
  ig::GemmArgs a{};
  a.M = 27 * pr.cin;
  a.N = pr.cout;
  a.K = (int)net->V[l];
  a.a = x.p; a.a_stride = x.stride; a.a_off = x.off; a.a_c = pr.cin;
  a.b = gv.p; a.b_stride = gv.stride; a.b_off = gv.off;
  a.ny = net->ny[l]; a.nx = net->nx[l]; a.nz = net->nz[l];
  const int tiles = (a.M + 127) / 128;
  const int splits = split_count(a.K, tiles);
  a.k_per_split = (int)(((a.K + splits - 1) / splits + 63) / 64 * 64);
  const int used = (a.K + a.k_per_split - 1) / a.k_per_split;
  if (int st = ensure_part(net, (size_t)used * a.M * a.N)) return st;
  a.outf = net->part;
  UCK(ig::launch(ig::A_WG_CONV3, ig::B_WG_ROWS, ig::E_PART, a, dim3(tiles, used, 1), s));
  k_wg_conv3<<<blocks_for(27 * pr.cin * pr.cout), 256, 0, s>>>(net->part, used, pr.cin, pr.cout, net->g + pr.off_w,
                                                               accumulate);
  UCK(cudaGetLastError());
  return colsum(net, gv, net->V[l], net->g + pr.off_b, accumulate, s);
}

// transposed convolution from level l+1 (coarse) into the left half of cat[l]
int tconv_fwd(unet_net* net, int l, const Param& pr, View x, cudaStream_t s) {
  ig::GemmArgs a{};
  a.M = (int)net->V[l + 1];
  a.N = pr.cout;
  a.K = pr.cin;
  a.a = x.p; a.a_stride = x.stride; a.a_off = x.off; a.a_c = pr.cin;
  a.b = pr.wf; a.b_stride = pr.cin; a.b_zstride = (long long)pr.cout * pr.cin;
  a.ny = net->ny[l + 1]; a.nx = net->nx[l + 1]; a.nz = net->nz[l + 1];
  a.bias = net->w + pr.off_b;
  a.out = net->cat[l]; a.out_stride = 2 * net->ch[l]; a.out_off = 0;
  a.out_child = 1;
  UCK(ig::launch(ig::A_ROWS, ig::B_GEMM_K, ig::E_BF16, a, dim3((a.M + 127) / 128, 1, 8), s));
  return UNET_OK;
}

// data gradient of the transposed convolution: G (left half of gcat, fine) -> coarse, masked
int tconv_bwd_data(unet_net* net, int l, const Param& pr, View gv, bf16* out, View mask, cudaStream_t s) {
  ig::GemmArgs a{};
  a.M = (int)net->V[l + 1];
  a.N = pr.cin;
  a.K = 8 * pr.cout;
  a.a = gv.p; a.a_stride = gv.stride; a.a_off = gv.off; a.a_c = pr.cout;
  a.b = pr.wb; a.b_stride = 8 * pr.cout;
  a.ny = net->ny[l + 1]; a.nx = net->nx[l + 1]; a.nz = net->nz[l + 1];
  a.out = out; a.out_stride = pr.cin; a.out_off = 0;
  a.mask = mask.p; a.mask_stride = mask.stride; a.mask_off = mask.off;
  UCK(ig::launch(ig::A_CHILD8, ig::B_GEMM_K, ig::E_BF16, a, dim3((a.M + 127) / 128), s));
  return UNET_OK;
}

int tconv_wgrad(unet_net* net, int l, const Param& pr, View x, View gv, int accumulate, cudaStream_t s) {
  ig::GemmArgs a{};
  a.M = pr.cin;
  a.N = pr.cout;
  a.K = (int)net->V[l + 1];
  a.a = x.p; a.a_stride = x.stride; a.a_off = x.off; a.a_c = pr.cin;
  a.b = gv.p; a.b_stride = gv.stride; a.b_off = gv.off;
  a.ny = net->ny[l + 1]; a.nx = net->nx[l + 1]; a.nz = net->nz[l + 1];
  const int tiles = (a.M + 127) / 128;
  const int splits = split_count(a.K, tiles * 8);
  a.k_per_split = (int)(((a.K + splits - 1) / splits + 63) / 64 * 64);
  const int used = (a.K + a.k_per_split - 1) / a.k_per_split;
  if (int st = ensure_part(net, (size_t)8 * used * a.M * a.N)) return st;
  a.outf = net->part;
  UCK(ig::launch(ig::A_WG_TCONV, ig::B_WG_CHILD, ig::E_PART, a, dim3(tiles, used, 8), s));
  k_wg_tconv<<<blocks_for(8 * pr.cin * pr.cout), 256, 0, s>>>(net->part, used, pr.cin, pr.cout, net->g + pr.off_w,
                                                              accumulate);
  UCK(cudaGetLastError());
  return colsum(net, gv, net->V[l], net->g + pr.off_b, accumulate, s);
}

int refresh_bf16(unet_net* net, cudaStream_t s) {
  for (Param& p : net->P) {
    if (p.kind == 0)
      k_bf16_conv3<<<blocks_for(p.n), 256, 0, s>>>(net->w + p.off_w, p.cin, p.cout, p.wf, p.wb);
    else if (p.kind == 1)
      k_bf16_tconv<<<blocks_for(p.n), 256, 0, s>>>(net->w + p.off_w, p.cin, p.cout, p.wf, p.wb);
  }
  UCK(cudaGetLastError());
  return UNET_OK;
}

}  // namespace

// ------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------

extern "C" {

const char* unet_last_error(const unet_net* net) { return net ? net->err.c_str() : "null network"; }

void unet_destroy(unet_net* net) {
  if (!net) return;
  for (Param& p : net->P) {
    if (p.wf) cudaFree(p.wf);
    if (p.wb) cudaFree(p.wb);
  }
  void* ptrs[] = {net->w, net->g, net->m, net->v, net->in0, net->xn, net->pred, net->gpred, net->bottom, net->gA,
                  net->gB, net->part, net->lpart, net->cpart, net->inv_s};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int l = 0; l < kMaxLevels; ++l) {
    void* q[] = {net->ea[l], net->cat[l], net->pool[l], net->arg[l], net->da[l], net->db[l], net->gcat[l]};
    for (void* p : q)
      if (p) cudaFree(p);
  }
  delete net;
}

int unet_create(int levels, const int* channels, int ny, int nx, int nz, unet_net** out) {
  if (!out) return UNET_ERR_ARG;
  *out = nullptr;
  if (levels < 2 || levels > kMaxLevels || !channels) return UNET_ERR_ARG;
  for (int l = 0; l < levels; ++l)
    if (channels[l] < 16 || channels[l] > 128 || (channels[l] & (channels[l] - 1))) return UNET_ERR_ARG;
  const int f = 1 << (levels - 1);
  if (ny <= 0 || nx <= 0 || nz <= 0 || ny % f || nx % f || nz % f) return UNET_ERR_ARG;
  unet_net* net = new unet_net();
  net->L = levels;
  for (int l = 0; l < levels; ++l) {
    net->ch[l] = channels[l];
    net->ny[l] = ny >> l;
    net->nx[l] = nx >> l;
    net->nz[l] = nz >> l;
    net->V[l] = (int64_t)net->ny[l] * net->nx[l] * net->nz[l];
  }
  // parameters (device layouts), in the order of the public parameter vector
  size_t off = 0;
  auto add = [&](int kind, int cin_true, int cout) {
    Param p;
    p.kind = kind;
    p.cin_true = cin_true;
    p.cin = kind == 0 ? ((cin_true + 7) & ~7) : cin_true;
    p.cout = cout;
    p.n = kind == 0 ? (size_t)cout * 27 * p.cin : kind == 1 ? (size_t)8 * cout * p.cin : (size_t)cin_true;
    p.off_w = off;
    off += p.n;
    p.off_b = off;
    off += kind == 2 ? 1 : cout;
    net->P.push_back(p);
  };
  int cin = 1;
  for (int l = 0; l < levels; ++l) {
    add(0, cin, channels[l]);
    add(0, channels[l], channels[l]);
    cin = channels[l];
  }
  for (int l = levels - 2; l >= 0; --l) {
    add(1, channels[l + 1], channels[l]);
    add(0, 2 * channels[l], channels[l]);
    add(0, channels[l], channels[l]);
  }
  add(2, channels[0], 1);
  net->n_master = off;
  int st = UNET_OK;
  auto A = [&](cudaError_t e) {
    if (e != cudaSuccess && st == UNET_OK) st = e == cudaErrorMemoryAllocation ? UNET_ERR_OOM : UNET_ERR_CUDA;
  };
  A(zalloc(&net->w, off));
  A(zalloc(&net->g, off));
  A(zalloc(&net->m, off));
  A(zalloc(&net->v, off));
  for (Param& p : net->P)
    if (p.kind != 2) {
      A(zalloc(&p.wf, p.n));
      A(zalloc(&p.wb, p.n));
    }
  const int64_t V0 = net->V[0];
  A(zalloc(&net->in0, (size_t)V0 * 8));
  A(zalloc(&net->xn, (size_t)V0));
  A(zalloc(&net->pred, (size_t)V0));
  A(zalloc(&net->gpred, (size_t)V0));
  size_t gmax = 0;
  for (int l = 0; l < levels; ++l) {
    const size_t Vl = (size_t)net->V[l], c = channels[l];
    A(zalloc(&net->ea[l], Vl * c));
    if (l < levels - 1) {
      A(zalloc(&net->cat[l], Vl * 2 * c));
      A(zalloc(&net->gcat[l], Vl * 2 * c));
      A(zalloc(&net->da[l], Vl * c));
      A(zalloc(&net->db[l], Vl * c));
    } else {
      A(zalloc(&net->bottom, Vl * c));
    }
    if (l > 0) {
      A(zalloc(&net->pool[l], Vl * channels[l - 1]));
      A(zalloc(&net->arg[l], Vl * channels[l - 1]));
    }
    gmax = std::max(gmax, Vl * 2 * c);
  }
  A(zalloc(&net->gA, gmax));
  A(zalloc(&net->gB, gmax));
  A(zalloc(&net->lpart, 1024));
  A(zalloc(&net->cpart, (size_t)kColsumBlocks * 256));
  A(zalloc(&net->inv_s, 1));
  if (st != UNET_OK) {
    unet_destroy(net);
    return st;
  }
  *out = net;
  return UNET_OK;
}

int64_t unet_num_params(const unet_net* net) {
  if (!net) return -1;
  int64_t n = 0;
  for (const Param& p : net->P) {
    const int64_t k = p.kind == 0 ? 27 : p.kind == 1 ? 8 : 1;
    n += (int64_t)p.cin_true * p.cout * k + (p.kind == 2 ? 1 : p.cout);
  }
  return n;
}

// Public parameter vector: per layer its weights then biases, in the layouts
//   conv3 W[co][ci][ky][kx][kz], tconv W[ci][co][ty][tx][tz], head W[ci]; biases [co].
int unet_set_params(unet_net* net, const float* host, int64_t n) {
  if (!net || !host || n != unet_num_params(net)) return UNET_ERR_ARG;
  std::vector<float> dev(net->n_master, 0.f);
  int64_t q = 0;
  for (const Param& p : net->P) {
    if (p.kind == 0) {
      for (int co = 0; co < p.cout; ++co)
        for (int ci = 0; ci < p.cin_true; ++ci)
          for (int t = 0; t < 27; ++t) dev[p.off_w + ((size_t)co * 27 + t) * p.cin + ci] = host[q++];
    } else if (p.kind == 1) {
      for (int ci = 0; ci < p.cin; ++ci)
        for (int co = 0; co < p.cout; ++co)
          for (int o = 0; o < 8; ++o) dev[p.off_w + ((size_t)o * p.cout + co) * p.cin + ci] = host[q++];
    } else {
      for (int ci = 0; ci < p.cin_true; ++ci) dev[p.off_w + ci] = host[q++];
    }
    const int nb = p.kind == 2 ? 1 : p.cout;
    for (int k = 0; k < nb; ++k) dev[p.off_b + k] = host[q++];
  }
  UCK(cudaMemcpy(net->w, dev.data(), dev.size() * sizeof(float), cudaMemcpyHostToDevice));
  UCK(cudaMemset(net->m, 0, net->n_master * sizeof(float)));
  UCK(cudaMemset(net->v, 0, net->n_master * sizeof(float)));
  net->adam_t = 0;
  if (int st = refresh_bf16(net, 0)) return st;
  UCK(cudaDeviceSynchronize());
  return UNET_OK;
}

// He-normal initialisation: weights ~ N(0, 2 / fan_in) (fan_in = cin * 27 for conv3, cin * 8 for
// the transposed convolution), biases and head zero, so the untrained network is the identity
// warm start pred = x/s.  Normal draws: Box-Muller on SplitMix64 uniforms (53-bit).
int unet_init(unet_net* net, uint64_t seed) {
  if (!net) return UNET_ERR_ARG;
  uint64_t k = 0;
  auto uniform = [&]() {
    uint64_t z = seed + (++k) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return ((z >> 11) + 0.5) * (1.0 / 9007199254740992.0);  // (0, 1)
  };
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<float> v((size_t)unet_num_params(net));
  size_t q = 0;
  for (const Param& p : net->P) {
    const size_t nw = p.kind == 0 ? (size_t)p.cout * p.cin_true * 27 : p.kind == 1 ? (size_t)8 * p.cout * p.cin : p.cin_true;
    const double sd = p.kind == 2 ? 0.0 : sqrt(2.0 / (p.kind == 0 ? 27.0 * p.cin_true : 8.0 * p.cin));
    for (size_t i = 0; i < nw; ++i) {
      const double r = sqrt(-2.0 * log(uniform())), t = two_pi * uniform();
      v[q++] = (float)(sd * r * cos(t));
    }
    const int nb = p.kind == 2 ? 1 : p.cout;
    for (int i = 0; i < nb; ++i) v[q++] = 0.f;
  }
  return unet_set_params(net, v.data(), (int64_t)v.size());
}

static int copy_vector_out(unet_net* net, const float* dsrc, float* host, int64_t n) {
  if (!net || !host || n != unet_num_params(net)) return UNET_ERR_ARG;
  std::vector<float> dev(net->n_master);
  UCK(cudaMemcpy(dev.data(), dsrc, dev.size() * sizeof(float), cudaMemcpyDeviceToHost));
  int64_t q = 0;
  for (const Param& p : net->P) {
    if (p.kind == 0) {
      for (int co = 0; co < p.cout; ++co)
        for (int ci = 0; ci < p.cin_true; ++ci)
          for (int t = 0; t < 27; ++t) host[q++] = dev[p.off_w + ((size_t)co * 27 + t) * p.cin + ci];
    } else if (p.kind == 1) {
      for (int ci = 0; ci < p.cin; ++ci)
        for (int co = 0; co < p.cout; ++co)
          for (int o = 0; o < 8; ++o) host[q++] = dev[p.off_w + ((size_t)o * p.cout + co) * p.cin + ci];
    } else {
      for (int ci = 0; ci < p.cin_true; ++ci) host[q++] = dev[p.off_w + ci];
    }
    const int nb = p.kind == 2 ? 1 : p.cout;
    for (int k = 0; k < nb; ++k) host[q++] = dev[p.off_b + k];
  }
  return UNET_OK;
}

int unet_get_params(unet_net* net, float* host, int64_t n) {
  if (!net) return UNET_ERR_ARG;
  return copy_vector_out(net, net->w, host, n);
}

int unet_get_grads(unet_net* net, float* host, int64_t n) {
  if (!net) return UNET_ERR_ARG;
  return copy_vector_out(net, net->g, host, n);
}

int unet_forward(unet_net* net, const float* x, float scale, float* pred, float* x0, void* stream) {
  if (!net || !x || !(scale == scale)) return UNET_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int L = net->L;
  const int64_t V0 = net->V[0];
  if (!(scale > 0)) k_sum_part<<<kMeanBlocks, 256, 0, s>>>(x, V0, net->lpart);
  k_inv_scale<<<1, 256, 0, s>>>(net->lpart, kMeanBlocks, V0, scale, net->inv_s);
  k_prep_input<<<blocks_for(V0), 256, 0, s>>>(x, net->inv_s, net->in0, net->xn, V0);
  UCK(cudaGetLastError());
  View h{net->in0, 8, 0, 8};
  for (int l = 0; l < L; ++l) {
    const int c = net->ch[l];
    if (l > 0) {
      const int cp = net->ch[l - 1];
      const bf16* src = (l - 1 < L - 1) ? net->cat[l - 1] : net->bottom;
      k_pool_fwd<<<blocks_for(net->V[l] * cp), 256, 0, s>>>(src, 2 * cp, cp, net->pool[l], cp, net->arg[l], cp, net->ny[l],
                                                            net->nx[l], net->nz[l]);
      UCK(cudaGetLastError());
      h = View{net->pool[l], cp, 0, cp};
    }
    if (int st = conv3_fwd(net, l, net->P[pi_enc(l, 0)], h, net->ea[l], c, 0, s)) return st;
    View ea{net->ea[l], c, 0, c};
    if (l < L - 1) {
      if (int st = conv3_fwd(net, l, net->P[pi_enc(l, 1)], ea, net->cat[l], 2 * c, c, s)) return st;
    } else {
      if (int st = conv3_fwd(net, l, net->P[pi_enc(l, 1)], ea, net->bottom, c, 0, s)) return st;
    }
  }
  View below{net->bottom, net->ch[L - 1], 0, net->ch[L - 1]};
  for (int l = L - 2; l >= 0; --l) {
    const int c = net->ch[l];
    if (int st = tconv_fwd(net, l, net->P[pi_up(net, l)], below, s)) return st;
    if (int st = conv3_fwd(net, l, net->P[pi_dec(net, l, 0)], View{net->cat[l], 2 * c, 0, 2 * c}, net->da[l], c, 0, s))
      return st;
    if (int st = conv3_fwd(net, l, net->P[pi_dec(net, l, 1)], View{net->da[l], c, 0, c}, net->db[l], c, 0, s)) return st;
    below = View{net->db[l], c, 0, c};
  }
  const Param& hd = net->P[pi_head(net)];
  k_head_fwd<<<blocks_for(V0), 256, 0, s>>>(net->db[0], net->ch[0], net->w + hd.off_w, net->w + hd.off_b, net->xn,
                                            net->pred, V0);
  UCK(cudaGetLastError());
  if (pred) UCK(cudaMemcpyAsync(pred, net->pred, V0 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  if (x0) {
    k_unscale<<<blocks_for(V0), 256, 0, s>>>(net->pred, net->inv_s, x0, V0);
    UCK(cudaGetLastError());
  }
  return UNET_OK;
}

int unet_backward(unet_net* net, const float* target, const float* gpred_in, int accumulate, double* loss, void* stream) {
  if (!net || (!target && !gpred_in)) return UNET_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int L = net->L;
  const int64_t V0 = net->V[0];
  if (!accumulate) net->grad_count = 0;
  ++net->grad_count;
  if (target) {
    const int nb = 512;
    k_mse<<<nb, 256, 0, s>>>(net->pred, target, net->inv_s, net->gpred, V0, net->lpart);
    UCK(cudaGetLastError());
    if (loss) {
      std::vector<double> h(nb);
      UCK(cudaMemcpyAsync(h.data(), net->lpart, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
      UCK(cudaStreamSynchronize(s));
      double lval = 0.0;
      for (double a : h) lval += a;
      *loss = lval / (double)V0;
    }
  } else {
    UCK(cudaMemcpyAsync(net->gpred, gpred_in, V0 * sizeof(float), cudaMemcpyDeviceToDevice, s));
  }
  // head: dW_c = sum_v gpred h_c, db = sum_v gpred; gradient of the last conv's pre-activation
  const Param& hd = net->P[pi_head(net)];
  const int c0 = net->ch[0];
  {
    const int threads = (256 / c0) * c0;
    k_colsum_part<bf16><<<kColsumBlocks, threads, threads * sizeof(float), s>>>(net->db[0], c0, 0, c0, V0, net->gpred,
                                                                                net->cpart);
    k_sum_parts<<<c0, 256, 0, s>>>(net->cpart, kColsumBlocks, c0, net->g + hd.off_w, accumulate);
    k_colsum_part<float><<<kColsumBlocks, 256, 256 * sizeof(float), s>>>(net->gpred, 1, 0, 1, V0, nullptr, net->cpart);
    k_sum_parts<<<1, 256, 0, s>>>(net->cpart, kColsumBlocks, 1, net->g + hd.off_b, accumulate);
    k_head_bwd<<<blocks_for(V0 * c0), 256, 0, s>>>(net->gpred, net->db[0], c0, net->w + hd.off_w, net->gA, V0);
    UCK(cudaGetLastError());
  }
  // decoder levels 0 .. L-2 (the reverse of their forward order); gA holds the gradient of the
  // pre-activation of the level's last conv
  for (int l = 0; l <= L - 2; ++l) {
    const int c = net->ch[l];
    const Param& pb = net->P[pi_dec(net, l, 1)];
    const Param& pa = net->P[pi_dec(net, l, 0)];
    const Param& pu = net->P[pi_up(net, l)];
    View gb{net->gA, c, 0, c};
    if (int st = conv3_wgrad(net, l, pb, View{net->da[l], c, 0, c}, gb, accumulate, s)) return st;
    if (int st = conv3_bwd_data(net, l, pb, gb, net->gB, c, 0, View{net->da[l], c, 0, c}, 0, s)) return st;
    View ga{net->gB, c, 0, c};
    if (int st = conv3_wgrad(net, l, pa, View{net->cat[l], 2 * c, 0, 2 * c}, ga, accumulate, s)) return st;
    // gradient of [up, skip]: the skip half masked by the skip (ReLU) output, the up half not
    if (int st = conv3_bwd_data(net, l, pa, ga, net->gcat[l], 2 * c, 0, View{net->cat[l], 2 * c, 0, 2 * c}, c, s))
      return st;
    // the transposed convolution that produced the up half, and the gradient of its input
    // (the output of the level below, a ReLU output)
    const int cb = net->ch[l + 1];
    const bf16* below = (l + 1 <= L - 2) ? net->db[l + 1] : net->bottom;
    View gu{net->gcat[l], 2 * c, 0, c};
    if (int st = tconv_wgrad(net, l, pu, View{below, cb, 0, cb}, gu, accumulate, s)) return st;
    if (int st = tconv_bwd_data(net, l, pu, gu, net->gA, View{below, cb, 0, cb}, s)) return st;
  }
  // encoder, bottom level first; gA holds the gradient of enc{L-1}b's pre-activation
  for (int l = L - 1; l >= 0; --l) {
    const int c = net->ch[l];
    const Param& pb = net->P[pi_enc(l, 1)];
    const Param& pa = net->P[pi_enc(l, 0)];
    View gb = (l == L - 1) ? View{net->gA, c, 0, c} : View{net->gcat[l], 2 * c, c, c};
    View ea{net->ea[l], c, 0, c};
    if (int st = conv3_wgrad(net, l, pb, ea, gb, accumulate, s)) return st;
    if (int st = conv3_bwd_data(net, l, pb, gb, net->gB, c, 0, ea, 0, s)) return st;
    View ga{net->gB, c, 0, c};
    const int cin = (l == 0) ? 8 : net->ch[l - 1];
    View xin = (l == 0) ? View{net->in0, 8, 0, 8} : View{net->pool[l], cin, 0, cin};
    if (int st = conv3_wgrad(net, l, pa, xin, ga, accumulate, s)) return st;
    if (l > 0) {
      // gradient at the pooled input (no ReLU there), then routed to the maxima of the level
      // above, whose skip-half gradient it joins (masked by the skip ReLU output)
      if (int st = conv3_bwd_data(net, l, pa, ga, net->gA, cin, 0, View{nullptr, 0, 0, 0}, 0, s)) return st;
      k_pool_bwd_add<<<blocks_for(net->V[l] * cin), 256, 0, s>>>(net->gA, cin, net->arg[l], net->cat[l - 1], 2 * cin, cin,
                                                                net->gcat[l - 1], 2 * cin, cin, cin, net->ny[l], net->nx[l],
                                                                net->nz[l]);
      UCK(cudaGetLastError());
    }
  }
  return UNET_OK;
}

int unet_adam_step(unet_net* net, float lr, void* stream) {
  if (!net || !(lr > 0) || net->grad_count <= 0) return UNET_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const float b1 = 0.9f, b2 = 0.999f;
  ++net->adam_t;
  const float bc1 = 1.f - powf(b1, (float)net->adam_t), bc2 = 1.f - powf(b2, (float)net->adam_t);
  k_adam<<<blocks_for((int64_t)net->n_master), 256, 0, s>>>(net->w, net->g, net->m, net->v, (int64_t)net->n_master, lr, b1,
                                                            b2, 1e-8f, bc1, bc2, 1.f / net->grad_count);
  UCK(cudaGetLastError());
  net->grad_count = 0;
  return refresh_bf16(net, s);
}

}  // extern "C"
