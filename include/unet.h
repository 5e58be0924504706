/*
 * unet.h -- C ABI of the learned warm start of libspdhg.so (no counterpart in the paper: a
 * network maps an early SPDHG iterate to a starting point x0 of Algorithm 2; the iteration and
 * its converged solution are unchanged).
 *
 * Tensors are BF16 (passed as uint16_t bit patterns), channels-last: element (voxel v, channel c)
 * of a tensor with row stride S and channel offset O is p[v * S + O + c]; voxels are numbered
 * like the image, v = (iy * nx + ix) * nz + iz.  All pointers are device pointers owned by the
 * caller; kernels are enqueued on `stream` (a cudaStream_t, NULL = legacy default stream).
 * Errors: UNET_OK (0) or a negative code; no call aborts the process.
 */
#ifndef UNET_H
#define UNET_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { UNET_OK = 0, UNET_ERR_ARG = -1, UNET_ERR_CUDA = -2, UNET_ERR_OOM = -3, UNET_ERR_TIMEOUT = -5 };
enum { UNET_GEMM_A_MN = 1, UNET_GEMM_B_MN = 2 };

/* D = A B^T on the tensor cores (tcgen05, BF16 inputs, FP32 accumulation), D row-major M x N.
 * A is M x K, stored row-major (A[m][k] at a[m*K + k]) or, with UNET_GEMM_A_MN, transposed
 * (a[k*M + m]); likewise B is N x K (b[n*K + k]) or with UNET_GEMM_B_MN b[k*N + n].
 * 16 <= N <= 256 with N % 16 == 0; K % 8 == 0; M % 8 == 0 when A is transposed. */
int unet_gemm(const uint16_t* a, const uint16_t* b, float* d, int M, int N, int K, int flags, void* stream);

typedef struct unet_net unet_net;

/* A 3-D U-Net for volumes of ny x nx x nz voxels (each divisible by 2^(levels-1)), 2 <= levels
 * <= 5, channels[l] in {16, 32, 64, 128}.  Encoder level l: conv3 + ReLU, conv3 + ReLU (3x3x3,
 * zero padding; 2x2x2 max-pooling before every level but the first); decoder level l = levels-2
 * .. 0: 2x2x2 stride-2 transposed convolution of the level below, concatenated [up, skip] with
 * the encoder output of level l, conv3 + ReLU, conv3 + ReLU; head pred = x/s + sum_c w_c h_c + b.
 * BF16 weights and activations, FP32 accumulation (tensor cores), FP32 master weights and Adam.
 * All buffers for the volume size are allocated here; parameters start at zero. */
int unet_create(int levels, const int* channels, int ny, int nx, int nz, unet_net** out);
void unet_destroy(unet_net* net);
const char* unet_last_error(const unet_net* net);

/* Number of parameters of the public parameter vector: per layer (encoder levels 0..L-1: conv a,
 * conv b; decoder levels L-2..0: up, conv a, conv b; head) its weights then its biases, with
 * conv weights W[co][ci][ky][kx][kz] (tap (ky,kx,kz) reads the voxel at offset (ky-1,kx-1,kz-1)),
 * transposed-conv weights W[ci][co][ty][tx][tz] (writes the child (2y+ty, 2x+tx, 2z+tz)), head
 * W[ci].  Returns -1 for a NULL net. */
int64_t unet_num_params(const unet_net* net);
/* Host vectors of unet_num_params floats.  set_params also resets the Adam moments. */
int unet_set_params(unet_net* net, const float* params, int64_t n);
int unet_get_params(unet_net* net, float* params, int64_t n);
/* He-normal initialisation from `seed`: weights ~ N(0, 2 / fan_in), biases and head zero (the
 * untrained network returns its input: x0 = x).  Resets the Adam moments. */
int unet_init(unet_net* net, uint64_t seed);
/* Accumulated gradients of the last unet_backward calls (sum over the accumulated samples). */
int unet_get_grads(unet_net* net, float* grads, int64_t n);

/* Forward pass on the FP32 image x (device, nx*ny*nz): input x/s with s = scale if scale > 0,
 * else s = mean(x) computed on the device.  pred (device, FP32, may be NULL) receives the
 * prediction in units of s, x0 (may be NULL) s * pred: the warm start. */
int unet_forward(unet_net* net, const float* x, float scale, float* pred, float* x0, void* stream);
/* Backward pass of the last forward: loss = mean((pred - target/scale)^2) with target a device
 * FP32 image (or, when target is NULL, the gradient gpred of any loss with respect to pred).
 * Gradients are added to the accumulated ones when accumulate != 0, else they replace them.
 * *loss (host, may be NULL) receives the loss (synchronises the stream). */
int unet_backward(unet_net* net, const float* target, const float* gpred, int accumulate, double* loss,
                  void* stream);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the accumulated gradient averaged over
 * the samples accumulated since the last step. */
int unet_adam_step(unet_net* net, float lr, void* stream);

/* UNET_ERR_TIMEOUT if any tensor-core kernel gave up a bounded wait since the library loaded
 * (its outputs are then invalid), else UNET_OK.  Synchronises the stream. */
int unet_device_error(void* stream);

#ifdef __cplusplus
}
#endif
#endif /* UNET_H */
