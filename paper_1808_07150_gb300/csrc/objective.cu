// FP64 reductions of the objective Psi (Problem "PET Reconstruction with Subsets"):
//   D(P x) = sum_j  y_j + r_j - b_j + b_j log(b_j / (y_j + r_j))      (Eq. EQU:LOCALDISTANCE,
//            with 0 log 0 = 0 and +inf where y_j + r_j <= 0 < b_j)
//   alpha R(x) for TV / dTV / aTV, or the TGV value at the current (u, w).
// The per-term arithmetic and the sums run in double precision.  Reductions are deterministic:
// a fixed grid of blocks accumulates grid-strided terms, each block reduces in a fixed tree, and
// one block sums the partials in order.
#include "internal.cuh"

namespace spdhg {

__device__ __forceinline__ double block_sum(double v, double* sh) {
  const int t = threadIdx.x;
  sh[t] = v;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (t < s) sh[t] += sh[t + s];
    __syncthreads();
  }
  return sh[0];
}

__global__ void k_finish_sum(const double* partial, int n, double* out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc += partial[i];
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) *out = s;
}

__global__ void k_finish_max(const double* partial, int n, double* out) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) acc = fmax(acc, partial[i]);
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

__global__ void k_data_term(const float* __restrict__ ax, const float* __restrict__ b,
                            const float* __restrict__ r, int64_t M, double* partial) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < M; j += (int64_t)gridDim.x * blockDim.x) {
    const double e = (double)ax[j] + (double)r[j];
    const double bj = b[j];
    double phi;
    if (bj > 0.0) phi = (e > 0.0) ? e - bj + bj * log(bj / e) : HUGE_VAL;
    else phi = e < 0.0 ? HUGE_VAL : e;
    acc += phi;
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// sum of squares (FP64) of v, for the power iteration of the operator norms
__global__ void k_sumsq(const float* __restrict__ v, int64_t n, double* partial) {
  __shared__ double sh[256];
  double acc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double a = v[j];
    acc += a * a;
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// v = y / sqrt(*ss)  (v = 0 if the norm is 0)
__global__ void k_normalize(const float* __restrict__ y, int64_t n, const double* __restrict__ ss, float* __restrict__ v) {
  const double q = *ss;
  const float inv = q > 0.0 ? (float)(1.0 / sqrt(q)) : 0.f;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
    v[j] = y[j] * inv;
}

cudaError_t launch_sumsq(const float* v, int64_t n, double* partial, int nblocks, double* out, cudaStream_t s) {
  k_sumsq<<<nblocks, 256, 0, s>>>(v, n, partial);
  k_finish_sum<<<1, 256, 0, s>>>(partial, nblocks, out);
  return cudaGetLastError();
}

cudaError_t launch_normalize(const float* y, int64_t n, const double* ss, float* v, cudaStream_t s) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 16) b = 152 * 16;
  k_normalize<<<(int)b, 256, 0, s>>>(y, n, ss, v);
  return cudaGetLastError();
}

cudaError_t launch_data_term(const float* ax, const float* b, const float* r, int64_t M,
                             double* partial, int nblocks, double* out, cudaStream_t s) {
  k_data_term<<<nblocks, 256, 0, s>>>(ax, b, r, M, partial);
  k_finish_sum<<<1, 256, 0, s>>>(partial, nblocks, out);
  return cudaGetLastError();
}

// forward differences (Neumann) of a float field at voxel (ix, iy, iz), in double
__device__ __forceinline__ void grad_d(const DevGeom& g, const float* u, int ix, int iy, int iz,
                                       int64_t j, double gr[3]) {
  const int sx = g.nz, sy = g.nx * g.nz;
  const double c = u[j];
  gr[0] = ix < g.nx - 1 ? (double)u[j + sx] - c : 0.0;
  gr[1] = iy < g.ny - 1 ? (double)u[j + sy] - c : 0.0;
  gr[2] = iz < g.nz - 1 ? (double)u[j + 1] - c : 0.0;
}

// d-_a w_c at j (backward difference, d- = -D^T)
__device__ __forceinline__ double dm_d(const DevGeom& g, const float* wc, int ax, int ix, int iy,
                                       int iz, int64_t j) {
  const int ja = ax == 0 ? ix : (ax == 1 ? iy : iz);
  const int na = ax == 0 ? g.nx : (ax == 1 ? g.ny : g.nz);
  const int st = ax == 0 ? g.nz : (ax == 1 ? g.nx * g.nz : 1);
  double r = 0.0;
  if (ja < na - 1) r += wc[j];
  if (ja > 0) r -= wc[j - st];
  return r;
}

__global__ void k_prior_term(DevGeom g, int kind, const float* __restrict__ x, const float* __restrict__ w,
                             const float* __restrict__ side, double gamma_d, double eta2, double* partial) {
  __shared__ double sh[256];
  const int64_t N = (int64_t)g.nx * g.ny * g.nz;
  double acc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    const int iz = (int)(j % g.nz);
    const int64_t t = j / g.nz;
    const int ix = (int)(t % g.nx);
    const int iy = (int)(t / g.nx);
    double gr[3];
    grad_d(g, x, ix, iy, iz, j, gr);
    if (kind == SPDHG_PRIOR_ATV) {
      acc += fabs(gr[0]) + fabs(gr[1]) + fabs(gr[2]);
    } else if (kind == SPDHG_PRIOR_TGV) {
      const double a0 = gr[0] - w[j], a1 = gr[1] - w[N + j], a2 = gr[2] - w[2 * N + j];
      acc += sqrt(a0 * a0 + a1 * a1 + a2 * a2);  // weighted by alpha0 on the host
    } else {
      if (kind == SPDHG_PRIOR_DTV) {
        double gv[3];
        grad_d(g, side, ix, iy, iz, j, gv);
        const double inv = 1.0 / sqrt(gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2] + eta2);
        const double xi0 = gv[0] * inv, xi1 = gv[1] * inv, xi2 = gv[2] * inv;
        const double d = gamma_d * (xi0 * gr[0] + xi1 * gr[1] + xi2 * gr[2]);
        gr[0] -= d * xi0;
        gr[1] -= d * xi1;
        gr[2] -= d * xi2;
      }
      acc += sqrt(gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
    }
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// sum_k |E w|_F (TGV second term; weighted by alpha1 on the host)
__global__ void k_tgv_sym_term(DevGeom g, const float* __restrict__ w, double* partial) {
  __shared__ double sh[256];
  const int64_t N = (int64_t)g.nx * g.ny * g.nz;
  double acc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    const int iz = (int)(j % g.nz);
    const int64_t t = j / g.nz;
    const int ix = (int)(t % g.nx);
    const int iy = (int)(t / g.nx);
    const float* w0 = w;
    const float* w1 = w + N;
    const float* w2 = w + 2 * N;
    const double e0 = dm_d(g, w0, 0, ix, iy, iz, j);
    const double e1 = dm_d(g, w1, 1, ix, iy, iz, j);
    const double e2 = dm_d(g, w2, 2, ix, iy, iz, j);
    const double e3 = 0.5 * (dm_d(g, w1, 0, ix, iy, iz, j) + dm_d(g, w0, 1, ix, iy, iz, j));
    const double e4 = 0.5 * (dm_d(g, w2, 0, ix, iy, iz, j) + dm_d(g, w0, 2, ix, iy, iz, j));
    const double e5 = 0.5 * (dm_d(g, w2, 1, ix, iy, iz, j) + dm_d(g, w1, 2, ix, iy, iz, j));
    acc += sqrt(e0 * e0 + e1 * e1 + e2 * e2 + 2.0 * (e3 * e3 + e4 * e4 + e5 * e5));
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

cudaError_t launch_prior_term(const DevGeom& g, int kind, const float* x, const float* w,
                              const float* side, float gamma_d, float eta2, double* partial,
                              int nblocks, double* out, cudaStream_t s) {
  k_prior_term<<<nblocks, 256, 0, s>>>(g, kind, x, w, side, (double)gamma_d, (double)eta2, partial);
  k_finish_sum<<<1, 256, 0, s>>>(partial, nblocks, out);
  if (kind == SPDHG_PRIOR_TGV) {
    k_tgv_sym_term<<<nblocks, 256, 0, s>>>(g, w, partial);
    k_finish_sum<<<1, 256, 0, s>>>(partial, nblocks, out + 1);
  }
  return cudaGetLastError();
}

__global__ void k_side_max_grad(DevGeom g, const float* __restrict__ v, double* partial) {
  __shared__ double sh[256];
  const int64_t N = (int64_t)g.nx * g.ny * g.nz;
  double acc = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    const int iz = (int)(j % g.nz);
    const int64_t t = j / g.nz;
    const int ix = (int)(t % g.nx);
    const int iy = (int)(t / g.nx);
    double gv[3];
    grad_d(g, v, ix, iy, iz, j, gv);
    acc = fmax(acc, sqrt(gv[0] * gv[0] + gv[1] * gv[1] + gv[2] * gv[2]));
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + s]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

cudaError_t launch_side_max_grad(const DevGeom& g, const float* side, double* partial, int nblocks,
                                 double* out, cudaStream_t s) {
  k_side_max_grad<<<nblocks, 256, 0, s>>>(g, side, partial);
  k_finish_max<<<1, 256, 0, s>>>(partial, nblocks, out);
  return cudaGetLastError();
}

// PSNR terms (Sec. 4): out[0] = sum_j (x_j - xs_j)^2, out[1] = max_j |xs_j|, both in FP64
__global__ void k_psnr_terms(const float* __restrict__ x, const float* __restrict__ xs, int64_t n,
                             double* partial_sq, double* partial_max) {
  __shared__ double sh[256];
  double acc = 0.0, mx = 0.0;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
    const double d = (double)x[j] - (double)xs[j];
    acc += d * d;
    mx = fmax(mx, fabs((double)xs[j]));
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial_sq[blockIdx.x] = s;
  __syncthreads();
  sh[threadIdx.x] = mx;
  __syncthreads();
  for (int k = blockDim.x / 2; k > 0; k >>= 1) {
    if (threadIdx.x < k) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + k]);
    __syncthreads();
  }
  if (threadIdx.x == 0) partial_max[blockIdx.x] = sh[0];
}

cudaError_t launch_psnr_terms(const float* x, const float* xs, int64_t n, double* partial, int nblocks,
                              double* out, cudaStream_t s) {
  k_psnr_terms<<<nblocks, 256, 0, s>>>(x, xs, n, partial, partial + nblocks);
  k_finish_sum<<<1, 256, 0, s>>>(partial, nblocks, out);
  k_finish_max<<<1, 256, 0, s>>>(partial + nblocks, nblocks, out + 1);
  return cudaGetLastError();
}

}  // namespace spdhg
