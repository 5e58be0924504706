// Prior block of SPDHG (block n of the generic problem, Eq. EQU:SETTING:TV):
//   q+ = prox_{sigma f_n*}(q + sigma A_n x),  dz = A_n^T (q+ - q),
// with A_n = grad (TV, aTV) or D grad (dTV), f_n = alpha||.||_{2,1} (TV, dTV) or alpha||.||_{1,1}
// (aTV), fused with the dual-sum update z += dz and the next primal step
// x = max(x - T (z + dz / p_n), 0).  grad is the forward difference with a zero last row
// (Neumann) at unit spacing.  The stencil reads x and q of the voxel and of its three lower
// neighbours, so x and q are ping-ponged (read *_in, write *_out) and tiles never race.
#include <algorithm>

#include "internal.cuh"

namespace spdhg {

// Dual update of one voxel: g = A_n x (forward differences; dTV: D g with
// D = I - gamma_d xi xi^T, xi = grad v / sqrt(|grad v|^2 + eta^2)), q+ = proj(q + sigma g),
// b = D^T (q+ - q).  Returns b and q+.
template <int KIND>
__device__ __forceinline__ void dual_update(const PriorArgs& a, const float gr_in[3], const float gv[3],
                                            const float qo[3], float b[3], float qn[3]) {
  float gr[3] = {gr_in[0], gr_in[1], gr_in[2]};
  float xi[3] = {0.f, 0.f, 0.f};
  if (KIND == SPDHG_PRIOR_DTV) {
    const float inv = __frsqrt_rn(fmaf(gv[0], gv[0], fmaf(gv[1], gv[1], fmaf(gv[2], gv[2], a.eta2))));
#pragma unroll
    for (int k = 0; k < 3; ++k) xi[k] = gv[k] * inv;
    const float gd = a.gamma_d * (xi[0] * gr[0] + xi[1] * gr[1] + xi[2] * gr[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) gr[k] -= gd * xi[k];
  }
  float qa[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) qa[k] = fmaf(a.sigma, gr[k], qo[k]);
  if (KIND == SPDHG_PRIOR_ATV) {
#pragma unroll
    for (int k = 0; k < 3; ++k) qn[k] = fminf(fmaxf(qa[k], -a.alpha), a.alpha);
  } else {
    const float nrm = sqrtf(qa[0] * qa[0] + qa[1] * qa[1] + qa[2] * qa[2]);
    const float sc = fmaxf(1.f, nrm / a.alpha);
#pragma unroll
    for (int k = 0; k < 3; ++k) qn[k] = qa[k] / sc;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) b[k] = qn[k] - qo[k];
  if (KIND == SPDHG_PRIOR_DTV) {
    const float d = a.gamma_d * (xi[0] * b[0] + xi[1] * b[1] + xi[2] * b[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) b[k] -= d * xi[k];
  }
}

// One block owns `cols - 1` voxel columns in x (plus one halo column on the lower side whose
// duals are recomputed, not written) and the whole z extent (warps along z, so every access is
// a contiguous 128-byte line), and marches along y over `ychunk` rows (plus one warm-up row).
// The dual change of the lower y neighbour is carried in registers, the lower x neighbour's in
// shared memory and the lower z neighbour's by a warp shuffle, so each voxel's dual is computed
// once (plus the halo) and every array is streamed once.
// Operands of one voxel row step, loaded one row ahead (software pipelining): the loads of
// row iy + 1 are in flight while row iy is computed.
struct RowLoads {
  float xz, xx, vz, vx, q0, q1, q2, zv, tv;
};

template <int KIND>
__device__ __forceinline__ void load_row(const PriorArgs& a, int64_t idx, int64_t N, int sx, bool hx, bool hz,
                                         bool owner, float xc, float vc, RowLoads& L) {
  L.xz = hz ? __ldg(a.x_in + idx + 1) : xc;
  L.xx = hx ? __ldg(a.x_in + idx + sx) : xc;
  if (KIND == SPDHG_PRIOR_DTV) {
    L.vz = hz ? __ldg(a.side + idx + 1) : vc;
    L.vx = hx ? __ldg(a.side + idx + sx) : vc;
  } else {
    L.vz = L.vx = 0.f;
  }
  L.q0 = __ldg(a.q_in + idx);
  L.q1 = __ldg(a.q_in + N + idx);
  L.q2 = __ldg(a.q_in + 2 * N + idx);
  L.zv = owner ? a.z[idx] : 0.f;  // z and T only matter where the block writes
  L.tv = owner ? __ldg(a.T + idx) : 0.f;
}

// One block owns `cols - 1` voxel columns in x (plus one halo column on the lower side whose
// duals are recomputed, not written) and the whole z extent (warps along z, so every access is
// a contiguous 128-byte line), and marches along y over `ychunk` rows (plus one warm-up row).
// The dual change of the lower y neighbour is carried in registers, the lower x neighbour's in
// shared memory and the lower z neighbour's by a warp shuffle, so each voxel's dual is computed
// once (plus the halo) and every array is streamed once.  Loads run one row (x, v: two rows)
// ahead of the arithmetic.
template <int KIND>
__global__ void __launch_bounds__(1024) k_prior(DevGeom g, PriorArgs a, int cols, int ychunk) {
  extern __shared__ float sh[];
  const int zw = (g.nz + 31) >> 5;           // warps per column
  float* sbx = sh;                            // [cols][zw * 32]: b_x of the current row
  float* sbz = sh + cols * zw * 32;           // [cols][zw]: b_z of lane 31 of each z-warp
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = w / zw, zi = w - c * zw;
  const int ix = blockIdx.x * (cols - 1) + c - 1;
  const int iz = zi * 32 + lane;
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int64_t N = (int64_t)nx * ny * nz;
  const int sx = nz;
  const int64_t sy = (int64_t)nx * nz;
  const bool live = ix >= 0 && ix < nx && iz < nz;
  const bool owner = live && c >= 1;
  const int y0 = blockIdx.y * ychunk, y1 = min(ny, y0 + ychunk);
  const bool hx = ix < nx - 1, hz = iz < nz - 1;

  int iy = y0 > 0 ? y0 - 1 : 0;
  int64_t idx = live ? ((int64_t)iy * nx + ix) * nz + iz : 0;
  float xc = 0.f, vc = 0.f, xn = 0.f, vn = 0.f;
  RowLoads cur{};
  if (live) {
    xc = __ldg(a.x_in + idx);
    if (KIND == SPDHG_PRIOR_DTV) vc = __ldg(a.side + idx);
    const bool hy = iy < ny - 1;
    xn = hy ? __ldg(a.x_in + idx + sy) : xc;
    if (KIND == SPDHG_PRIOR_DTV) vn = hy ? __ldg(a.side + idx + sy) : vc;
    load_row<KIND>(a, idx, N, sx, hx, hz, owner, xc, vc, cur);
  }
  float by_prev = 0.f;
  for (; iy < y1; ++iy, idx += sy) {
    const bool hy = iy < ny - 1;
    // prefetch: operands of row iy + 1, and x, v of row iy + 2
    RowLoads nxt = cur;
    float xnn = xn, vnn = vn;
    const bool more = live && iy + 1 < y1;
    if (more) {
      load_row<KIND>(a, idx + sy, N, sx, hx, hz, owner, xn, vn, nxt);
      const bool hy1 = iy + 1 < ny - 1;
      xnn = hy1 ? __ldg(a.x_in + idx + 2 * sy) : xn;
      if (KIND == SPDHG_PRIOR_DTV) vnn = hy1 ? __ldg(a.side + idx + 2 * sy) : vn;
    }
    float b[3] = {0.f, 0.f, 0.f}, qn[3] = {0.f, 0.f, 0.f};
    if (live) {
      const float gr[3] = {cur.xx - xc, hy ? xn - xc : 0.f, cur.xz - xc};
      float gv[3] = {0.f, 0.f, 0.f};
      if (KIND == SPDHG_PRIOR_DTV) {
        gv[0] = cur.vx - vc;
        gv[1] = hy ? vn - vc : 0.f;
        gv[2] = cur.vz - vc;
      }
      const float qo[3] = {cur.q0, cur.q1, cur.q2};
      dual_update<KIND>(a, gr, gv, qo, b, qn);
    }
    const float bz_lo = __shfl_up_sync(0xffffffffu, b[2], 1);
    sbx[c * zw * 32 + zi * 32 + lane] = b[0];
    if (lane == 31) sbz[c * zw + zi] = b[2];
    __syncthreads();
    if (owner && iy >= y0) {
      a.q_out[idx] = qn[0];
      a.q_out[N + idx] = qn[1];
      a.q_out[2 * N + idx] = qn[2];
      // dz = A_n^T dq = sum_a [k_a >= 1] b_a(k - e_a) - [k_a < n_a - 1] b_a(k)
      float dz = 0.f;
      if (ix > 0) dz += sbx[(c - 1) * zw * 32 + zi * 32 + lane];
      if (iy > 0) dz += by_prev;
      if (iz > 0) dz += lane > 0 ? bz_lo : sbz[c * zw + zi - 1];
      if (hx) dz -= b[0];
      if (hy) dz -= b[1];
      if (hz) dz -= b[2];
      const float zn = cur.zv + dz;
      a.z[idx] = zn;
      a.x_out[idx] = fmaxf(xc - cur.tv * fmaf(dz, a.inv_p, zn), 0.f);
    }
    by_prev = b[1];
    xc = xn;
    vc = vn;
    xn = xnn;
    vn = vnn;
    cur = nxt;
    __syncthreads();
  }
}

cudaError_t launch_prior(const DevGeom& g, const PriorArgs& a, cudaStream_t s) {
  const int zw = (g.nz + 31) / 32;
  if (zw > 16) return cudaErrorInvalidValue;
  const int cols = g.tune[SPDHG_TUNE_PRIOR_COLS] ? g.tune[SPDHG_TUNE_PRIOR_COLS]
                                                 : std::max(2, std::min(16 / zw, g.nx + 1));
  const int ychunk = g.tune[SPDHG_TUNE_PRIOR_YCHUNK] ? g.tune[SPDHG_TUNE_PRIOR_YCHUNK] : 16;
  if (cols * zw > 32) return cudaErrorInvalidValue;
  const size_t smem = (size_t)cols * zw * 33 * sizeof(float);
  dim3 grid((g.nx + cols - 2) / (cols - 1), (g.ny + ychunk - 1) / ychunk);
  const int threads = cols * zw * 32;
  switch (a.kind) {
    case SPDHG_PRIOR_TV: k_prior<SPDHG_PRIOR_TV><<<grid, threads, smem, s>>>(g, a, cols, ychunk); break;
    case SPDHG_PRIOR_DTV: k_prior<SPDHG_PRIOR_DTV><<<grid, threads, smem, s>>>(g, a, cols, ychunk); break;
    case SPDHG_PRIOR_ATV: k_prior<SPDHG_PRIOR_ATV><<<grid, threads, smem, s>>>(g, a, cols, ychunk); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// TGV (Sec. 4.3): x = (u, w); block n-1: A = (grad, -I), f = alpha0 ||.||_{2,1};
// block n: A = (0, E), f = alpha1 ||.||_{2,1} with E the symmetrised gradient built from the
// backward difference d-_a = -D_a^T (components xx, yy, zz, xy, xz, yz; off-diagonals count
// twice in the norm).
// ---------------------------------------------------------------------------------------

__global__ void k_w_step(int64_t n, float* __restrict__ w, const float* __restrict__ zw, float Tw) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    w[i] = w[i] - Tw * zw[i];
}

cudaError_t launch_w_step(const DevGeom& g, float* w, const float* zw, float Tw, cudaStream_t s) {
  const int64_t n = 3 * (int64_t)g.nx * g.ny * g.nz;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  k_w_step<<<(int)blocks, 256, 0, s>>>(n, w, zw, Tw);
  return cudaGetLastError();
}

// block 0: q+ = proj_{alpha0}(q + sigma (grad u - w)); dq = q+ - q; dzu = grad^T dq, dzw = -dq
struct Tgv0 {
  const DevGeom& g;
  const TgvArgs& a;
  int64_t N;
  int sx, sy;
  __device__ __forceinline__ void dual(int jx, int jy, int jz, int64_t j, float b[3], float qn[3]) const {
    const float* u = a.u_in;
    const float c = u[j];
    float gr[3];
    gr[0] = jx < g.nx - 1 ? u[j + sx] - c : 0.f;
    gr[1] = jy < g.ny - 1 ? u[j + sy] - c : 0.f;
    gr[2] = jz < g.nz - 1 ? u[j + 1] - c : 0.f;
    float qo[3], qa[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      qo[k] = a.q_in[k * N + j];
      qa[k] = fmaf(a.sigma, gr[k] - a.w_in[k * N + j], qo[k]);
    }
    const float nrm = sqrtf(qa[0] * qa[0] + qa[1] * qa[1] + qa[2] * qa[2]);
    const float sc = fmaxf(1.f, nrm / a.alpha);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      qn[k] = qa[k] / sc;
      b[k] = qn[k] - qo[k];
    }
  }
};

__global__ void __launch_bounds__(256) k_tgv0(DevGeom g, TgvArgs a) {
  const int64_t N = (int64_t)g.nx * g.ny * g.nz;
  Tgv0 st{g, a, N, g.nz, g.nx * g.nz};
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N; idx += (int64_t)gridDim.x * blockDim.x) {
    const int iz = (int)(idx % g.nz);
    const int64_t t = idx / g.nz;
    const int ix = (int)(t % g.nx);
    const int iy = (int)(t / g.nx);
    float b[3], qn[3], bm[3], tmp[3];
    st.dual(ix, iy, iz, idx, b, qn);
    float dz = 0.f;
    if (ix < g.nx - 1) dz -= b[0];
    if (iy < g.ny - 1) dz -= b[1];
    if (iz < g.nz - 1) dz -= b[2];
    if (ix > 0) { st.dual(ix - 1, iy, iz, idx - st.sx, bm, tmp); dz += bm[0]; }
    if (iy > 0) { st.dual(ix, iy - 1, iz, idx - st.sy, bm, tmp); dz += bm[1]; }
    if (iz > 0) { st.dual(ix, iy, iz - 1, idx - 1, bm, tmp); dz += bm[2]; }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      a.q_out[k * N + idx] = qn[k];
      // w part: dzw = -dq;  zw += dzw;  w = w - Tw (zw + dzw / p)
      const float dzw = -b[k];
      const float zwn = a.zw[k * N + idx] + dzw;
      a.zw[k * N + idx] = zwn;
      a.w_out[k * N + idx] = a.w_in[k * N + idx] - a.Tw * fmaf(dzw, a.inv_p, zwn);
    }
    const float zn = a.zu[idx] + dz;
    a.zu[idx] = zn;
    a.u_out[idx] = fmaxf(a.u_in[idx] - a.Tu[idx] * fmaf(dz, a.inv_p, zn), 0.f);
  }
}

// block 1: q+ = proj_{alpha1}(q + sigma E w); dq; dzw = E^T dq; u only takes its primal step.
struct Tgv1 {
  const DevGeom& g;
  const TgvArgs& a;
  int64_t N;
  int sx, sy;
  // backward difference of w component c along axis ax at voxel j (d-_a = -D_a^T)
  __device__ __forceinline__ float dm(int c, int ax, int jx, int jy, int jz, int64_t j) const {
    const float* wc = a.w_in + c * N;
    const int ja = ax == 0 ? jx : (ax == 1 ? jy : jz);
    const int na = ax == 0 ? g.nx : (ax == 1 ? g.ny : g.nz);
    const int st = ax == 0 ? sx : (ax == 1 ? sy : 1);
    float r = 0.f;
    if (ja < na - 1) r += wc[j];
    if (ja > 0) r -= wc[j - st];
    return r;
  }
  __device__ __forceinline__ void dual(int jx, int jy, int jz, int64_t j, float b[6], float qn[6]) const {
    float e[6];
    e[0] = dm(0, 0, jx, jy, jz, j);
    e[1] = dm(1, 1, jx, jy, jz, j);
    e[2] = dm(2, 2, jx, jy, jz, j);
    e[3] = 0.5f * (dm(1, 0, jx, jy, jz, j) + dm(0, 1, jx, jy, jz, j));
    e[4] = 0.5f * (dm(2, 0, jx, jy, jz, j) + dm(0, 2, jx, jy, jz, j));
    e[5] = 0.5f * (dm(2, 1, jx, jy, jz, j) + dm(1, 2, jx, jy, jz, j));
    float qo[6], qa[6];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      qo[k] = a.q_in[k * N + j];
      qa[k] = fmaf(a.sigma, e[k], qo[k]);
    }
    const float n2 = qa[0] * qa[0] + qa[1] * qa[1] + qa[2] * qa[2] +
                     2.f * (qa[3] * qa[3] + qa[4] * qa[4] + qa[5] * qa[5]);
    const float sc = fmaxf(1.f, sqrtf(n2) / a.alpha);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      qn[k] = qa[k] / sc;
      b[k] = qn[k] - qo[k];
    }
  }
};

__global__ void __launch_bounds__(256) k_tgv1(DevGeom g, TgvArgs a) {
  const int64_t N = (int64_t)g.nx * g.ny * g.nz;
  Tgv1 st{g, a, N, g.nz, g.nx * g.nz};
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N; idx += (int64_t)gridDim.x * blockDim.x) {
    const int iz = (int)(idx % g.nz);
    const int64_t t = idx / g.nz;
    const int ix = (int)(t % g.nx);
    const int iy = (int)(t / g.nx);
    float b[6], qn[6], bp[6], tmp[6];
    st.dual(ix, iy, iz, idx, b, qn);
#pragma unroll
    for (int k = 0; k < 6; ++k) a.q_out[k * N + idx] = qn[k];
    // (d-_a)^T = -D_a:  ((d-_a)^T p)(k) = p(k) - p(k + e_a) for k_a < n_a - 1, else 0.
    // E^T dq:  w_c += sum over entries (a,b) of E containing d-_a w_c, weights 1 (diag) or 1
    // (off-diagonal: 2 in the inner product times the 1/2 of the definition).
    float up[3][6];  // dq at k + e_a for a = x, y, z
    const bool hx = ix < g.nx - 1, hy = iy < g.ny - 1, hz = iz < g.nz - 1;
    if (hx) st.dual(ix + 1, iy, iz, idx + st.sx, up[0], tmp);
    if (hy) st.dual(ix, iy + 1, iz, idx + st.sy, up[1], tmp);
    if (hz) st.dual(ix, iy, iz + 1, idx + 1, up[2], tmp);
    auto dmT = [&](int comp, int ax) -> float {
      const bool h = ax == 0 ? hx : (ax == 1 ? hy : hz);
      return h ? b[comp] - up[ax][comp] : 0.f;
    };
    float dzw[3];
    dzw[0] = dmT(0, 0) + dmT(3, 1) + dmT(4, 2);
    dzw[1] = dmT(1, 1) + dmT(3, 0) + dmT(5, 2);
    dzw[2] = dmT(2, 2) + dmT(4, 0) + dmT(5, 1);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const float zwn = a.zw[k * N + idx] + dzw[k];
      a.zw[k * N + idx] = zwn;
      a.w_out[k * N + idx] = a.w_in[k * N + idx] - a.Tw * fmaf(dzw[k], a.inv_p, zwn);
    }
    // u: no change of z_u in this block; zbar_u = z_u
    a.u_out[idx] = fmaxf(a.u_in[idx] - a.Tu[idx] * a.zu[idx], 0.f);
  }
}

cudaError_t launch_tgv(const DevGeom& g, const TgvArgs& a, cudaStream_t s) {
  const int64_t N = (int64_t)g.nx * g.ny * g.nz;
  int64_t blocks = (N + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (a.block == 0) k_tgv0<<<(int)blocks, 256, 0, s>>>(g, a);
  else k_tgv1<<<(int)blocks, 256, 0, s>>>(g, a);
  return cudaGetLastError();
}

}  // namespace spdhg
