// Prior block of SPDHG (block n of the generic problem, Eq. EQU:SETTING:TV):
//   q+ = prox_{sigma f_n*}(q + sigma A_n x),  dz = A_n^T (q+ - q),
// with A_n = grad (TV, aTV) or D grad (dTV), f_n = alpha||.||_{2,1} (TV, dTV) or alpha||.||_{1,1}
// (aTV), fused with the dual-sum update z += dz and the next primal step
// x = max(x - T (z + dz / p_n), 0).  grad is the forward difference with a zero last row
// (Neumann) at unit spacing.  The stencil reads x and q of the voxel and of its three lower
// neighbours, so x and q are ping-ponged (read *_in, write *_out) and tiles never race.
#include "internal.cuh"

namespace spdhg {

template <int KIND>
struct PriorStencil {
  const DevGeom& g;
  const PriorArgs& a;
  int64_t N;
  int sx, sy;

  __device__ __forceinline__ void xi_at(int jx, int jy, int jz, int64_t j, float xi[3]) const {
    const float* v = a.side;
    const float c = v[j];
    const float gx = jx < g.nx - 1 ? v[j + sx] - c : 0.f;
    const float gy = jy < g.ny - 1 ? v[j + sy] - c : 0.f;
    const float gz = jz < g.nz - 1 ? v[j + 1] - c : 0.f;
    const float inv = __frsqrt_rn(fmaf(gx, gx, fmaf(gy, gy, fmaf(gz, gz, a.eta2))));
    xi[0] = gx * inv;
    xi[1] = gy * inv;
    xi[2] = gz * inv;
  }

  // b = D (q+ - q) at voxel j (D = I for TV / aTV); optionally returns q+.
  __device__ __forceinline__ void dual(int jx, int jy, int jz, int64_t j, float b[3], float qn[3]) const {
    const float* x = a.x_in;
    const float c = x[j];
    float gr[3];
    gr[0] = jx < g.nx - 1 ? x[j + sx] - c : 0.f;
    gr[1] = jy < g.ny - 1 ? x[j + sy] - c : 0.f;
    gr[2] = jz < g.nz - 1 ? x[j + 1] - c : 0.f;
    float xi[3] = {0.f, 0.f, 0.f};
    if (KIND == SPDHG_PRIOR_DTV) {
      xi_at(jx, jy, jz, j, xi);
      const float d = xi[0] * gr[0] + xi[1] * gr[1] + xi[2] * gr[2];
      const float gd = a.gamma_d * d;
#pragma unroll
      for (int k = 0; k < 3; ++k) gr[k] -= gd * xi[k];
    }
    float qo[3], qa[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      qo[k] = a.q_in[k * N + j];
      qa[k] = fmaf(a.sigma, gr[k], qo[k]);
    }
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
};

template <int KIND>
__global__ void __launch_bounds__(256) k_prior(DevGeom g, PriorArgs a) {
  const int64_t N = (int64_t)g.nx * g.ny * g.nz;
  PriorStencil<KIND> st{g, a, N, g.nz, g.nx * g.nz};
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N; idx += (int64_t)gridDim.x * blockDim.x) {
    const int iz = (int)(idx % g.nz);
    const int64_t t = idx / g.nz;
    const int ix = (int)(t % g.nx);
    const int iy = (int)(t / g.nx);
    float b[3], qn[3], bm[3], tmp[3];
    st.dual(ix, iy, iz, idx, b, qn);
#pragma unroll
    for (int k = 0; k < 3; ++k) a.q_out[k * N + idx] = qn[k];
    // dz = A_n^T dq:  sum_a [k_a >= 1] b_a(k - e_a) - [k_a < n_a - 1] b_a(k)
    float dz = 0.f;
    if (ix < g.nx - 1) dz -= b[0];
    if (iy < g.ny - 1) dz -= b[1];
    if (iz < g.nz - 1) dz -= b[2];
    if (ix > 0) {
      st.dual(ix - 1, iy, iz, idx - st.sx, bm, tmp);
      dz += bm[0];
    }
    if (iy > 0) {
      st.dual(ix, iy - 1, iz, idx - st.sy, bm, tmp);
      dz += bm[1];
    }
    if (iz > 0) {
      st.dual(ix, iy, iz - 1, idx - 1, bm, tmp);
      dz += bm[2];
    }
    const float zn = a.z[idx] + dz;
    a.z[idx] = zn;
    a.x_out[idx] = fmaxf(a.x_in[idx] - a.T[idx] * fmaf(dz, a.inv_p, zn), 0.f);
  }
}

cudaError_t launch_prior(const DevGeom& g, const PriorArgs& a, cudaStream_t s) {
  const int64_t N = (int64_t)g.nx * g.ny * g.nz;
  int64_t blocks = (N + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  switch (a.kind) {
    case SPDHG_PRIOR_TV: k_prior<SPDHG_PRIOR_TV><<<(int)blocks, 256, 0, s>>>(g, a); break;
    case SPDHG_PRIOR_DTV: k_prior<SPDHG_PRIOR_DTV><<<(int)blocks, 256, 0, s>>>(g, a); break;
    case SPDHG_PRIOR_ATV: k_prior<SPDHG_PRIOR_ATV><<<(int)blocks, 256, 0, s>>>(g, a); break;
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
