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
// b = D^T (q+ - q).  The ball projection q+ = qa min(1, alpha / |qa|) uses one reciprocal
// square root.  Returns b and q+.
template <int KIND>
__device__ __forceinline__ void dual_update(const PriorArgs& a, const float gr_in[3], const float gv[3],
                                            const float qo[3], float b[3], float qn[3]) {
  float gr[3] = {gr_in[0], gr_in[1], gr_in[2]};
  float xi[3] = {0.f, 0.f, 0.f};
  if (KIND == SPDHG_PRIOR_DTV) {
    const float inv = rsqrtf(fmaf(gv[0], gv[0], fmaf(gv[1], gv[1], fmaf(gv[2], gv[2], a.eta2))));
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
    const float n2 = fmaf(qa[0], qa[0], fmaf(qa[1], qa[1], qa[2] * qa[2]));
    const float sc = fminf(1.f, a.alpha * rsqrtf(n2));  // n2 = 0 gives +inf -> 1
#pragma unroll
    for (int k = 0; k < 3; ++k) qn[k] = qa[k] * sc;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) b[k] = qn[k] - qo[k];
  if (KIND == SPDHG_PRIOR_DTV) {
    const float d = a.gamma_d * (xi[0] * b[0] + xi[1] * b[1] + xi[2] * b[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) b[k] -= d * xi[k];
  }
}

// 4-byte asynchronous global -> shared copy; src_bytes = 0 fills the destination with zero.
// `base` is a valid address of the same array, used as the (unread) source when !valid.
__device__ __forceinline__ void cp_async4(float* dst, const float* base, int off, bool valid) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  const float* src = valid ? base + off : base;
  const int n = valid ? 4 : 0;
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(d), "l"(src), "r"(n) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Row pipeline depth STAGES: rows iy and iy + 1 of x (and v) are used, the next STAGES - 2 rows
// are loading.

// One block owns `cols - 1` voxel columns in x (plus one halo column on the lower side whose
// duals are recomputed, not written) and the whole z extent, and marches along y over `ychunk`
// rows (plus one warm-up row).  A thread holds VZ voxels of one column, z = z0 + lane + 32 k
// (k < VZ), so every warp access is a contiguous 128-byte line and the per-row work of the
// thread (addresses, barriers, pipeline control) is shared by VZ voxels.  x and v, whose
// neighbours other threads need, are staged in shared memory by a STAGES-deep cp.async pipeline
// (each thread copies its own voxels, the halo warps also one upper halo column); q, z and T are
// read by their own thread only and go straight into registers, one row ahead.  The lower y
// neighbour's dual change is carried in a register and the lower x / z neighbours' through
// shared memory.  Every array is read from HBM once per row.
template <int KIND, int STAGES, int VZ>
__global__ void __launch_bounds__(1024) k_prior(DevGeom g, PriorArgs a, int cols, int ychunk) {
  extern __shared__ float sh[];
  const int zw = (g.nz + 32 * VZ - 1) / (32 * VZ);  // warps per column
  const int zc = zw * 32 * VZ;                      // staged z extent
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int c = w / zw, zi = w - c * zw;
  const int iz0 = zi * 32 * VZ + lane;              // voxel k of this thread: iz0 + 32 k
  const int nx = g.nx, ny = g.ny, nz = g.nz;
  const int N = nx * ny * nz;
  const int sy = nx * nz;
  const int x0 = blockIdx.x * (cols - 1) - 1;       // x of column 0 (the lower halo)
  const int ix = x0 + c;
  const bool col_live = ix >= 0 && ix < nx;
  const bool col_owner = col_live && c >= 1;
  const int y0 = blockIdx.y * ychunk, y1 = min(ny, y0 + ychunk);
  const int ys = y0 > 0 ? y0 - 1 : 0;               // first row computed (warm-up row for y0 > 0)
  const int ylast = min(y1, ny - 1);                // last row whose x / v are needed
  const bool hx = ix < nx - 1;
  const bool dtv = KIND == SPDHG_PRIOR_DTV;
  const int ixh = x0 + cols;                        // upper halo column (x, v only)
  const bool colh = ixh < nx;

  // stage layout per row: x, v: (cols + 1) x zc
  const int xv_sz = (cols + 1) * zc;
  const int stage_sz = dtv ? 2 * xv_sz : xv_sz;
  float* sbx = sh + STAGES * stage_sz;              // [cols][zc] b_x of the current row
  float* sbz = sbx + cols * zc;                     // [cols][zc] b_z of the current row
  const int me = c * zc + iz0;

  auto issue_row = [&](int row) {
    float* st = sh + (row % STAGES) * stage_sz;
    const int base = row * sy + ix * nz + iz0;      // only dereferenced when valid
#pragma unroll
    for (int k = 0; k < VZ; ++k) {
      const bool lv = col_live && iz0 + 32 * k < nz;
      cp_async4(st + me + 32 * k, a.x_in, base + 32 * k, lv);
      if (dtv) cp_async4(st + xv_sz + me + 32 * k, a.side, base + 32 * k, lv);
    }
    if (c == 0) {  // upper halo column: x and v of x0 + cols
      const int bh = row * sy + ixh * nz + iz0;
#pragma unroll
      for (int k = 0; k < VZ; ++k) {
        const bool vh = colh && iz0 + 32 * k < nz;
        cp_async4(st + cols * zc + iz0 + 32 * k, a.x_in, bh + 32 * k, vh);
        if (dtv) cp_async4(st + xv_sz + cols * zc + iz0 + 32 * k, a.side, bh + 32 * k, vh);
      }
    }
  };
  // q of every live voxel (the halo column's duals are recomputed), z and T of the owned ones
  float qr[VZ][3], zr[VZ], Tr[VZ];
  auto load_regs = [&](int row) {
    const int base = row * sy + ix * nz + iz0;
#pragma unroll
    for (int k = 0; k < VZ; ++k) {
      const bool lv = col_live && iz0 + 32 * k < nz;
      const bool ow = lv && c >= 1;
      const int i = base + 32 * k;
      qr[k][0] = lv ? a.q_in[i] : 0.f;
      qr[k][1] = lv ? a.q_in[N + i] : 0.f;
      qr[k][2] = lv ? a.q_in[2 * N + i] : 0.f;
      zr[k] = ow ? a.z[i] : 0.f;
      Tr[k] = ow ? a.T[i] : 0.f;
    }
  };

  for (int k = 0; k < STAGES - 1; ++k) {
    if (ys + k <= ylast) issue_row(ys + k);
    cp_async_commit();
  }
  load_regs(ys);
  float by_prev[VZ];
#pragma unroll
  for (int k = 0; k < VZ; ++k) by_prev[k] = 0.f;
  for (int iy = ys; iy < y1; ++iy) {
    if (iy + STAGES - 1 <= ylast) issue_row(iy + STAGES - 1);
    cp_async_commit();
    // this row's q, z, T; the next row's are requested before this row's arithmetic
    float qo[VZ][3], zo[VZ], To[VZ];
#pragma unroll
    for (int k = 0; k < VZ; ++k) {
      qo[k][0] = qr[k][0];
      qo[k][1] = qr[k][1];
      qo[k][2] = qr[k][2];
      zo[k] = zr[k];
      To[k] = Tr[k];
    }
    if (iy + 1 < y1) load_regs(iy + 1);
    cp_async_wait<STAGES - 2>();  // rows iy and iy + 1 of x, v have landed
    __syncthreads();
    const float* st = sh + (iy % STAGES) * stage_sz;
    const float* sn = sh + ((iy + 1) % STAGES) * stage_sz;
    const bool hy = iy < ny - 1;
    float b[VZ][3], qn[VZ][3], xc[VZ];
#pragma unroll
    for (int k = 0; k < VZ; ++k) {
      const int iz = iz0 + 32 * k, m = me + 32 * k;
      const bool lv = col_live && iz < nz, hz = iz < nz - 1;
      b[k][0] = b[k][1] = b[k][2] = 0.f;
      qn[k][0] = qn[k][1] = qn[k][2] = 0.f;
      xc[k] = st[m];
      if (lv) {
        const float gr[3] = {hx ? st[m + zc] - xc[k] : 0.f, hy ? sn[m] - xc[k] : 0.f, hz ? st[m + 1] - xc[k] : 0.f};
        float gv[3] = {0.f, 0.f, 0.f};
        if (dtv) {
          const float* sv = st + xv_sz;
          const float vc = sv[m];
          gv[0] = hx ? sv[m + zc] - vc : 0.f;
          gv[1] = hy ? sn[xv_sz + m] - vc : 0.f;
          gv[2] = hz ? sv[m + 1] - vc : 0.f;
        }
        dual_update<KIND>(a, gr, gv, qo[k], b[k], qn[k]);
      }
      sbx[m] = b[k][0];
      sbz[m] = b[k][2];
    }
    __syncthreads();
    if (col_owner && iy >= y0) {
#pragma unroll
      for (int k = 0; k < VZ; ++k) {
        const int iz = iz0 + 32 * k, m = me + 32 * k;
        if (iz >= nz) continue;
        const int idx = iy * sy + ix * nz + iz;
        a.q_out[idx] = qn[k][0];
        a.q_out[N + idx] = qn[k][1];
        a.q_out[2 * N + idx] = qn[k][2];
        // dz = A_n^T dq = sum_a [k_a >= 1] b_a(k - e_a) - [k_a < n_a - 1] b_a(k)
        float dz = 0.f;
        if (ix > 0) dz += sbx[m - zc];
        if (iy > 0) dz += by_prev[k];
        if (iz > 0) dz += sbz[m - 1];
        if (hx) dz -= b[k][0];
        if (hy) dz -= b[k][1];
        if (iz < nz - 1) dz -= b[k][2];
        const float zn = zo[k] + dz;
        a.z[idx] = zn;
        a.x_out[idx] = prox_nonneg(xc[k] - To[k] * fmaf(dz, a.inv_p, zn));
      }
    }
#pragma unroll
    for (int k = 0; k < VZ; ++k) by_prev[k] = b[k][1];
    __syncthreads();  // stage iy % S is refilled by the next iteration's copy
  }
  cp_async_wait<0>();
}

// voxels per thread along z (more columns per block: a smaller halo share, but fewer blocks)
static int prior_vz(const DevGeom& g) { return g.tune[SPDHG_TUNE_PRIOR_VZ] ? g.tune[SPDHG_TUNE_PRIOR_VZ] : 1; }

// launch shape of the prior kernel at the current knobs; false where they do not fit together
static bool prior_shape(const DevGeom& g, bool dtv, int* vz_out, int* zw_out, int* cols_out, int* ychunk_out,
                        int* stages_out, size_t* smem_out) {
  const int vz = prior_vz(g);
  if (vz != 1 && vz != 2 && vz != 4) return false;
  const int zw = (g.nz + 32 * vz - 1) / (32 * vz);
  if (zw > 16) return false;
  const int cols = g.tune[SPDHG_TUNE_PRIOR_COLS] ? g.tune[SPDHG_TUNE_PRIOR_COLS]
                                                 : std::max(2, std::min(std::min(16, 32 / zw), g.nx + 1));
  const int gx = (g.nx + cols - 2) / (cols - 1);
  const int chunks = std::max(1, std::min(g.ny, 152 / gx));
  const int ychunk = g.tune[SPDHG_TUNE_PRIOR_YCHUNK] ? g.tune[SPDHG_TUNE_PRIOR_YCHUNK] : (g.ny + chunks - 1) / chunks;
  const int stages = g.tune[SPDHG_TUNE_PRIOR_STAGES] ? g.tune[SPDHG_TUNE_PRIOR_STAGES] : 4;
  if (cols * zw > 32 || (stages != 3 && stages != 4)) return false;
  const size_t zc = (size_t)zw * 32 * vz;
  const size_t stage = (size_t)(dtv ? 2 : 1) * (cols + 1) * zc;
  const size_t smem = (stages * stage + 2 * (size_t)cols * zc) * sizeof(float);
  if (smem > 227 * 1024) return false;
  *vz_out = vz; *zw_out = zw; *cols_out = cols; *ychunk_out = ychunk; *stages_out = stages; *smem_out = smem;
  return true;
}

bool prior_launch_ok(const DevGeom& g, int kind) {
  int vz, zw, cols, ychunk, stages;
  size_t smem;
  return prior_shape(g, kind == SPDHG_PRIOR_DTV, &vz, &zw, &cols, &ychunk, &stages, &smem);
}

cudaError_t launch_prior(const DevGeom& g, const PriorArgs& a, cudaStream_t s) {
  int vz, zw, cols, ychunk, stages;
  size_t smem;
  if (!prior_shape(g, a.kind == SPDHG_PRIOR_DTV, &vz, &zw, &cols, &ychunk, &stages, &smem)) return cudaErrorInvalidValue;
  dim3 grid((g.nx + cols - 2) / (cols - 1), (g.ny + ychunk - 1) / ychunk);
  const int threads = cols * zw * 32;
  auto launch = [&](auto kern) -> cudaError_t {
    cudaError_t e = allow_dynamic_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<grid, threads, smem, s>>>(g, a, cols, ychunk);
    return cudaGetLastError();
  };
  auto by_shape = [&](auto k31, auto k32, auto k34, auto k41, auto k42, auto k44) -> cudaError_t {
    if (stages == 3) return vz == 1 ? launch(k31) : (vz == 2 ? launch(k32) : launch(k34));
    return vz == 1 ? launch(k41) : (vz == 2 ? launch(k42) : launch(k44));
  };
#define SPDHG_PRIOR_SHAPES(K) \
  k_prior<K, 3, 1>, k_prior<K, 3, 2>, k_prior<K, 3, 4>, k_prior<K, 4, 1>, k_prior<K, 4, 2>, k_prior<K, 4, 4>
  switch (a.kind) {
    case SPDHG_PRIOR_TV: return by_shape(SPDHG_PRIOR_SHAPES(SPDHG_PRIOR_TV));
    case SPDHG_PRIOR_DTV: return by_shape(SPDHG_PRIOR_SHAPES(SPDHG_PRIOR_DTV));
    case SPDHG_PRIOR_ATV: return by_shape(SPDHG_PRIOR_SHAPES(SPDHG_PRIOR_ATV));
    default: return cudaErrorInvalidValue;
  }
#undef SPDHG_PRIOR_SHAPES
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

// Each TGV block runs in two passes: the dual pass computes q+ = proj(q + sigma A x) and the dual
// change b = q+ - q once per voxel (written to a scratch array), the primal pass forms A^T b from
// b and its neighbours and takes the z, w and u steps.  The arithmetic per voxel, and the order
// of every sum, is that of computing the neighbours' dual changes in place.

// block 0: q+ = proj_{alpha0}(q + sigma (grad u - w)); b = q+ - q
__global__ void __launch_bounds__(256) k_tgv0_dual(DevGeom g, TgvArgs a) {
  const int64_t N = (int64_t)g.nx * g.ny * g.nz;
  const int sx = g.nz, sy = g.nx * g.nz;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    const int jz = (int)(j % g.nz);
    const int64_t t = j / g.nz;
    const int jx = (int)(t % g.nx), jy = (int)(t / g.nx);
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
      const float qn = qa[k] / sc;
      a.q_out[k * N + j] = qn;
      a.bscr[k * N + j] = qn - qo[k];
    }
  }
}

// block 0: dzu = grad^T b, dzw = -b; z and primal steps of u and w
__global__ void __launch_bounds__(256) k_tgv0_primal(DevGeom g, TgvArgs a) {
  const int64_t N = (int64_t)g.nx * g.ny * g.nz;
  const int sx = g.nz, sy = g.nx * g.nz;
  const float* bs = a.bscr;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N; idx += (int64_t)gridDim.x * blockDim.x) {
    const int iz = (int)(idx % g.nz);
    const int64_t t = idx / g.nz;
    const int ix = (int)(t % g.nx), iy = (int)(t / g.nx);
    const float b[3] = {bs[idx], bs[N + idx], bs[2 * N + idx]};
    float dz = 0.f;
    if (ix < g.nx - 1) dz -= b[0];
    if (iy < g.ny - 1) dz -= b[1];
    if (iz < g.nz - 1) dz -= b[2];
    if (ix > 0) dz += bs[idx - sx];
    if (iy > 0) dz += bs[N + idx - sy];
    if (iz > 0) dz += bs[2 * N + idx - 1];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      // w part: dzw = -dq;  zw += dzw;  w = w - Tw (zw + dzw / p)
      const float dzw = -b[k];
      const float zwn = a.zw[k * N + idx] + dzw;
      a.zw[k * N + idx] = zwn;
      a.w_out[k * N + idx] = a.w_in[k * N + idx] - a.Tw * fmaf(dzw, a.inv_p, zwn);
    }
    const float zn = a.zu[idx] + dz;
    a.zu[idx] = zn;
    a.u_out[idx] = prox_nonneg(a.u_in[idx] - a.Tu[idx] * fmaf(dz, a.inv_p, zn));
  }
}

// backward difference of w component c along axis ax at voxel j (d-_a = -D_a^T)
__device__ __forceinline__ float tgv_dm(const TgvArgs& a, const DevGeom& g, int64_t N, int c, int ax, int ja,
                                        int na, int st, int64_t j) {
  const float* wc = a.w_in + c * N;
  float r = 0.f;
  if (ja < na - 1) r += wc[j];
  if (ja > 0) r -= wc[j - st];
  return r;
}

// block 1: q+ = proj_{alpha1}(q + sigma E w) (Frobenius ball, off-diagonals counted twice)
__global__ void __launch_bounds__(256) k_tgv1_dual(DevGeom g, TgvArgs a) {
  const int64_t N = (int64_t)g.nx * g.ny * g.nz;
  const int sx = g.nz, sy = g.nx * g.nz;
  for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < N; j += (int64_t)gridDim.x * blockDim.x) {
    const int jz = (int)(j % g.nz);
    const int64_t t = j / g.nz;
    const int jx = (int)(t % g.nx), jy = (int)(t / g.nx);
    auto dm = [&](int c, int ax) {
      return ax == 0 ? tgv_dm(a, g, N, c, 0, jx, g.nx, sx, j)
                     : (ax == 1 ? tgv_dm(a, g, N, c, 1, jy, g.ny, sy, j) : tgv_dm(a, g, N, c, 2, jz, g.nz, 1, j));
    };
    float e[6];
    e[0] = dm(0, 0);
    e[1] = dm(1, 1);
    e[2] = dm(2, 2);
    e[3] = 0.5f * (dm(1, 0) + dm(0, 1));
    e[4] = 0.5f * (dm(2, 0) + dm(0, 2));
    e[5] = 0.5f * (dm(2, 1) + dm(1, 2));
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
      const float qn = qa[k] / sc;
      a.q_out[k * N + j] = qn;
      a.bscr[k * N + j] = qn - qo[k];
    }
  }
}

// block 1: dzw = E^T b; z and primal step of w; u takes its primal step with zbar_u = z_u
__global__ void __launch_bounds__(256) k_tgv1_primal(DevGeom g, TgvArgs a) {
  const int64_t N = (int64_t)g.nx * g.ny * g.nz;
  const int sx = g.nz, sy = g.nx * g.nz;
  const float* bs = a.bscr;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < N; idx += (int64_t)gridDim.x * blockDim.x) {
    const int iz = (int)(idx % g.nz);
    const int64_t t = idx / g.nz;
    const int ix = (int)(t % g.nx), iy = (int)(t / g.nx);
    const bool hx = ix < g.nx - 1, hy = iy < g.ny - 1, hz = iz < g.nz - 1;
    // (d-_a)^T = -D_a:  ((d-_a)^T p)(k) = p(k) - p(k + e_a) for k_a < n_a - 1, else 0.
    // E^T dq:  w_c += sum over entries (a,b) of E containing d-_a w_c, weights 1 (diag) or 1
    // (off-diagonal: 2 in the inner product times the 1/2 of the definition).
    auto dmT = [&](int comp, int ax) -> float {
      const bool h = ax == 0 ? hx : (ax == 1 ? hy : hz);
      const int st = ax == 0 ? sx : (ax == 1 ? sy : 1);
      return h ? bs[comp * N + idx] - bs[comp * N + idx + st] : 0.f;
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
    a.u_out[idx] = prox_nonneg(a.u_in[idx] - a.Tu[idx] * a.zu[idx]);
  }
}

cudaError_t launch_tgv(const DevGeom& g, const TgvArgs& a, cudaStream_t s) {
  const int64_t N = (int64_t)g.nx * g.ny * g.nz;
  int64_t blocks = (N + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  if (!a.bscr) return cudaErrorInvalidValue;
  if (a.block == 0) {
    k_tgv0_dual<<<(int)blocks, 256, 0, s>>>(g, a);
    k_tgv0_primal<<<(int)blocks, 256, 0, s>>>(g, a);
  } else {
    k_tgv1_dual<<<(int)blocks, 256, 0, s>>>(g, a);
    k_tgv1_primal<<<(int)blocks, 256, 0, s>>>(g, a);
  }
  return cudaGetLastError();
}

}  // namespace spdhg
