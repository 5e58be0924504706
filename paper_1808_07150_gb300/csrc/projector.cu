// Ray-driven forward projector (fused with the KL dual prox) and gather-based backprojector
// (fused with the dual-sum update and the next primal step) for SPDHG on a cylindrical PET
// scanner.  Both directions evaluate the same exact line-integral model
//     (L x)_j = sum_k |LOR_j  intersect voxel_k| x_k
// through one factorisation:
//   * transaxially, a LOR (view v, radial bin r) is a 2-D line; its intersection with pixel
//     (ix, iy) is a parameter interval [ta, tb] (pixel_interval);
//   * axially, the LORs of one michelogram segment differ only by a shift of exactly one slice
//     per plane, so inside a pixel the LOR of plane q meets slab iz = q - j with a length that
//     depends only on j, the segment and [ta, tb] (segment_taps).
// Forward and back projection call these two functions with the same inputs, so each
// (LOR, voxel) length is bit-identical in both directions and the backprojector is the exact
// transpose of the projector (up to the order of the sums).  No float atomics are used: the
// forward kernel owns one LOR line per block, the backward kernel one voxel column per thread
// group.
#include "internal.cuh"

namespace spdhg {

struct Line {
  float ox, oy, dx, dy, inv_dx, inv_dy, h;
};

// Transaxial line of (view v, radial bin r): P(t) = (ox + t dx, oy + t dy), t in [-h, h].
__device__ __forceinline__ Line make_line(const DevGeom& g, int v, int r) {
  const float2 cs = g.view_cs[v];
  Line L;
  const float s = __fmul_rn(__fsub_rn((float)r, g.half_R), g.d_radial);
  L.ox = __fmul_rn(s, cs.x);
  L.oy = __fmul_rn(s, cs.y);
  L.dx = -cs.y;
  L.dy = cs.x;
  L.inv_dx = (L.dx != 0.f) ? __frcp_rn(L.dx) : 0.f;
  L.inv_dy = (L.dy != 0.f) ? __frcp_rn(L.dy) : 0.f;
  L.h = __fsqrt_rn(__fsub_rn(g.radius2, __fmul_rn(s, s)));
  return L;
}

__device__ __forceinline__ float grid_x(const DevGeom& g, int i) { return __fmaf_rn((float)i, g.vx, g.lox); }
__device__ __forceinline__ float grid_y(const DevGeom& g, int i) { return __fmaf_rn((float)i, g.vx, g.loy); }

// [ta, tb] = {t in [-h, h] : P(t) in pixel (ix, iy)}; false if empty.  A line lying in a grid
// line belongs to the pixel whose lower edge holds it.
__device__ __forceinline__ bool pixel_interval(const DevGeom& g, const Line& L, int ix, int iy,
                                               float& ta, float& tb) {
  float lo = -L.h, hi = L.h;
  const float X0 = grid_x(g, ix), X1 = grid_x(g, ix + 1);
  if (L.dx == 0.f) {
    if (!(X0 <= L.ox && L.ox < X1)) return false;
  } else {
    const float t0 = __fmul_rn(__fsub_rn(X0, L.ox), L.inv_dx);
    const float t1 = __fmul_rn(__fsub_rn(X1, L.ox), L.inv_dx);
    lo = fmaxf(lo, fminf(t0, t1));
    hi = fminf(hi, fmaxf(t0, t1));
  }
  const float Y0 = grid_y(g, iy), Y1 = grid_y(g, iy + 1);
  if (L.dy == 0.f) {
    if (!(Y0 <= L.oy && L.oy < Y1)) return false;
  } else {
    const float t0 = __fmul_rn(__fsub_rn(Y0, L.oy), L.inv_dy);
    const float t1 = __fmul_rn(__fsub_rn(Y1, L.oy), L.inv_dy);
    lo = fmaxf(lo, fminf(t0, t1));
    hi = fminf(hi, fmaxf(t0, t1));
  }
  ta = lo;
  tb = hi;
  return hi > lo;
}

// Axial constants of a LOR line for one segment: slab coordinate zeta(t) = f + j + kappa t.
struct SegLine {
  float f, kappa, inv_kappa, scale;
};

__device__ __forceinline__ SegLine seg_line(const DevGeom& g, const Line& L, int gi) {
  const SegDev sd = g.seg[gi];
  const float slope = __fdiv_rn(sd.dz, __fmul_rn(2.f, L.h));
  SegLine S;
  S.f = sd.f;
  S.kappa = __fdiv_rn(slope, g.vz);
  S.inv_kappa = (S.kappa != 0.f) ? __frcp_rn(S.kappa) : 0.f;
  const float n2 = __fadd_rn(__fadd_rn(__fmul_rn(L.dx, L.dx), __fmul_rn(L.dy, L.dy)), __fmul_rn(slope, slope));
  S.scale = __fdiv_rn(__fsqrt_rn(n2), g.vx);  // |dP/dt| in voxel units
  return S;
}

// Lengths (voxel units) of the plane-q LOR in slabs iz = q - (j0 + k), k < NT, for the pixel
// interval [ta, tb].  Returns j0.
template <int NT>
__device__ __forceinline__ int segment_taps(const SegLine& S, float ta, float tb, float* Lk) {
  if (S.kappa == 0.f) {
    const int j0 = -(int)floorf(S.f);  // f + j0 in [0, 1): the slab holding the LOR
    Lk[0] = __fmul_rn(__fsub_rn(tb, ta), S.scale);
#pragma unroll
    for (int k = 1; k < NT; ++k) Lk[k] = 0.f;
    return j0;
  }
  const float ka = __fmul_rn(S.kappa, ta), kb = __fmul_rn(S.kappa, tb);
  const float B = __fadd_rn(S.f, fmaxf(ka, kb));
  const int j0 = (int)floorf(-B) + 1;  // smallest j with f + j + max(kappa t) > 0
#pragma unroll
  for (int k = 0; k < NT; ++k) {
    const float u0 = -__fadd_rn(S.f, (float)(j0 + k));  // zeta = 0  at  t = u0 / kappa
    const float u1 = __fadd_rn(u0, 1.f);               // zeta = 1  at  t = u1 / kappa
    const float t0 = __fmul_rn(u0, S.inv_kappa), t1 = __fmul_rn(u1, S.inv_kappa);
    const float lo = fmaxf(ta, fminf(t0, t1)), hi = fminf(tb, fmaxf(t0, t1));
    Lk[k] = hi > lo ? __fmul_rn(__fsub_rn(hi, lo), S.scale) : 0.f;
  }
  return j0;
}

// ---------------------------------------------------------------------------------------
// forward projection: one block per transaxial line (view, radial bin), threads over planes
// ---------------------------------------------------------------------------------------

struct Entry {
  int col;  // iy * nx + ix, or -1
  float ta, tb;
};

// The (at most two) pixels of `row` along the dominant axis crossed by the line.
__device__ __forceinline__ void row_entries(const DevGeom& g, const Line& L, bool ydom, int row,
                                            Entry& e0, Entry& e1) {
  e0.col = -1;
  e1.col = -1;
  const float inv_d = ydom ? L.inv_dy : L.inv_dx;
  const float o = ydom ? L.oy : L.ox;
  const float G0 = ydom ? grid_y(g, row) : grid_x(g, row);
  const float G1 = ydom ? grid_y(g, row + 1) : grid_x(g, row + 1);
  const float t0 = __fmul_rn(__fsub_rn(G0, o), inv_d), t1 = __fmul_rn(__fsub_rn(G1, o), inv_d);
  const float tlo = fmaxf(-L.h, fminf(t0, t1)), thi = fminf(L.h, fmaxf(t0, t1));
  if (!(thi > tlo)) return;
  const float oc = ydom ? L.ox : L.oy;   // coordinate across the row
  const float dc = ydom ? L.dx : L.dy;
  const float lo = ydom ? g.lox : g.loy;
  const int nc = ydom ? g.nx : g.ny;
  int c0;
  if (dc == 0.f) {
    c0 = (int)floorf(__fmul_rn(__fsub_rn(oc, lo), g.inv_vx));
    const float C0 = __fmaf_rn((float)c0, g.vx, lo), C1 = __fmaf_rn((float)(c0 + 1), g.vx, lo);
    if (C0 > oc) --c0;
    else if (C1 <= oc) ++c0;
  } else {
    const float ca = __fmaf_rn(tlo, dc, oc), cb = __fmaf_rn(thi, dc, oc);
    c0 = (int)floorf(__fmul_rn(__fsub_rn(fminf(ca, cb), lo), g.inv_vx));
  }
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int c = c0 + k;
    if (c < 0 || c >= nc) continue;
    const int ix = ydom ? c : row, iy = ydom ? row : c;
    float ta, tb;
    if (pixel_interval(g, L, ix, iy, ta, tb)) {
      Entry& e = k ? e1 : e0;
      e.col = iy * g.nx + ix;
      e.ta = ta;
      e.tb = tb;
    }
  }
}

template <int NT, int PPT, int MODE>
__global__ void __launch_bounds__(512) k_forward(DevGeom g, int subset, int rpc, FwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ SegLine sl[kMaxSeg];
  const int n_ent = 2 * rpc;
  Entry* ent = reinterpret_cast<Entry*>(smem);
  int* tapJ = reinterpret_cast<int*>(ent + n_ent);
  float* tapL = reinterpret_cast<float*>(tapJ + g.n_seg * n_ent);

  const int line = blockIdx.x;
  const int l = line / g.R, r = line - (line / g.R) * g.R;
  const int v = subset_view(g, subset, l);
  const Line L = make_line(g, v, r);
  if (threadIdx.x < g.n_seg) sl[threadIdx.x] = seg_line(g, L, threadIdx.x);

  int pseg[PPT], pq[PPT];
  float acc[PPT], chord[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int p = threadIdx.x + k * blockDim.x;
    acc[k] = 0.f;
    chord[k] = 0.f;
    if (p < g.P) {
      const int gi = g.plane_seg[p];
      pseg[k] = gi;
      pq[k] = p - g.seg[gi].p0;
    } else {
      pseg[k] = -1;
      pq[k] = 0;
    }
  }
  const bool ydom = fabsf(L.dy) >= fabsf(L.dx);
  const int nrows = ydom ? g.ny : g.nx;
  const int nz = g.nz;
  __syncthreads();

  for (int row0 = 0; row0 < nrows; row0 += rpc) {
    for (int t = threadIdx.x; t < rpc; t += blockDim.x) {
      Entry e0, e1;
      e0.col = -1;
      e1.col = -1;
      if (row0 + t < nrows) row_entries(g, L, ydom, row0 + t, e0, e1);
      ent[2 * t] = e0;
      ent[2 * t + 1] = e1;
    }
    __syncthreads();
    for (int it = threadIdx.x; it < g.n_seg * n_ent; it += blockDim.x) {
      const int gi = it / n_ent, e = it - gi * n_ent;
      const Entry en = ent[e];
      float Lk[NT];
      int j0 = 0;
      if (en.col >= 0) {
        j0 = segment_taps<NT>(sl[gi], en.ta, en.tb, Lk);
      } else {
#pragma unroll
        for (int k = 0; k < NT; ++k) Lk[k] = 0.f;
      }
      tapJ[it] = j0;
#pragma unroll
      for (int k = 0; k < NT; ++k) tapL[it * NT + k] = Lk[k];
    }
    __syncthreads();
    for (int e = 0; e < n_ent; ++e) {
      const int col = ent[e].col;
      if (col < 0) continue;
      const float* __restrict__ xc = a.x + (size_t)col * nz;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (pseg[k] < 0) continue;
        const int it = pseg[k] * n_ent + e;
        const int iz = pq[k] - tapJ[it];
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          const float Lt = tapL[it * NT + t];
          const int izt = iz - t;
          if (izt >= 0 && izt < nz) {
            acc[k] = fmaf(Lt, __ldg(xc + izt), acc[k]);
            if (MODE != FWD_PROJECT) chord[k] += Lt;
          }
        }
      }
    }
    __syncthreads();
  }

#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int p = threadIdx.x + k * blockDim.x;
    if (p >= g.P) continue;
    const size_t j = ((size_t)v * g.R + r) * g.P + p;
    const float mu = a.mult ? a.mult[j] : 1.f;
    if (MODE == FWD_PROJECT) {
      a.out[j] = mu * acc[k];
    } else if (MODE == FWD_SIGMA) {
      const float a1 = mu * chord[k];
      a.out[j] = a1 > 0.f ? a.gamma_rho / a1 : 0.f;
    } else {
      // KL dual prox on this bin:  y+ = prox_{sigma varphi*}(y + sigma (P_i x)_j), evaluated as
      // 2 (w - sigma b) / (w + 1 + sqrt((w - 1)^2 + 4 sigma b)),  w = y + sigma ((P_i x)_j + r_j),
      // which equals 1/2 [w + 1 - sqrt((w - 1)^2 + 4 sigma b)] without its cancellation.
      const float a1 = mu * chord[k];
      const float sigma = a1 > 0.f ? a.gamma_rho / a1 : 0.f;
      const float yj = a.y[j];
      const float bj = a.b[j];
      const float w = fmaf(sigma, fmaf(mu, acc[k], a.r[j]), yj);
      const float sb = sigma * bj;
      const float wm = w - 1.f;
      const float root = sqrtf(fmaf(wm, wm, 4.f * sb));
      const float yn = 2.f * (w - sb) / (w + 1.f + root);
      a.y[j] = yn;
      a.wdy[((size_t)l * g.R + r) * g.P + p] = mu * (yn - yj);
    }
  }
}

// ---------------------------------------------------------------------------------------
// backprojection: one thread group per voxel column (ix, iy), threads over iz
// ---------------------------------------------------------------------------------------

template <int NT>
struct Item {
  int base;  // subset-local sinogram index of (view, radial, first plane of the segment)
  int n;     // planes in the segment (0: no contribution)
  int j0;
  float L[NT];
};

template <int NT, int MODE>
__global__ void __launch_bounds__(256) k_backward(DevGeom g, int subset, int tpc, int cpb, int vchunk,
                                                  BwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int per_view = g.nr_max * g.n_seg;
  const int items_per_col = vchunk * per_view;
  Item<NT>* items = reinterpret_cast<Item<NT>*>(smem) + (threadIdx.x / tpc) * items_per_col;
  const int tz = threadIdx.x % tpc;
  const int col = blockIdx.x * cpb + threadIdx.x / tpc;
  const bool live = col < g.nx * g.ny;
  const int iy = live ? col / g.nx : 0, ix = live ? col - iy * g.nx : 0;
  const int nviews = subset_views(g, subset);
  const float xc = __fmaf_rn((float)ix + 0.5f, g.vx, g.lox);
  const float yc = __fmaf_rn((float)iy + 0.5f, g.vx, g.loy);
  const float inv_dr = 1.f / g.d_radial;
  const int nz = g.nz;
  float acc = 0.f;  // tpc >= nz: one voxel per thread

  for (int l0 = 0; l0 < nviews; l0 += vchunk) {
    const int nv = min(vchunk, nviews - l0);
    for (int it = tz; it < nv * per_view; it += tpc) {
      const int gi = it % g.n_seg;
      const int rest = it / g.n_seg;
      const int ri = rest % g.nr_max;
      const int l = l0 + rest / g.nr_max;
      Item<NT> I;
      I.n = 0;
      I.base = 0;
      I.j0 = 0;
#pragma unroll
      for (int k = 0; k < NT; ++k) I.L[k] = 0.f;
      if (live) {
        const int v = subset_view(g, subset, l);
        const float2 cs = g.view_cs[v];
        const float sc = xc * cs.x + yc * cs.y;
        const float half = 0.5f * g.vx * (fabsf(cs.x) + fabsf(cs.y));
        const int rlo = (int)ceilf((sc - half) * inv_dr + g.half_R) - 1;
        const int rhi = (int)floorf((sc + half) * inv_dr + g.half_R) + 1;
        const int r = rlo + ri;
        if (r >= 0 && r < g.R && r <= rhi) {
          const Line L = make_line(g, v, r);
          float ta, tb;
          if (pixel_interval(g, L, ix, iy, ta, tb)) {
            const SegLine S = seg_line(g, L, gi);
            I.j0 = segment_taps<NT>(S, ta, tb, I.L);
            I.base = (l * g.R + r) * g.P + g.seg[gi].p0;
            I.n = g.seg[gi].n;
          }
        }
      }
      items[it] = I;
    }
    __syncthreads();
    if (live && tz < nz) {
      for (int it = 0; it < nv * per_view; ++it) {
        const Item<NT> I = items[it];
        if (I.n == 0) continue;
        const int q = tz + I.j0;
#pragma unroll
        for (int k = 0; k < NT; ++k) {
          const int qk = q + k;
          if (qk >= 0 && qk < I.n) acc = fmaf(I.L[k], __ldg(a.w + I.base + qk), acc);
        }
      }
    }
    __syncthreads();
  }
  if (!live || tz >= nz) return;
  const size_t idx = (size_t)col * nz + tz;
  if (MODE == BWD_OUT) {
    a.out[idx] = acc;
  } else if (MODE == BWD_SENS) {
    // T_i = rho p_i / (gamma (P_i^T 1)); +inf (kept) where the subset does not see the voxel
    if (acc > 0.f) a.T[idx] = fminf(a.T[idx], a.sens_num / acc);
  } else {
    // z = z + dz;  zbar = z + dz / p_i;  next primal step x = max(x - T zbar, 0)
    const float zn = a.z[idx] + acc;
    a.z[idx] = zn;
    a.x[idx] = fmaxf(a.x[idx] - a.T[idx] * fmaf(acc, a.inv_p, zn), 0.f);
  }
}

__global__ void k_gather_subset(DevGeom g, int subset, const float* __restrict__ y,
                                const float* __restrict__ mult, float* __restrict__ w) {
  const int64_t per_view = (int64_t)g.R * g.P;
  const int64_t n = (int64_t)subset_views(g, subset) * per_view;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(i / per_view);
    const int64_t j = (int64_t)subset_view(g, subset, l) * per_view + (i - l * per_view);
    w[i] = mult ? y[j] * mult[j] : y[j];
  }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------

static int fwd_threads(int P, int* ppt) {
  int t = (P + 2) / 3;
  t = ((t + 31) / 32) * 32;
  t = t < 128 ? 128 : (t > 512 ? 512 : t);
  int k = (P + t - 1) / t;
  *ppt = k < 1 ? 1 : k;
  return t;
}

template <int NT, int PPT, int MODE>
static cudaError_t fwd_launch(const DevGeom& g, int subset, const FwdArgs& a, cudaStream_t s, int threads) {
  int rpc = 64;
  auto bytes = [&](int rows) {
    return (size_t)(2 * rows) * (sizeof(Entry) + (size_t)g.n_seg * sizeof(int) + (size_t)g.n_seg * NT * sizeof(float));
  };
  while (rpc > 8 && bytes(rpc) > 40 * 1024) rpc /= 2;
  const size_t smem = bytes(rpc);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_forward<NT, PPT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int lines = subset_views(g, subset) * g.R;
  if (lines == 0) return cudaSuccess;
  k_forward<NT, PPT, MODE><<<lines, threads, smem, s>>>(g, subset, rpc, a);
  return cudaGetLastError();
}

template <int NT, int MODE>
static cudaError_t fwd_ppt(const DevGeom& g, int subset, const FwdArgs& a, cudaStream_t s) {
  int ppt;
  const int threads = fwd_threads(g.P, &ppt);
  switch (ppt) {
    case 1: return fwd_launch<NT, 1, MODE>(g, subset, a, s, threads);
    case 2: return fwd_launch<NT, 2, MODE>(g, subset, a, s, threads);
    case 3: return fwd_launch<NT, 3, MODE>(g, subset, a, s, threads);
    case 4: return fwd_launch<NT, 4, MODE>(g, subset, a, s, threads);
    default: return cudaErrorInvalidValue;
  }
}

template <int MODE>
static cudaError_t fwd_nt(const DevGeom& g, int subset, const FwdArgs& a, cudaStream_t s) {
  switch (g.taps) {
    case 1: return fwd_ppt<1, MODE>(g, subset, a, s);
    case 2: return fwd_ppt<2, MODE>(g, subset, a, s);
    case 3: return fwd_ppt<3, MODE>(g, subset, a, s);
    case 4: return fwd_ppt<4, MODE>(g, subset, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_forward(const DevGeom& g, int subset, int mode, const FwdArgs& a, cudaStream_t s) {
  switch (mode) {
    case FWD_PROJECT: return fwd_nt<FWD_PROJECT>(g, subset, a, s);
    case FWD_SIGMA: return fwd_nt<FWD_SIGMA>(g, subset, a, s);
    case FWD_DATA: return fwd_nt<FWD_DATA>(g, subset, a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <int NT, int MODE>
static cudaError_t bwd_launch(const DevGeom& g, int subset, const BwdArgs& a, cudaStream_t s) {
  int tpc = ((g.nz + 31) / 32) * 32;
  if (tpc > 256) return cudaErrorInvalidValue;
  const int cpb = 256 / tpc;
  const int per_view = g.nr_max * g.n_seg;
  const int budget = 160;  // items per column and chunk
  int vchunk = budget / per_view;
  if (vchunk < 1) vchunk = 1;
  const int nviews = subset_views(g, subset);
  if (vchunk > nviews) vchunk = nviews > 0 ? nviews : 1;
  const size_t smem = (size_t)cpb * vchunk * per_view * sizeof(Item<NT>);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_backward<NT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int cols = g.nx * g.ny;
  const int blocks = (cols + cpb - 1) / cpb;
  k_backward<NT, MODE><<<blocks, cpb * tpc, smem, s>>>(g, subset, tpc, cpb, vchunk, a);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t bwd_nt(const DevGeom& g, int subset, const BwdArgs& a, cudaStream_t s) {
  switch (g.taps) {
    case 1: return bwd_launch<1, MODE>(g, subset, a, s);
    case 2: return bwd_launch<2, MODE>(g, subset, a, s);
    case 3: return bwd_launch<3, MODE>(g, subset, a, s);
    case 4: return bwd_launch<4, MODE>(g, subset, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_backward(const DevGeom& g, int subset, int mode, const BwdArgs& a, cudaStream_t s) {
  switch (mode) {
    case BWD_OUT: return bwd_nt<BWD_OUT>(g, subset, a, s);
    case BWD_SENS: return bwd_nt<BWD_SENS>(g, subset, a, s);
    case BWD_UPDATE: return bwd_nt<BWD_UPDATE>(g, subset, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gather_subset(const DevGeom& g, int subset, const float* y, const float* mult,
                                 float* w_local, cudaStream_t s) {
  const int64_t n = (int64_t)subset_views(g, subset) * g.R * g.P;
  if (n == 0) return cudaSuccess;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_gather_subset<<<blocks, 256, 0, s>>>(g, subset, y, mult, w_local);
  return cudaGetLastError();
}

}  // namespace spdhg
