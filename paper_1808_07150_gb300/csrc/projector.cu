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

// Error-free transformations (Knuth two-sum, FMA two-product): a + b = s + e, a * b = p + e.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

// Transaxial line of (view v, radial bin r) in pixel units: the points X n_perp with
// X . (c, s) = s_r, parameter t along (-s, c), t in [-h, h]  (all as double-float pairs).
struct Line {
  float c_hi, c_lo, s_hi, s_lo;
  float sp_hi, sp_lo, h_hi, h_lo;
};

__device__ __forceinline__ Line make_line(const DevGeom& g, int v, int r) {
  const float4 a = g.view[v];
  const float4 b = g.rad[r];
  return Line{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
}

// Intersection of a line with pixel (ix, iy), expressed relative to the foot point of the
// pixel centre on the line: t in tc + [ua, ub], tc = tch + tcl.  The offset of the line from
// the pixel centre and tc are evaluated with error-free transformations, so [ua, ub] is
// resolved to FP32 precision of quantities of order one pixel.  A line lying in a grid line
// belongs to the pixel whose lower edge holds it.
struct PixInt {
  float ua, ub, tch, tcl;
};

__device__ __forceinline__ bool pixel_interval(const DevGeom& g, const Line& L, int ix, int iy, PixInt& out) {
  const float Xc = (float)ix + 0.5f - 0.5f * (float)g.nx;  // pixel centre (exact)
  const float Yc = (float)iy + 0.5f - 0.5f * (float)g.ny;
  float p1, e1, p2, e2, S, eS, D, eD;
  // delta = Xc c + Yc s - s_r: signed distance of the pixel centre from the line
  two_prod(Xc, L.c_hi, p1, e1);
  two_prod(Yc, L.s_hi, p2, e2);
  two_sum(p1, p2, S, eS);
  two_sum(S, -L.sp_hi, D, eD);
  const float delta = __fadd_rn(D, __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), __fadd_rn(eS, eD)),
                                              __fsub_rn(__fmaf_rn(Xc, L.c_lo, __fmul_rn(Yc, L.s_lo)), L.sp_lo)));
  // tc = Yc c - Xc s: line parameter of the foot point
  two_prod(Yc, L.c_hi, p1, e1);
  two_prod(-Xc, L.s_hi, p2, e2);
  two_sum(p1, p2, S, eS);
  two_sum(S, __fadd_rn(__fadd_rn(__fadd_rn(e1, e2), eS), __fsub_rn(__fmul_rn(Yc, L.c_lo), __fmul_rn(Xc, L.s_lo))),
          out.tch, out.tcl);
  // segment ends t = -h, h relative to tc
  float lo = __fadd_rn(__fsub_rn(-L.h_hi, out.tch), __fsub_rn(-L.h_lo, out.tcl));
  float hi = __fadd_rn(__fsub_rn(L.h_hi, out.tch), __fsub_rn(L.h_lo, out.tcl));
  const float ex = __fmul_rn(-delta, L.c_hi), ey = __fmul_rn(-delta, L.s_hi);  // foot point - centre
  const float dx = -L.s_hi, dy = L.c_hi;
  if (dx == 0.f) {
    if (!(ex >= -0.5f && ex < 0.5f)) return false;
  } else {
    const float u1 = __fdiv_rn(__fsub_rn(-0.5f, ex), dx), u2 = __fdiv_rn(__fsub_rn(0.5f, ex), dx);
    lo = fmaxf(lo, fminf(u1, u2));
    hi = fminf(hi, fmaxf(u1, u2));
  }
  if (dy == 0.f) {
    if (!(ey >= -0.5f && ey < 0.5f)) return false;
  } else {
    const float u1 = __fdiv_rn(__fsub_rn(-0.5f, ey), dy), u2 = __fdiv_rn(__fsub_rn(0.5f, ey), dy);
    lo = fmaxf(lo, fminf(u1, u2));
    hi = fminf(hi, fmaxf(u1, u2));
  }
  out.ua = lo;
  out.ub = hi;
  return hi > lo;
}

// Lengths (voxel units) of the plane-q LOR of segment gi in slabs iz = q - (j0 + k), k < NT,
// inside the pixel interval I.  The LOR's slab coordinate at the foot point,
// zeta_c = f + kappa tc, is split exactly into an integer n0 and a fraction in [0, 1); the
// crossings are then solved in local quantities of order one.  Returns j0.
template <int NT>
__device__ __forceinline__ int segment_taps(const DevGeom& g, int r, int gi, const PixInt& I, float* Lk) {
  const float4 rs = g.rs[r * g.n_seg + gi];
  const SegDev sd = g.seg[gi];
  const float kh = rs.x, kl = rs.y, scale = rs.z;
  float p, e, s1, e1;
  two_prod(kh, I.tch, p, e);
  e = __fadd_rn(e, __fmaf_rn(kh, I.tcl, __fmul_rn(kl, I.tch)));
  two_sum(sd.f_hi, p, s1, e1);
  float n0 = floorf(s1);
  float frac = __fadd_rn(__fsub_rn(s1, n0), __fadd_rn(__fadd_rn(e1, e), sd.f_lo));
  if (frac >= 1.f) {
    frac -= 1.f;
    n0 += 1.f;
  } else if (frac < 0.f) {
    frac += 1.f;
    n0 -= 1.f;
  }
  const int in0 = (int)n0;
  if (kh == 0.f) {
    Lk[0] = __fmul_rn(__fsub_rn(I.ub, I.ua), scale);
#pragma unroll
    for (int k = 1; k < NT; ++k) Lk[k] = 0.f;
    return -in0;  // frac in [0, 1): the LOR stays in one slab
  }
  const float ka = __fmul_rn(kh, I.ua), kb = __fmul_rn(kh, I.ub);
  const float B = __fadd_rn(frac, fmaxf(ka, kb));
  const int j0l = (int)floorf(-B) + 1;  // smallest local j with frac + j + max(kappa u) > 0
  const float inv_k = __frcp_rn(kh);
#pragma unroll
  for (int k = 0; k < NT; ++k) {
    const float u0 = -__fadd_rn(frac, (float)(j0l + k));  // zeta = 0 at u = u0 / kappa
    const float u1 = __fadd_rn(u0, 1.f);                  // zeta = 1 at u = u1 / kappa
    const float t0 = __fmul_rn(u0, inv_k), t1 = __fmul_rn(u1, inv_k);
    const float lo = fmaxf(I.ua, fminf(t0, t1)), hi = fminf(I.ub, fmaxf(t0, t1));
    Lk[k] = hi > lo ? __fmul_rn(__fsub_rn(hi, lo), scale) : 0.f;
  }
  return j0l - in0;
}

// ---------------------------------------------------------------------------------------
// forward projection: one block per transaxial line (view, radial bin), threads over planes
// ---------------------------------------------------------------------------------------

struct Entry {
  int col;  // iy * nx + ix
  PixInt I;
};

constexpr int kCandPerRow = 4;

// Pixels of `row` (along the dominant axis of the line) that the line crosses.  Candidates come
// from approximate arithmetic (one pixel of margin on each side); pixel_interval decides exactly.
__device__ __forceinline__ int row_entries(const DevGeom& g, const Line& L, bool ydom, int row, Entry* e) {
  const float c = L.c_hi, s = L.s_hi, sp = L.sp_hi, h = L.h_hi;
  float t0, t1;
  if (ydom) {  // y in [Y0, Y0 + 1);  y(t) = sp s + t c
    const float Y0 = (float)row - 0.5f * (float)g.ny;
    t0 = (Y0 - sp * s) / c;
    t1 = (Y0 + 1.f - sp * s) / c;
  } else {     // x in [X0, X0 + 1);  x(t) = sp c - t s
    const float X0 = (float)row - 0.5f * (float)g.nx;
    t0 = (sp * c - X0) / s;
    t1 = (sp * c - X0 - 1.f) / s;
  }
  const float tlo = fmaxf(fminf(t0, t1), -h - 1e-2f), thi = fminf(fmaxf(t0, t1), h + 1e-2f);
  if (thi < tlo) return 0;
  const float ca = ydom ? sp * c - tlo * s : sp * s + tlo * c;
  const float cb = ydom ? sp * c - thi * s : sp * s + thi * c;
  const float half = 0.5f * (float)(ydom ? g.nx : g.ny);
  const int nc = ydom ? g.nx : g.ny;
  const int cmin = max((int)floorf(fminf(ca, cb) + half) - 1, 0);
  const int cmax = min((int)floorf(fmaxf(ca, cb) + half) + 1, nc - 1);
  int n = 0;
  for (int cc = cmin; cc <= cmax && n < kCandPerRow; ++cc) {
    const int ix = ydom ? cc : row, iy = ydom ? row : cc;
    PixInt I;
    if (pixel_interval(g, L, ix, iy, I)) {
      e[n].col = iy * g.nx + ix;
      e[n].I = I;
      ++n;
    }
  }
  return n;
}

template <int NT, int PPT, int MODE>
__global__ void __launch_bounds__(512) k_forward(DevGeom g, int subset, int rpc, int split, FwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int warp_tot[2];
  __shared__ int n_ent_sh;
  const int cap = kCandPerRow * rpc;
  Entry* ent = reinterpret_cast<Entry*>(smem);
  int* tapJ = reinterpret_cast<int*>(ent + cap);   // j0 | (nt << 24) per (segment, entry)
  float* tapL = reinterpret_cast<float*>(tapJ + g.n_seg * cap);

  // block = (line, part): `split` blocks share the planes of one LOR line
  const int line = blockIdx.x / split, part = blockIdx.x - line * split;
  const int l = line / g.R, r = line - (line / g.R) * g.R;
  const int v = subset_view(g, subset, l);
  const Line L = make_line(g, v, r);
  const int per_part = (g.P + split - 1) / split;
  const int p_lo = part * per_part, p_hi = min(g.P, p_lo + per_part);
  const int g_lo = g.plane_seg[min(p_lo, g.P - 1)], g_hi = g.plane_seg[max(p_hi - 1, 0)];

  int pseg[PPT], pq[PPT];
  float acc[PPT], chord[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int p = p_lo + threadIdx.x + k * blockDim.x;
    acc[k] = 0.f;
    chord[k] = 0.f;
    if (p < p_hi) {
      const int gi = g.plane_seg[p];
      pseg[k] = gi;
      pq[k] = p - g.seg[gi].p0;
    } else {
      pseg[k] = -1;
      pq[k] = 0;
    }
  }
  const bool ydom = fabsf(L.c_hi) >= fabsf(L.s_hi);  // |dy| >= |dx|: walk the rows of y
  const int nrows = ydom ? g.ny : g.nx;
  const int nz = g.nz;
  const int nseg_part = g_hi - g_lo + 1;

  for (int row0 = 0; row0 < nrows; row0 += rpc) {
    // 1. rows -> exact pixel intervals, compacted with a two-warp prefix sum (rpc <= 64)
    Entry loc[kCandPerRow];
    int cnt = 0;
    if (threadIdx.x < rpc && row0 + (int)threadIdx.x < nrows) cnt = row_entries(g, L, ydom, row0 + threadIdx.x, loc);
    int incl = 0;
    if (threadIdx.x < 64) {
      const int lane = threadIdx.x & 31;
      incl = cnt;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane == 31) warp_tot[threadIdx.x >> 5] = incl;
    }
    __syncthreads();
    if (threadIdx.x < 64) {
      const int off = incl - cnt + (threadIdx.x >= 32 ? warp_tot[0] : 0);
      for (int k = 0; k < cnt; ++k) ent[off + k] = loc[k];
      if (threadIdx.x == 0) n_ent_sh = warp_tot[0] + (rpc > 32 ? warp_tot[1] : 0);
    }
    __syncthreads();
    const int n_ent = n_ent_sh;
    // 2. axial taps of every (entry, segment of this block's planes)
    for (int it = threadIdx.x; it < nseg_part * n_ent; it += blockDim.x) {
      const int gi = g_lo + it / n_ent, e = it - (it / n_ent) * n_ent;
      float Lk[NT];
      const int j0 = segment_taps<NT>(g, r, gi, ent[e].I, Lk);
      int nt = NT;
      while (nt > 1 && Lk[nt - 1] == 0.f) --nt;
      const int slot = gi * cap + e;
      tapJ[slot] = (j0 & 0xffffff) | (nt << 24);
#pragma unroll
      for (int k = 0; k < NT; ++k) tapL[slot * NT + k] = Lk[k];
    }
    __syncthreads();
    // 3. accumulate the planes of this thread over the entries
    for (int e = 0; e < n_ent; ++e) {
      const float* __restrict__ xc = a.x + (size_t)ent[e].col * nz;
#pragma unroll
      for (int k = 0; k < PPT; ++k) {
        if (pseg[k] < 0) continue;
        const int slot = pseg[k] * cap + e;
        const int jn = tapJ[slot];
        const int nt = jn >> 24;
        const int iz = pq[k] - ((jn << 8) >> 8);  // sign-extended j0
#pragma unroll
        for (int t = 0; t < NT; ++t) {
          if (t < nt) {
            const float Lt = tapL[slot * NT + t];
            const int izt = iz - t;
            if ((unsigned)izt < (unsigned)nz) {
              acc[k] = fmaf(Lt, __ldg(xc + izt), acc[k]);
              if (MODE != FWD_PROJECT) chord[k] += Lt;
            }
          }
        }
      }
    }
    __syncthreads();
  }

#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int p = p_lo + threadIdx.x + k * blockDim.x;
    if (p >= p_hi) continue;
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
  int n;     // planes in the segment
  int j0;
  int nt;    // taps actually used (trailing zero-length taps dropped)
  float L[NT];
};

struct PixItem {
  int l, r;  // view (subset-local) and radial bin
  PixInt I;
};

// Candidate (view, bin) pairs of the pixel footprint handled per chunk by the first warp of a
// column; the pairs that intersect the pixel are compacted with a warp ballot.
constexpr int kPairsPerChunk = 32;

template <int NT, int MODE>
__global__ void __launch_bounds__(256) k_backward(DevGeom g, int subset, int tpc, int cpb, int vchunk,
                                                  BwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int n_pairs_sh[8];
  const int items_per_col = kPairsPerChunk * g.n_seg;
  const int cb = threadIdx.x / tpc;
  PixItem* pix = reinterpret_cast<PixItem*>(smem) + cb * kPairsPerChunk;
  Item<NT>* items = reinterpret_cast<Item<NT>*>(reinterpret_cast<PixItem*>(smem) + cpb * kPairsPerChunk) +
                    cb * items_per_col;
  const int tz = threadIdx.x % tpc;
  const int col = blockIdx.x * cpb + cb;
  const bool live = col < g.nx * g.ny;
  const int iy = live ? col / g.nx : 0, ix = live ? col - iy * g.nx : 0;
  const int nviews = subset_views(g, subset);
  const float Xc = (float)ix + 0.5f - 0.5f * (float)g.nx;
  const float Yc = (float)iy + 0.5f - 0.5f * (float)g.ny;
  const int nz = g.nz;
  float acc = 0.f;  // tpc >= nz: one voxel per thread

  for (int l0 = 0; l0 < nviews; l0 += vchunk) {
    const int nv = min(vchunk, nviews - l0);
    // 1. footprint pairs -> exact pixel intervals, compacted (first warp of the column)
    if (tz < 32) {
      PixItem P;
      bool ok = false;
      if (live && tz < nv * g.nr_max) {
        const int l = l0 + tz / g.nr_max, ri = tz % g.nr_max;
        const int v = subset_view(g, subset, l);
        const float4 cs = g.view[v];
        const float sc = Xc * cs.x + Yc * cs.z;
        const float hw = 0.5f * (fabsf(cs.x) + fabsf(cs.z));
        const int rlo = (int)ceilf((sc - hw) * g.inv_drp + g.half_R) - 1;
        const int rhi = (int)floorf((sc + hw) * g.inv_drp + g.half_R) + 1;
        const int r = rlo + ri;
        if (r >= 0 && r < g.R && r <= rhi) {
          const Line L = make_line(g, v, r);
          ok = pixel_interval(g, L, ix, iy, P.I);
          P.l = l;
          P.r = r;
        }
      }
      const unsigned mask = __ballot_sync(0xffffffffu, ok);
      if (ok) pix[__popc(mask & ((1u << tz) - 1u))] = P;
      if (tz == 0) n_pairs_sh[cb] = __popc(mask);
    }
    __syncthreads();
    const int np = n_pairs_sh[cb];
    // 2. axial taps per (pair, segment)
    for (int it = tz; it < np * g.n_seg; it += tpc) {
      const int pi = it / g.n_seg, gi = it - pi * g.n_seg;
      const PixItem P = pix[pi];
      Item<NT> I;
      I.j0 = segment_taps<NT>(g, P.r, gi, P.I, I.L);
      I.base = (P.l * g.R + P.r) * g.P + g.seg[gi].p0;
      I.n = g.seg[gi].n;
      int nt = NT;
      while (nt > 1 && I.L[nt - 1] == 0.f) --nt;
      I.nt = nt;
      items[it] = I;
    }
    __syncthreads();
    // 3. gather along contiguous plane runs
    if (live && tz < nz) {
      const int ni = np * g.n_seg;
      for (int it = 0; it < ni; ++it) {
        const Item<NT> I = items[it];
        const int q = tz + I.j0;
        const float* __restrict__ wp = a.w + I.base;
#pragma unroll
        for (int k = 0; k < NT; ++k) {
          if (k < I.nt) {
            const int qk = q + k;
            if ((unsigned)qk < (unsigned)I.n) acc = fmaf(I.L[k], __ldg(wp + qk), acc);
          }
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

static int fwd_split(const DevGeom& g) {
  if (g.tune[SPDHG_TUNE_FWD_SPLIT]) return g.tune[SPDHG_TUNE_FWD_SPLIT];
  return g.P >= 512 ? 4 : (g.P >= 256 ? 2 : 1);  // enough blocks per SM for long plane lists
}

static int fwd_threads(int planes, int* ppt) {
  int t = (planes + 2) / 3;
  t = ((t + 31) / 32) * 32;
  t = t < 128 ? 128 : (t > 512 ? 512 : t);
  int k = (planes + t - 1) / t;
  *ppt = k < 1 ? 1 : k;
  return t;
}

template <int NT, int PPT, int MODE>
static cudaError_t fwd_launch(const DevGeom& g, int subset, const FwdArgs& a, cudaStream_t s, int threads, int split) {
  auto bytes = [&](int rows) {
    const size_t cap = (size_t)kCandPerRow * rows;
    return cap * (sizeof(Entry) + (size_t)g.n_seg * sizeof(int) + (size_t)g.n_seg * NT * sizeof(float));
  };
  int rpc = 64;
  while (rpc > 8 && bytes(rpc) > 40 * 1024) rpc /= 2;
  const size_t smem = bytes(rpc);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_forward<NT, PPT, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  const int lines = subset_views(g, subset) * g.R;
  if (lines == 0) return cudaSuccess;
  k_forward<NT, PPT, MODE><<<lines * split, threads, smem, s>>>(g, subset, rpc, split, a);
  return cudaGetLastError();
}

template <int NT, int MODE>
static cudaError_t fwd_ppt(const DevGeom& g, int subset, const FwdArgs& a, cudaStream_t s) {
  int split = fwd_split(g);
  if (split > g.P) split = g.P;
  int ppt;
  const int threads = fwd_threads((g.P + split - 1) / split, &ppt);
  switch (ppt) {
    case 1: return fwd_launch<NT, 1, MODE>(g, subset, a, s, threads, split);
    case 2: return fwd_launch<NT, 2, MODE>(g, subset, a, s, threads, split);
    case 3: return fwd_launch<NT, 3, MODE>(g, subset, a, s, threads, split);
    case 4: return fwd_launch<NT, 4, MODE>(g, subset, a, s, threads, split);
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
  int cpb = tpc >= 128 ? 1 : 256 / tpc;
  if (g.tune[SPDHG_TUNE_BWD_COLS] && g.tune[SPDHG_TUNE_BWD_COLS] * tpc <= 256) cpb = g.tune[SPDHG_TUNE_BWD_COLS];
  int vchunk = kPairsPerChunk / g.nr_max;  // views whose footprint pairs fit one warp
  if (vchunk < 1) return cudaErrorInvalidValue;
  const int nviews = subset_views(g, subset);
  if (vchunk > nviews) vchunk = nviews > 0 ? nviews : 1;
  const size_t smem = (size_t)cpb * kPairsPerChunk * (sizeof(PixItem) + (size_t)g.n_seg * sizeof(Item<NT>));
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
