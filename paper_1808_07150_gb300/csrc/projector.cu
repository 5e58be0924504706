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
#include <algorithm>
#include <type_traits>

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
  float inv_dx, inv_dy;  // 1 / (-s_hi), 1 / c_hi (0 for a zero component)
};

__device__ __forceinline__ Line make_line(const DevGeom& g, int v, int r) {
  const float4 a = g.view[v];
  const float4 b = g.rad[r];
  const float2 iv = g.view_inv[v];
  return Line{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, iv.x, iv.y};
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
    const float u1 = __fmul_rn(__fsub_rn(-0.5f, ex), L.inv_dx), u2 = __fmul_rn(__fsub_rn(0.5f, ex), L.inv_dx);
    lo = fmaxf(lo, fminf(u1, u2));
    hi = fminf(hi, fmaxf(u1, u2));
  }
  if (dy == 0.f) {
    if (!(ey >= -0.5f && ey < 0.5f)) return false;
  } else {
    const float u1 = __fmul_rn(__fsub_rn(-0.5f, ey), L.inv_dy), u2 = __fmul_rn(__fsub_rn(0.5f, ey), L.inv_dy);
    lo = fmaxf(lo, fminf(u1, u2));
    hi = fminf(hi, fmaxf(u1, u2));
  }
  out.ua = lo;
  out.ub = hi;
  return hi > lo;
}

// Lengths (voxel units) of the plane-q LOR of component ci in slabs iz = q - (j0 + k), k < NT,
// inside the pixel interval I.  The LOR's slab coordinate at the foot point,
// zeta_c = f + kappa tc, is split exactly into an integer n0 and a fraction in [0, 1); the
// crossings are then solved in local quantities of order one.  Returns j0.
template <int NT>
__device__ __forceinline__ int segment_taps(const DevGeom& g, int r, int ci, const PixInt& I, float* Lk) {
  // ci: the LOR component (its axial tilt); the plane mid-points are those of its segment
  const float4 rs = g.rs[r * g.n_comp + ci];
  const SegDev sd = g.seg[g.comp[ci].seg];
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

// Asynchronous global -> shared copies (4 and 16 bytes).
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

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

constexpr int kFwdChunk = 32;  // pixel entries per double-buffered chunk
constexpr int kRunsPerWarp = 2;  // 32-plane runs per warp (lane = plane within a run)
// Entry groups: when a line has few plane runs (a shallow volume), several warps share each run,
// each taking every egroups-th pixel entry, and their partial sums are added in group order.
constexpr int kFwdMaxGroupWarps = 7;  // warps of groups 1.. (their sums are staged in shared)

// Block-wide exclusive prefix sum of one int per thread (blockDim <= 1024); returns the
// exclusive prefix and writes the total to *total.  Uses `scratch` (>= 33 ints of shared).
__device__ __forceinline__ int block_exclusive_scan(int v, int* scratch, int* total) {
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) scratch[wi] = incl;
  __syncthreads();
  if (wi == 0) {
    int t = lane < nw ? scratch[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) scratch[lane] = t;  // inclusive warp totals
    if (lane == 31) scratch[32] = t;
  }
  __syncthreads();
  const int excl = incl - v + (wi > 0 ? scratch[wi - 1] : 0);
  *total = scratch[32];
  __syncthreads();
  return excl;
}

// Axial taps of one (pixel entry, segment) pair as the gather reads them: lengths of taps
// 0..NT-1 and, in `off`, the offset of plane 0's tap 0 in the staged x column (low 28 bits) and
// the entry's own tap count (top bits; lengths past it are zero).
struct TapRec {
  float l0, l1, l2;
  int off;
};
struct TapRec4 {  // geometries whose LORs cross four slices inside a pixel
  float l0, l1, l2;
  int off;
  float l3, pad0, pad1, pad2;
};
template <int NT>
using TapRecT = typename std::conditional<(NT > 3), TapRec4, TapRec>::type;
constexpr int kOffBits = 28;
constexpr int kOffMask = (1 << kOffBits) - 1;

__device__ __forceinline__ float2 ffma2_bcast(float l, float xa, float xb, float2 acc) {
  return __ffma2_rn(make_float2(l, l), make_float2(xa, xb), acc);
}

// sum_t L_t x[-t] over the entry's taps (scalar; one plane)
template <int NT, class Rec>
__device__ __forceinline__ float taps_dot(const Rec& t, int nt, const float* xp, float acc) {
  acc = fmaf(t.l0, xp[0], acc);
  if (NT > 1 && nt > 1) {
    acc = fmaf(t.l1, xp[-1], acc);
    if (NT > 2 && nt > 2) {
      acc = fmaf(t.l2, xp[-2], acc);
      if constexpr (NT > 3) {
        if (nt > 3) acc = fmaf(t.l3, xp[-3], acc);
      }
    }
  }
  return acc;
}

// Forward projection.  Block (line, row part, plane part) owns the rows [row_lo, row_hi) of one
// transaxial LOR line (view, radial bin) and a contiguous range of the line's plane runs (32
// consecutive planes of one segment, segment-major); warp w owns two neighbouring runs and lane l
// plane q0 + l of each.  All threads first find the pixels the line crosses in those rows (exact
// intervals, compacted); the entries are then processed in chunks of kFwdChunk: the x columns of
// chunk c+1 are copied to shared memory (cp.async) inside zero frames wide enough for every tap
// of every plane of the segments (the axial bound of the geometry, so no plane needs a range
// test), and its axial taps computed while chunk c is accumulated.  When both runs of a warp lie
// in one segment, one tap record serves both and a packed FP32 FMA accumulates the two planes.
// When a line has few runs, egroups warps share each pair of runs, warp group k taking the
// entries k, k + egroups, ... of every chunk; group 0 adds the other groups' sums in group order.
// When several row parts share a line, each writes partial plane sums and the last one to finish
// reduces them in a fixed order.
template <int NT, int MODE, bool GROUPS>
__global__ void __launch_bounds__(512) k_forward(DevGeom g, int subset, int ecap, int rsplit, int xs_stride,
                                                 int runs_per_part, int ncomp_tab, int chunk, int egroups_arg,
                                                 FwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int scan_scratch[33];
  const int FL = g.fz_lo;
  float* xs = reinterpret_cast<float*>(smem);                                  // [2][chunk][xs_stride]
  using Rec = TapRecT<NT>;
  Rec* taps = reinterpret_cast<Rec*>(xs + 2 * chunk * xs_stride);              // [2][ncomp_tab][chunk]
  Entry* ent = reinterpret_cast<Entry*>(taps + 2 * ncomp_tab * chunk);         // [ecap]
  float* group_acc = reinterpret_cast<float*>(ent + ecap);  // [egroups - 1][nrw][2][32] partial sums
  const int nz = g.nz;

  const int line = blockIdx.x, rpart = blockIdx.y, ppart = blockIdx.z;
  const int l = line / g.R, r = line - l * g.R;
  const int v = subset_view(g, subset, l);
  const Line L = make_line(g, v, r);

  // this thread's planes: lane of runs rf + 2w and rf + 2w + 1 of the plane part, w = wi mod
  // nrw; warp wi takes every egroups-th pixel entry from entry wi / nrw on
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const int egroups = GROUPS ? egroups_arg : 1;
  const int nrw = GROUPS ? nw / egroups : nw, rw = GROUPS ? wi % nrw : wi, eg = GROUPS ? wi / nrw : 0;
  const int rfirst = ppart * runs_per_part;
  const int rlast = min(g.n_runs, rfirst + runs_per_part) - 1;
  const int g_lo = g.runs[rfirst].x, g_hi = g.runs[rlast].x;
  // the LOR components of the block's segments, c_lo .. c_hi
  const int c_lo = g.seg[g_lo].c0, c_hi = g.seg[g_hi].c0 + g.seg[g_hi].nc - 1;
  int gs_[kRunsPerWarp], qv_[kRunsPerWarp], qr_[kRunsPerWarp];
  unsigned incl_[kRunsPerWarp];                  // mashed: components of the segment this plane sums
  bool valid_[kRunsPerWarp];
#pragma unroll
  for (int k = 0; k < kRunsPerWarp; ++k) {
    const int run = rfirst + kRunsPerWarp * rw + k;
    const int2 ru = g.runs[min(run, rlast)];
    const SegDev sd = g.seg[ru.x];
    gs_[k] = ru.x;
    qv_[k] = ru.y + lane;                        // the plane of this lane
    valid_[k] = run <= rlast && qv_[k] < sd.n;
    qr_[k] = min(qv_[k], sd.n - 1);              // the plane read (inside the segment's frames)
    incl_[k] = 0u;
    if (g.mashed)
      for (int c = 0; c < sd.nc; ++c) {
        const CompDev cd = g.comp[sd.c0 + c];
        const int dq = qv_[k] - cd.qlo;
        if (qv_[k] < cd.qhi && dq >= 0 && (dq & cd.smask) == 0) incl_[k] |= 1u << c;
      }
  }
  const bool same = gs_[0] == gs_[1];            // warp-uniform

  // zero frames of the staged columns (never overwritten); SIGMA stages ones: the projection of
  // the constant image is the chord of each LOR inside the image
  for (int i = threadIdx.x; i < 2 * chunk * xs_stride; i += blockDim.x) {
    const int k = i % xs_stride;
    if (MODE == FWD_SIGMA) xs[i] = (k >= FL && k < FL + nz) ? 1.f : 0.f;
    else if (k < FL || k >= FL + nz) xs[i] = 0.f;
  }
  const bool ydom = fabsf(L.c_hi) >= fabsf(L.s_hi);  // |dy| >= |dx|: walk the rows of y
  const int nrows_all = ydom ? g.ny : g.nx;
  const int rows_per_part = (nrows_all + rsplit - 1) / rsplit;
  const int row_lo = rpart * rows_per_part, row_hi = min(nrows_all, row_lo + rows_per_part);

  // A. this block's rows -> exact pixel intervals, compacted into ent[]
  int n_ent = 0;
  for (int row0 = row_lo; row0 < row_hi; row0 += blockDim.x) {
    Entry loc[kCandPerRow];
    const int row = row0 + threadIdx.x;
    const int cnt = row < row_hi ? row_entries(g, L, ydom, row, loc) : 0;
    int total;
    const int off = n_ent + block_exclusive_scan(cnt, scan_scratch, &total);
    for (int k = 0; k < cnt; ++k)
      if (off + k < ecap) ent[off + k] = loc[k];
    n_ent = min(n_ent + total, ecap);
  }
  __syncthreads();

  const int ncb = c_hi - c_lo + 1;
  auto stage = [&](int c) {  // x columns + taps of chunk c into buffer c & 1
    const int buf = c & 1;
    const int e0 = c * chunk, ne = min(chunk, n_ent - e0);
    float* xb = xs + buf * chunk * xs_stride;
    if (MODE != FWD_SIGMA) {
      // one warp per entry, lanes along z
      for (int e = wi; e < ne; e += nw) {
        const float* src = a.x + (size_t)ent[e0 + e].col * nz;
        float* dst = xb + e * xs_stride + FL;
        for (int iz = lane; iz < nz; iz += 32) cp_async4(dst + iz, src + iz);
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    Rec* tb = taps + buf * ncomp_tab * chunk;
    for (int it = threadIdx.x; it < ncb * ne; it += blockDim.x) {
      const int gs = it / ne, e = it - gs * ne;
      float Lk[4] = {0.f, 0.f, 0.f, 0.f};
      int j0 = segment_taps<NT>(g, r, c_lo + gs, ent[e0 + e].I, Lk);
      // the geometry's axial bound keeps every read inside the framed column; the clamp only
      // guards shared memory should a rounding case fall outside it
      const CompDev cd = g.comp[c_lo + gs];
      j0 = min(max(j0, cd.jlo), cd.jhi);
      int nt = NT;
      while (nt > 1 && Lk[nt - 1] == 0.f) --nt;
      Rec& rec = tb[gs * chunk + e];
      rec.l0 = Lk[0];
      rec.l1 = NT > 1 ? Lk[1] : 0.f;
      rec.l2 = NT > 2 ? Lk[2] : 0.f;
      rec.off = (e * xs_stride + FL - j0) | (nt << kOffBits);
      if constexpr (NT > 3) rec.l3 = Lk[3];
    }
  };

  float acc[kRunsPerWarp] = {0.f, 0.f};
  const int nchunks = (n_ent + chunk - 1) / chunk;
  if (nchunks > 0) stage(0);
  for (int c = 0; c < nchunks; ++c) {
    if (c + 1 < nchunks) {
      stage(c + 1);
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    const int buf = c & 1;
    const int ne = min(chunk, n_ent - c * chunk);
    const int nk = !GROUPS ? ne : (ne > eg ? (ne - eg + egroups - 1) / egroups : 0);  // entries eg + k egroups
    const float* xb = xs + buf * chunk * xs_stride;
    if (g.mashed) {
      // each plane sums the components of its segment it includes (exact mashing)
#pragma unroll
      for (int k = 0; k < kRunsPerWarp; ++k) {
        const SegDev sd = g.seg[gs_[k]];
        const Rec* trk = taps + buf * ncomp_tab * chunk + (sd.c0 - c_lo) * chunk;
        float sk = 0.f;
        for (int ci = 0; ci < sd.nc; ++ci) {
          const bool in = (incl_[k] >> ci) & 1u;
          const Rec* tc = trk + ci * chunk;
          float sc = 0.f;
          for (int kk = 0; kk < nk; ++kk) {
            const Rec t = tc[eg + kk * egroups];
            sc = taps_dot<NT>(t, NT > 1 ? (t.off >> kOffBits) : 1, xb + (t.off & kOffMask) + qr_[k], sc);
          }
          sk += in ? sc : 0.f;
        }
        acc[k] += sk;
      }
      __syncthreads();
      continue;
    }
    const Rec* tr0 = taps + buf * ncomp_tab * chunk + (gs_[0] - g_lo) * chunk;
    if (same) {
      float2 s2 = make_float2(0.f, 0.f);
#pragma unroll 1
      for (int k = 0; k < nk; ++k) {
        const Rec t = tr0[eg + k * egroups];
        const int off = t.off & kOffMask, nt = NT > 1 ? (t.off >> kOffBits) : 1;
        const float* xa = xb + off + qr_[0];
        // the warp's second run is the next 32 planes of the segment: a constant offset.  Lanes
        // past the segment's last plane read up to 31 slots beyond their column (the next
        // column, or the tap records after the last buffer) and are never written
        const float* xc = xa + 32;
        s2 = ffma2_bcast(t.l0, xa[0], xc[0], s2);
        if (NT > 1 && nt > 1) {
          s2 = ffma2_bcast(t.l1, xa[-1], xc[-1], s2);
          if (NT > 2 && nt > 2) {
            s2 = ffma2_bcast(t.l2, xa[-2], xc[-2], s2);
            if constexpr (NT > 3) {
              if (nt > 3) s2 = ffma2_bcast(t.l3, xa[-3], xc[-3], s2);
            }
          }
        }
      }
      acc[0] += s2.x;
      acc[1] += s2.y;
    } else {
      const Rec* tr1 = taps + buf * ncomp_tab * chunk + (gs_[1] - g_lo) * chunk;
      float s0 = 0.f, s1 = 0.f;
      for (int k = 0; k < nk; ++k) {
        const int e = eg + k * egroups;
        const Rec t0 = tr0[e], t1 = tr1[e];
        s0 = taps_dot<NT>(t0, NT > 1 ? (t0.off >> kOffBits) : 1, xb + (t0.off & kOffMask) + qr_[0], s0);
        s1 = taps_dot<NT>(t1, NT > 1 ? (t1.off >> kOffBits) : 1, xb + (t1.off & kOffMask) + qr_[1], s1);
      }
      acc[0] += s0;
      acc[1] += s1;
    }
    __syncthreads();
  }

  if (GROUPS) {
    // entry groups 1.. hand their partial sums to group 0, which adds them in group order
    if (eg > 0) {
#pragma unroll
      for (int k = 0; k < kRunsPerWarp; ++k) group_acc[(((eg - 1) * nrw + rw) * kRunsPerWarp + k) * 32 + lane] = acc[k];
    }
    __syncthreads();
    if (eg == 0) {
      for (int q = 1; q < egroups; ++q) {
#pragma unroll
        for (int k = 0; k < kRunsPerWarp; ++k) acc[k] += group_acc[(((q - 1) * nrw + rw) * kRunsPerWarp + k) * 32 + lane];
      }
    } else {
#pragma unroll
      for (int k = 0; k < kRunsPerWarp; ++k) valid_[k] = false;  // group 0 writes the planes
    }
  }

  if (rsplit > 1) {
    // publish this block's partial sums; the last row part of the (line, plane part) reduces them
    __shared__ unsigned last_sh;
    const size_t pbase = ((size_t)line * rsplit + rpart) * g.P;
#pragma unroll
    for (int k = 0; k < kRunsPerWarp; ++k)
      if (valid_[k]) a.part_acc[pbase + g.seg[gs_[k]].p0 + qv_[k]] = acc[k];
    __threadfence();
    __syncthreads();
    const size_t ticket = (size_t)line * gridDim.z + ppart;
    if (threadIdx.x == 0) last_sh = (atomicAdd(a.tickets + ticket, 1u) == (unsigned)rsplit - 1u) ? 1u : 0u;
    __syncthreads();
    if (!last_sh) return;
    __threadfence();
#pragma unroll
    for (int k = 0; k < kRunsPerWarp; ++k) {
      if (!valid_[k]) continue;
      float sa = 0.f;
      for (int q = 0; q < rsplit; ++q)  // fixed order: deterministic
        sa += __ldcg(a.part_acc + ((size_t)line * rsplit + q) * g.P + g.seg[gs_[k]].p0 + qv_[k]);
      acc[k] = sa;
    }
    if (threadIdx.x == 0) a.tickets[ticket] = 0u;  // ready for the next launch
  }

#pragma unroll
  for (int k = 0; k < kRunsPerWarp; ++k) {
    if (!valid_[k]) continue;
    const int p = g.seg[gs_[k]].p0 + qv_[k];
    const size_t j = ((size_t)v * g.R + r) * g.P + p;
    const size_t jl = ((size_t)l * g.R + r) * g.P + p;  // subset-local index (= j for bin subsets)
    if (!bin_in_subset(g, subset, j)) {  // a bin of another subset: not written; no dual change
      if (MODE == FWD_DATA || MODE == FWD_EM) a.wdy[jl] = 0.f;
      continue;
    }
    const float mu = a.mult ? a.mult[j] : 1.f;
    if (MODE == FWD_EM) {
      // EM ratio backprojected by P^T = L^T diag(mult): mult_j b_j / ((P x)_j + r_j)  (Eq. EQU:OSEM)
      const float bj = a.b[j];
      a.wdy[jl] = bj > 0.f ? mu * bj / fmaf(mu, acc[k], a.r[j]) : 0.f;
    } else if (MODE == FWD_PROJECT) {
      a.out[j] = mu * acc[k];
    } else if (MODE == FWD_SIGMA) {
      // sigma_j = gamma rho / (P_i 1)_j,  (P_i 1)_j = mult_j * chord_j  (Eq. EQU:STEPSIZE:PRECOND)
      const float a1 = mu * acc[k];
      a.out[j] = a1 > 0.f ? a.gamma_rho / a1 : 0.f;
    } else {
      // KL dual prox on this bin:  y+ = prox_{sigma varphi*}(y + sigma (P_i x)_j), evaluated as
      // 2 (w - sigma b) / (w + 1 + sqrt((w - 1)^2 + 4 sigma b)),  w = y + sigma ((P_i x)_j + r_j),
      // which equals 1/2 [w + 1 - sqrt((w - 1)^2 + 4 sigma b)] without its cancellation.
      const float sigma = a.sigma[j];
      const float yj = a.y[j];
      const float bj = a.b[j];
      const float w = fmaf(sigma, fmaf(mu, acc[k], a.r[j]), yj);
      const float sb = sigma * bj;
      const float wm = w - 1.f;
      const float root = sqrtf(fmaf(wm, wm, 4.f * sb));
      const float yn = 2.f * (w - sb) / (w + 1.f + root);
      a.y[j] = yn;
      a.wdy[jl] = mu * (yn - yj);
    }
  }
}

// ---------------------------------------------------------------------------------------
// backprojection: one thread group per voxel column (ix, iy), threads over iz
// ---------------------------------------------------------------------------------------

struct PixItem {
  int l, r;  // view (subset-local) and radial bin
  PixInt I;
};

constexpr int kBwdTileX = 4;             // block = kBwdTileX x kBwdTileY voxel columns, one warp each
constexpr int kBwdTileY = 4;
constexpr int kBwdWarps = kBwdTileX * kBwdTileY;
constexpr int kBwdBlocksPerSM = 64 / kBwdWarps;      // resident blocks, up to 128 slices (4 voxels a lane)
constexpr int kBwdBlocksPerSM8 = 48 / kBwdWarps;     // more slices (8 accumulators a lane)
constexpr int kBwdMaxItems = 64;         // (pair, segment) items per column and view

// Gather of one column's items on an unmashed geometry, bucket b holding the items with b + 1
// taps: voxel iz (lane + 32 k) adds sum_t L_t sw[x + iz + t] where its first tap's plane
// iz + j0 lies in [-PAD, n) (the segment's frames supply the zeros of the other taps).
template <int NT, int ZK>
__device__ __forceinline__ void gather_items(const float* sw, const float4* myL, const int4* myM, const int* bs,
                                             int lane, float* acc) {
#pragma unroll
  for (int b = 0; b < NT; ++b) {
    for (int it = bs[b]; it < bs[b + 1]; ++it) {
      const float4 Lv = myL[it];
      const int4 M = myM[it];
      const float* src0 = sw + M.x;
#pragma unroll
      for (int k = 0; k < ZK; ++k) {
        const int iz = lane + 32 * k;
        if ((unsigned)(iz + M.y) < (unsigned)M.z) {
          const float* src = src0 + iz;
          float sum = Lv.x * src[0];
          if (b >= 1) sum = fmaf(Lv.y, src[1], sum);
          if (b >= 2) sum = fmaf(Lv.z, src[2], sum);
          if (b >= 3) sum = fmaf(Lv.w, src[3], sum);
          acc[k] += sum;
        }
      }
    }
  }
}

// Backprojection.  A block owns a 4 x 4 tile of voxel columns; for each view of the subset it
// stages the contiguous radial rows w[view][r_min..r_max][0..P) that the tile's footprints
// touch into shared memory (cp.async, overlapped with the geometry below; the first view's copies
// are issued before anything else), each segment's plane run framed by NT-1 zeros so that taps
// leaving the segment read zeros.  Each warp owns one column: its lanes find the footprint (bin,
// pixel interval) pairs, compact them with a ballot, compute the axial taps of every (pair,
// segment) item, and then gather along contiguous plane runs from shared memory, lane = iz mod
// 32, ZK voxels per lane.  With TAB the items, in the same order, are read from the table
// spdhg_setup builds (k_bwd_items) instead of being computed.  In BWD_UPDATE the epilogue's x, z,
// T lines are requested into L2 at block start, and after the last view each warp goes on to its
// epilogue without waiting for the others.  Up to 128 slices (ZK <= 4) four blocks share an SM
// (32 registers per thread); with eight accumulators per lane, three.
template <int NT, int ZK, int MODE, bool MASHED, bool TAB>
__global__ void __launch_bounds__(kBwdWarps * 32, ZK <= 4 ? kBwdBlocksPerSM : kBwdBlocksPerSM8) k_backward(DevGeom g, int subset, int nr_tile, int p_pad,
                                                             int bcap, int cpb, BwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int PAD = NT - 1;
  const int icap = bcap;  // items per warp (all buckets)
  float* sw = reinterpret_cast<float*>(smem);                                  // nr_tile x p_pad
  float4* itL = reinterpret_cast<float4*>(sw + ((nr_tile * p_pad + 3) & ~3));  // [warp][icap]
  int4* itM = reinterpret_cast<int4*>(itL + kBwdWarps * icap);
  PixItem* pix = reinterpret_cast<PixItem*>(itM + kBwdWarps * icap);          // [warp][nr_max]
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  float4* myL = itL + wi * icap;
  int4* myM = itM + wi * icap;
  PixItem* mypix = pix + wi * g.nr_max;
  const int nviews = subset_views(g, subset);
  const int nz = g.nz;
  const int tx0 = blockIdx.x * kBwdTileX, ty0 = blockIdx.y * kBwdTileY;
  const int ix = tx0 + (wi % kBwdTileX), iy = ty0 + (wi / kBwdTileX);
  const bool live = ix < g.nx && iy < g.ny;
  const float Xc = (float)ix + 0.5f - 0.5f * (float)g.nx;
  const float Yc = (float)iy + 0.5f - 0.5f * (float)g.ny;
  const float X0 = (float)tx0 + 0.5f - 0.5f * (float)g.nx, Y0 = (float)ty0 + 0.5f - 0.5f * (float)g.ny;
  const float X1 = X0 + (float)(kBwdTileX - 1), Y1 = Y0 + (float)(kBwdTileY - 1);
  float acc[ZK];
#pragma unroll
  for (int k = 0; k < ZK; ++k) acc[k] = 0.f;
  // 1. rows r_min..r_max of view l of the subset -> their slots in the staged rows (each segment's
  //    planes framed by zeros); the radial rows are those of the whole tile's footprints (its
  //    extreme pixel centres).  The first view's copies are issued before anything else.
  auto rows_of = [&](int l, int* rmin) {
    const float4 cs = g.view[subset_view(g, subset, l)];
    const float hw = 0.5f * (fabsf(cs.x) + fabsf(cs.z));
    const float s00 = X0 * cs.x + Y0 * cs.z, s01 = X0 * cs.x + Y1 * cs.z;
    const float s10 = X1 * cs.x + Y0 * cs.z, s11 = X1 * cs.x + Y1 * cs.z;
    const float smin = fminf(fminf(s00, s01), fminf(s10, s11)), smax = fmaxf(fmaxf(s00, s01), fmaxf(s10, s11));
    const int r_min = max(0, (int)ceilf((smin - hw) * g.inv_drp + g.half_R) - 1);
    *rmin = r_min;
    return min(g.R - 1, min(r_min + nr_tile - 1, (int)floorf((smax + hw) * g.inv_drp + g.half_R) + 1));
  };
  auto stage = [&](int l) {
    int r_min;
    const int r_max = rows_of(l, &r_min);
    const float* src = a.w + ((size_t)l * g.R + r_min) * g.P;
    const int nr = r_max - r_min + 1;
    for (int p = threadIdx.x; p < g.P; p += blockDim.x) {
      const int dst = __ldg(g.stage_pos + p);
      for (int rr = 0; rr < nr; ++rr) cp_async4(sw + rr * p_pad + dst, src + rr * g.P + p);
    }
  };
  if (nviews > 0) stage(0);
  if constexpr (MODE == BWD_UPDATE) {
    // the epilogue's x, z, T lines of the block's columns are requested into L2 now, so that
    // their DRAM reads overlap the staging and the gather
    const int lines = (nz + 31) / 32;
    for (int q = threadIdx.x; q < kBwdWarps * 3 * lines; q += blockDim.x) {
      const int col = q / (3 * lines), rem = q - col * 3 * lines, arr = rem / lines, seg = rem - arr * lines;
      const int cx = tx0 + (col % kBwdTileX), cy = ty0 + (col / kBwdTileX);
      if (cx < g.nx && cy < g.ny) {
        const float* base = arr == 0 ? (const float*)a.x : (arr == 1 ? (const float*)a.z : a.T);
        asm volatile("prefetch.global.L2 [%0];" ::"l"(base + ((size_t)cy * g.nx + cx) * nz + 32 * seg));
      }
    }
  }
  // the zero frames of the staged rows (written once; the copies never touch them)
  if constexpr (PAD > 0) {
    for (int i = threadIdx.x; i < nr_tile * g.n_seg * 2 * PAD; i += blockDim.x) {
      const int rr = i / (g.n_seg * 2 * PAD), rem = i - rr * (g.n_seg * 2 * PAD);
      const int gi = rem / (2 * PAD), k = rem - gi * (2 * PAD);
      const SegDev sd = g.seg[gi];
      const int start = sd.p0 + 2 * gi * PAD;  // first slot of the segment's frame
      sw[rr * p_pad + (k < PAD ? start + k : start + PAD + sd.n + (k - PAD))] = 0.f;
    }
  }
  __syncthreads();

  for (int l = 0; l < nviews; ++l) {
    const int v = subset_view(g, subset, l);
    const float4 cs = g.view[v];
    const float hw = 0.5f * (fabsf(cs.x) + fabsf(cs.z));
    int r_min;
    const int r_max = rows_of(l, &r_min);
    if (l > 0) stage(l);
    int bs[5] = {0, 0, 0, 0, 0};  // bucket b (items with b + 1 taps) spans [bs[b], bs[b + 1])
    if constexpr (TAB) {
      // 2-3. this column's items, in the order the code below computes them, from the table
      const int2 h = a.hdr[((size_t)v * gridDim.x * gridDim.y + (size_t)blockIdx.y * gridDim.x + blockIdx.x) *
                               kBwdWarps + wi];
      const int n = h.y >> 16;
      bs[1] = h.y & 0xFF;
      if (NT > 2) bs[2] = (h.y >> 8) & 0xFF;
      bs[NT] = n;
      for (int it = lane; it < n; it += 32) {
        const float4 e = a.items[(size_t)(unsigned)h.x + it];
        const unsigned pk = __float_as_uint(e.w);
        const int idx = (int)(pk >> 25);
        myL[it] = make_float4(e.x, e.y, e.z, 0.f);
        if constexpr (MASHED) {
          const CompDev cd = g.comp[idx];
          myM[it] = make_int4((int)(pk & 0xFFFFu), (int)((pk >> 16) & 0x1FFu) - 256, cd.qhi - cd.qlo, cd.smask);
        } else {
          myM[it] = make_int4((int)(pk & 0xFFFFu), (int)((pk >> 16) & 0x1FFu) - 256, g.seg[idx].n + PAD, 0);
        }
      }
    }
    // 2. footprint pairs of this warp's column (overlaps the copy)
    PixItem P;
    bool ok = false;
    if (!TAB && live && lane < g.nr_max) {
      const float sc = Xc * cs.x + Yc * cs.z;
      const int rlo = (int)ceilf((sc - hw) * g.inv_drp + g.half_R) - 1;
      const int rhi = (int)floorf((sc + hw) * g.inv_drp + g.half_R) + 1;
      const int r = rlo + lane;
      if (r >= r_min && r <= r_max && r <= rhi) {
        const Line L = make_line(g, v, r);
        ok = pixel_interval(g, L, ix, iy, P.I);
        P.l = l;
        P.r = r;
      }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, ok);
    if (!TAB && ok) mypix[__popc(mask & ((1u << lane) - 1u))] = P;
    const int np = __popc(mask);
    __syncwarp();
    // 3. axial taps per (pair, component), ordered by tap count: a lane holds up to two items,
    //    ballots count each tap-count bucket, and the items are written bucket after bucket.  The
    //    components are taken in batches of cpb (one batch unless the bins are mashed).
    for (int cf = 0; cf < (MASHED ? g.n_comp : 1); cf += cpb) {
    const int ccount = MASHED ? min(cpb, g.n_comp - cf) : g.n_comp;
    const int ni = TAB ? 0 : min(np * ccount, bcap);
    float4 Lv2[2];
    int4 Mv2[2];
    int nt2[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int it = lane + 32 * h;
      Lv2[h] = make_float4(0.f, 0.f, 0.f, 0.f);
      Mv2[h] = make_int4(0, 0, 0, 0);
      if (it < ni) {
        const int pi = it / ccount, ci = cf + (it - pi * ccount);
        const PixItem Q = mypix[pi];
        float Lk[4] = {0.f, 0.f, 0.f, 0.f};
        const int j0 = segment_taps<NT>(g, Q.r, ci, Q.I, Lk);
        int nt = NT;
        while (nt > 1 && Lk[nt - 1] == 0.f) --nt;
        const CompDev cd = g.comp[ci];
        const int gi = cd.seg;
        const SegDev sd = g.seg[gi];
        Lv2[h] = make_float4(Lk[0], Lk[1], Lk[2], Lk[3]);
        // voxel iz, tap t reads plane q = iz + j0 + t at sw[x + iz + t]; without mashing some tap is
        // inside the segment while -PAD <= iz + j0 < n, and the frame supplies zeros for the
        // others; a mashed component keeps the taps of the planes that include it
        const int x = (Q.r - r_min) * p_pad + sd.p0 + (2 * gi + 1) * PAD + j0;
        Mv2[h] = MASHED ? make_int4(x, j0 - cd.qlo, cd.qhi - cd.qlo, cd.smask)
                        : make_int4(x, j0 + PAD, sd.n + PAD, 0);
        nt2[h] = nt;
      }
    }
    if (!TAB) {
      int off = 0;
#pragma unroll
      for (int b = 0; b < NT; ++b) {
        const unsigned m0 = __ballot_sync(0xffffffffu, nt2[0] == b + 1);
        const unsigned m1 = __ballot_sync(0xffffffffu, nt2[1] == b + 1);
        const unsigned below = (1u << lane) - 1u;
        if (nt2[0] == b + 1) {
          const int slot = off + __popc(m0 & below);
          myL[slot] = Lv2[0];
          myM[slot] = Mv2[0];
        }
        if (nt2[1] == b + 1) {
          const int slot = off + __popc(m0) + __popc(m1 & below);
          myL[slot] = Lv2[1];
          myM[slot] = Mv2[1];
        }
        bs[b] = off;
        off += __popc(m0) + __popc(m1);
      }
      bs[NT] = off;
    }
    if (!MASHED || cf == 0) {
      cp_async_commit_wait_all();
      __syncthreads();
    } else {
      __syncwarp();
    }
    // 4. gather: one branch-free loop per tap count
    if (live && !MASHED) {
      gather_items<NT, ZK>(sw, myL, myM, bs, lane, acc);
    } else if (live) {
      // mashed: tap t of voxel iz counts when its plane includes the component
#pragma unroll
      for (int b = 0; b < NT; ++b) {
        for (int it = bs[b]; it < bs[b + 1]; ++it) {
          const float4 Lv = myL[it];
          const int4 M = myM[it];
          const float* src0 = sw + M.x;
          const float Lt[4] = {Lv.x, Lv.y, Lv.z, Lv.w};
#pragma unroll
          for (int k = 0; k < ZK; ++k) {
            const int iz = lane + 32 * k;
            float sum = 0.f;
#pragma unroll
            for (int t = 0; t <= b; ++t) {
              const int rel = iz + t + M.y;  // plane - qlo
              if ((unsigned)rel < (unsigned)M.z && (rel & M.w) == 0) sum = fmaf(Lt[t], src0[iz + t], sum);
            }
            acc[k] += sum;
          }
        }
      }
    }
    if (MASHED) __syncwarp();  // the items are replaced by the next batch's
    }  // component batches
    // the staged rows are replaced by the next view's; after the last view each warp goes on to
    // its epilogue as soon as its own gather is done, so that the early warps' loads and stores
    // overlap the others' gathers
    if (l + 1 < nviews) __syncthreads();
  }
  if (!live) return;
#pragma unroll
  for (int k = 0; k < ZK; ++k) {
    const int iz = lane + 32 * k;
    if (iz >= nz) continue;
    const size_t idx = ((size_t)iy * g.nx + ix) * nz + iz;
    if (MODE == BWD_OUT) {
      a.out[idx] = acc[k];
    } else if (MODE == BWD_SENS) {
      // T_i = rho p_i / (gamma (P_i^T 1)); +inf (kept) where the subset does not see the voxel
      if (acc[k] > 0.f) a.T[idx] = fminf(a.T[idx], a.sens_num / acc[k]);
    } else if (MODE == BWD_EM) {
      // u <- u / (P_i^T 1) * P_i^T (b_i / (P_i u + r_i)), 0 where the subset does not see the voxel
      const float sens = a.T[idx];
      a.x[idx] = sens > 0.f ? a.x[idx] * acc[k] / sens : 0.f;
    } else {
      // z = z + dz;  zbar = z + dz / p_i;  next primal step x = max(x - T zbar, 0)
      const float zn = a.z[idx] + acc[k];
      a.z[idx] = zn;
      a.x[idx] = prox_nonneg(a.x[idx] - a.T[idx] * fmaf(acc[k], a.inv_p, zn));
    }
  }
}

// ---------------------------------------------------------------------------------------
// tap-item table of the backprojector: the (pair, component) items of every view, tile and
// column, computed once by the code the kernel runs and read back by k_backward<..., TAB>
// ---------------------------------------------------------------------------------------

constexpr int kTabMaxPairs = 16;  // candidate radial bins per column and view (nr_max <= 16)

template <int NT, int PASS>
__global__ void __launch_bounds__(kBwdWarps * 32) k_bwd_items(DevGeom g, int nr_tile, int p_pad, int bcap,
                                                           unsigned char* cnt, unsigned* bad, const unsigned* starts,
                                                           const unsigned* view_base, float4* items, int2* hdr) {
  __shared__ PixItem pix[kBwdWarps][kTabMaxPairs];
  constexpr int PAD = NT - 1;
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int tx0 = blockIdx.x * kBwdTileX, ty0 = blockIdx.y * kBwdTileY;
  const int ix = tx0 + (wi % kBwdTileX), iy = ty0 + (wi / kBwdTileX);
  const bool live = ix < g.nx && iy < g.ny;
  const float Xc = (float)ix + 0.5f - 0.5f * (float)g.nx;
  const float Yc = (float)iy + 0.5f - 0.5f * (float)g.ny;
  const float X0 = (float)tx0 + 0.5f - 0.5f * (float)g.nx, Y0 = (float)ty0 + 0.5f - 0.5f * (float)g.ny;
  const float X1 = X0 + (float)(kBwdTileX - 1), Y1 = Y0 + (float)(kBwdTileY - 1);
  const int v = blockIdx.z;
  const size_t col = ((size_t)v * gridDim.x * gridDim.y + (size_t)blockIdx.y * gridDim.x + blockIdx.x) * kBwdWarps + wi;
  PixItem* mypix = pix[wi];
  // the same arithmetic as k_backward for view v
  const float4 cs = g.view[v];
  const float hw = 0.5f * (fabsf(cs.x) + fabsf(cs.z));
  const float s00 = X0 * cs.x + Y0 * cs.z, s01 = X0 * cs.x + Y1 * cs.z;
  const float s10 = X1 * cs.x + Y0 * cs.z, s11 = X1 * cs.x + Y1 * cs.z;
  const float smin = fminf(fminf(s00, s01), fminf(s10, s11)), smax = fmaxf(fmaxf(s00, s01), fmaxf(s10, s11));
  const int r_min = max(0, (int)ceilf((smin - hw) * g.inv_drp + g.half_R) - 1);
  const int r_max = min(g.R - 1, min(r_min + nr_tile - 1, (int)floorf((smax + hw) * g.inv_drp + g.half_R) + 1));
  PixItem P;
  bool ok = false;
  if (live && lane < g.nr_max) {
    const float sc = Xc * cs.x + Yc * cs.z;
    const int rlo = (int)ceilf((sc - hw) * g.inv_drp + g.half_R) - 1;
    const int rhi = (int)floorf((sc + hw) * g.inv_drp + g.half_R) + 1;
    const int r = rlo + lane;
    if (r >= r_min && r <= r_max && r <= rhi) {
      const Line L = make_line(g, v, r);
      ok = pixel_interval(g, L, ix, iy, P.I);
      P.l = v;
      P.r = r;
    }
  }
  const unsigned mask = __ballot_sync(0xffffffffu, ok);
  if (ok) mypix[__popc(mask & ((1u << lane) - 1u))] = P;
  const int np = __popc(mask);
  __syncwarp();
  const int ccount = g.n_comp;
  const int ni = min(np * ccount, bcap);
  float4 It[2];
  int nt2[2] = {0, 0};
  bool misfit = false;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int it = lane + 32 * h;
    It[h] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (it < ni) {
      const int pi = it / ccount, ci = it - pi * ccount;
      const PixItem Q = mypix[pi];
      float Lk[4] = {0.f, 0.f, 0.f, 0.f};
      const int j0 = segment_taps<NT>(g, Q.r, ci, Q.I, Lk);
      int nt = NT;
      while (nt > 1 && Lk[nt - 1] == 0.f) --nt;
      const CompDev cd = g.comp[ci];
      const int gi = cd.seg;
      const SegDev sd = g.seg[gi];
      const int x = (Q.r - r_min) * p_pad + sd.p0 + (2 * gi + 1) * PAD + j0;
      // first tap's offset: to the segment's frame (unmashed) or to the component's first plane
      // (mashed, whose bound and parity come from the component), and which of the two indexes
      const int jp = (g.mashed ? j0 - cd.qlo : j0 + PAD) + 256;
      const int idx = g.mashed ? ci : gi;
      misfit = misfit || x < 0 || x >= 65536 || jp < 0 || jp >= 512 || idx >= 128;
      const unsigned packed = ((unsigned)x & 0xFFFFu) | (((unsigned)jp & 0x1FFu) << 16) | ((unsigned)idx << 25);
      It[h] = make_float4(Lk[0], Lk[1], Lk[2], __uint_as_float(packed));
      nt2[h] = nt;
    }
  }
  int bs[4] = {0, 0, 0, 0};
  unsigned base = 0;
  if (PASS == 1) base = view_base[v] + starts[col];
  {
    int off = 0;
#pragma unroll
    for (int b = 0; b < NT; ++b) {
      const unsigned m0 = __ballot_sync(0xffffffffu, nt2[0] == b + 1);
      const unsigned m1 = __ballot_sync(0xffffffffu, nt2[1] == b + 1);
      const unsigned below = (1u << lane) - 1u;
      if (PASS == 1) {
        if (nt2[0] == b + 1) items[base + off + __popc(m0 & below)] = It[0];
        if (nt2[1] == b + 1) items[base + off + __popc(m0) + __popc(m1 & below)] = It[1];
      }
      off += __popc(m0) + __popc(m1);
      bs[b + 1] = off;
    }
  }
  if (PASS == 0) {
    if (__any_sync(0xffffffffu, misfit) && lane == 0) atomicOr(bad, 1u);
    if (lane == 0) cnt[col] = (unsigned char)bs[NT];
  } else if (lane == 0) {
    const int n1 = bs[1], n12 = NT > 2 ? bs[2] : bs[NT], n = bs[NT];
    hdr[col] = make_int2((int)base, n1 | (n12 << 8) | (n << 16));
  }
}

// per view: exclusive prefix sums of the columns' item counts, and the view's total
__global__ void __launch_bounds__(1024) k_bwd_table_scan(const unsigned char* cnt, size_t cols_per_view,
                                                         unsigned* starts, unsigned* totals) {
  __shared__ int scratch[33];
  const size_t v = blockIdx.x;
  const unsigned char* c = cnt + v * cols_per_view;
  unsigned* st = starts + v * cols_per_view;
  const size_t per = (cols_per_view + blockDim.x - 1) / blockDim.x;
  const size_t lo = min(cols_per_view, threadIdx.x * per), hi = min(cols_per_view, lo + per);
  int sum = 0;
  for (size_t k = lo; k < hi; ++k) sum += c[k];
  int total;
  int run = block_exclusive_scan(sum, scratch, &total);
  for (size_t k = lo; k < hi; ++k) {
    st[k] = (unsigned)run;
    run += c[k];
  }
  if (threadIdx.x == 0) totals[v] = (unsigned)total;
}

// one table record per (pair, component) item of a single batch: mashed geometries qualify when
// all their components fit in one batch of the backprojector
bool backward_table_possible(const DevGeom& g) {
  const int max_pairs = (int)floorf(1.4143f * g.inv_drp) + 2;
  return !g.bins && g.taps <= 3 && g.nr_max <= kTabMaxPairs && max_pairs * g.n_comp <= kBwdMaxItems;
}

static int bwd_rows_per_tile(const DevGeom& g);

template <int PASS>
static cudaError_t table_pass(const DevGeom& g, unsigned char* cnt, unsigned* bad, const unsigned* starts,
                              const unsigned* view_base, float4* items, int2* hdr, cudaStream_t s) {
  if (!backward_table_possible(g)) return cudaErrorInvalidValue;
  const int max_pairs = (int)floorf(1.4143f * g.inv_drp) + 2;
  const int bcap = max_pairs * g.n_comp;
  const int nr_tile = bwd_rows_per_tile(g);
  const int NT = g.taps;
  const int p_pad = g.P + 2 * (NT - 1) * g.n_seg;
  dim3 grid((g.nx + kBwdTileX - 1) / kBwdTileX, (g.ny + kBwdTileY - 1) / kBwdTileY, g.V);
  switch (NT) {
    case 1: k_bwd_items<1, PASS><<<grid, kBwdWarps * 32, 0, s>>>(g, nr_tile, p_pad, bcap, cnt, bad, starts, view_base, items, hdr); break;
    case 2: k_bwd_items<2, PASS><<<grid, kBwdWarps * 32, 0, s>>>(g, nr_tile, p_pad, bcap, cnt, bad, starts, view_base, items, hdr); break;
    default: k_bwd_items<3, PASS><<<grid, kBwdWarps * 32, 0, s>>>(g, nr_tile, p_pad, bcap, cnt, bad, starts, view_base, items, hdr); break;
  }
  return cudaGetLastError();
}

cudaError_t backward_table_count(const DevGeom& g, unsigned char* cnt, unsigned* bad, cudaStream_t s) {
  return table_pass<0>(g, cnt, bad, nullptr, nullptr, nullptr, nullptr, s);
}

cudaError_t backward_table_starts(const DevGeom& g, const unsigned char* cnt, unsigned* starts,
                                  unsigned* view_totals, cudaStream_t s) {
  const size_t cols = (size_t)((g.nx + kBwdTileX - 1) / kBwdTileX) * ((g.ny + kBwdTileY - 1) / kBwdTileY) * kBwdWarps;
  k_bwd_table_scan<<<g.V, 1024, 0, s>>>(cnt, cols, starts, view_totals);
  return cudaGetLastError();
}

cudaError_t backward_table_fill(const DevGeom& g, const unsigned* starts, const unsigned* view_base,
                                float4* items, int2* hdr, cudaStream_t s) {
  return table_pass<1>(g, nullptr, nullptr, starts, view_base, items, hdr, s);
}

__global__ void k_gather_subset(DevGeom g, int subset, const float* __restrict__ y,
                                const float* __restrict__ mult, float* __restrict__ w) {
  const int64_t per_view = (int64_t)g.R * g.P;
  const int64_t n = (int64_t)subset_views(g, subset) * per_view;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int l = (int)(i / per_view);
    const int64_t j = (int64_t)subset_view(g, subset, l) * per_view + (i - l * per_view);
    const float v = (y ? y[j] : 1.f) * (mult ? mult[j] : 1.f);
    w[i] = bin_in_subset(g, subset, (size_t)j) ? v : 0.f;
  }
}

// ---------------------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------------------

int forward_split(const DevGeom& g, int subset) {
  if (g.tune[SPDHG_TUNE_FWD_SPLIT]) return g.tune[SPDHG_TUNE_FWD_SPLIT];
  // enough blocks for every SM: one LOR line per block is too few for small subsets
  const int lines = subset_views(g, subset) * g.R * forward_parts(g);
  const int nrows = g.nx > g.ny ? g.nx : g.ny;
  int split = 1;
  while (split < 8 && lines * split < 152 && nrows / (split * 2) >= 32) split *= 2;
  return split;
}

// plane runs per block: two per warp, at most 16 warps
static int forward_runs_per_part(const DevGeom& g) {
  const int w = g.tune[SPDHG_TUNE_FWD_WARPS] ? g.tune[SPDHG_TUNE_FWD_WARPS] : 16;
  return w * kRunsPerWarp;
}

int forward_parts(const DevGeom& g) {
  const int rpp = forward_runs_per_part(g);
  return (g.n_runs + rpp - 1) / rpp;
}

// entry groups per block: at least four warps per block when the runs of a part need fewer
int forward_entry_groups(const DevGeom& g) {
  const int rpp = forward_runs_per_part(g);
  const int nrw = (std::min(rpp, g.n_runs) + kRunsPerWarp - 1) / kRunsPerWarp;
  int eg = g.tune[SPDHG_TUNE_FWD_GROUPS] ? g.tune[SPDHG_TUNE_FWD_GROUPS] : std::max(1, 4 / nrw);
  while (eg > 1 && ((eg - 1) * nrw > kFwdMaxGroupWarps || nrw * eg > 16)) --eg;
  return eg;
}

template <int NT, int MODE>
static cudaError_t fwd_launch(const DevGeom& g, int subset, const FwdArgs& a, cudaStream_t s) {
  const int xs_stride = g.fz_stride;
  const int nrows = g.nx > g.ny ? g.nx : g.ny;
  const int ecap = 3 * nrows + 8;  // a line crosses at most two pixels per row of its dominant axis
  const int rpp = forward_runs_per_part(g);
  const int parts = (g.n_runs + rpp - 1) / rpp;
  const int nrw = (std::min(rpp, g.n_runs) + kRunsPerWarp - 1) / kRunsPerWarp;  // warps per entry group
  const int egroups = forward_entry_groups(g);
  if (egroups < 1 || (egroups - 1) * nrw > kFwdMaxGroupWarps || nrw * egroups > 16) return cudaErrorInvalidValue;
  const int threads = 32 * nrw * egroups;
  // a block computes the taps of the components of the segments its runs span
  const int ncomp_tab = g.max_part_comps[rpp / kRunsPerWarp];
  // entries per chunk: 32, fewer when a block holds the taps of many components (mashing)
  int chunk = kFwdChunk;
  while (chunk > 4 && (size_t)2 * ncomp_tab * chunk * sizeof(TapRecT<NT>) > 48 * 1024) chunk /= 2;
  const size_t smem = (size_t)2 * chunk * xs_stride * sizeof(float) +
                      (size_t)2 * ncomp_tab * chunk * sizeof(TapRecT<NT>) + (size_t)ecap * sizeof(Entry) +
                      (size_t)(egroups - 1) * nrw * kRunsPerWarp * 32 * sizeof(float);
  if (smem > 200 * 1024 || (size_t)chunk * xs_stride >= ((size_t)1 << kOffBits)) return cudaErrorInvalidValue;
  if (MODE == FWD_DATA && !a.sigma) return cudaErrorInvalidValue;
  if ((MODE == FWD_DATA || MODE == FWD_EM) && (!a.b || !a.r || !a.wdy)) return cudaErrorInvalidValue;
  auto kern = egroups > 1 ? k_forward<NT, MODE, true> : k_forward<NT, MODE, false>;
  {
    cudaError_t e = allow_dynamic_smem(kern, smem);
    if (e != cudaSuccess) return e;
  }
  const int lines = subset_views(g, subset) * g.R;
  if (lines == 0) return cudaSuccess;
  const int rsplit = forward_split(g, subset);
  if (rsplit > 1 && (!a.part_acc || !a.tickets || (size_t)lines * rsplit * g.P > a.part_cap ||
                     (size_t)lines * parts > a.ticket_cap))
    return cudaErrorInvalidValue;
  dim3 grid(lines, rsplit, parts);
  kern<<<grid, threads, smem, s>>>(g, subset, ecap, rsplit, xs_stride, rpp, ncomp_tab, chunk, egroups, a);
  return cudaGetLastError();
}

template <int MODE>
static cudaError_t fwd_nt(const DevGeom& g, int subset, const FwdArgs& a, cudaStream_t s) {
  switch (g.taps) {
    case 1: return fwd_launch<1, MODE>(g, subset, a, s);
    case 2: return fwd_launch<2, MODE>(g, subset, a, s);
    case 3: return fwd_launch<3, MODE>(g, subset, a, s);
    case 4: return fwd_launch<4, MODE>(g, subset, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_forward(const DevGeom& g, int subset, int mode, const FwdArgs& a, cudaStream_t s) {
  switch (mode) {
    case FWD_PROJECT: return fwd_nt<FWD_PROJECT>(g, subset, a, s);
    case FWD_SIGMA: return fwd_nt<FWD_SIGMA>(g, subset, a, s);
    case FWD_DATA: return fwd_nt<FWD_DATA>(g, subset, a, s);
    case FWD_EM: return fwd_nt<FWD_EM>(g, subset, a, s);
    default: return cudaErrorInvalidValue;
  }
}

static int bwd_rows_per_tile(const DevGeom& g) {
  // radial rows a tile's footprints can touch: the projection of the tile's pixel centres spans
  // (TX - 1)|c| + (TY - 1)|s| pixels and a footprint |c| + |s| more, at most sqrt(TX^2 + TY^2);
  // the kernel's rounding (ceil - 1 .. floor + 1) adds three rows, one more is margin
  const float diag = kBwdTileX == kBwdTileY ? kBwdTileX * 1.4143f
                                            : sqrtf((float)(kBwdTileX * kBwdTileX + kBwdTileY * kBwdTileY)) * 1.0001f;
  return (int)floorf(diag * g.inv_drp) + 4;
}

template <int NT, int ZK, int MODE, bool MASHED>
static cudaError_t bwd_launch(const DevGeom& g, int subset, const BwdArgs& a, cudaStream_t s) {
  // at most floor(sqrt(2) vx / d_radial) + 2 bins of one view cross a pixel
  const int max_pairs = (int)floorf(1.4143f * g.inv_drp) + 2;
  // components per batch and items per warp and batch (two per lane at most)
  const int cpb = std::min(g.n_comp, kBwdMaxItems / max_pairs);
  const int bcap = max_pairs * cpb;
  if (g.nr_max > 32 || cpb < 1 || bcap > kBwdMaxItems) return cudaErrorInvalidValue;
  const int nr_tile = bwd_rows_per_tile(g);
  const int p_pad = g.P + 2 * (NT - 1) * g.n_seg;  // each segment framed by NT-1 zeros
  const size_t sw_floats = ((size_t)nr_tile * p_pad + 3) & ~(size_t)3;
  const size_t smem = sw_floats * sizeof(float) + (size_t)kBwdWarps * bcap * (sizeof(float4) + sizeof(int4)) +
                      (size_t)kBwdWarps * g.nr_max * sizeof(PixItem);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  // the table holds one batch of items: mashed geometries with more components run without it
  const bool tab = a.items && MODE == BWD_UPDATE && NT <= 3 && cpb == g.n_comp;
  if (a.items && (MODE != BWD_UPDATE || NT > 3)) return cudaErrorInvalidValue;
  const int tiles_x = (g.nx + kBwdTileX - 1) / kBwdTileX, tiles_y = (g.ny + kBwdTileY - 1) / kBwdTileY;
  auto kern = tab ? k_backward<NT, ZK, MODE, MASHED, (MODE == BWD_UPDATE && NT <= 3)>
                  : k_backward<NT, ZK, MODE, MASHED, false>;
  {
    cudaError_t e = allow_dynamic_smem(kern, smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid(tiles_x, tiles_y);
  kern<<<grid, kBwdWarps * 32, smem, s>>>(g, subset, nr_tile, p_pad, bcap, cpb, a);
  return cudaGetLastError();
}

template <int NT, int MODE, bool MASHED>
static cudaError_t bwd_zk(const DevGeom& g, int subset, const BwdArgs& a, cudaStream_t s) {
  const int zk = (g.nz + 31) / 32;
  if (zk <= 1) return bwd_launch<NT, 1, MODE, MASHED>(g, subset, a, s);
  if (zk <= 2) return bwd_launch<NT, 2, MODE, MASHED>(g, subset, a, s);
  if (zk <= 4) return bwd_launch<NT, 4, MODE, MASHED>(g, subset, a, s);
  if (zk <= 8) return bwd_launch<NT, 8, MODE, MASHED>(g, subset, a, s);
  return cudaErrorInvalidValue;
}

template <int NT, int MODE>
static cudaError_t bwd_mashed(const DevGeom& g, int subset, const BwdArgs& a, cudaStream_t s) {
  return g.mashed ? bwd_zk<NT, MODE, true>(g, subset, a, s) : bwd_zk<NT, MODE, false>(g, subset, a, s);
}

template <int MODE>
static cudaError_t bwd_nt(const DevGeom& g, int subset, const BwdArgs& a, cudaStream_t s) {
  switch (g.taps) {
    case 1: return bwd_mashed<1, MODE>(g, subset, a, s);
    case 2: return bwd_mashed<2, MODE>(g, subset, a, s);
    case 3: return bwd_mashed<3, MODE>(g, subset, a, s);
    case 4: return bwd_mashed<4, MODE>(g, subset, a, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_backward(const DevGeom& g, int subset, int mode, const BwdArgs& a, cudaStream_t s) {
  switch (mode) {
    case BWD_OUT: return bwd_nt<BWD_OUT>(g, subset, a, s);
    case BWD_SENS: return bwd_nt<BWD_SENS>(g, subset, a, s);
    case BWD_UPDATE: return bwd_nt<BWD_UPDATE>(g, subset, a, s);
    case BWD_EM: return bwd_nt<BWD_EM>(g, subset, a, s);
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
