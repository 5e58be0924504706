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

// Forward projection.  A block owns the rows [row_lo, row_hi) of one transaxial LOR line
// (view, radial bin) and all its planes.  All threads first find the pixels the line crosses in
// those rows (exact intervals, compacted); the entries are then processed in chunks of
// kFwdChunk: the x columns of chunk c+1 are copied to shared memory (cp.async, with NT-1 zeros
// on each side so that taps leaving the image read zeros) and its axial taps computed while
// chunk c is accumulated, one thread per plane.  When several blocks share a line, each writes
// partial plane sums and the last one to finish reduces them in a fixed order.
template <int NT, int PPT, int MODE>
__global__ void __launch_bounds__(512) k_forward(DevGeom g, int subset, int ecap, int split, int xs_stride,
                                                 FwdArgs a, float* part_acc, float* part_chord,
                                                 unsigned* tickets) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int scan_scratch[33];
  constexpr int PAD = NT - 1;
  float* xs = reinterpret_cast<float*>(smem);                             // [2][kFwdChunk][xs_stride]
  float4* tapL = reinterpret_cast<float4*>(xs + 2 * kFwdChunk * xs_stride);  // [2][n_seg][kFwdChunk]
  int4* tapM = reinterpret_cast<int4*>(tapL + 2 * g.n_seg * kFwdChunk);      // [2][n_seg][kFwdChunk]
  Entry* ent = reinterpret_cast<Entry*>(tapM + 2 * g.n_seg * kFwdChunk);     // [ecap]
  const int nz = g.nz;

  const int line = blockIdx.x / split, part = blockIdx.x - line * split;
  const int l = line / g.R, r = line - (line / g.R) * g.R;
  const int v = subset_view(g, subset, l);
  const Line L = make_line(g, v, r);

  // planes of this thread: lane of warp-sized runs of one segment (run = PPT * warp + k, so the
  // runs of a warp are neighbours in the run table and usually share their segment)
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  int pseg[PPT], pq[PPT], pp[PPT];
  bool pvalid[PPT];
  float acc[PPT], chord[PPT];
#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    const int run = wi * PPT + k;
    acc[k] = 0.f;
    chord[k] = 0.f;
    pseg[k] = -1;
    pq[k] = 0;
    pp[k] = 0;
    pvalid[k] = false;
    if (run < g.n_runs) {
      const int2 ru = g.runs[run];
      const SegDev sd = g.seg[ru.x];
      pseg[k] = ru.x;
      pq[k] = ru.y + lane;
      pp[k] = sd.p0 + pq[k];
      pvalid[k] = pq[k] < sd.n;
    }
  }
  // zero pads of the staged columns (never overwritten by the copies)
  if constexpr (PAD > 0) {
    for (int i = threadIdx.x; i < 2 * kFwdChunk * 2 * PAD; i += blockDim.x) {
      const int col = i / (2 * PAD), k = i - col * (2 * PAD);
      xs[col * xs_stride + (k < PAD ? k : nz + k)] = 0.f;
    }
  }
  const bool ydom = fabsf(L.c_hi) >= fabsf(L.s_hi);  // |dy| >= |dx|: walk the rows of y
  const int nrows_all = ydom ? g.ny : g.nx;
  const int rows_per_part = (nrows_all + split - 1) / split;
  const int row_lo = part * rows_per_part, row_hi = min(nrows_all, row_lo + rows_per_part);

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

  auto stage = [&](int c) {  // x columns + taps of chunk c into buffer c & 1
    const int buf = c & 1;
    const int e0 = c * kFwdChunk, ne = min(kFwdChunk, n_ent - e0);
    float* xb = xs + buf * kFwdChunk * xs_stride;
    // one warp per entry, lanes along z: no division or entry lookup per staged value
    const int nw = blockDim.x >> 5;
    for (int e = wi; e < ne; e += nw) {
      const float* src = a.x + (size_t)ent[e0 + e].col * nz;
      float* dst = xb + e * xs_stride + PAD;
      for (int iz = lane; iz < nz; iz += 32) cp_async4(dst + iz, src + iz);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    float4* tl = tapL + buf * g.n_seg * kFwdChunk;
    int4* tm = tapM + buf * g.n_seg * kFwdChunk;
    for (int it = threadIdx.x; it < g.n_seg * ne; it += blockDim.x) {
      const int gs = it / ne, e = it - gs * ne;
      float Lk[4] = {0.f, 0.f, 0.f, 0.f};
      const int j0 = segment_taps<NT>(g, r, gs, ent[e0 + e].I, Lk);
      int nt = NT;
      while (nt > 1 && Lk[nt - 1] == 0.f) --nt;
      const int slot = gs * kFwdChunk + e;
      tl[slot] = make_float4(Lk[0], Lk[1], Lk[2], Lk[3]);
      // plane q, tap t reads xs[e * stride + PAD + q - j0 - t]; useful while 0 <= q - j0 < nz + PAD
      tm[slot] = make_int4(e * xs_stride + PAD - j0, j0, nt, 0);
    }
  };

  const int nchunks = (n_ent + kFwdChunk - 1) / kFwdChunk;
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
    const int ne = min(kFwdChunk, n_ent - c * kFwdChunk);
    const float* xb = xs + buf * kFwdChunk * xs_stride;
    const float4* tl = tapL + buf * g.n_seg * kFwdChunk;
    const int4* tm = tapM + buf * g.n_seg * kFwdChunk;
    // all runs of this warp in one segment (warp-uniform): one load of each entry's taps serves them
    bool same = pseg[0] >= 0;
#pragma unroll
    for (int k = 1; k < PPT; ++k) same = same && (pseg[k] < 0 || pseg[k] == pseg[0]);
    if (MODE != FWD_SIGMA && PPT > 1 && same) {
      const float4* tlk = tl + pseg[0] * kFwdChunk;
      const int4* tmk = tm + pseg[0] * kFwdChunk;
      float sum[PPT];
#pragma unroll
      for (int k = 0; k < PPT; ++k) sum[k] = 0.f;
      for (int e = 0; e < ne; ++e) {
        const int4 M = tmk[e];
        const float4 Lv = tlk[e];
        const float* xe = xb + M.x;
        if (NT == 1 || M.z == 1) {  // tap count is uniform across the warp
#pragma unroll
          for (int k = 0; k < PPT; ++k)
            if (pseg[k] >= 0 && (unsigned)(pq[k] - M.y) < (unsigned)(nz + PAD)) sum[k] = fmaf(Lv.x, xe[pq[k]], sum[k]);
        } else if (NT == 2 || M.z == 2) {
#pragma unroll
          for (int k = 0; k < PPT; ++k)
            if (pseg[k] >= 0 && (unsigned)(pq[k] - M.y) < (unsigned)(nz + PAD)) {
              const float* xp = xe + pq[k];
              sum[k] = fmaf(Lv.y, xp[-1], fmaf(Lv.x, xp[0], sum[k]));
            }
        } else if (NT == 3 || M.z == 3) {
#pragma unroll
          for (int k = 0; k < PPT; ++k)
            if (pseg[k] >= 0 && (unsigned)(pq[k] - M.y) < (unsigned)(nz + PAD)) {
              const float* xp = xe + pq[k];
              sum[k] = fmaf(Lv.z, xp[-2], fmaf(Lv.y, xp[-1], fmaf(Lv.x, xp[0], sum[k])));
            }
        } else {
#pragma unroll
          for (int k = 0; k < PPT; ++k)
            if (pseg[k] >= 0 && (unsigned)(pq[k] - M.y) < (unsigned)(nz + PAD)) {
              const float* xp = xe + pq[k];
              sum[k] = fmaf(Lv.w, xp[-3], fmaf(Lv.z, xp[-2], fmaf(Lv.y, xp[-1], fmaf(Lv.x, xp[0], sum[k]))));
            }
        }
      }
#pragma unroll
      for (int k = 0; k < PPT; ++k) acc[k] += sum[k];
    }
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      if (MODE != FWD_SIGMA && PPT > 1 && same) break;  // done above
      if (pseg[k] < 0) break;  // warp-uniform: no more runs for this warp
      const float4* tlk = tl + pseg[k] * kFwdChunk;
      const int4* tmk = tm + pseg[k] * kFwdChunk;
      const int q = pq[k];
      float sum = 0.f;
      for (int e = 0; e < ne; ++e) {
        const int4 M = tmk[e];     // warp broadcast: one segment per warp
        const float4 Lv = tlk[e];
        const int d = q - M.y;
        const bool in = (unsigned)d < (unsigned)(nz + PAD);
        const float* xp = xb + M.x + q;  // taps t read xp[-t], inside the zero-padded column
        if (MODE == FWD_SIGMA) {  // chord of the LOR inside the image: taps whose slab exists
          if (in)
            chord[k] += (d < nz ? Lv.x : 0.f) + (NT > 1 && d >= 1 && d - 1 < nz ? Lv.y : 0.f) +
                        (NT > 2 && d >= 2 && d - 2 < nz ? Lv.z : 0.f) + (NT > 3 && d >= 3 && d - 3 < nz ? Lv.w : 0.f);
        } else if (NT == 1 || M.z == 1) {  // tap count is uniform across the warp
          if (in) sum = fmaf(Lv.x, xp[0], sum);
        } else if (NT == 2 || M.z == 2) {
          if (in) sum = fmaf(Lv.y, xp[-1], fmaf(Lv.x, xp[0], sum));
        } else if (NT == 3 || M.z == 3) {
          if (in) sum = fmaf(Lv.z, xp[-2], fmaf(Lv.y, xp[-1], fmaf(Lv.x, xp[0], sum)));
        } else {
          if (in) sum = fmaf(Lv.w, xp[-3], fmaf(Lv.z, xp[-2], fmaf(Lv.y, xp[-1], fmaf(Lv.x, xp[0], sum))));
        }
      }
      acc[k] += sum;
    }
    __syncthreads();
  }

  if (split > 1) {
    // publish this block's partial sums; the last block of the line reduces them
    __shared__ unsigned last_sh;
    const size_t pbase = ((size_t)line * split + part) * g.P;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      if (!pvalid[k]) continue;
      const int p = pp[k];
      part_acc[pbase + p] = acc[k];
      if (MODE == FWD_SIGMA) part_chord[pbase + p] = chord[k];
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) last_sh = (atomicAdd(tickets + line, 1u) == (unsigned)split - 1u) ? 1u : 0u;
    __syncthreads();
    if (!last_sh) return;
    __threadfence();
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
      if (!pvalid[k]) continue;
      const int p = pp[k];
      float sa = 0.f, sc = 0.f;
      for (int q = 0; q < split; ++q) {  // fixed order: deterministic
        const size_t o = ((size_t)line * split + q) * g.P + p;
        sa += __ldcg(part_acc + o);
        if (MODE == FWD_SIGMA) sc += __ldcg(part_chord + o);
      }
      acc[k] = sa;
      chord[k] = sc;
    }
    if (threadIdx.x == 0) tickets[line] = 0u;  // ready for the next launch
  }

#pragma unroll
  for (int k = 0; k < PPT; ++k) {
    if (!pvalid[k]) continue;
    const int p = pp[k];
    const size_t j = ((size_t)v * g.R + r) * g.P + p;
    const float mu = a.mult ? a.mult[j] : 1.f;
    if (MODE == FWD_PROJECT) {
      a.out[j] = mu * acc[k];
    } else if (MODE == FWD_SIGMA) {
      // sigma_j = gamma rho / (P_i 1)_j,  (P_i 1)_j = mult_j * chord_j  (Eq. EQU:STEPSIZE:PRECOND)
      const float a1 = mu * chord[k];
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
      a.wdy[((size_t)l * g.R + r) * g.P + p] = mu * (yn - yj);
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

constexpr int kBwdTile = 4;              // block = kBwdTile x kBwdTile voxel columns, one warp each
constexpr int kBwdWarps = kBwdTile * kBwdTile;
constexpr int kBwdMaxItems = 64;         // (pair, segment) items per column and view

// Backprojection.  A block owns a 4 x 4 tile of voxel columns; for each view of the subset it
// stages the contiguous radial rows w[view][r_min..r_max][0..P) that the tile's footprints
// touch into shared memory (cp.async, overlapped with the geometry below), each segment's plane
// run framed by NT-1 zeros so that taps leaving the segment read zeros.  Each warp owns one
// column: its lanes find the footprint (bin, pixel interval) pairs, compact them with a ballot,
// compute the axial taps of every (pair, segment) item, and then gather along contiguous plane
// runs from shared memory, lane = iz mod 32, ZK voxels per lane.  Up to 128 slices (ZK <= 4) four
// blocks share an SM (32 registers per thread); with eight accumulators per lane, three.
template <int NT, int ZK, int MODE>
__global__ void __launch_bounds__(kBwdWarps * 32, ZK <= 4 ? 4 : 3) k_backward(DevGeom g, int subset, int nr_tile, int p_pad,
                                                             int bcap, BwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  constexpr int PAD = NT - 1;
  const int icap = bcap;  // items per warp (all buckets)
  float* sw = reinterpret_cast<float*>(smem);                                  // nr_tile x p_pad
  float4* itL = reinterpret_cast<float4*>(sw + ((nr_tile * p_pad + 3) & ~3));  // [warp][icap]
  int4* itM = reinterpret_cast<int4*>(itL + kBwdWarps * icap);
  PixItem* pix = reinterpret_cast<PixItem*>(itM + kBwdWarps * icap);          // [warp][nr_max]
  int* seg_of = reinterpret_cast<int*>(pix + kBwdWarps * g.nr_max);           // [P]: padded position
  const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
  const int tx0 = blockIdx.x * kBwdTile, ty0 = blockIdx.y * kBwdTile;
  const int ix = tx0 + (wi % kBwdTile), iy = ty0 + (wi / kBwdTile);
  const bool live = ix < g.nx && iy < g.ny;
  const float Xc = (float)ix + 0.5f - 0.5f * (float)g.nx;
  const float Yc = (float)iy + 0.5f - 0.5f * (float)g.ny;
  const float X0 = (float)tx0 + 0.5f - 0.5f * (float)g.nx, Y0 = (float)ty0 + 0.5f - 0.5f * (float)g.ny;
  const float X1 = X0 + (float)(kBwdTile - 1), Y1 = Y0 + (float)(kBwdTile - 1);
  float4* myL = itL + wi * icap;
  int4* myM = itM + wi * icap;
  PixItem* mypix = pix + wi * g.nr_max;
  const int nviews = subset_views(g, subset);
  const int nz = g.nz;
  float acc[ZK];
#pragma unroll
  for (int k = 0; k < ZK; ++k) acc[k] = 0.f;
  // padded position of every plane, and the zero frames of the staged rows (written once)
  for (int p = threadIdx.x; p < g.P; p += blockDim.x) seg_of[p] = p + (2 * g.plane_seg[p] + 1) * PAD;
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
    // radial rows of the whole tile (footprints of its extreme pixel centres)
    const float s00 = X0 * cs.x + Y0 * cs.z, s01 = X0 * cs.x + Y1 * cs.z;
    const float s10 = X1 * cs.x + Y0 * cs.z, s11 = X1 * cs.x + Y1 * cs.z;
    const float smin = fminf(fminf(s00, s01), fminf(s10, s11)), smax = fmaxf(fmaxf(s00, s01), fmaxf(s10, s11));
    const int r_min = max(0, (int)ceilf((smin - hw) * g.inv_drp + g.half_R) - 1);
    const int r_max = min(g.R - 1, min(r_min + nr_tile - 1, (int)floorf((smax + hw) * g.inv_drp + g.half_R) + 1));
    // 1. stage rows r_min..r_max of this view into their padded slots
    {
      const float* src = a.w + ((size_t)l * g.R + r_min) * g.P;
      const int nr = r_max - r_min + 1;
      for (int p = threadIdx.x; p < g.P; p += blockDim.x) {
        const int dst = seg_of[p];
        for (int rr = 0; rr < nr; ++rr) cp_async4(sw + rr * p_pad + dst, src + rr * g.P + p);
      }
    }
    // 2. footprint pairs of this warp's column (overlaps the copy)
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
        P.l = l;
        P.r = r;
      }
    }
    const unsigned mask = __ballot_sync(0xffffffffu, ok);
    if (ok) mypix[__popc(mask & ((1u << lane) - 1u))] = P;
    const int np = __popc(mask);
    __syncwarp();
    // 3. axial taps per (pair, segment), ordered by tap count: a lane holds up to two items,
    //    ballots count each tap-count bucket, and the items are written bucket after bucket
    const int ni = min(np * g.n_seg, bcap);
    float4 Lv2[2];
    int4 Mv2[2];
    int nt2[2] = {0, 0};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int it = lane + 32 * h;
      Lv2[h] = make_float4(0.f, 0.f, 0.f, 0.f);
      Mv2[h] = make_int4(0, 0, 0, 0);
      if (it < ni) {
        const int pi = it / g.n_seg, gi = it - pi * g.n_seg;
        const PixItem Q = mypix[pi];
        float Lk[4] = {0.f, 0.f, 0.f, 0.f};
        const int j0 = segment_taps<NT>(g, Q.r, gi, Q.I, Lk);
        int nt = NT;
        while (nt > 1 && Lk[nt - 1] == 0.f) --nt;
        const SegDev sd = g.seg[gi];
        Lv2[h] = make_float4(Lk[0], Lk[1], Lk[2], Lk[3]);
        // voxel iz, tap t reads plane q = iz + j0 + t at sw[x + iz + t]; some tap is inside the
        // segment while -PAD <= iz + j0 < n, and the frame supplies zeros for the others
        Mv2[h] = make_int4((Q.r - r_min) * p_pad + sd.p0 + (2 * gi + 1) * PAD + j0, j0 + PAD, sd.n + PAD, nt);
        nt2[h] = nt;
      }
    }
    int bs[5] = {0, 0, 0, 0, 0};  // bucket b (items with b + 1 taps) spans [bs[b], bs[b + 1])
    {
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
    cp_async_commit_wait_all();
    __syncthreads();
    // 4. gather: one branch-free loop per tap count
    if (live) {
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
    __syncthreads();  // the staged rows are replaced by the next view's
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
    } else {
      // z = z + dz;  zbar = z + dz / p_i;  next primal step x = max(x - T zbar, 0)
      const float zn = a.z[idx] + acc[k];
      a.z[idx] = zn;
      a.x[idx] = fmaxf(a.x[idx] - a.T[idx] * fmaf(acc[k], a.inv_p, zn), 0.f);
    }
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

int forward_split(const DevGeom& g, int subset) {
  if (g.tune[SPDHG_TUNE_FWD_SPLIT]) return g.tune[SPDHG_TUNE_FWD_SPLIT];
  // enough blocks for every SM: one LOR line per block is too few for small subsets
  const int lines = subset_views(g, subset) * g.R;
  const int nrows = g.nx > g.ny ? g.nx : g.ny;
  int split = 1;
  while (split < 8 && lines * split < 152 && nrows / (split * 2) >= 32) split *= 2;
  return split;
}

template <int NT, int PPT, int MODE>
static cudaError_t fwd_launch(const DevGeom& g, int subset, const FwdArgs& a, cudaStream_t s, int threads, int split) {
  const int xs_stride = g.nz + 2 * (NT - 1);  // staged x column with zero pads
  const int nrows = g.nx > g.ny ? g.nx : g.ny;
  const int ecap = 3 * nrows + 8;  // a line crosses at most two pixels per row of its dominant axis
  const size_t smem = (size_t)2 * kFwdChunk * xs_stride * sizeof(float) +
                      (size_t)2 * g.n_seg * kFwdChunk * (sizeof(float4) + sizeof(int4)) + (size_t)ecap * sizeof(Entry);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  if (MODE == FWD_DATA && !a.sigma) return cudaErrorInvalidValue;
  {
    cudaError_t e = allow_dynamic_smem(k_forward<NT, PPT, MODE>, smem);
    if (e != cudaSuccess) return e;
  }
  const int lines = subset_views(g, subset) * g.R;
  if (lines == 0) return cudaSuccess;
  if (split > 1 && (!a.part_acc || !a.part_chord || !a.tickets || (size_t)lines * split * g.P > a.part_cap ||
                    (size_t)lines > a.ticket_cap))
    return cudaErrorInvalidValue;
  k_forward<NT, PPT, MODE><<<lines * split, threads, smem, s>>>(g, subset, ecap, split, xs_stride, a, a.part_acc,
                                                                a.part_chord, a.tickets);
  return cudaGetLastError();
}

template <int NT, int MODE>
static cudaError_t fwd_ppt(const DevGeom& g, int subset, const FwdArgs& a, cudaStream_t s) {
  const int split = forward_split(g, subset);
  const int nwarps = g.tune[SPDHG_TUNE_FWD_WARPS] ? g.tune[SPDHG_TUNE_FWD_WARPS]
                                                  : (g.n_runs < 16 ? (g.n_runs < 4 ? 4 : g.n_runs) : 16);
  const int ppt = (g.n_runs + nwarps - 1) / nwarps;                      // runs per warp
  const int threads = nwarps * 32;
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

static int bwd_rows_per_tile(const DevGeom& g) {
  // radial rows a tile's footprints can touch: the projection of the tile's pixel centres spans
  // (kBwdTile - 1)(|c| + |s|) pixels and a footprint |c| + |s| more, at most kBwdTile sqrt(2);
  // the kernel's rounding (ceil - 1 .. floor + 1) adds three rows, one more is margin
  return (int)floorf(kBwdTile * 1.4143f * g.inv_drp) + 4;
}

template <int NT, int ZK, int MODE>
static cudaError_t bwd_launch(const DevGeom& g, int subset, const BwdArgs& a, cudaStream_t s) {
  // at most floor(sqrt(2) vx / d_radial) + 2 bins of one view cross a pixel
  const int max_pairs = (int)floorf(1.4143f * g.inv_drp) + 2;
  // items per warp and view (two per lane at most)
  const int bcap = max_pairs * g.n_seg;
  if (g.nr_max > 32 || bcap > kBwdMaxItems) return cudaErrorInvalidValue;
  const int nr_tile = bwd_rows_per_tile(g);
  const int p_pad = g.P + 2 * (NT - 1) * g.n_seg;  // each segment framed by NT-1 zeros
  const size_t sw_floats = ((size_t)nr_tile * p_pad + 3) & ~(size_t)3;
  const size_t smem = sw_floats * sizeof(float) + (size_t)kBwdWarps * bcap * (sizeof(float4) + sizeof(int4)) +
                      (size_t)kBwdWarps * g.nr_max * sizeof(PixItem) + (size_t)g.P * sizeof(int);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  auto kern = k_backward<NT, ZK, MODE>;
  {
    cudaError_t e = allow_dynamic_smem(kern, smem);
    if (e != cudaSuccess) return e;
  }
  dim3 grid((g.nx + kBwdTile - 1) / kBwdTile, (g.ny + kBwdTile - 1) / kBwdTile);
  kern<<<grid, kBwdWarps * 32, smem, s>>>(g, subset, nr_tile, p_pad, bcap, a);
  return cudaGetLastError();
}

template <int NT, int MODE>
static cudaError_t bwd_zk(const DevGeom& g, int subset, const BwdArgs& a, cudaStream_t s) {
  const int zk = (g.nz + 31) / 32;
  if (zk <= 1) return bwd_launch<NT, 1, MODE>(g, subset, a, s);
  if (zk <= 2) return bwd_launch<NT, 2, MODE>(g, subset, a, s);
  if (zk <= 4) return bwd_launch<NT, 4, MODE>(g, subset, a, s);
  if (zk <= 8) return bwd_launch<NT, 8, MODE>(g, subset, a, s);
  return cudaErrorInvalidValue;
}

template <int MODE>
static cudaError_t bwd_nt(const DevGeom& g, int subset, const BwdArgs& a, cudaStream_t s) {
  switch (g.taps) {
    case 1: return bwd_zk<1, MODE>(g, subset, a, s);
    case 2: return bwd_zk<2, MODE>(g, subset, a, s);
    case 3: return bwd_zk<3, MODE>(g, subset, a, s);
    case 4: return bwd_zk<4, MODE>(g, subset, a, s);
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
