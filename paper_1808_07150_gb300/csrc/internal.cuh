// Internal declarations shared by the CUDA translation units of libspdhg.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/spdhg.h"

namespace spdhg {

constexpr int kMaxSeg = 32;       // segments held in the per-line shared tables
constexpr int kMaxTaps = 4;       // slices an oblique LOR may cross inside one transaxial pixel

// Per-segment constants.  Plane q of segment g has its LOR mid-point at slab coordinate
// f + q (in units of vz measured from the lower image face, so slab iz is [iz, iz+1)); f is
// held as a double-float pair f_hi + f_lo.
struct SegDev {
  int p0;      // first plane index of the segment in the sinogram
  int n;       // planes in the segment
  float f_hi, f_lo;
  int c0, nc;  // the segment's LOR components: c0 .. c0 + nc - 1
};

// One LOR component of a segment's bins (exact mashing; without mashing every segment has one
// component that every plane includes).  Plane q of the segment includes it when
// qlo <= q < qhi and ((q - qlo) & smask) == 0 (step 1: smask 0, step 2: smask 1).
struct CompDev {
  int seg;
  int qlo, qhi, smask;
  int jlo, jhi;  // range of the tap offset j0 of any pixel of any LOR of the component (host bound)
};

// Geometry passed by value to every kernel.  Transaxial quantities are in pixel units (mm / vx);
// every table entry that enters a length is a double-float pair (hi + lo) so that the position of
// a LOR relative to a pixel is resolved far below FP32 rounding of the absolute coordinates.
struct DevGeom {
  int nx, ny, nz;
  int R, V, P, m;        // radial bins, views, planes, subsets
  int bins;              // 1: bin-interleaved subsets (every subset spans all views), 0: view subsets
  int n_seg;
  int n_comp;            // LOR components (= n_seg without mashing)
  int mashed;            // 1: some bin sums several LORs or some plane lacks a component
  int taps;              // maximum slices a LOR crosses inside one pixel
  int nr_max;            // maximum candidate radial bins per pixel and view
  float half_R;          // (R - 1) / 2
  float inv_drp;         // vx / d_radial: radial bins per pixel unit
  const float4* view;    // per view: cos_hi, cos_lo, sin_hi, sin_lo (exact zeros on the axes)
  const float2* view_inv;  // per view: 1 / (-sin_hi), 1 / cos_hi (0 where the component is 0)
  const float4* rad;     // per radial bin: s_hi, s_lo, h_hi, h_lo (s = signed offset, h = half chord)
  const float4* rs;      // per (radial bin, component): kappa_hi, kappa_lo, len_scale, 0
  const SegDev* seg;
  const CompDev* comp;
  const int* stage_pos;  // plane -> its slot in the backprojector's staged rows (frames included)
  int n_runs;            // plane runs of the forward projector: run k = planes [q0, q0 + 32) of one segment
  const int2* runs;      // (segment, q0) per run, segment-major
  int max_part_comps[17];  // forward: most components one block spans, by warps per block
  int fz_lo;             // forward staging: zero slabs below each staged x column
  int fz_stride;         // forward staging: floats per staged x column (frames included)
  int tune[SPDHG_TUNE_KNOBS];  // launch-shape overrides (0: built-in heuristic)
};

// Lets `kern` take more than 48 KB of dynamic shared memory.  The attribute belongs to the
// function, not to a launch, so it is raised once per device to the largest value the function
// admits (the opt-in maximum less its static shared memory) instead of to this launch's size:
// launches and captured graph nodes of contexts with different sizes then never invalidate one
// another.  Occupancy still follows each launch's own size.
cudaError_t allow_dynamic_smem_fn(const void* kern, size_t smem);
template <class K>
cudaError_t allow_dynamic_smem(K kern, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return allow_dynamic_smem_fn(reinterpret_cast<const void*>(kern), smem);
}

// Proximal map of the non-negativity constraint, max(v, 0) (Sec. 2.2, the Example after the prox
// definition), written so that a
// NaN stays NaN: fmaxf(NaN, 0) would return 0 and hide a state that has stopped being finite
// from the objective check that reports divergence.
__host__ __device__ __forceinline__ float prox_nonneg(float v) { return v < 0.f ? 0.f : v; }

// Views a subset's projection traverses: i, i+m, ... for view subsets; every view for bin
// subsets and for subset < 0 (all bins).
__host__ __device__ inline int subset_views(const DevGeom& g, int subset) {
  return (subset < 0 || g.bins) ? g.V : (g.V - subset + g.m - 1) / g.m;
}
__host__ __device__ inline int subset_view(const DevGeom& g, int subset, int l) {
  return (subset < 0 || g.bins) ? l : subset + l * g.m;
}
// Whether bin j (flattened sinogram index) belongs to `subset` (always for view subsets, whose
// traversal already visits only their views, and for subset < 0).
__host__ __device__ inline bool bin_in_subset(const DevGeom& g, int subset, size_t j) {
  return subset < 0 || !g.bins || (int)(j % (size_t)g.m) == subset;
}

struct Ctx;

// ---------------------------------------------------------------------------------------
// projector launches (projector.cu)
// ---------------------------------------------------------------------------------------
enum FwdMode { FWD_PROJECT = 0, FWD_SIGMA = 1, FWD_DATA = 2, FWD_EM = 3 };
enum BwdMode { BWD_OUT = 0, BWD_SENS = 1, BWD_UPDATE = 2, BWD_EM = 3 };

struct FwdArgs {
  const float* x;        // image
  float* out;            // FWD_PROJECT: y (full sinogram); FWD_SIGMA: sigma (full sinogram)
  const float* mult;     // may be null (ones)
  // FWD_DATA
  const float* b;
  const float* r;
  float* y;              // dual, full sinogram
  float* wdy;            // subset-local mult * (y+ - y); FWD_EM: mult * b / (P x + r)
  const float* sigma;    // FWD_DATA: per-bin dual step sigma_j (full sinogram)
  float gamma_rho;       // gamma * rho
  // row-split scratch: partial plane sums [line][part][P] and one ticket per line (zeroed)
  float* part_acc;
  unsigned* tickets;
  size_t part_cap;       // floats in each partial buffer
  size_t ticket_cap;     // tickets (one per line and plane part)
};
// row parts per LOR line the forward projector uses for `subset` (1: no scratch needed)
int forward_split(const DevGeom& g, int subset);
// plane parts per LOR line (blocks that share the rows of a line, each with its own planes)
int forward_parts(const DevGeom& g);
int forward_entry_groups(const DevGeom& g);

struct BwdArgs {
  const float* w;        // subset-local sinogram (mult already applied)
  float* out;            // BWD_OUT: image (overwritten)
  float* T;              // BWD_SENS: running min; BWD_UPDATE: step image; BWD_EM: sensitivity P_i^T 1
  float sens_num;        // BWD_SENS: rho p_i / gamma
  float* x;              // BWD_UPDATE, BWD_EM
  float* z;
  float inv_p;
  // BWD_UPDATE: the tap items of every (view, tile, column), built once (null: computed in the
  // kernel); see backward_table_count / _fill
  const float4* items;
  const int2* hdr;
};

// Tap-item table of the backprojector: for every view, 4 x 4 tile and column the (pair, segment)
// items the kernel would compute, in its order.  Items are float4 (L0, L1, L2, packed): packed =
// shared offset (16 bits) | (j0 + taps - 1 + 256) << 16 (9 bits) | segment << 25 (7 bits).  Header
// per column: (first item, n1 | (n1 + n2) << 8 | n << 16) with n_k the items of k taps.
// Pass 0 counts the items per column into `cnt` (bytes) and flags an item that does not fit the
// packing in *bad; pass 1 fills the items and headers from the per-column starts.
cudaError_t backward_table_count(const DevGeom& g, unsigned char* cnt, unsigned* bad, cudaStream_t s);
cudaError_t backward_table_starts(const DevGeom& g, const unsigned char* cnt, unsigned* starts,
                                  unsigned* view_totals, cudaStream_t s);
cudaError_t backward_table_fill(const DevGeom& g, const unsigned* starts, const unsigned* view_base,
                                float4* items, int2* hdr, cudaStream_t s);
// whether the geometry admits the table (unmashed, at most 3 taps, packing limits)
bool backward_table_possible(const DevGeom& g);

cudaError_t launch_forward(const DevGeom& g, int subset, int mode, const FwdArgs& a, cudaStream_t s);
cudaError_t launch_backward(const DevGeom& g, int subset, int mode, const BwdArgs& a, cudaStream_t s);
// w_local = y * mult over the bins of subset i (y or mult null: ones); for bin subsets the
// buffer spans the whole sinogram and the other subsets' bins are 0
cudaError_t launch_gather_subset(const DevGeom& g, int subset, const float* y, const float* mult,
                                 float* w_local, cudaStream_t s);

// ---------------------------------------------------------------------------------------
// prior (prior.cu)
// ---------------------------------------------------------------------------------------
struct PriorArgs {
  int kind;              // SPDHG_PRIOR_TV / DTV / ATV
  const float* x_in;
  float* x_out;
  const float* q_in;     // 3N
  float* q_out;
  float* z;
  const float* T;
  const float* side;     // dTV side image v
  float sigma, alpha, inv_p, gamma_d, eta2;
};
cudaError_t launch_prior(const DevGeom& g, const PriorArgs& a, cudaStream_t s);
// whether the prior kernel's launch-shape knobs fit together (voxels per thread, columns, rows)
bool prior_launch_ok(const DevGeom& g, int kind);

struct TgvArgs {
  int block;             // 0: A = (grad, -I), 1: A = (0, E)
  const float* u_in; float* u_out;
  const float* w_in; float* w_out;      // 3N each
  const float* q_in; float* q_out;      // 3N (block 0) or 6N (block 1)
  float* zu; float* zw;
  const float* Tu; float Tw;
  float sigma, alpha, inv_p;
  float* bscr;                          // scratch: the dual change b (3N or 6N)
};
// the block's dual pass and primal pass (two kernels)
cudaError_t launch_tgv(const DevGeom& g, const TgvArgs& a, cudaStream_t s);
// data iteration for TGV also steps w: w -= Tw * zbar_w with zbar_w = zw (no new w-dual change)
cudaError_t launch_w_step(const DevGeom& g, float* w, const float* zw, float Tw, cudaStream_t s);

// ---------------------------------------------------------------------------------------
// objective (objective.cu)
// ---------------------------------------------------------------------------------------
cudaError_t launch_data_term(const float* ax, const float* b, const float* r, int64_t M,
                             double* partial, int nblocks, double* out, cudaStream_t s);
cudaError_t launch_prior_term(const DevGeom& g, int kind, const float* x, const float* w,
                              const float* side, float gamma_d, float eta2, double* partial,
                              int nblocks, double* out, cudaStream_t s);
cudaError_t launch_side_max_grad(const DevGeom& g, const float* side, double* partial, int nblocks,
                                 double* out, cudaStream_t s);
// *out = sum_j v_j^2 (FP64, deterministic);  v = y / sqrt(*ss)
cudaError_t launch_sumsq(const float* v, int64_t n, double* partial, int nblocks, double* out, cudaStream_t s);
cudaError_t launch_normalize(const float* y, int64_t n, const double* ss, float* v, cudaStream_t s);
// out[0] = sum (x - xs)^2, out[1] = max |xs| (FP64); `partial` holds 2 * nblocks doubles
cudaError_t launch_psnr_terms(const float* x, const float* xs, int64_t n, double* partial, int nblocks,
                              double* out, cudaStream_t s);

// ---------------------------------------------------------------------------------------
// iteration driver (api.cu) and epoch graphs (graph.cu)
// ---------------------------------------------------------------------------------------
// enqueues the kernels of one SPDHG iteration on block i and advances the ping-pong parities
int enqueue_block(spdhg_ctx* ctx, int i, cudaStream_t s);
// row-split scratch of the forward projector for `subset` into a (allocated on first need)
int forward_scratch(spdhg_ctx* ctx, int subset, FwdArgs& a, cudaStream_t s);
// allocates the forward row-split scratch for the full projection and every subset
int prepare_all_forward(spdhg_ctx* ctx, cudaStream_t s);
struct GraphCache;
void graph_cache_free(spdhg_ctx* ctx);

// Quality log and stopping rule shared by spdhg_run and spdhg_run_batch: the relative objective
// (Psi(x^k) - Psi*) / (Psi(0) - Psi*) and PSNR(x^k, x*) of Sec. 4, evaluated in FP64 on the GPU.
struct RunLog {
  int every = 0;         // evaluate after every `every` epochs (0: never)
  double psi0 = 0.0;     // Psi(0), when a target gap is set
  double ms = 0.0;       // solver device time so far
  bool stopped = false;  // the target gap was reached
};
// after spdhg_setup: fills the report's defaults and evaluates the start (index 0)
int runlog_begin(spdhg_ctx* ctx, const spdhg_params& p, spdhg_report* rep, RunLog& L, cudaStream_t s);
// after epoch e (1-based) that took epoch_ms of device time
int runlog_epoch(spdhg_ctx* ctx, const spdhg_params& p, spdhg_report* rep, RunLog& L, int e, double epoch_ms,
                 cudaStream_t s);

// device allocations of a context, charged to its memory limit (cudaErrorMemoryAllocation past it)
cudaError_t ctx_malloc(spdhg_ctx* ctx, void** p, size_t bytes);
void ctx_free(spdhg_ctx* ctx, void* p);

}  // namespace spdhg

// The opaque context of the C ABI.
struct spdhg_ctx {
  spdhg_geometry geom{};
  std::vector<int> seg_n;
  std::vector<double> seg_zmid0, seg_dzmid, seg_dz;
  std::vector<int> comp_seg, comp_qlo, comp_qhi, comp_step;
  std::vector<double> comp_dz;
  spdhg::DevGeom dg{};
  int64_t N = 0, M = 0, max_subset_bins = 0;
  int device = 0;
  // device tables
  float4* d_view = nullptr;
  float4* d_rad = nullptr;
  float4* d_rs = nullptr;
  int2* d_runs = nullptr;
  float2* d_view_inv = nullptr;
  spdhg::SegDev* d_seg = nullptr;
  spdhg::CompDev* d_comp = nullptr;
  int* d_stage_pos = nullptr;
  // data
  float *b = nullptr, *r = nullptr, *mult = nullptr, *side = nullptr;
  bool has_data = false, has_mult = false, has_side = false;
  // state
  float* x[2] = {nullptr, nullptr};
  int xcur = 0;
  float *z = nullptr, *T = nullptr, *y = nullptr, *wdy = nullptr;
  float* sigma = nullptr;      // per-bin dual step sigma_j, computed by spdhg_setup
  float* q[2] = {nullptr, nullptr};
  int qcur = 0;
  // TGV
  float* w[2] = {nullptr, nullptr};
  int wcur = 0;
  float* zw = nullptr;
  float* q2[2] = {nullptr, nullptr};
  float* tgv_b = nullptr;      // TGV dual change of the current prior block (6N)
  int q2cur = 0;
  float Tw = 0.f;
  // scratch
  float* tmp_sino = nullptr;   // M floats (objective, sigma export)
  float* tmp_img = nullptr;    // N floats (objective of a host image, Psi(0), x* of spdhg_psnr)
  float* tmp_img2 = nullptr;   // N floats (x of spdhg_psnr from the host)
  float* em_sens = nullptr;    // OSEM / MLEM sensitivity images P_i^T 1 (m x N, or N for MLEM)
  float4* bwd_items = nullptr; // backprojector tap-item table (see backward_table_count / _fill)
  int2* bwd_hdr = nullptr;
  int bwd_table = -1;          // -1 not tried, 0 not built (does not fit / not possible), 1 built
  int em_sens_kind = -1;       // which set em_sens holds: 0 OSEM, 1 MLEM, -1 none (reset by set_data)
  float* fwd_part = nullptr;   // forward row-split partial sums (2 x fwd_part_cap floats)
  unsigned* fwd_tickets = nullptr;
  size_t fwd_part_cap = 0, fwd_ticket_cap = 0;
  double* red = nullptr;       // FP64 partial sums
  double* red_out = nullptr;   // FP64 results (4)
  int red_blocks = 1024;
  // parameters of the last setup
  bool is_setup = false;
  spdhg_params params{};
  std::vector<double> probs;
  std::vector<float> sigma_prior;
  double eta2 = 0.0;
  int64_t iterations = 0;
  std::string err;
  // per-launch profiler
  bool profiling = false;
  struct ProfRec { int kind; cudaEvent_t a, b; };
  std::vector<ProfRec> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[SPDHG_KERNEL_KINDS] = {0, 0, 0, 0, 0};
  int64_t prof_n[SPDHG_KERNEL_KINDS] = {0, 0, 0, 0, 0};
  // captured iteration templates of the epoch graphs; graph_gen changes whenever an argument
  // the kernels receive (parameters, buffers, launch shapes) may have changed
  spdhg::GraphCache* gcache = nullptr;
  uint64_t graph_gen = 0;
  std::vector<double> graph_sig;
  // device memory the context holds, and its limit (0: none)
  size_t mem_used = 0, mem_limit = 0;
  std::unordered_map<void*, size_t> mem_size;
};
