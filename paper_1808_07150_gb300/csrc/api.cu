// C ABI of libspdhg: context management, data upload, projector entry points, step-size
// setup, the SPDHG iteration driver, the sampler and the FP64 objective.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "internal.cuh"

using namespace spdhg;

// Device allocations of a context are charged to its memory limit (spdhg_set_memory_limit): one
// that would take the context past the limit fails as an out-of-memory error, as the driver's
// own would, and leaves the context usable.
cudaError_t spdhg::ctx_malloc(spdhg_ctx* ctx, void** p, size_t bytes) {
  if (ctx->mem_limit && ctx->mem_used + bytes > ctx->mem_limit) return cudaErrorMemoryAllocation;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) {
    ctx->mem_used += bytes;
    ctx->mem_size[*p] = bytes;
  }
  return e;
}

void spdhg::ctx_free(spdhg_ctx* ctx, void* p) {
  if (!p) return;
  auto it = ctx->mem_size.find(p);
  if (it != ctx->mem_size.end()) {
    ctx->mem_used -= it->second;
    ctx->mem_size.erase(it);
  }
  cudaFree(p);
}

namespace {

int fail(spdhg_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? SPDHG_ERR_OOM : SPDHG_ERR_CUDA,     \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                        \
  } while (0)

template <class T>
cudaError_t dalloc(spdhg_ctx* ctx, T** p, size_t n) {
  if (*p) return cudaSuccess;
  return ctx_malloc(ctx, (void**)p, n * sizeof(T) + 16);
}

__global__ void k_fill(float* p, int64_t n, float v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

// per-bin value of the bin's subset (bin subsets: bin j belongs to subset j mod m)
__global__ void k_fill_bins(float* p, int64_t n, int m, const float* per_subset) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = per_subset[i % m];
}

__global__ void k_clamp_copy(float* dst, const float* src, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = prox_nonneg(src[i]);
}

// T = min(T, t_prior); voxels that no block sees (+inf) get T = 0.
__global__ void k_finalize_T(float* T, int64_t n, float t_prior) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    float t = fminf(T[i], t_prior);
    T[i] = isinf(t) ? 0.f : t;
  }
}

// counts values that are non-finite or violate the bound (mode 0: >= 0, mode 1: > 0)
__global__ void k_validate(const float* p, int64_t n, int mode, unsigned long long* bad) {
  unsigned long long cnt = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float v = p[i];
    const bool ok = isfinite(v) && (mode == 0 ? v >= 0.f : v > 0.f);
    cnt += ok ? 0ull : 1ull;
  }
  if (cnt) atomicAdd(bad, cnt);
}

int grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 32));
}

uint64_t splitmix64(uint64_t seed, uint64_t k) {
  uint64_t z = seed + (k + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

double grad_norm(int nx, int ny, int nz) {
  // largest eigenvalue of the Neumann Laplacian of n points: 4 sin^2(pi (n-1) / (2n))
  const double pi = 3.14159265358979323846;
  double s = 0.0;
  for (int n : {nx, ny, nz}) s += 4.0 * pow(sin(pi * (n - 1) / (2.0 * n)), 2);
  return sqrt(s);
}

int n_prior_blocks(int prior) {
  switch (prior) {
    case SPDHG_PRIOR_NONE: return 0;
    case SPDHG_PRIOR_TGV: return 2;
    default: return 1;
  }
}

std::vector<double> block_probs(int m, int prior, int sampling) {
  const int nb = n_prior_blocks(prior);
  const int n = m + nb;
  std::vector<double> p(n);
  if (nb == 0 || sampling == SPDHG_SAMPLING_UNIFORM) {
    for (auto& v : p) v = 1.0 / n;
  } else {
    for (int i = 0; i < m; ++i) p[i] = 1.0 / (2.0 * m);
    for (int i = m; i < n; ++i) p[i] = 0.5 / nb;
  }
  return p;
}

int check_device(spdhg_ctx* ctx) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return fail(ctx, SPDHG_ERR_CUDA, "cudaGetDevice failed");
  if (dev != ctx->device) return fail(ctx, SPDHG_ERR_STATE, "current CUDA device differs from the context's device");
  return SPDHG_OK;
}

cudaEvent_t prof_event(spdhg_ctx* ctx) {
  if (!ctx->prof_pool.empty()) {
    cudaEvent_t e = ctx->prof_pool.back();
    ctx->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Records an event pair around one kernel launch when profiling is on.
struct ProfScope {
  spdhg_ctx* ctx;
  int kind;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(spdhg_ctx* c, int k, cudaStream_t st) : ctx(c), kind(k), s(st) {
    if (ctx->profiling) {
      a = prof_event(ctx);
      cudaEventRecord(a, s);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = prof_event(ctx);
      cudaEventRecord(b, s);
      ctx->prof_pending.push_back({kind, a, b});
    }
  }
};

int copy_in(spdhg_ctx* ctx, float* dst, const float* src, int64_t n, int where, cudaStream_t s) {
  CK(cudaMemcpyAsync(dst, src, n * sizeof(float), where == SPDHG_WHERE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  return SPDHG_OK;
}

int copy_out(spdhg_ctx* ctx, void* dst, const float* src, int64_t n, int where, cudaStream_t s) {
  CK(cudaMemcpyAsync(dst, src, n * sizeof(float), where == SPDHG_WHERE_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s));
  if (where == SPDHG_WHERE_HOST) CK(cudaStreamSynchronize(s));
  return SPDHG_OK;
}

// Row-split scratch of the forward projector for `subset` (allocated on first need).
int prepare_forward(spdhg_ctx* ctx, int subset, FwdArgs& a, cudaStream_t s) {
  const int split = forward_split(ctx->dg, subset);
  if (split <= 1) return SPDHG_OK;
  const size_t lines = (size_t)subset_views(ctx->dg, subset) * ctx->dg.R;
  const size_t tickets = lines * forward_parts(ctx->dg);
  const size_t need = lines * split * ctx->dg.P;
  if (need > ctx->fwd_part_cap) {
    ++ctx->graph_gen;  // captured iterations hold the old address
    ctx_free(ctx, ctx->fwd_part);
    ctx->fwd_part = nullptr;
    ctx->fwd_part_cap = 0;
    CK(ctx_malloc(ctx, (void**)&ctx->fwd_part, need * sizeof(float)));
    ctx->fwd_part_cap = need;
  }
  if (tickets > ctx->fwd_ticket_cap) {
    ++ctx->graph_gen;
    ctx_free(ctx, ctx->fwd_tickets);
    ctx->fwd_tickets = nullptr;
    ctx->fwd_ticket_cap = 0;
    CK(ctx_malloc(ctx, (void**)&ctx->fwd_tickets, tickets * sizeof(unsigned)));
    CK(cudaMemsetAsync(ctx->fwd_tickets, 0, tickets * sizeof(unsigned), s));
    ctx->fwd_ticket_cap = tickets;
  }
  a.part_acc = ctx->fwd_part;
  a.tickets = ctx->fwd_tickets;
  a.part_cap = ctx->fwd_part_cap;
  a.ticket_cap = ctx->fwd_ticket_cap;
  return SPDHG_OK;
}

// ||P_i|| by power iteration on P_i^T P_i (scalar step sizes, Eq. EQU:STEPSIZE:SCALAR): P_i is
// non-negative, so the iteration from the constant unit vector converges to its Perron vector.
// The eigenvalue estimate is read every kNormCheck steps; the iteration stops once it changes by
// less than kNormTol (relative) over those steps, or after kNormMax steps.  FP64 norms, the
// normalisation done on the device.  Uses x[1], tmp_img, tmp_sino and wdy as scratch (before
// spdhg_setup writes the initial state).
constexpr int kNormCheck = 10, kNormMax = 2000;
constexpr double kNormTol = 1e-7;

int subset_norm(spdhg_ctx* ctx, int i, cudaStream_t s, double* out) {
  const int64_t N = ctx->N;
  float* v = ctx->x[1];
  float* y = ctx->tmp_img;
  const float* mult = ctx->has_mult ? ctx->mult : nullptr;
  k_fill<<<grid_for(N), 256, 0, s>>>(v, N, (float)(1.0 / sqrt((double)N)));
  CK(cudaGetLastError());
  double prev = -1.0, ss = 0.0;
  for (int it = 0; it < kNormMax; ++it) {
    FwdArgs fa{};
    fa.x = v;
    fa.out = ctx->tmp_sino;
    fa.mult = mult;
    if (int st = prepare_forward(ctx, i, fa, s)) return st;
    CK(launch_forward(ctx->dg, i, FWD_PROJECT, fa, s));
    CK(launch_gather_subset(ctx->dg, i, ctx->tmp_sino, mult, ctx->wdy, s));
    BwdArgs ba{};
    ba.w = ctx->wdy;
    ba.out = y;
    CK(launch_backward(ctx->dg, i, BWD_OUT, ba, s));
    CK(launch_sumsq(y, N, ctx->red, ctx->red_blocks, ctx->red_out + 3, s));
    CK(launch_normalize(y, N, ctx->red_out + 3, v, s));
    if ((it + 1) % kNormCheck == 0) {
      CK(cudaMemcpyAsync(&ss, ctx->red_out + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      const double lam = sqrt(ss);  // ||P^T P v|| with ||v|| = 1: the largest eigenvalue of P^T P
      if (prev > 0.0 && fabs(lam - prev) <= kNormTol * lam) break;
      prev = lam;
    }
  }
  CK(cudaMemcpyAsync(&ss, ctx->red_out + 3, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *out = sqrt(sqrt(ss));
  return SPDHG_OK;
}

}  // namespace

// Enqueues the kernels of one SPDHG iteration (Algorithm 2) on block i and advances the
// ping-pong parities.  Used by spdhg_iterate and, under stream capture, by the epoch graphs.
int spdhg::enqueue_block(spdhg_ctx* ctx, int i, cudaStream_t s) {
  const int m = ctx->geom.n_subsets;
  const spdhg_params& p = ctx->params;
  const float inv_p = (float)(1.0 / ctx->probs[i]);
  if (i < m) {
    FwdArgs fa{};
    fa.x = ctx->x[ctx->xcur];
    fa.mult = ctx->has_mult ? ctx->mult : nullptr;
    fa.b = ctx->b;
    fa.r = ctx->r;
    fa.y = ctx->y;
    fa.wdy = ctx->wdy;
    fa.sigma = ctx->sigma;
    fa.gamma_rho = (float)(p.gamma * p.rho);
    if (int st = prepare_forward(ctx, i, fa, s)) return st;
    {
      ProfScope ps(ctx, SPDHG_KERNEL_FORWARD, s);
      CK(launch_forward(ctx->dg, i, FWD_DATA, fa, s));
    }
    BwdArgs ba{};
    ba.w = ctx->wdy;
    ba.x = ctx->x[ctx->xcur];
    ba.z = ctx->z;
    ba.T = ctx->T;
    ba.inv_p = inv_p;
    if (ctx->bwd_table == 1) {
      ba.items = ctx->bwd_items;
      ba.hdr = ctx->bwd_hdr;
    }
    {
      ProfScope ps(ctx, SPDHG_KERNEL_BACKWARD, s);
      CK(launch_backward(ctx->dg, i, BWD_UPDATE, ba, s));
    }
    if (p.prior == SPDHG_PRIOR_TGV) {
      ProfScope ps(ctx, SPDHG_KERNEL_WSTEP, s);
      CK(launch_w_step(ctx->dg, ctx->w[ctx->wcur], ctx->zw, ctx->Tw, s));
    }
  } else if (p.prior == SPDHG_PRIOR_TGV) {
    const int kblk = i - m;
    TgvArgs ta{};
    ta.block = kblk;
    ta.u_in = ctx->x[ctx->xcur];
    ta.u_out = ctx->x[1 - ctx->xcur];
    ta.w_in = ctx->w[ctx->wcur];
    ta.w_out = ctx->w[1 - ctx->wcur];
    if (kblk == 0) {
      ta.q_in = ctx->q[ctx->qcur];
      ta.q_out = ctx->q[1 - ctx->qcur];
      ta.alpha = (float)p.alpha0;
    } else {
      ta.q_in = ctx->q2[ctx->q2cur];
      ta.q_out = ctx->q2[1 - ctx->q2cur];
      ta.alpha = (float)p.alpha1;
    }
    ta.zu = ctx->z;
    ta.zw = ctx->zw;
    ta.Tu = ctx->T;
    ta.Tw = ctx->Tw;
    ta.sigma = ctx->sigma_prior[kblk];
    ta.inv_p = inv_p;
    ta.bscr = ctx->tgv_b;
    {
      ProfScope ps(ctx, SPDHG_KERNEL_TGV, s);
      CK(launch_tgv(ctx->dg, ta, s));
    }
    ctx->xcur ^= 1;
    ctx->wcur ^= 1;
    if (kblk == 0) ctx->qcur ^= 1;
    else ctx->q2cur ^= 1;
  } else {
    PriorArgs pa{};
    pa.kind = p.prior;
    pa.x_in = ctx->x[ctx->xcur];
    pa.x_out = ctx->x[1 - ctx->xcur];
    pa.q_in = ctx->q[ctx->qcur];
    pa.q_out = ctx->q[1 - ctx->qcur];
    pa.z = ctx->z;
    pa.T = ctx->T;
    pa.side = ctx->side;
    pa.sigma = ctx->sigma_prior[0];
    pa.alpha = (float)p.alpha;
    pa.inv_p = inv_p;
    pa.gamma_d = (float)p.dtv_gamma;
    pa.eta2 = (float)ctx->eta2;
    {
      ProfScope ps(ctx, SPDHG_KERNEL_PRIOR, s);
      CK(launch_prior(ctx->dg, pa, s));
    }
    ctx->xcur ^= 1;
    ctx->qcur ^= 1;
  }
  ++ctx->iterations;
  return SPDHG_OK;
}

cudaError_t spdhg::allow_dynamic_smem_fn(const void* kern, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, int> limit;  // (device, function) -> bytes allowed
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  auto it = limit.find({dev, kern});
  if (it == limit.end()) {
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    cudaFuncAttributes fa{};
    if ((e = cudaFuncGetAttributes(&fa, kern)) != cudaSuccess) return e;
    const int lim = optin - (int)fa.sharedSizeBytes;
    if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, lim)) != cudaSuccess) return e;
    it = limit.emplace(std::make_pair(dev, kern), lim).first;
  }
  return smem <= (size_t)it->second ? cudaSuccess : cudaErrorInvalidValue;
}

// Builds the backprojector's tap-item table once per context (geometry only): counted, scanned per
// view, then filled by the same code the kernel runs.  Not built when the geometry does not admit
// it, when the knob switches it off, or when it would take more than 40 % of the free device
// memory (the kernel then computes the items itself; the results are the same bits either way).
static int build_bwd_table(spdhg_ctx* ctx, cudaStream_t s) {
  if (ctx->bwd_table >= 0) return SPDHG_OK;
  ctx->bwd_table = 0;
  const DevGeom& g = ctx->dg;
  if (g.tune[SPDHG_TUNE_BWD_TABLE] == 1 || !backward_table_possible(g)) return SPDHG_OK;
  const size_t cols = (size_t)((g.nx + 3) / 4) * ((g.ny + 3) / 4) * 16;
  const size_t V = (size_t)g.V;
  unsigned char* cnt = nullptr;
  unsigned *bad = nullptr, *starts = nullptr, *totals = nullptr;
  int status = SPDHG_OK;
  auto release = [&]() {
    ctx_free(ctx, cnt);
    ctx_free(ctx, bad);
    ctx_free(ctx, starts);
    ctx_free(ctx, totals);
  };
  if (ctx_malloc(ctx, (void**)&cnt, V * cols) != cudaSuccess || ctx_malloc(ctx, (void**)&bad, sizeof(unsigned)) != cudaSuccess ||
      ctx_malloc(ctx, (void**)&starts, V * cols * sizeof(unsigned)) != cudaSuccess ||
      ctx_malloc(ctx, (void**)&totals, V * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    release();
    return SPDHG_OK;  // no room for the table: the kernel computes the items
  }
  cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned), s);
  if (e == cudaSuccess) e = backward_table_count(g, cnt, bad, s);
  if (e == cudaSuccess) e = backward_table_starts(g, cnt, starts, totals, s);
  std::vector<unsigned> tot(V);
  unsigned hbad = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(tot.data(), totals, V * sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    release();
    return fail(ctx, SPDHG_ERR_CUDA, std::string("backprojector table: ") + cudaGetErrorString(e));
  }
  std::vector<unsigned> base(V);
  uint64_t total = 0;
  for (size_t v = 0; v < V; ++v) {
    base[v] = (unsigned)total;
    total += tot[v];
  }
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const size_t need = (size_t)total * sizeof(float4) + V * cols * sizeof(int2);
  if (hbad || total >= (1ull << 32) || need > free_b / 10 * 4 ||
      (ctx->mem_limit && ctx->mem_used + need > ctx->mem_limit)) {
    release();
    return SPDHG_OK;
  }
  if (ctx_malloc(ctx, (void**)&ctx->bwd_items, (size_t)total * sizeof(float4) + 16) != cudaSuccess ||
      ctx_malloc(ctx, (void**)&ctx->bwd_hdr, V * cols * sizeof(int2)) != cudaSuccess) {
    cudaGetLastError();
    ctx_free(ctx, ctx->bwd_items);
    ctx_free(ctx, ctx->bwd_hdr);
    ctx->bwd_items = nullptr;
    ctx->bwd_hdr = nullptr;
    release();
    return SPDHG_OK;
  }
  e = cudaMemcpyAsync(totals, base.data(), V * sizeof(unsigned), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = backward_table_fill(g, starts, totals, ctx->bwd_items, ctx->bwd_hdr, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  release();
  if (e != cudaSuccess) return fail(ctx, SPDHG_ERR_CUDA, std::string("backprojector table: ") + cudaGetErrorString(e));
  ctx->bwd_table = 1;
  ++ctx->graph_gen;
  return status;
}

// Drops the table (a knob changed); the next spdhg_setup decides again.
static void drop_bwd_table(spdhg_ctx* ctx) {
  ctx_free(ctx, ctx->bwd_items);
  ctx_free(ctx, ctx->bwd_hdr);
  ctx->bwd_items = nullptr;
  ctx->bwd_hdr = nullptr;
  ctx->bwd_table = -1;
  ++ctx->graph_gen;
}

int spdhg::forward_scratch(spdhg_ctx* ctx, int subset, FwdArgs& a, cudaStream_t s) {
  return prepare_forward(ctx, subset, a, s);
}

// Allocates the forward row-split scratch of every subset now, so that no allocation or memset
// happens while an iteration is captured into a graph.
int spdhg::prepare_all_forward(spdhg_ctx* ctx, cudaStream_t s) {
  for (int i = -1; i < ctx->geom.n_subsets; ++i) {
    FwdArgs a{};
    if (int st = prepare_forward(ctx, i, a, s)) return st;
  }
  return SPDHG_OK;
}

extern "C" {

int spdhg_create_geometry(const spdhg_geometry* geom, spdhg_ctx** out) { return spdhg_create(geom, out); }

int spdhg_create(const spdhg_geometry* geom, spdhg_ctx** out) {
  if (!out) return SPDHG_ERR_ARG;
  *out = nullptr;
  if (!geom || !geom->seg_n || !geom->seg_zmid0 || !geom->seg_dzmid || !geom->seg_dz) return SPDHG_ERR_ARG;
  const spdhg_geometry& g = *geom;
  if (g.nx < 1 || g.ny < 1 || g.nz < 1 || g.n_radial < 1 || g.n_views < 1 || g.n_segments < 1 ||
      g.n_subsets < 1 || !(g.vx > 0) || !(g.vy > 0) || !(g.vz > 0) || !(g.d_radial > 0) || !(g.radius > 0) ||
      (g.subset_kind != SPDHG_SUBSETS_VIEWS && g.subset_kind != SPDHG_SUBSETS_BINS) ||
      (g.subset_kind == SPDHG_SUBSETS_VIEWS && g.n_subsets > g.n_views))
    return SPDHG_ERR_ARG;
  if (fabs(g.vx - g.vy) > 1e-9 * g.vx) return SPDHG_ERR_UNSUPPORTED;
  if (g.n_segments > kMaxSeg || g.nz > 256) return SPDHG_ERR_UNSUPPORTED;
  const double smax = 0.5 * (g.n_radial - 1) * g.d_radial;
  if (!(g.radius > smax)) return SPDHG_ERR_UNSUPPORTED;
  int P = 0;
  double kappa_max = 0.0;
  const double hmin = sqrt(g.radius * g.radius - smax * smax);
  for (int k = 0; k < g.n_segments; ++k) {
    if (g.seg_n[k] < 1) return SPDHG_ERR_ARG;
    if (g.seg_n[k] > 1 && fabs(g.seg_dzmid[k] - g.vz) > 1e-9 * g.vz) return SPDHG_ERR_UNSUPPORTED;
    P += g.seg_n[k];
  }
  // LOR components: the given ones (exact mashing), or one per segment covering every plane
  std::vector<int> c_seg, c_qlo, c_qhi, c_step;
  std::vector<double> c_dz;
  if (g.n_components > 0) {
    if (!g.comp_seg || !g.comp_dz || !g.comp_qlo || !g.comp_qhi || !g.comp_step) return SPDHG_ERR_ARG;
    int prev = 0;
    std::vector<int> per_seg(g.n_segments, 0);
    for (int c = 0; c < g.n_components; ++c) {
      const int k = g.comp_seg[c];
      if (k < prev || k >= g.n_segments || g.comp_qlo[c] < 0 || g.comp_qhi[c] > g.seg_n[k] ||
          g.comp_qlo[c] >= g.comp_qhi[c] || (g.comp_step[c] != 1 && g.comp_step[c] != 2) || !isfinite(g.comp_dz[c]))
        return SPDHG_ERR_ARG;
      prev = k;
      if (++per_seg[k] > 32) return SPDHG_ERR_UNSUPPORTED;
      c_seg.push_back(k);
      c_dz.push_back(g.comp_dz[c]);
      c_qlo.push_back(g.comp_qlo[c]);
      c_qhi.push_back(g.comp_qhi[c]);
      c_step.push_back(g.comp_step[c]);
    }
    for (int k = 0; k < g.n_segments; ++k)
      if (per_seg[k] == 0) return SPDHG_ERR_ARG;
  } else {
    for (int k = 0; k < g.n_segments; ++k) {
      c_seg.push_back(k);
      c_dz.push_back(g.seg_dz[k]);
      c_qlo.push_back(0);
      c_qhi.push_back(g.seg_n[k]);
      c_step.push_back(1);
    }
  }
  const int C = (int)c_seg.size();
  bool mashed = false;
  {
    std::vector<int> per_seg(g.n_segments, 0);
    for (int c = 0; c < C; ++c) {
      ++per_seg[c_seg[c]];
      if (c_qlo[c] != 0 || c_qhi[c] != g.seg_n[c_seg[c]] || c_step[c] != 1) mashed = true;
    }
    for (int k = 0; k < g.n_segments; ++k) mashed = mashed || per_seg[k] > 1;
  }
  for (int c = 0; c < C; ++c) kappa_max = std::max(kappa_max, fabs(c_dz[c]) / (2.0 * hmin * g.vz));
  if (P > 8192) return SPDHG_ERR_UNSUPPORTED;
  // kernels index images (up to 6 components) and sinograms with 32-bit integers
  if ((double)g.nx * g.ny * g.nz * 6 >= 2147483647.0 || (double)g.n_views * g.n_radial * P >= 2147483647.0)
    return SPDHG_ERR_UNSUPPORTED;
  const double dt_max = sqrt(2.0) * g.vx;  // longest transaxial chord of a pixel
  const int taps = kappa_max == 0.0 ? 1 : (int)ceil(1.0 + kappa_max * dt_max * (1.0 + 1e-6));
  if (taps > kMaxTaps) return SPDHG_ERR_UNSUPPORTED;
  const int nr_max = (int)floor(sqrt(2.0) * g.vx / g.d_radial) + 4;
  if (nr_max > 16) return SPDHG_ERR_UNSUPPORTED;

  spdhg_ctx* ctx = new spdhg_ctx();
  ctx->geom = g;
  ctx->seg_n.assign(g.seg_n, g.seg_n + g.n_segments);
  ctx->seg_zmid0.assign(g.seg_zmid0, g.seg_zmid0 + g.n_segments);
  ctx->seg_dzmid.assign(g.seg_dzmid, g.seg_dzmid + g.n_segments);
  ctx->seg_dz.assign(g.seg_dz, g.seg_dz + g.n_segments);
  ctx->geom.seg_n = ctx->seg_n.data();
  ctx->geom.seg_zmid0 = ctx->seg_zmid0.data();
  ctx->geom.seg_dzmid = ctx->seg_dzmid.data();
  ctx->geom.seg_dz = ctx->seg_dz.data();
  ctx->comp_seg = c_seg;
  ctx->comp_dz = c_dz;
  ctx->comp_qlo = c_qlo;
  ctx->comp_qhi = c_qhi;
  ctx->comp_step = c_step;
  ctx->geom.n_components = g.n_components > 0 ? C : 0;
  ctx->geom.comp_seg = g.n_components > 0 ? ctx->comp_seg.data() : nullptr;
  ctx->geom.comp_dz = g.n_components > 0 ? ctx->comp_dz.data() : nullptr;
  ctx->geom.comp_qlo = g.n_components > 0 ? ctx->comp_qlo.data() : nullptr;
  ctx->geom.comp_qhi = g.n_components > 0 ? ctx->comp_qhi.data() : nullptr;
  ctx->geom.comp_step = g.n_components > 0 ? ctx->comp_step.data() : nullptr;
  cudaGetDevice(&ctx->device);
  ctx->N = (int64_t)g.nx * g.ny * g.nz;
  ctx->M = (int64_t)g.n_views * g.n_radial * P;
  // a view subset's local sinogram holds its views; a bin subset's spans the whole sinogram
  ctx->max_subset_bins = g.subset_kind == SPDHG_SUBSETS_BINS
                             ? ctx->M
                             : (int64_t)((g.n_views + g.n_subsets - 1) / g.n_subsets) * g.n_radial * P;
  if (g.subset_kind == SPDHG_SUBSETS_BINS && ctx->M < g.n_subsets) {
    delete ctx;
    return SPDHG_ERR_ARG;
  }

  // device tables (FP64 on the host, stored as double-float pairs hi + lo)
  const double pi = 3.14159265358979323846;
  auto split = [](double v, float& hi, float& lo) {
    hi = (float)v;
    lo = (float)(v - (double)hi);
  };
  const int R = g.n_radial, V = g.n_views, S = g.n_segments;
  std::vector<float4> view(V), rad(R), rs((size_t)R * C);
  std::vector<float2> view_inv(V);
  for (int v = 0; v < V; ++v) {
    double c = cos(pi * v / V), sn = sin(pi * v / V);
    if (fabs(c) < 1e-12) c = 0.0;
    if (fabs(sn) < 1e-12) sn = 0.0;
    float4 t;
    split(c, t.x, t.y);
    split(sn, t.z, t.w);
    view[v] = t;
    // reciprocals of the FP32 direction components, rounded once on the host
    view_inv[v] = make_float2(t.z != 0.f ? (float)(1.0 / -(double)t.z) : 0.f, t.x != 0.f ? (float)(1.0 / (double)t.x) : 0.f);
  }
  for (int r = 0; r < R; ++r) {
    const double s = (r - 0.5 * (R - 1)) * g.d_radial;
    const double h = sqrt(g.radius * g.radius - s * s);
    float4 t;
    split(s / g.vx, t.x, t.y);
    split(h / g.vx, t.z, t.w);
    rad[r] = t;
    for (int c = 0; c < C; ++c) {
      const double slope = c_dz[c] / (2.0 * h);      // dz/dt of the component's LOR
      float4 u;
      split(slope * g.vx / g.vz, u.x, u.y);          // slab units per pixel unit of t
      u.z = (float)sqrt(1.0 + slope * slope);        // 3-D length per transaxial length
      u.w = 0.f;
      rs[(size_t)r * C + c] = u;
    }
  }
  const double loz = -0.5 * g.nz * g.vz;
  std::vector<SegDev> seg(S);
  std::vector<CompDev> comp(C);
  std::vector<int> stage_pos(P);
  int p0 = 0;
  int fz_lo = taps - 1, fz_stride = g.nz;
  for (int k = 0; k < S; ++k) {
    seg[k].p0 = p0;
    seg[k].n = g.seg_n[k];
    split((g.seg_zmid0[k] - loz) / g.vz, seg[k].f_hi, seg[k].f_lo);
    seg[k].c0 = -1;
    seg[k].nc = 0;
    // the backprojector's staged slot of each plane: segment k's planes follow 2k + 1 frames
    for (int q = 0; q < g.seg_n[k]; ++q) stage_pos[p0 + q] = p0 + q + (2 * k + 1) * (taps - 1);
    p0 += g.seg_n[k];
  }
  for (int c = 0; c < C; ++c) {
    const int k = c_seg[c];
    if (seg[k].c0 < 0) seg[k].c0 = c;
    ++seg[k].nc;
    comp[c].seg = k;
    comp[c].qlo = c_qlo[c];
    comp[c].qhi = c_qhi[c];
    comp[c].smask = c_step[c] - 1;
    // Axial bound of the forward gather: along the component's LOR of plane 0 the slab coordinate
    // is f + kappa t with |t| <= h, so every slab it touches lies in [floor(f - |kappa| h),
    // floor(f + |kappa| h)]; the tap offset j0 (plane 0's top slab is -j0) lies within that range
    // widened by two slabs for rounding.  The staged columns get frames that hold every read.
    const double f = (g.seg_zmid0[k] - loz) / g.vz;
    const double span = fabs(c_dz[c]) / (2.0 * g.vz);  // |kappa| h in slabs (independent of h)
    comp[c].jlo = -(int)floor(f + span) - 2;
    comp[c].jhi = -(int)floor(f - span) + 2;
    fz_lo = std::max(fz_lo, comp[c].jhi + taps - 1);
  }
  // plane q (read as min(q, n - 1)) reads slabs q - j0 - t: the highest is n - 1 - jlo
  for (int c = 0; c < C; ++c) fz_stride = std::max(fz_stride, g.seg_n[c_seg[c]] + 3 - comp[c].jlo);
  fz_stride += fz_lo;
  fz_stride = std::max(fz_stride, fz_lo + g.nz);
  std::vector<int2> runs;
  for (int k = 0; k < S; ++k)
    for (int q0 = 0; q0 < g.seg_n[k]; q0 += 32) runs.push_back(make_int2(k, q0));
  auto cleanup_fail = [&](cudaError_t e) {
    spdhg_destroy(ctx);
    return e == cudaErrorMemoryAllocation ? SPDHG_ERR_OOM : SPDHG_ERR_CUDA;
  };
  cudaError_t e;
  if ((e = ctx_malloc(ctx, (void**)&ctx->d_view, sizeof(float4) * V)) != cudaSuccess) return cleanup_fail(e);
  if ((e = ctx_malloc(ctx, (void**)&ctx->d_rad, sizeof(float4) * R)) != cudaSuccess) return cleanup_fail(e);
  if ((e = ctx_malloc(ctx, (void**)&ctx->d_rs, sizeof(float4) * R * C)) != cudaSuccess) return cleanup_fail(e);
  if ((e = ctx_malloc(ctx, (void**)&ctx->d_comp, sizeof(CompDev) * C)) != cudaSuccess) return cleanup_fail(e);
  if ((e = cudaMemcpy(ctx->d_comp, comp.data(), sizeof(CompDev) * C, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e);
  if ((e = ctx_malloc(ctx, (void**)&ctx->d_seg, sizeof(SegDev) * S)) != cudaSuccess) return cleanup_fail(e);
  if ((e = ctx_malloc(ctx, (void**)&ctx->d_stage_pos, sizeof(int) * P)) != cudaSuccess) return cleanup_fail(e);
  if ((e = cudaMemcpy(ctx->d_view, view.data(), sizeof(float4) * V, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e);
  if ((e = cudaMemcpy(ctx->d_rad, rad.data(), sizeof(float4) * R, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e);
  if ((e = cudaMemcpy(ctx->d_rs, rs.data(), sizeof(float4) * R * C, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e);
  if ((e = cudaMemcpy(ctx->d_seg, seg.data(), sizeof(SegDev) * S, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e);
  if ((e = cudaMemcpy(ctx->d_stage_pos, stage_pos.data(), sizeof(int) * P, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e);
  if ((e = ctx_malloc(ctx, (void**)&ctx->d_runs, sizeof(int2) * runs.size())) != cudaSuccess) return cleanup_fail(e);
  if ((e = ctx_malloc(ctx, (void**)&ctx->d_view_inv, sizeof(float2) * V)) != cudaSuccess) return cleanup_fail(e);
  if ((e = cudaMemcpy(ctx->d_view_inv, view_inv.data(), sizeof(float2) * V, cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e);
  if ((e = cudaMemcpy(ctx->d_runs, runs.data(), sizeof(int2) * runs.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return cleanup_fail(e);

  DevGeom& d = ctx->dg;
  d.nx = g.nx;
  d.ny = g.ny;
  d.nz = g.nz;
  d.R = R;
  d.V = V;
  d.P = P;
  d.m = g.n_subsets;
  d.bins = g.subset_kind == SPDHG_SUBSETS_BINS ? 1 : 0;
  d.n_seg = S;
  d.n_comp = C;
  d.mashed = mashed ? 1 : 0;
  d.comp = ctx->d_comp;
  d.taps = taps;
  d.nr_max = nr_max;
  d.half_R = (float)(0.5 * (R - 1));
  d.inv_drp = (float)(g.vx / g.d_radial);
  d.view = ctx->d_view;
  d.view_inv = ctx->d_view_inv;
  d.rad = ctx->d_rad;
  d.rs = ctx->d_rs;
  d.seg = ctx->d_seg;
  d.stage_pos = ctx->d_stage_pos;
  d.n_runs = (int)runs.size();
  d.runs = ctx->d_runs;
  for (int w = 0; w <= 16; ++w) {
    // components spanned by the blocks of the forward projector with w warps (2 runs each)
    int mx = 1;
    const int rpp = 2 * std::max(w, 1);
    for (size_t r0 = 0; r0 < runs.size(); r0 += rpp) {
      const size_t r1 = std::min(runs.size(), r0 + rpp) - 1;
      const int glo = runs[r0].x, ghi = runs[r1].x;
      mx = std::max(mx, seg[ghi].c0 + seg[ghi].nc - seg[glo].c0);
    }
    d.max_part_comps[w] = mx;
  }
  d.fz_lo = fz_lo;
  d.fz_stride = fz_stride;
  *out = ctx;
  return SPDHG_OK;
}

void spdhg_destroy(spdhg_ctx* ctx) {
  if (!ctx) return;
  void* ptrs[] = {ctx->d_view, ctx->d_view_inv, ctx->d_rad, ctx->d_rs, ctx->d_runs, ctx->d_seg, ctx->d_comp, ctx->d_stage_pos, ctx->b, ctx->r, ctx->mult, ctx->side,
                  ctx->x[0], ctx->x[1], ctx->z, ctx->T, ctx->y, ctx->sigma, ctx->wdy, ctx->q[0], ctx->q[1],
                  ctx->w[0], ctx->w[1], ctx->zw, ctx->q2[0], ctx->q2[1], ctx->tgv_b, ctx->tmp_sino, ctx->tmp_img, ctx->tmp_img2, ctx->em_sens, ctx->bwd_items, ctx->bwd_hdr, ctx->fwd_part, ctx->fwd_tickets,
                  ctx->red, ctx->red_out};
  for (void* p : ptrs) ctx_free(ctx, p);
  for (auto& r : ctx->prof_pending) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
  spdhg::graph_cache_free(ctx);
  delete ctx;
}

const char* spdhg_last_error(const spdhg_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

int spdhg_sizes(const spdhg_ctx* ctx, int64_t* n_voxels, int64_t* n_bins, int* n_blocks) {
  if (!ctx) return SPDHG_ERR_ARG;
  if (n_voxels) *n_voxels = ctx->N;
  if (n_bins) *n_bins = ctx->M;
  if (n_blocks) *n_blocks = ctx->is_setup ? (int)ctx->probs.size() : ctx->geom.n_subsets;
  return SPDHG_OK;
}

int spdhg_set_data(spdhg_ctx* ctx, const float* b, const float* r, const float* mult, const float* side,
                   int where) {
  if (!ctx) return SPDHG_ERR_ARG;
  if (!b || !r || (where != SPDHG_WHERE_HOST && where != SPDHG_WHERE_DEVICE)) return fail(ctx, SPDHG_ERR_ARG, "b and r are required");
  if (int st = check_device(ctx)) return st;
  CK(dalloc(ctx, &ctx->b, ctx->M));
  CK(dalloc(ctx, &ctx->r, ctx->M));
  CK(dalloc(ctx, &ctx->red, 2048));
  CK(dalloc(ctx, &ctx->red_out, 8));
  cudaStream_t s = 0;
  if (int st = copy_in(ctx, ctx->b, b, ctx->M, where, s)) return st;
  if (int st = copy_in(ctx, ctx->r, r, ctx->M, where, s)) return st;
  ctx->has_mult = mult != nullptr;
  if (mult) {
    CK(dalloc(ctx, &ctx->mult, ctx->M));
    if (int st = copy_in(ctx, ctx->mult, mult, ctx->M, where, s)) return st;
  }
  ctx->has_side = side != nullptr;
  if (side) {
    CK(dalloc(ctx, &ctx->side, ctx->N));
    if (int st = copy_in(ctx, ctx->side, side, ctx->N, where, s)) return st;
  }
  unsigned long long* bad = reinterpret_cast<unsigned long long*>(ctx->red_out);
  CK(cudaMemsetAsync(bad, 0, 8 * sizeof(double), s));
  k_validate<<<grid_for(ctx->M), 256, 0, s>>>(ctx->b, ctx->M, 0, bad);
  k_validate<<<grid_for(ctx->M), 256, 0, s>>>(ctx->r, ctx->M, 0, bad + 1);
  if (mult) k_validate<<<grid_for(ctx->M), 256, 0, s>>>(ctx->mult, ctx->M, 1, bad + 2);
  if (side) k_validate<<<grid_for(ctx->N), 256, 0, s>>>(ctx->side, ctx->N, 0, bad + 3);
  CK(cudaGetLastError());
  unsigned long long h[4];
  CK(cudaMemcpy(h, bad, sizeof(h), cudaMemcpyDeviceToHost));
  if (h[0] || h[1] || h[2] || h[3]) {
    ctx->has_data = false;
    char msg[256];
    snprintf(msg, sizeof msg, "invalid data: %llu bad b, %llu bad r, %llu bad mult (<=0), %llu bad side", h[0], h[1], h[2], h[3]);
    return fail(ctx, SPDHG_ERR_DATA, msg);
  }
  ctx->has_data = true;
  ctx->is_setup = false;
  ctx->em_sens_kind = -1;  // sensitivities follow the multipliers
  ++ctx->graph_gen;  // mult may have switched between a buffer and none
  return SPDHG_OK;
}

int spdhg_project(spdhg_ctx* ctx, const float* x, float* y, int subset, void* stream) {
  if (!ctx || !x || !y) return SPDHG_ERR_ARG;
  if (subset < -1 || subset >= ctx->geom.n_subsets) return fail(ctx, SPDHG_ERR_ARG, "subset out of range");
  if (int st = check_device(ctx)) return st;
  FwdArgs a{};
  a.x = x;
  a.out = y;
  a.mult = ctx->has_mult ? ctx->mult : nullptr;
  if (int st = prepare_forward(ctx, subset, a, (cudaStream_t)stream)) return st;
  CK(launch_forward(ctx->dg, subset, FWD_PROJECT, a, (cudaStream_t)stream));
  return SPDHG_OK;
}

int spdhg_backproject(spdhg_ctx* ctx, const float* y, float* x, int subset, void* stream) {
  if (!ctx || !x || !y) return SPDHG_ERR_ARG;
  if (subset < -1 || subset >= ctx->geom.n_subsets) return fail(ctx, SPDHG_ERR_ARG, "subset out of range");
  if (int st = check_device(ctx)) return st;
  cudaStream_t s = (cudaStream_t)stream;
  // subset -1 uses a full-size scratch sinogram
  float* w = nullptr;
  if (subset < 0) {
    CK(dalloc(ctx, &ctx->tmp_sino, ctx->M));
    w = ctx->tmp_sino;
  } else {
    CK(dalloc(ctx, &ctx->wdy, ctx->max_subset_bins));
    w = ctx->wdy;
  }
  CK(launch_gather_subset(ctx->dg, subset, y, ctx->has_mult ? ctx->mult : nullptr, w, s));
  BwdArgs a{};
  a.w = w;
  a.out = x;
  CK(launch_backward(ctx->dg, subset, BWD_OUT, a, s));
  return SPDHG_OK;
}

int spdhg_probabilities(const spdhg_ctx* ctx, double* probs, int* n_blocks) {
  if (!ctx || !n_blocks) return SPDHG_ERR_ARG;
  if (!ctx->is_setup) return SPDHG_ERR_STATE;
  *n_blocks = (int)ctx->probs.size();
  if (probs)
    for (size_t i = 0; i < ctx->probs.size(); ++i) probs[i] = ctx->probs[i];
  return SPDHG_OK;
}

int spdhg_sample(uint64_t seed, uint64_t offset, int n, const double* probs, int n_blocks, int32_t* out) {
  if (n < 0 || n_blocks < 1 || !probs || (n > 0 && !out)) return SPDHG_ERR_ARG;
  std::vector<double> cum(n_blocks);
  double acc = 0.0;
  for (int i = 0; i < n_blocks; ++i) {
    if (!(probs[i] >= 0.0)) return SPDHG_ERR_ARG;
    acc += probs[i];
    cum[i] = acc;
  }
  for (int k = 0; k < n; ++k) {
    const double u = (double)(splitmix64(seed, offset + (uint64_t)k) >> 11) * (1.0 / 9007199254740992.0);
    int i = 0;
    while (i < n_blocks - 1 && !(u < cum[i])) ++i;
    out[k] = i;
  }
  return SPDHG_OK;
}

int spdhg_setup(spdhg_ctx* ctx, const spdhg_params* params, const float* x0, int where, void* stream) {
  if (!ctx || !params) return SPDHG_ERR_ARG;
  if (int st = check_device(ctx)) return st;
  if (!ctx->has_data) return fail(ctx, SPDHG_ERR_STATE, "spdhg_set_data must be called before spdhg_setup");
  spdhg_params p = *params;
  if (!(p.rho > 0)) p.rho = 0.99;
  if (!(p.gamma > 0)) p.gamma = 1.0;
  if (p.prior < SPDHG_PRIOR_NONE || p.prior > SPDHG_PRIOR_TGV) return fail(ctx, SPDHG_ERR_ARG, "unknown prior");
  if (!(p.rho < 1.0)) return fail(ctx, SPDHG_ERR_ARG, "rho must be < 1");
  if (p.prior == SPDHG_PRIOR_DTV && !ctx->has_side) return fail(ctx, SPDHG_ERR_STATE, "dTV needs a side image (spdhg_set_data)");
  if (p.prior == SPDHG_PRIOR_DTV && !(p.dtv_gamma >= 0.0 && p.dtv_gamma < 1.0)) return fail(ctx, SPDHG_ERR_ARG, "dtv_gamma must be in [0, 1)");
  if (p.prior == SPDHG_PRIOR_TGV ? !(p.alpha0 > 0 && p.alpha1 > 0) : (p.prior != SPDHG_PRIOR_NONE && !(p.alpha > 0)))
    return fail(ctx, SPDHG_ERR_ARG, "prior weights must be positive");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = ctx->N, M = ctx->M;
  const int m = ctx->geom.n_subsets;

  CK(dalloc(ctx, &ctx->x[0], N));
  CK(dalloc(ctx, &ctx->x[1], N));
  CK(dalloc(ctx, &ctx->z, N));
  CK(dalloc(ctx, &ctx->T, N));
  CK(dalloc(ctx, &ctx->y, M));
  CK(dalloc(ctx, &ctx->sigma, M));
  CK(dalloc(ctx, &ctx->wdy, ctx->max_subset_bins));
  const bool tgv = p.prior == SPDHG_PRIOR_TGV;
  if (p.prior != SPDHG_PRIOR_NONE) {
    CK(dalloc(ctx, &ctx->q[0], 3 * N));
    CK(dalloc(ctx, &ctx->q[1], 3 * N));
  }
  if (tgv) {
    CK(dalloc(ctx, &ctx->w[0], 3 * N));
    CK(dalloc(ctx, &ctx->w[1], 3 * N));
    CK(dalloc(ctx, &ctx->zw, 3 * N));
    CK(dalloc(ctx, &ctx->tgv_b, 6 * N));
    CK(dalloc(ctx, &ctx->q2[0], 6 * N));
    CK(dalloc(ctx, &ctx->q2[1], 6 * N));
  }

  if (p.sampling == SPDHG_SAMPLING_CUSTOM) {
    if (!p.probs) return fail(ctx, SPDHG_ERR_ARG, "custom sampling needs params.probs");
    const int nb = m + n_prior_blocks(p.prior);
    double tot = 0.0;
    for (int i = 0; i < nb; ++i) {
      if (!(p.probs[i] > 0.0) || !isfinite(p.probs[i])) return fail(ctx, SPDHG_ERR_ARG, "custom probabilities must be positive");
      tot += p.probs[i];
    }
    if (fabs(tot - 1.0) > 1e-9) return fail(ctx, SPDHG_ERR_ARG, "custom probabilities must sum to one");
  } else if (p.sampling != SPDHG_SAMPLING_BALANCED && p.sampling != SPDHG_SAMPLING_UNIFORM) {
    return fail(ctx, SPDHG_ERR_ARG, "unknown sampling");
  }
  ctx->params = p;
  ctx->params.probs = nullptr;  // the caller's array is not kept
  ctx->probs = block_probs(m, p.prior, p.sampling);
  if (p.sampling == SPDHG_SAMPLING_CUSTOM) ctx->probs.assign(p.probs, p.probs + ctx->probs.size());
  const double gn = grad_norm(ctx->geom.nx, ctx->geom.ny, ctx->geom.nz);

  // scalar data steps (Eq. EQU:STEPSIZE:SCALAR): sigma_i = gamma rho / ||P_i||, T_i = rho p_i /
  // (gamma ||P_i||), with ||P_i|| by power iteration
  std::vector<double> norms;
  if (!p.precond) {
    CK(dalloc(ctx, &ctx->tmp_sino, M));
    CK(dalloc(ctx, &ctx->tmp_img, N));
    double t_data = INFINITY;
    for (int i = 0; i < m; ++i) {
      double nrm = 0.0;
      if (int st = subset_norm(ctx, i, s, &nrm)) return st;
      norms.push_back(nrm);
      if (nrm > 0.0) t_data = std::min(t_data, p.rho * ctx->probs[i] / (p.gamma * nrm));
    }
    k_fill<<<grid_for(N), 256, 0, s>>>(ctx->T, N, (float)t_data);
    CK(cudaGetLastError());
  }
  // T = min over data blocks of rho p_i / (gamma P_i^T 1)  (Eq. EQU:STEPSIZE:PRECOND)
  if (p.precond) {
    k_fill<<<grid_for(N), 256, 0, s>>>(ctx->T, N, INFINITY);
    CK(cudaGetLastError());
  }
  for (int i = 0; i < (p.precond ? m : 0); ++i) {
    CK(launch_gather_subset(ctx->dg, i, nullptr, ctx->has_mult ? ctx->mult : nullptr, ctx->wdy, s));
    BwdArgs a{};
    a.w = ctx->wdy;
    a.T = ctx->T;
    a.sens_num = (float)(p.rho * ctx->probs[i] / p.gamma);
    CK(launch_backward(ctx->dg, i, BWD_SENS, a, s));
  }
  // prior blocks: scalar steps (Eq. EQU:STEPSIZE:SCALAR)
  ctx->sigma_prior.clear();
  float t_prior = INFINITY;
  if (tgv) {
    const double n0 = sqrt(gn * gn + 1.0), n1 = gn;  // ||(grad, -I)||, bound on ||E||
    const double T0 = p.rho * ctx->probs[m] / (p.gamma * n0), T1 = p.rho * ctx->probs[m + 1] / (p.gamma * n1);
    ctx->sigma_prior = {(float)(p.gamma * p.rho / n0), (float)(p.gamma * p.rho / n1)};
    t_prior = (float)T0;
    ctx->Tw = (float)std::min(T0, T1);
  } else if (p.prior != SPDHG_PRIOR_NONE) {
    ctx->sigma_prior = {(float)(p.gamma * p.rho / gn)};
    t_prior = (float)(p.rho * ctx->probs[m] / (p.gamma * gn));
  }
  k_finalize_T<<<grid_for(N), 256, 0, s>>>(ctx->T, N, t_prior);
  CK(cudaGetLastError());
  // sigma_j = gamma rho / (P 1)_j for every bin (Eq. EQU:STEPSIZE:PRECOND), stored once; scalar
  // steps: gamma rho / ||P_i|| on every bin of subset i
  if (!p.precond && ctx->dg.bins) {
    std::vector<float> sig_i(m);
    for (int i = 0; i < m; ++i) sig_i[i] = norms[i] > 0.0 ? (float)(p.gamma * p.rho / norms[i]) : 0.f;
    CK(dalloc(ctx, &ctx->tmp_img, N));  // m <= N floats of per-subset steps
    if (m > N) return fail(ctx, SPDHG_ERR_UNSUPPORTED, "more bin subsets than voxels");
    CK(cudaMemcpyAsync(ctx->tmp_img, sig_i.data(), m * sizeof(float), cudaMemcpyHostToDevice, s));
    k_fill_bins<<<grid_for(M), 256, 0, s>>>(ctx->sigma, M, m, ctx->tmp_img);
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(s));
  } else if (!p.precond) {
    const int64_t RP = (int64_t)ctx->dg.R * ctx->dg.P;
    for (int v = 0; v < ctx->dg.V; ++v) {
      const double nrm = norms[v % m];
      k_fill<<<grid_for(RP), 256, 0, s>>>(ctx->sigma + v * RP, RP, nrm > 0.0 ? (float)(p.gamma * p.rho / nrm) : 0.f);
    }
    CK(cudaGetLastError());
  } else {
    FwdArgs a{};
    a.x = ctx->x[0];  // unused by the sigma pass
    a.out = ctx->sigma;
    a.mult = ctx->has_mult ? ctx->mult : nullptr;
    a.gamma_rho = (float)(p.gamma * p.rho);
    if (int st = prepare_forward(ctx, -1, a, s)) return st;
    CK(launch_forward(ctx->dg, -1, FWD_SIGMA, a, s));
  }

  if (p.prior == SPDHG_PRIOR_DTV) {
    CK(launch_side_max_grad(ctx->dg, ctx->side, ctx->red, ctx->red_blocks, ctx->red_out, s));
    double gmax = 0.0;
    CK(cudaMemcpyAsync(&gmax, ctx->red_out, sizeof(double), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const double eta = gmax > 0 ? p.dtv_eta_frac * gmax : 1.0;
    ctx->eta2 = eta * eta;
  }

  // captured graph iterations stay valid while the scalars their kernels receive do not change
  {
    std::vector<double> sig = {(double)p.prior, p.alpha, p.alpha0, p.alpha1, p.dtv_gamma, p.gamma * p.rho,
                               ctx->eta2, (double)ctx->Tw, (double)p.sampling};
    sig.insert(sig.end(), ctx->probs.begin(), ctx->probs.end());
    sig.insert(sig.end(), ctx->sigma_prior.begin(), ctx->sigma_prior.end());
    if (sig != ctx->graph_sig) {
      ctx->graph_sig = sig;
      ++ctx->graph_gen;
    }
  }

  // initial state: x = max(x0, 0), y = z = q = 0
  ctx->xcur = 0;
  ctx->qcur = 0;
  ctx->wcur = 0;
  ctx->q2cur = 0;
  if (x0) {
    if (where == SPDHG_WHERE_HOST) {
      CK(cudaMemcpyAsync(ctx->x[1], x0, N * sizeof(float), cudaMemcpyHostToDevice, s));
      k_clamp_copy<<<grid_for(N), 256, 0, s>>>(ctx->x[0], ctx->x[1], N);
    } else {
      k_clamp_copy<<<grid_for(N), 256, 0, s>>>(ctx->x[0], x0, N);
    }
    CK(cudaGetLastError());
  } else {
    CK(cudaMemsetAsync(ctx->x[0], 0, N * sizeof(float), s));
  }
  CK(cudaMemsetAsync(ctx->z, 0, N * sizeof(float), s));
  CK(cudaMemsetAsync(ctx->y, 0, M * sizeof(float), s));
  if (p.prior != SPDHG_PRIOR_NONE) CK(cudaMemsetAsync(ctx->q[0], 0, 3 * N * sizeof(float), s));
  if (tgv) {
    CK(cudaMemsetAsync(ctx->w[0], 0, 3 * N * sizeof(float), s));
    CK(cudaMemsetAsync(ctx->zw, 0, 3 * N * sizeof(float), s));
    CK(cudaMemsetAsync(ctx->q2[0], 0, 6 * N * sizeof(float), s));
  }
  ctx->iterations = 0;
  if (int st = build_bwd_table(ctx, s)) return st;
  ctx->is_setup = true;
  return SPDHG_OK;
}

int spdhg_iterate(spdhg_ctx* ctx, const int32_t* blocks, int n, void* stream) {
  if (!ctx || (n > 0 && !blocks) || n < 0) return SPDHG_ERR_ARG;
  if (!ctx->is_setup) return fail(ctx, SPDHG_ERR_STATE, "spdhg_setup must be called before spdhg_iterate");
  if (int st = check_device(ctx)) return st;
  const int nblk = (int)ctx->probs.size();
  for (int k = 0; k < n; ++k)
    if (blocks[k] < 0 || blocks[k] >= nblk) return fail(ctx, SPDHG_ERR_ARG, "block index out of range");
  for (int k = 0; k < n; ++k)
    if (int st = spdhg::enqueue_block(ctx, blocks[k], (cudaStream_t)stream)) return st;
  return SPDHG_OK;
}

int spdhg_get(spdhg_ctx* ctx, int what, void* dst, int where, void* stream) {
  if (!ctx || !dst) return SPDHG_ERR_ARG;
  if (int st = check_device(ctx)) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = ctx->N, M = ctx->M;
  if (!ctx->is_setup) return fail(ctx, SPDHG_ERR_STATE, "no state before spdhg_setup");
  const bool tgv = ctx->params.prior == SPDHG_PRIOR_TGV;
  switch (what) {
    case SPDHG_STATE_X: return copy_out(ctx, dst, ctx->x[ctx->xcur], N, where, s);
    case SPDHG_STATE_Z: return copy_out(ctx, dst, ctx->z, N, where, s);
    case SPDHG_STATE_T: return copy_out(ctx, dst, ctx->T, N, where, s);
    case SPDHG_STATE_Y: return copy_out(ctx, dst, ctx->y, M, where, s);
    case SPDHG_STATE_Q:
      if (ctx->params.prior == SPDHG_PRIOR_NONE) return fail(ctx, SPDHG_ERR_STATE, "no prior dual");
      return copy_out(ctx, dst, ctx->q[ctx->qcur], 3 * N, where, s);
    case SPDHG_STATE_W:
      if (!tgv) return fail(ctx, SPDHG_ERR_STATE, "no TGV state");
      return copy_out(ctx, dst, ctx->w[ctx->wcur], 3 * N, where, s);
    case SPDHG_STATE_ZW:
      if (!tgv) return fail(ctx, SPDHG_ERR_STATE, "no TGV state");
      return copy_out(ctx, dst, ctx->zw, 3 * N, where, s);
    case SPDHG_STATE_Q2:
      if (!tgv) return fail(ctx, SPDHG_ERR_STATE, "no TGV state");
      return copy_out(ctx, dst, ctx->q2[ctx->q2cur], 6 * N, where, s);
    case SPDHG_STATE_SIGMA: return copy_out(ctx, dst, ctx->sigma, M, where, s);
    default: return fail(ctx, SPDHG_ERR_ARG, "unknown state array");
  }
}

int spdhg_set(spdhg_ctx* ctx, int what, const void* src, int where, void* stream) {
  if (!ctx || !src || (where != SPDHG_WHERE_HOST && where != SPDHG_WHERE_DEVICE)) return SPDHG_ERR_ARG;
  if (int st = check_device(ctx)) return st;
  if (!ctx->is_setup) return fail(ctx, SPDHG_ERR_STATE, "no state before spdhg_setup");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = ctx->N, M = ctx->M;
  const bool tgv = ctx->params.prior == SPDHG_PRIOR_TGV;
  const float* f = static_cast<const float*>(src);
  switch (what) {
    case SPDHG_STATE_X: {
      // the primal iterate that opens the next iteration: kept non-negative
      float* dst = ctx->x[ctx->xcur];
      if (where == SPDHG_WHERE_HOST) {
        if (int st = copy_in(ctx, ctx->x[1 - ctx->xcur], f, N, where, s)) return st;
        f = ctx->x[1 - ctx->xcur];
      }
      k_clamp_copy<<<grid_for(N), 256, 0, s>>>(dst, f, N);
      CK(cudaGetLastError());
      return SPDHG_OK;
    }
    case SPDHG_STATE_Z: return copy_in(ctx, ctx->z, f, N, where, s);
    case SPDHG_STATE_Y: return copy_in(ctx, ctx->y, f, M, where, s);
    case SPDHG_STATE_Q:
      if (ctx->params.prior == SPDHG_PRIOR_NONE) return fail(ctx, SPDHG_ERR_STATE, "no prior dual");
      return copy_in(ctx, ctx->q[ctx->qcur], f, 3 * N, where, s);
    case SPDHG_STATE_W:
      if (!tgv) return fail(ctx, SPDHG_ERR_STATE, "no TGV state");
      return copy_in(ctx, ctx->w[ctx->wcur], f, 3 * N, where, s);
    case SPDHG_STATE_ZW:
      if (!tgv) return fail(ctx, SPDHG_ERR_STATE, "no TGV state");
      return copy_in(ctx, ctx->zw, f, 3 * N, where, s);
    case SPDHG_STATE_Q2:
      if (!tgv) return fail(ctx, SPDHG_ERR_STATE, "no TGV state");
      return copy_in(ctx, ctx->q2[ctx->q2cur], f, 6 * N, where, s);
    default: return fail(ctx, SPDHG_ERR_ARG, "state array cannot be set (T and SIGMA follow from the data)");
  }
}

int spdhg_objective(spdhg_ctx* ctx, const float* x, int where, double out[3], void* stream) {
  if (!ctx || !out) return SPDHG_ERR_ARG;
  if (int st = check_device(ctx)) return st;
  if (!ctx->has_data) return fail(ctx, SPDHG_ERR_STATE, "no data");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = ctx->N, M = ctx->M;
  CK(dalloc(ctx, &ctx->tmp_sino, M));
  const float* xd = x;
  if (!x) {
    if (!ctx->is_setup) return fail(ctx, SPDHG_ERR_STATE, "no iterate before spdhg_setup");
    xd = ctx->x[ctx->xcur];
  } else if (where == SPDHG_WHERE_HOST) {
    CK(dalloc(ctx, &ctx->tmp_img, N));
    CK(cudaMemcpyAsync(ctx->tmp_img, x, N * sizeof(float),
                       where == SPDHG_WHERE_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
    xd = ctx->tmp_img;
  }
  FwdArgs a{};
  a.x = xd;
  a.out = ctx->tmp_sino;
  a.mult = ctx->has_mult ? ctx->mult : nullptr;
  if (int st = prepare_forward(ctx, -1, a, s)) return st;
  CK(launch_forward(ctx->dg, -1, FWD_PROJECT, a, s));
  CK(launch_data_term(ctx->tmp_sino, ctx->b, ctx->r, M, ctx->red, ctx->red_blocks, ctx->red_out, s));
  int kind = ctx->is_setup ? ctx->params.prior : SPDHG_PRIOR_NONE;
  if (kind == SPDHG_PRIOR_TGV && x) kind = SPDHG_PRIOR_NONE;  // w unknown for an external u
  if (kind != SPDHG_PRIOR_NONE) {
    const float* w = kind == SPDHG_PRIOR_TGV ? ctx->w[ctx->wcur] : nullptr;
    CK(launch_prior_term(ctx->dg, kind, xd, w, ctx->side, (float)ctx->params.dtv_gamma, (float)ctx->eta2,
                         ctx->red, ctx->red_blocks, ctx->red_out + 1, s));
  }
  double h[3] = {0, 0, 0};
  CK(cudaMemcpyAsync(h, ctx->red_out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double prior = 0.0;
  const spdhg_params& p = ctx->params;
  if (kind == SPDHG_PRIOR_TGV) prior = p.alpha0 * h[1] + p.alpha1 * h[2];
  else if (kind != SPDHG_PRIOR_NONE) prior = p.alpha * h[1];
  out[0] = h[0];
  out[1] = prior;
  out[2] = h[0] + prior;
  return SPDHG_OK;
}

int spdhg_psnr(spdhg_ctx* ctx, const float* x, const float* x_star, int where, double* out, void* stream) {
  if (!ctx || !x_star || !out || (where != SPDHG_WHERE_HOST && where != SPDHG_WHERE_DEVICE)) return SPDHG_ERR_ARG;
  if (int st = check_device(ctx)) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = ctx->N;
  const float* xd = x;
  const float* xs = x_star;
  if (!x) {
    if (!ctx->is_setup) return fail(ctx, SPDHG_ERR_STATE, "no iterate before spdhg_setup");
    xd = ctx->x[ctx->xcur];
  } else if (where == SPDHG_WHERE_HOST) {
    CK(dalloc(ctx, &ctx->tmp_img2, N));
    CK(cudaMemcpyAsync(ctx->tmp_img2, x, N * sizeof(float), cudaMemcpyHostToDevice, s));
    xd = ctx->tmp_img2;
  }
  if (where == SPDHG_WHERE_HOST) {
    CK(dalloc(ctx, &ctx->tmp_img, N));
    CK(cudaMemcpyAsync(ctx->tmp_img, x_star, N * sizeof(float), cudaMemcpyHostToDevice, s));
    xs = ctx->tmp_img;
  }
  CK(launch_psnr_terms(xd, xs, N, ctx->red, ctx->red_blocks, ctx->red_out + 4, s));
  double h[2] = {0, 0};
  CK(cudaMemcpyAsync(h, ctx->red_out + 4, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // PSNR(x, x*) = 20 log10(||x*||_inf / ||x - x*||_2)  (Sec. 4, log read as base 10)
  *out = 20.0 * log10(h[1] / sqrt(h[0]));
  return SPDHG_OK;
}

}  // extern "C"

int spdhg::runlog_begin(spdhg_ctx* ctx, const spdhg_params& p, spdhg_report* rep, RunLog& L, cudaStream_t s) {
  const bool target = p.target_gap > 0.0;
  if (target && !isfinite(p.psi_star)) return fail(ctx, SPDHG_ERR_ARG, "target_gap needs a finite psi_star");
  if (p.x_star) {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, p.x_star) != cudaSuccess || pa.type != cudaMemoryTypeDevice) {
      cudaGetLastError();
      return fail(ctx, SPDHG_ERR_ARG, "x_star must be device memory");
    }
  }
  L = RunLog{};
  L.every = p.objective_every > 0 ? p.objective_every : ((target || p.x_star) ? 1 : 0);
  if (rep) {
    rep->epochs_done = 0;
    rep->iterations_done = 0;
    rep->stop_epoch = -1;
    rep->ms_to_stop = NAN;
    rep->psi_zero = NAN;
    if (rep->objective)
      for (int e = 0; e <= p.epochs; ++e) rep->objective[e] = NAN;
    if (rep->psnr)
      for (int e = 0; e <= p.epochs; ++e) rep->psnr[e] = NAN;
  }
  if (target) {
    // Psi(0): the zero image, for the normaliser of every run (warm starts included)
    CK(dalloc(ctx, &ctx->tmp_img, ctx->N));
    CK(cudaMemsetAsync(ctx->tmp_img, 0, ctx->N * sizeof(float), s));
    double o[3];
    if (int st = spdhg_objective(ctx, ctx->tmp_img, SPDHG_WHERE_DEVICE, o, s)) return st;
    L.psi0 = o[2];
    if (rep) rep->psi_zero = o[2];
  }
  if (rep && rep->objective && L.every > 0) {
    double o[3];
    if (int st = spdhg_objective(ctx, nullptr, SPDHG_WHERE_DEVICE, o, s)) return st;
    rep->objective[0] = o[2];
  }
  if (rep && rep->psnr && p.x_star) {
    double v;
    if (int st = spdhg_psnr(ctx, nullptr, p.x_star, SPDHG_WHERE_DEVICE, &v, s)) return st;
    rep->psnr[0] = v;
  }
  return SPDHG_OK;
}

int spdhg::runlog_epoch(spdhg_ctx* ctx, const spdhg_params& p, spdhg_report* rep, RunLog& L, int e, double epoch_ms,
                        cudaStream_t s) {
  L.ms += epoch_ms;
  if (L.every <= 0 || e % L.every) return SPDHG_OK;
  double o[3];
  if (int st = spdhg_objective(ctx, nullptr, SPDHG_WHERE_DEVICE, o, s)) return st;
  if (rep && rep->objective) rep->objective[e] = o[2];
  if (!isfinite(o[2])) return fail(ctx, SPDHG_ERR_DIVERGED, "objective is not finite");
  if (rep && rep->psnr && p.x_star) {
    double v;
    if (int st = spdhg_psnr(ctx, nullptr, p.x_star, SPDHG_WHERE_DEVICE, &v, s)) return st;
    rep->psnr[e] = v;
  }
  if (p.target_gap > 0.0 && (o[2] - p.psi_star) <= p.target_gap * (L.psi0 - p.psi_star)) {
    L.stopped = true;
    if (rep) {
      rep->stop_epoch = e;
      rep->ms_to_stop = L.ms;
    }
  }
  return SPDHG_OK;
}

extern "C" {

int spdhg_run(spdhg_ctx* ctx, const spdhg_params* params, float* x_inout, int where, spdhg_report* rep,
              void* stream) {
  if (!ctx || !params || params->epochs < 0) return SPDHG_ERR_ARG;
  if (params->graph) return spdhg_run_batch(&ctx, params, &x_inout, where, 1, rep, stream);
  cudaStream_t s = (cudaStream_t)stream;
  if (int st = spdhg_setup(ctx, params, x_inout, where, stream)) return st;
  const int m = ctx->geom.n_subsets;
  double pdata = 0.0;
  for (int i = 0; i < m; ++i) pdata += ctx->probs[i];
  const int ipe = (int)llround(m / pdata);
  std::vector<int32_t> seq(ipe);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  RunLog L;
  int status = runlog_begin(ctx, *params, rep, L, s);
  const bool timed = (rep && rep->epoch_ms) || params->target_gap > 0.0;
  for (int ep = 0; ep < params->epochs && status == SPDHG_OK; ++ep) {
    spdhg_sample(ctx->params.seed, (uint64_t)ep * ipe, ipe, ctx->probs.data(), (int)ctx->probs.size(), seq.data());
    if (cudaEventRecord(e0, s) != cudaSuccess) { status = fail(ctx, SPDHG_ERR_CUDA, "event record"); break; }
    if ((status = spdhg_iterate(ctx, seq.data(), ipe, stream))) break;
    if (cudaEventRecord(e1, s) != cudaSuccess) { status = fail(ctx, SPDHG_ERR_CUDA, "event record"); break; }
    float ms = 0.f;
    if (timed) {
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep && rep->epoch_ms) rep->epoch_ms[ep] = ms;
    }
    if (rep) {
      rep->epochs_done = ep + 1;
      rep->iterations_done = (int64_t)(ep + 1) * ipe;
    }
    if ((status = runlog_epoch(ctx, *params, rep, L, ep + 1, ms, s))) break;
    if (L.stopped) break;
  }
  if (status == SPDHG_OK && x_inout) status = copy_out(ctx, x_inout, ctx->x[ctx->xcur], ctx->N, where, s);
  if (status == SPDHG_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) status = fail(ctx, SPDHG_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return status;
}

int spdhg_osem(spdhg_ctx* ctx, const spdhg_params* params, int mlem, float* x_inout, int where, spdhg_report* rep,
               void* stream) {
  if (!ctx || !params || params->epochs < 0 || (x_inout && where != SPDHG_WHERE_HOST && where != SPDHG_WHERE_DEVICE))
    return SPDHG_ERR_ARG;
  if (int st = check_device(ctx)) return st;
  if (!ctx->has_data) return fail(ctx, SPDHG_ERR_STATE, "spdhg_set_data must be called before spdhg_osem");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = ctx->N;
  const int m = mlem ? 1 : ctx->geom.n_subsets;
  CK(dalloc(ctx, &ctx->x[0], N));
  CK(dalloc(ctx, &ctx->x[1], N));
  CK(dalloc(ctx, &ctx->wdy, mlem ? ctx->M : ctx->max_subset_bins));
  if (mlem && ctx->max_subset_bins < ctx->M) {
    // MLEM needs a full-size ratio sinogram
    CK(dalloc(ctx, &ctx->tmp_sino, ctx->M));
  }
  float* ratio = (mlem && ctx->max_subset_bins < ctx->M) ? ctx->tmp_sino : ctx->wdy;
  // sensitivity images P_i^T 1 (Eq. EQU:OSEM), or P^T 1 (Eq. EQU:MLEM)
  const int kind = mlem ? 1 : 0;
  if (ctx->em_sens_kind != kind) {
    ctx_free(ctx, ctx->em_sens);
    ctx->em_sens = nullptr;
    ctx->em_sens_kind = -1;
    CK(ctx_malloc(ctx, (void**)&ctx->em_sens, (size_t)m * N * sizeof(float)));
    for (int i = 0; i < m; ++i) {
      const int sub = mlem ? -1 : i;
      CK(launch_gather_subset(ctx->dg, sub, nullptr, ctx->has_mult ? ctx->mult : nullptr, ratio, s));
      BwdArgs a{};
      a.w = ratio;
      a.out = ctx->em_sens + (size_t)i * N;
      CK(launch_backward(ctx->dg, sub, BWD_OUT, a, s));
    }
    ctx->em_sens_kind = kind;
  }
  // the iterate: u0 from the caller, or ones (Eq. EQU:MLEM needs a positive start)
  float* u = ctx->x[0];
  ctx->xcur = 0;
  if (x_inout) {
    if (int st = copy_in(ctx, u, x_inout, N, where, s)) return st;
  } else {
    k_fill<<<grid_for(N), 256, 0, s>>>(u, N, 1.f);
    CK(cudaGetLastError());
  }
  // the objective of an EM run is the data term alone
  spdhg_params p = *params;
  p.prior = SPDHG_PRIOR_NONE;
  p.probs = nullptr;
  ctx->params = p;
  ctx->is_setup = true;
  ++ctx->graph_gen;
  ctx->probs = block_probs(ctx->geom.n_subsets, SPDHG_PRIOR_NONE, SPDHG_SAMPLING_UNIFORM);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  RunLog L;
  int status = runlog_begin(ctx, p, rep, L, s);
  const bool timed = (rep && rep->epoch_ms) || p.target_gap > 0.0;
  for (int ep = 0; ep < p.epochs && status == SPDHG_OK; ++ep) {
    if (cudaEventRecord(e0, s) != cudaSuccess) { status = fail(ctx, SPDHG_ERR_CUDA, "event record"); break; }
    for (int k = 0; k < m && status == SPDHG_OK; ++k) {
      const int sub = mlem ? -1 : k;  // i = k mod m (Eq. EQU:OSEM)
      FwdArgs fa{};
      fa.x = u;
      fa.mult = ctx->has_mult ? ctx->mult : nullptr;
      fa.b = ctx->b;
      fa.r = ctx->r;
      fa.wdy = ratio;
      if ((status = prepare_forward(ctx, sub, fa, s))) break;
      cudaError_t e = launch_forward(ctx->dg, sub, FWD_EM, fa, s);
      if (e == cudaSuccess) {
        BwdArgs ba{};
        ba.w = ratio;
        ba.x = u;
        ba.T = ctx->em_sens + (size_t)(mlem ? 0 : k) * N;
        e = launch_backward(ctx->dg, sub, BWD_EM, ba, s);
      }
      if (e != cudaSuccess) status = fail(ctx, SPDHG_ERR_CUDA, std::string("EM iteration: ") + cudaGetErrorString(e));
    }
    if (status) break;
    if (cudaEventRecord(e1, s) != cudaSuccess) { status = fail(ctx, SPDHG_ERR_CUDA, "event record"); break; }
    float ms = 0.f;
    if (timed) {
      cudaEventSynchronize(e1);
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep && rep->epoch_ms) rep->epoch_ms[ep] = ms;
    }
    if (rep) {
      rep->epochs_done = ep + 1;
      rep->iterations_done = (int64_t)(ep + 1) * m;
    }
    if ((status = runlog_epoch(ctx, p, rep, L, ep + 1, ms, s))) break;
    if (L.stopped) break;
  }
  if (status == SPDHG_OK && x_inout) status = copy_out(ctx, x_inout, u, N, where, s);
  if (status == SPDHG_OK) {
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) status = fail(ctx, SPDHG_ERR_CUDA, cudaGetErrorString(e));
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return status;
}

int spdhg_set_memory_limit(spdhg_ctx* ctx, uint64_t limit_bytes, uint64_t* used) {
  if (!ctx) return SPDHG_ERR_ARG;
  ctx->mem_limit = (size_t)limit_bytes;
  if (used) *used = ctx->mem_used;
  return SPDHG_OK;
}

int spdhg_tune(spdhg_ctx* ctx, int knob, int value) {
  if (!ctx || knob < 0 || knob >= SPDHG_TUNE_KNOBS || value < 0) return SPDHG_ERR_ARG;
  switch (knob) {
    case SPDHG_TUNE_PRIOR_COLS:
      // the launch checks cols against the warps of a column at the current voxels per thread
      if (value != 0 && (value < 2 || value > 32)) return fail(ctx, SPDHG_ERR_ARG, "prior cols out of range");
      break;
    case SPDHG_TUNE_PRIOR_VZ:
      if (value != 0 && value != 1 && value != 2 && value != 4)
        return fail(ctx, SPDHG_ERR_ARG, "prior voxels per thread must be 1, 2 or 4");
      break;
    case SPDHG_TUNE_PRIOR_STAGES:
      if (value != 0 && value != 3 && value != 4) return fail(ctx, SPDHG_ERR_ARG, "prior stages must be 3 or 4");
      break;
    case SPDHG_TUNE_PRIOR_YCHUNK:
      if (value > 1 << 20) return fail(ctx, SPDHG_ERR_ARG, "ychunk out of range");
      break;
    case SPDHG_TUNE_FWD_SPLIT:
      if (value > 16) return fail(ctx, SPDHG_ERR_ARG, "forward split out of range");
      break;
    case SPDHG_TUNE_BWD_TABLE:
      if (value > 1) return fail(ctx, SPDHG_ERR_ARG, "backprojector table knob must be 0 or 1");
      if (ctx->dg.tune[knob] != value) drop_bwd_table(ctx);
      break;
    case SPDHG_TUNE_FWD_GROUPS:
      if (value > 8) return fail(ctx, SPDHG_ERR_ARG, "forward entry groups must be 1 .. 8");
      break;
    case SPDHG_TUNE_FWD_WARPS:
      if (value != 0 && value != 1 && value != 2 && value != 4 && value != 8 && value != 16)
        return fail(ctx, SPDHG_ERR_ARG, "forward warps must be 1, 2, 4, 8 or 16");
      break;
    default: break;
  }
  if (ctx->dg.tune[knob] != value) ++ctx->graph_gen;
  ctx->dg.tune[knob] = value;
  return SPDHG_OK;
}

int spdhg_profile(spdhg_ctx* ctx, int enable) {
  if (!ctx) return SPDHG_ERR_ARG;
  for (auto& r : ctx->prof_pending) {
    ctx->prof_pool.push_back(r.a);
    ctx->prof_pool.push_back(r.b);
  }
  ctx->prof_pending.clear();
  for (int k = 0; k < SPDHG_KERNEL_KINDS; ++k) {
    ctx->prof_ms[k] = 0.0;
    ctx->prof_n[k] = 0;
  }
  ctx->profiling = enable != 0;
  return SPDHG_OK;
}

int spdhg_profile_read(spdhg_ctx* ctx, double* ms, int64_t* launches, int n) {
  if (!ctx || n < 0 || n > SPDHG_KERNEL_KINDS) return SPDHG_ERR_ARG;
  for (auto& r : ctx->prof_pending) {
    CK(cudaEventSynchronize(r.b));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, r.a, r.b));
    ctx->prof_ms[r.kind] += t;
    ctx->prof_n[r.kind] += 1;
    ctx->prof_pool.push_back(r.a);
    ctx->prof_pool.push_back(r.b);
  }
  ctx->prof_pending.clear();
  for (int k = 0; k < n; ++k) {
    if (ms) ms[k] = ctx->prof_ms[k];
    if (launches) launches[k] = ctx->prof_n[k];
  }
  return SPDHG_OK;
}

}  // extern "C"
