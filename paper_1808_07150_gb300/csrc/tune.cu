// Autotuner of the launch-shape knobs (spdhg_tune): coordinate descent over the admissible
// values of each knob, each candidate timed with CUDA events on the kernel it shapes.  The
// timed launches read the context's current state and data and write only scratch (a copy of
// the dual y, the subset-local wdy buffer, the idle halves of the x and q ping-pong pairs and a
// copy of z), so tuning does not change the reconstruction.
#include <math.h>

#include <string>
#include <vector>

#include "internal.cuh"

using namespace spdhg;

namespace {

int fail(spdhg_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define TCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? SPDHG_ERR_OOM : SPDHG_ERR_CUDA,      \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

struct Timer {
  cudaEvent_t a = nullptr, b = nullptr;
  ~Timer() {
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
  }
};

// ms per launch of the forward (subset 0, the largest) or of the prior kernel
int time_kernel(spdhg_ctx* ctx, bool forward, int reps, cudaStream_t s, Timer& tm, double* ms) {
  const spdhg_params& p = ctx->params;
  auto launch = [&]() -> int {
    if (forward) {
      FwdArgs fa{};
      fa.x = ctx->x[ctx->xcur];
      fa.mult = ctx->has_mult ? ctx->mult : nullptr;
      fa.b = ctx->b;
      fa.r = ctx->r;
      fa.y = ctx->tmp_sino;
      fa.wdy = ctx->wdy;
      fa.sigma = ctx->sigma;
      fa.gamma_rho = (float)(p.gamma * p.rho);
      if (int st = forward_scratch(ctx, 0, fa, s)) return st;
      TCK(launch_forward(ctx->dg, 0, FWD_DATA, fa, s));
    } else {
      PriorArgs pa{};
      pa.kind = p.prior;
      pa.x_in = ctx->x[ctx->xcur];
      pa.x_out = ctx->x[1 - ctx->xcur];
      pa.q_in = ctx->q[ctx->qcur];
      pa.q_out = ctx->q[1 - ctx->qcur];
      pa.z = ctx->tmp_img;
      pa.T = ctx->T;
      pa.side = ctx->side;
      pa.sigma = ctx->sigma_prior[0];
      pa.alpha = (float)p.alpha;
      pa.inv_p = (float)(1.0 / ctx->probs[ctx->geom.n_subsets]);
      pa.gamma_d = (float)p.dtv_gamma;
      pa.eta2 = (float)ctx->eta2;
      TCK(launch_prior(ctx->dg, pa, s));
    }
    return SPDHG_OK;
  };
  if (int st = launch()) return st;  // warm-up (also sets the kernel's shared-memory attribute)
  // best of three trials of `reps` back-to-back launches: short kernels are timed against
  // host launch gaps and clock ramps, which only ever add time
  *ms = INFINITY;
  for (int trial = 0; trial < 3; ++trial) {
    TCK(cudaEventRecord(tm.a, s));
    for (int k = 0; k < reps; ++k)
      if (int st = launch()) return st;
    TCK(cudaEventRecord(tm.b, s));
    TCK(cudaEventSynchronize(tm.b));
    float t = 0.f;
    TCK(cudaEventElapsedTime(&t, tm.a, tm.b));
    *ms = fmin(*ms, (double)t / reps);
  }
  return SPDHG_OK;
}

}  // namespace

extern "C" int spdhg_autotune(spdhg_ctx* ctx, int reps, int* chosen, void* stream) {
  if (!ctx) return SPDHG_ERR_ARG;
  if (!ctx->is_setup) return fail(ctx, SPDHG_ERR_STATE, "spdhg_setup must be called before spdhg_autotune");
  if (reps <= 0) reps = 10;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != ctx->device)
    return fail(ctx, SPDHG_ERR_STATE, "current CUDA device differs from the context's device");
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t N = ctx->N, M = ctx->M;
  if (!ctx->tmp_sino) TCK(ctx_malloc(ctx, (void**)&ctx->tmp_sino, M * sizeof(float) + 16));
  if (!ctx->tmp_img) TCK(ctx_malloc(ctx, (void**)&ctx->tmp_img, N * sizeof(float) + 16));
  TCK(cudaMemcpyAsync(ctx->tmp_sino, ctx->y, M * sizeof(float), cudaMemcpyDeviceToDevice, s));
  TCK(cudaMemcpyAsync(ctx->tmp_img, ctx->z, N * sizeof(float), cudaMemcpyDeviceToDevice, s));
  Timer tm;
  TCK(cudaEventCreate(&tm.a));
  TCK(cudaEventCreate(&tm.b));

  const DevGeom& g = ctx->dg;
  const int nrows = g.nx > g.ny ? g.nx : g.ny;
  const bool stencil = ctx->params.prior == SPDHG_PRIOR_TV || ctx->params.prior == SPDHG_PRIOR_DTV ||
                       ctx->params.prior == SPDHG_PRIOR_ATV;
  struct Knob {
    int id;
    bool forward;
    std::vector<int> values;
  };
  std::vector<Knob> knobs;
  {
    Knob k{SPDHG_TUNE_FWD_WARPS, true, {}};
    for (int w : {2, 4, 8, 16})
      if (w == 2 || (g.n_runs + 1) / 2 > w / 2) k.values.push_back(w);
    knobs.push_back(k);
  }
  {
    // entry groups only where a line's plane runs leave the block with few warps
    Knob k{SPDHG_TUNE_FWD_GROUPS, true, {}};
    if (g.n_runs <= 6)
      for (int eg : {1, 2, 4, 8}) k.values.push_back(eg);
    knobs.push_back(k);
  }
  {
    Knob k{SPDHG_TUNE_FWD_SPLIT, true, {}};
    for (int sp : {1, 2, 4, 8})
      if (sp == 1 || nrows / sp >= 32) k.values.push_back(sp);
    knobs.push_back(k);
  }
  if (stencil) {
    Knob vz{SPDHG_TUNE_PRIOR_VZ, false, {1, 2, 4}};
    knobs.push_back(vz);
    // columns per block: the launch admits cols x (warps per column) <= 32 at the chosen voxels
    // per thread; candidates that do not fit are skipped below
    Knob c{SPDHG_TUNE_PRIOR_COLS, false, {}};
    for (int v : {2, 3, 4, 6, 8, 12, 16, 32})
      if (v <= g.nx + 1) c.values.push_back(v);
    knobs.push_back(c);
    Knob st{SPDHG_TUNE_PRIOR_STAGES, false, {3, 4}};
    knobs.push_back(st);
    Knob y{SPDHG_TUNE_PRIOR_YCHUNK, false, {}};
    for (int v : {16, 32, 64, 128, 256})
      if (v / 2 < g.ny) y.values.push_back(v);
    knobs.push_back(y);
  }
  for (const Knob& k : knobs) {
    if (k.values.size() < 2) continue;
    const int keep = g.tune[k.id];
    int best = keep;
    // the current setting is the one to beat (a candidate list need not hold the built-in choice)
    double best_ms = INFINITY;
    if (k.forward || prior_launch_ok(ctx->dg, ctx->params.prior))
      if (int st = time_kernel(ctx, k.forward, reps, s, tm, &best_ms)) return st;
    for (int v : k.values) {
      if (spdhg_tune(ctx, k.id, v) != SPDHG_OK) continue;
      if (!k.forward && !prior_launch_ok(ctx->dg, ctx->params.prior)) continue;
      double ms = 0.0;
      if (int st = time_kernel(ctx, k.forward, reps, s, tm, &ms)) {
        spdhg_tune(ctx, k.id, keep);
        return st;
      }
      if (ms < best_ms) {
        best_ms = ms;
        best = v;
      }
    }
    if (int st = spdhg_tune(ctx, k.id, best)) return st;
  }
  if (chosen)
    for (int k = 0; k < SPDHG_TUNE_KNOBS; ++k) chosen[k] = ctx->dg.tune[k];
  TCK(cudaStreamSynchronize(s));
  return SPDHG_OK;
}
