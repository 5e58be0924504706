// Epoch graphs: every epoch of one or many reconstructions runs as ONE CUDA graph launch.
//
// The sampled block sequence changes every epoch (Algorithm 2 draws i_k at random), so the
// graph has a fixed topology and the sequence is written into it from the host:
//   * each iteration of each reconstruction owns a fixed set of kernel-node "slots" (forward,
//     backward, [w step,] prior [, second prior pass for TGV]), chained in iteration order; the reconstructions are
//     independent branches of the same graph, so small problems run side by side on the SMs;
//   * the kernels of one iteration on block i (with the current ping-pong parities of x, q, w)
//     are captured once from the eager launch path (enqueue_block) into a small template graph;
//     its kernel-node parameters are what a slot receives;
//   * per epoch the host sets each slot to the template of the sampled block
//     (cudaGraphExecKernelNodeSetParams) or disables it (cudaGraphNodeSetEnabled), then the
//     whole batch is launched once.  Updates only affect later launches, so the host prepares
//     epoch e+1 while epoch e runs.
// The graph runs exactly the kernels, launch shapes and arguments of the eager path, so a run
// is bit-identical to spdhg_iterate on the same sequence.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "internal.cuh"

namespace spdhg {

namespace {

enum Slot { SLOT_FWD = 0, SLOT_BWD = 1, SLOT_WSTEP = 2, SLOT_PRIOR = 3, SLOT_PRIOR2 = 4, SLOT_KINDS = 5 };

int fail(spdhg_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

#define GCK(ctx, call)                                                                         \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? SPDHG_ERR_OOM : SPDHG_ERR_CUDA,      \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

// parity bits of the ping-pong pairs
constexpr int PX = 1, PQ = 2, PW = 4, PQ2 = 8;

int parity_of(const spdhg_ctx* c) {
  return (c->xcur ? PX : 0) | (c->qcur ? PQ : 0) | (c->wcur ? PW : 0) | (c->q2cur ? PQ2 : 0);
}
void set_parity(spdhg_ctx* c, int p) {
  c->xcur = (p & PX) ? 1 : 0;
  c->qcur = (p & PQ) ? 1 : 0;
  c->wcur = (p & PW) ? 1 : 0;
  c->q2cur = (p & PQ2) ? 1 : 0;
}

}  // namespace

// One captured iteration: its kernel nodes (1-3), the slot each belongs to, and how the
// iteration flips the parities.
struct Template {
  cudaGraph_t g = nullptr;  // owns the argument storage `p[k].kernelParams` points into
  int n = 0;
  int slot[3] = {0, 0, 0};
  cudaKernelNodeParams p[3];
  int par_xor = 0;
};

struct GraphCache {
  uint64_t gen = ~0ull;
  std::map<int64_t, Template> tpl;
  cudaStream_t cap = nullptr;  // capture stream
  void clear() {
    for (auto& kv : tpl)
      if (kv.second.g) cudaGraphDestroy(kv.second.g);
    tpl.clear();
  }
  ~GraphCache() {
    clear();
    if (cap) cudaStreamDestroy(cap);
  }
};

void graph_cache_free(spdhg_ctx* ctx) {
  delete ctx->gcache;
  ctx->gcache = nullptr;
}

namespace {

int n_slots(const spdhg_ctx* c, int* slots) {
  int n = 0;
  slots[n++] = SLOT_FWD;
  slots[n++] = SLOT_BWD;
  if (c->params.prior == SPDHG_PRIOR_TGV) slots[n++] = SLOT_WSTEP;
  if (c->params.prior != SPDHG_PRIOR_NONE) slots[n++] = SLOT_PRIOR;
  if (c->params.prior == SPDHG_PRIOR_TGV) slots[n++] = SLOT_PRIOR2;  // TGV: dual pass + primal pass
  return n;
}

// parity bits the kernels of block i read
int parity_mask(const spdhg_ctx* c, int i) {
  const bool tgv = c->params.prior == SPDHG_PRIOR_TGV;
  if (i < c->geom.n_subsets) return PX | (tgv ? PW : 0);
  if (!tgv) return PX | PQ;
  return PX | PW | (i == c->geom.n_subsets ? PQ : PQ2);
}

// Captures the kernels enqueue_block launches for block i at parity `par`.
int capture(spdhg_ctx* ctx, int i, int par, Template& t) {
  GraphCache* gc = ctx->gcache;
  if (!gc->cap) GCK(ctx, cudaStreamCreateWithFlags(&gc->cap, cudaStreamNonBlocking));
  GCK(ctx, cudaStreamBeginCapture(gc->cap, cudaStreamCaptureModeRelaxed));
  const int saved_par = parity_of(ctx);
  const int64_t saved_it = ctx->iterations;
  const bool saved_prof = ctx->profiling;
  ctx->profiling = false;
  set_parity(ctx, par);
  const int st = enqueue_block(ctx, i, gc->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(gc->cap, &g);
  const int par_after = parity_of(ctx);
  set_parity(ctx, saved_par);
  ctx->iterations = saved_it;
  ctx->profiling = saved_prof;
  if (st != SPDHG_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return st != SPDHG_OK ? st : fail(ctx, SPDHG_ERR_CUDA, std::string("iteration capture: ") + cudaGetErrorString(e));
  }
  t.g = g;
  t.par_xor = par ^ par_after;
  // walk the captured chain from its root
  const bool data = i < ctx->geom.n_subsets;
  const bool tgv = ctx->params.prior == SPDHG_PRIOR_TGV;
  const int expect = data ? (tgv ? 3 : 2) : (tgv ? 2 : 1);
  static const int data_slots[3] = {SLOT_FWD, SLOT_BWD, SLOT_WSTEP};
  cudaGraphNode_t node = nullptr;
  size_t nn = 1;
  GCK(ctx, cudaGraphGetRootNodes(g, &node, &nn));
  size_t total = 0;
  GCK(ctx, cudaGraphGetNodes(g, nullptr, &total));
  if (nn != 1 || (int)total != expect) return fail(ctx, SPDHG_ERR_STATE, "captured iteration has an unexpected shape");
  for (int k = 0; k < expect; ++k) {
    cudaGraphNodeType ty;
    GCK(ctx, cudaGraphNodeGetType(node, &ty));
    if (ty != cudaGraphNodeTypeKernel) return fail(ctx, SPDHG_ERR_STATE, "captured iteration holds a non-kernel node");
    GCK(ctx, cudaGraphKernelNodeGetParams(node, &t.p[k]));
    t.slot[k] = data ? data_slots[k] : (k == 0 ? SLOT_PRIOR : SLOT_PRIOR2);
    if (k + 1 < expect) {
      size_t nd = 1;
      cudaGraphNode_t next = nullptr;
      GCK(ctx, cudaGraphNodeGetDependentNodes(node, &next, nullptr, &nd));
      if (nd != 1 || !next) return fail(ctx, SPDHG_ERR_STATE, "captured iteration is not a chain");
      node = next;
    }
  }
  t.n = expect;
  return SPDHG_OK;
}

int get_template(spdhg_ctx* ctx, int i, int par, const Template** out) {
  if (!ctx->gcache) ctx->gcache = new GraphCache();
  GraphCache* gc = ctx->gcache;
  if (gc->gen != ctx->graph_gen) {
    gc->clear();
    gc->gen = ctx->graph_gen;
  }
  const int key_par = par & parity_mask(ctx, i);
  const int64_t key = (int64_t)i * 16 + key_par;
  auto it = gc->tpl.find(key);
  if (it == gc->tpl.end()) {
    Template t;
    if (int st = capture(ctx, i, key_par, t)) {
      if (t.g) cudaGraphDestroy(t.g);
      return st;
    }
    it = gc->tpl.emplace(key, t).first;
  }
  *out = &it->second;
  return SPDHG_OK;
}

// The branch of one reconstruction in the epoch graph.
struct Branch {
  spdhg_ctx* ctx = nullptr;
  int ipe = 0;                              // iterations per epoch
  int nslot = 0;
  int slots[SLOT_KINDS];
  std::vector<cudaGraphNode_t> node;        // [ipe][nslot]
  std::vector<const Template*> cur;         // template whose parameters the node holds
  std::vector<char> on;                     // node enabled
  uint64_t gen = ~0ull;                     // template generation `cur` refers to
};

struct EpochGraph {
  cudaGraph_t g = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<Branch> br;
  ~EpochGraph() {
    if (exec) cudaGraphExecDestroy(exec);
    if (g) cudaGraphDestroy(g);
  }
};

int build(EpochGraph& eg, spdhg_ctx* err_ctx) {
  GCK(err_ctx, cudaGraphCreate(&eg.g, 0));
  for (Branch& b : eg.br) {
    spdhg_ctx* ctx = b.ctx;
    b.nslot = n_slots(ctx, b.slots);
    // placeholder parameters of each slot: any template holding that slot
    cudaKernelNodeParams init[SLOT_KINDS];
    bool have[SLOT_KINDS] = {false, false, false, false, false};
    const Template* t = nullptr;
    const int par = parity_of(ctx);
    if (int st = get_template(ctx, 0, par, &t)) return st;
    for (int k = 0; k < t->n; ++k) { init[t->slot[k]] = t->p[k]; have[t->slot[k]] = true; }
    if (ctx->params.prior != SPDHG_PRIOR_NONE) {
      if (int st = get_template(ctx, ctx->geom.n_subsets, par, &t)) return st;
      for (int k = 0; k < t->n; ++k) {
        init[t->slot[k]] = t->p[k];
        have[t->slot[k]] = true;
      }
    }
    for (int j = 0; j < b.nslot; ++j)
      if (!have[b.slots[j]]) return fail(ctx, SPDHG_ERR_STATE, "no template for a graph slot");
    b.node.assign((size_t)b.ipe * b.nslot, nullptr);
    b.cur.assign(b.node.size(), nullptr);
    b.on.assign(b.node.size(), 1);
    cudaGraphNode_t prev = nullptr;
    for (size_t k = 0; k < b.node.size(); ++k) {
      const cudaKernelNodeParams& p = init[b.slots[k % b.nslot]];
      GCK(ctx, cudaGraphAddKernelNode(&b.node[k], eg.g, prev ? &prev : nullptr, prev ? 1 : 0, &p));
      prev = b.node[k];
    }
  }
  GCK(err_ctx, cudaGraphInstantiate(&eg.exec, eg.g, 0));
  return SPDHG_OK;
}

int set_node(spdhg_ctx* ctx, EpochGraph& eg, Branch& b, size_t k, const Template* t, int tk) {
  if (t) {
    if (b.cur[k] != t) {
      GCK(ctx, cudaGraphExecKernelNodeSetParams(eg.exec, b.node[k], &t->p[tk]));
      b.cur[k] = t;
    }
    if (!b.on[k]) {
      GCK(ctx, cudaGraphNodeSetEnabled(eg.exec, b.node[k], 1));
      b.on[k] = 1;
    }
  } else if (b.on[k]) {
    GCK(ctx, cudaGraphNodeSetEnabled(eg.exec, b.node[k], 0));
    b.on[k] = 0;
  }
  return SPDHG_OK;
}

// Writes one epoch of block indices into the branch (seq = NULL: the branch idles).
int update(EpochGraph& eg, Branch& b, const int32_t* seq) {
  spdhg_ctx* ctx = b.ctx;
  if (b.gen != ctx->graph_gen) {
    // the templates were (or will be) recaptured: every node gets its parameters again
    std::fill(b.cur.begin(), b.cur.end(), nullptr);
    b.gen = ctx->graph_gen;
  }
  int par = parity_of(ctx);
  for (int k = 0; k < b.ipe; ++k) {
    const Template* t = nullptr;
    if (seq)
      if (int st = get_template(ctx, seq[k], par, &t)) return st;
    for (int j = 0; j < b.nslot; ++j) {
      int tk = -1;
      if (t)
        for (int q = 0; q < t->n; ++q)
          if (t->slot[q] == b.slots[j]) tk = q;
      if (int st = set_node(ctx, eg, b, (size_t)k * b.nslot + j, tk >= 0 ? t : nullptr, tk)) return st;
    }
    if (t) par ^= t->par_xor;
  }
  if (seq) {
    set_parity(ctx, par);
    ctx->iterations += b.ipe;
  }
  return SPDHG_OK;
}

int iterations_per_epoch(const spdhg_ctx* ctx) {
  double pdata = 0.0;
  for (int i = 0; i < ctx->geom.n_subsets; ++i) pdata += ctx->probs[i];
  return (int)llround(ctx->geom.n_subsets / pdata);
}

}  // namespace
}  // namespace spdhg

using namespace spdhg;

extern "C" int spdhg_run_batch(spdhg_ctx* const* ctxs, const spdhg_params* params, float* const* x_inout,
                               int where, int n, spdhg_report* reports, void* stream) {
  if (!ctxs || !params || n <= 0) return SPDHG_ERR_ARG;
  for (int r = 0; r < n; ++r) {
    if (!ctxs[r] || params[r].epochs < 0) return SPDHG_ERR_ARG;
    for (int q = 0; q < r; ++q)
      if (ctxs[q] == ctxs[r]) return fail(ctxs[r], SPDHG_ERR_ARG, "a context appears twice in the batch");
    if (ctxs[r]->device != ctxs[0]->device) return fail(ctxs[r], SPDHG_ERR_ARG, "batch contexts live on different devices");
  }
  cudaStream_t s = (cudaStream_t)stream;
  EpochGraph eg;
  eg.br.resize(n);
  std::vector<RunLog> logs(n);
  int epochs = 0;
  for (int r = 0; r < n; ++r) {
    spdhg_ctx* ctx = ctxs[r];
    if (int st = spdhg_setup(ctx, &params[r], x_inout ? x_inout[r] : nullptr, where, stream)) return st;
    if (int st = prepare_all_forward(ctx, s)) return st;
    eg.br[r].ctx = ctx;
    eg.br[r].ipe = iterations_per_epoch(ctx);
    epochs = std::max(epochs, params[r].epochs);
    if (int st = runlog_begin(ctx, params[r], reports ? &reports[r] : nullptr, logs[r], s)) return st;
  }
  if (int st = build(eg, ctxs[0])) return st;
  std::vector<cudaEvent_t> ev(2 * (size_t)epochs, nullptr);
  int status = SPDHG_OK;
  std::vector<int32_t> seq;
  auto active = [&](int r, int e) { return e < params[r].epochs && !logs[r].stopped; };
  bool timed_now = false;
  for (int r = 0; r < n; ++r) timed_now = timed_now || params[r].target_gap > 0.0;
  std::vector<int> ran(n, 0);  // epochs each context has run
  for (int e = 0; e < epochs && status == SPDHG_OK; ++e) {
    bool any = false;
    for (int r = 0; r < n; ++r) any = any || active(r, e);
    if (!any) break;  // every context has finished or reached its target
    for (int r = 0; r < n && status == SPDHG_OK; ++r) {
      Branch& b = eg.br[r];
      const bool act = active(r, e);
      if (act) {
        seq.resize(b.ipe);
        spdhg_sample(b.ctx->params.seed, (uint64_t)e * b.ipe, b.ipe, b.ctx->probs.data(), (int)b.ctx->probs.size(),
                     seq.data());
      }
      status = update(eg, b, act ? seq.data() : nullptr);
    }
    if (status) break;
    for (int k = 0; k < 2 && status == SPDHG_OK; ++k)
      if (cudaEventCreate(&ev[2 * e + k]) != cudaSuccess) status = fail(ctxs[0], SPDHG_ERR_CUDA, "event create");
    if (status) break;
    cudaEventRecord(ev[2 * e], s);
    cudaError_t le = cudaGraphLaunch(eg.exec, s);
    if (le != cudaSuccess) { status = fail(ctxs[0], SPDHG_ERR_CUDA, std::string("cudaGraphLaunch: ") + cudaGetErrorString(le)); break; }
    cudaEventRecord(ev[2 * e + 1], s);
    // the epoch's device time is read now only when a stopping rule needs it; otherwise the host
    // goes on preparing the next epoch while this one runs, and the times are read at the end
    float ms = 0.f;
    if (timed_now && (cudaEventSynchronize(ev[2 * e + 1]) != cudaSuccess ||
                      cudaEventElapsedTime(&ms, ev[2 * e], ev[2 * e + 1]) != cudaSuccess))
      ms = NAN;
    for (int r = 0; r < n && status == SPDHG_OK; ++r) {
      if (!active(r, e)) continue;
      ran[r] = e + 1;
      if (reports) {
        reports[r].epochs_done = e + 1;
        reports[r].iterations_done = (int64_t)(e + 1) * eg.br[r].ipe;
      }
      status = runlog_epoch(ctxs[r], params[r], reports ? &reports[r] : nullptr, logs[r], e + 1, ms, s);
    }
  }
  if (status == SPDHG_OK) {
    cudaError_t se = cudaStreamSynchronize(s);
    if (se != cudaSuccess) status = fail(ctxs[0], SPDHG_ERR_CUDA, cudaGetErrorString(se));
  }
  if (status == SPDHG_OK && reports) {
    for (int e = 0; e < epochs; ++e) {
      if (!ev[2 * e]) break;
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, ev[2 * e], ev[2 * e + 1]) != cudaSuccess) ms = NAN;
      for (int r = 0; r < n; ++r)
        if (reports[r].epoch_ms && e < ran[r]) reports[r].epoch_ms[e] = ms;
    }
  }
  for (cudaEvent_t x : ev)
    if (x) cudaEventDestroy(x);
  if (status == SPDHG_OK && x_inout)
    for (int r = 0; r < n && status == SPDHG_OK; ++r)
      if (x_inout[r]) status = spdhg_get(ctxs[r], SPDHG_STATE_X, x_inout[r], where, stream);
  if (status == SPDHG_OK) {
    cudaError_t se = cudaStreamSynchronize(s);
    if (se != cudaSuccess) status = fail(ctxs[0], SPDHG_ERR_CUDA, cudaGetErrorString(se));
  }
  return status;
}
