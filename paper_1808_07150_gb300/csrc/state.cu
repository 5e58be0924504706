// Checkpoint files of a reconstruction: spdhg_save_state / spdhg_load_state.
//
// File layout (little-endian as written by the host): an 8-byte magic "SPDHGST1", then int64
// N (voxels), M (bins), n_subsets, prior kind, iterations, and the spdhg_params fields that decide
// the step sizes and the iteration (prior weights, dTV parameters, sampling, precond, rho,
// gamma) as doubles / int64; then the FP32 arrays x, z, y and, with a prior, q (3N), and for TGV
// w (3N), zw (3N), q2 (6N).  T and sigma are not stored: spdhg_setup derives them from the data
// and the parameters, which the loading context must share.
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "internal.cuh"

namespace {

const char kMagic[8] = {'S', 'P', 'D', 'H', 'G', 'S', 'T', '1'};

int fail(spdhg_ctx* c, int code, const std::string& msg) {
  if (c) c->err = msg;
  return code;
}

// the parameters a checkpoint must agree on (the run length, objective cadence, sampler seed
// and launch mode are free)
std::vector<double> param_signature(const spdhg_params& p) {
  return {(double)p.prior, p.alpha, p.alpha0, p.alpha1, p.dtv_gamma, p.dtv_eta_frac,
          (double)p.sampling, (double)p.precond, p.rho, p.gamma};
}

struct Arr {
  float* dev;
  int64_t n;
};

std::vector<Arr> state_arrays(spdhg_ctx* c) {
  const int64_t N = c->N, M = c->M;
  std::vector<Arr> a = {{c->x[c->xcur], N}, {c->z, N}, {c->y, M}};
  if (c->params.prior != SPDHG_PRIOR_NONE) a.push_back({c->q[c->qcur], 3 * N});
  if (c->params.prior == SPDHG_PRIOR_TGV) {
    a.push_back({c->w[c->wcur], 3 * N});
    a.push_back({c->zw, 3 * N});
    a.push_back({c->q2[c->q2cur], 6 * N});
  }
  return a;
}

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

}  // namespace

extern "C" int spdhg_save_state(spdhg_ctx* ctx, const char* path) {
  if (!ctx || !path) return SPDHG_ERR_ARG;
  if (!ctx->is_setup) return fail(ctx, SPDHG_ERR_STATE, "no state before spdhg_setup");
  File fh;
  fh.f = fopen(path, "wb");
  if (!fh.f) return fail(ctx, SPDHG_ERR_ARG, std::string("cannot open ") + path + " for writing");
  const int64_t head[5] = {ctx->N, ctx->M, ctx->geom.n_subsets, ctx->params.prior, ctx->iterations};
  const std::vector<double> sig = param_signature(ctx->params);
  bool ok = fwrite(kMagic, 1, 8, fh.f) == 8 && fwrite(head, sizeof(head), 1, fh.f) == 1 &&
            fwrite(sig.data(), sizeof(double), sig.size(), fh.f) == sig.size();
  std::vector<float> h;
  for (const Arr& a : state_arrays(ctx)) {
    h.resize((size_t)a.n);
    cudaError_t e = cudaMemcpy(h.data(), a.dev, (size_t)a.n * sizeof(float), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(ctx, SPDHG_ERR_CUDA, std::string("state copy: ") + cudaGetErrorString(e));
    ok = ok && fwrite(h.data(), sizeof(float), h.size(), fh.f) == h.size();
  }
  if (!ok) return fail(ctx, SPDHG_ERR_ARG, std::string("short write to ") + path);
  return SPDHG_OK;
}

extern "C" int spdhg_load_state(spdhg_ctx* ctx, const char* path) {
  if (!ctx || !path) return SPDHG_ERR_ARG;
  if (!ctx->is_setup) return fail(ctx, SPDHG_ERR_STATE, "spdhg_setup (with the saved run's parameters) must come first");
  File fh;
  fh.f = fopen(path, "rb");
  if (!fh.f) return fail(ctx, SPDHG_ERR_ARG, std::string("cannot open ") + path);
  char magic[8];
  int64_t head[5];
  std::vector<double> sig(param_signature(ctx->params).size());
  if (fread(magic, 1, 8, fh.f) != 8 || memcmp(magic, kMagic, 8) != 0 || fread(head, sizeof(head), 1, fh.f) != 1 ||
      fread(sig.data(), sizeof(double), sig.size(), fh.f) != sig.size())
    return fail(ctx, SPDHG_ERR_DATA, std::string(path) + " is not a state file of this library");
  if (head[0] != ctx->N || head[1] != ctx->M || head[2] != ctx->geom.n_subsets)
    return fail(ctx, SPDHG_ERR_STATE, "the state file belongs to another geometry");
  if (head[3] != ctx->params.prior || sig != param_signature(ctx->params))
    return fail(ctx, SPDHG_ERR_STATE, "the state file was written with other parameters");
  std::vector<float> h;
  for (const Arr& a : state_arrays(ctx)) {
    h.resize((size_t)a.n);
    if (fread(h.data(), sizeof(float), h.size(), fh.f) != h.size())
      return fail(ctx, SPDHG_ERR_DATA, std::string(path) + " is truncated");
    cudaError_t e = cudaMemcpy(a.dev, h.data(), (size_t)a.n * sizeof(float), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(ctx, SPDHG_ERR_CUDA, std::string("state copy: ") + cudaGetErrorString(e));
  }
  ctx->iterations = head[4];
  return SPDHG_OK;
}
