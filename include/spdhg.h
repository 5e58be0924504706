/*
 * spdhg.h -- C ABI of the GB300 SPDHG+ PET reconstruction library (libspdhg.so).
 *
 * Method: Ehrhardt, Markiewicz, Schoenlieb, "Faster PET reconstruction with non-smooth priors
 * by randomization and preconditioning".  The library solves
 *     min_{u >= 0}  sum_i D_i(P_i u) + alpha R(u)                 (Sec. 2.1, Problem "PET
 *                                                                    Reconstruction with Subsets")
 * with SPDHG (Algorithm 2), preconditioned step sizes (Eq. EQU:STEPSIZE:PRECOND) and balanced
 * sampling (Sec. 4.2).  All arithmetic runs in the library's CUDA kernels on the current device.
 *
 * Conventions
 *   image     x[iy][ix][iz], z fastest; voxel (ix,iy,iz) = [X_ix, X_ix+1) x [Y_iy, Y_iy+1) x
 *             [Z_iz, Z_iz+1), X_i = -nx*vx/2 + i*vx (same for y, z); float32.
 *   sinogram  y[view][radial][plane], plane fastest; float32.  View v has angle v*pi/n_views,
 *             radial bin r sits at s = (r - (n_radial-1)/2) * d_radial.
 *   planes    grouped in segments (fixed axial tilt); plane q of segment g has its LOR mid-point
 *             at z = seg_zmid0[g] + q*seg_dzmid[g] and its two ends seg_dz[g] apart axially.
 *   LOR       P(t) = (s cos - t sin, s sin + t cos, z_mid + t dz/(2h)), t in [-h, h],
 *             h = sqrt(radius^2 - s^2): the chord between two points of the detector cylinder.
 *   projector (L x)_j = sum_k |LOR_j intersect voxel_k| x_k, lengths in units of vx; a line lying
 *             in a grid plane belongs to the voxel whose lower face holds it.  P = diag(mult) L:
 *             the per-bin multiplier carries the geometric, attenuation and normalisation
 *             factors of the projection model (Sec. 1.2).
 *   subsets   view-interleaved: subset i = views v with v mod n_subsets == i (Sec. 4 forms the
 *             subsets from evenly spaced view angles), or bin-interleaved (subset_kind).
 *   blocks    SPDHG block indices 0..m-1 are the data subsets; m (and m+1 for TGV) the prior.
 *
 * Errors: every call returns SPDHG_OK (0) or a negative spdhg_status; no call aborts the process.
 * The message of the last failure on a context is available from spdhg_last_error().  CUDA
 * errors raised by a kernel launched through a context are reported as SPDHG_ERR_CUDA.
 * Ownership: the context owns every buffer it allocates (released by spdhg_destroy); the caller
 * owns every pointer it passes and the library keeps none of them after the call returns.
 * Streams: `stream` is a cudaStream_t (NULL = legacy default stream); kernels of a call are
 * enqueued on it in order, and calls that return data to host memory synchronise it.
 */
#ifndef SPDHG_H
#define SPDHG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct spdhg_ctx spdhg_ctx;

typedef enum {
  SPDHG_OK = 0,
  SPDHG_ERR_ARG = -1,         /* invalid argument (null pointer, out-of-range index, bad size) */
  SPDHG_ERR_CUDA = -2,        /* a CUDA runtime call or kernel failed */
  SPDHG_ERR_OOM = -3,         /* device allocation failed */
  SPDHG_ERR_DATA = -4,        /* non-finite or negative data, non-positive multiplier */
  SPDHG_ERR_TIMEOUT = -5,     /* a bounded device-side wait expired */
  SPDHG_ERR_DIVERGED = -6,    /* the FP64 objective became non-finite */
  SPDHG_ERR_STATE = -7,       /* call order violated (e.g. iterate before setup) */
  SPDHG_ERR_UNSUPPORTED = -8  /* geometry outside what the kernels handle (see spdhg_create) */
} spdhg_status;

enum { SPDHG_WHERE_HOST = 0, SPDHG_WHERE_DEVICE = 1 };

/* Scanner + image description.  Arrays are read during spdhg_create only. */
typedef struct {
  int nx, ny, nz;             /* image size in voxels */
  double vx, vy, vz;          /* voxel size in mm; vx == vy is required */
  int n_radial;               /* radial bins per view */
  double d_radial;            /* radial bin spacing, mm */
  int n_views;                /* views over [0, pi) */
  double radius;              /* detector cylinder radius, mm; > max |s| */
  int n_segments;
  const int* seg_n;           /* planes per segment (sinogram plane order is segment-major) */
  const double* seg_zmid0;    /* LOR mid-point z of the segment's first plane, mm */
  const double* seg_dzmid;    /* plane spacing within the segment; must equal vz if seg_n > 1 */
  const double* seg_dz;       /* axial separation z2 - z1 of the segment's LOR ends, mm */
  int n_subsets;              /* m, number of data subsets */
  int n_components;           /* exact mashing (0: none, every bin is the single LOR of its segment,
                                 seg_dz): the LOR components summed into the bins.  Component c
                                 belongs to segment comp_seg[c] (non-decreasing; every segment has
                                 at least one); plane q of that segment includes its LOR (the
                                 plane's mid-point, axial separation comp_dz[c] mm) when
                                 comp_qlo[c] <= q < comp_qhi[c] and (q - comp_qlo[c]) is a
                                 multiple of comp_step[c] (1 or 2).  Span-11 data are mashed this
                                 way from the ring-pair LORs of span 1 (Sec. 1) */
  const int* comp_seg;
  const double* comp_dz;
  const int* comp_qlo;
  const int* comp_qhi;
  const int* comp_step;
  int subset_kind;            /* SPDHG_SUBSETS_VIEWS (0): subset i = views v with v mod m == i;
                                 SPDHG_SUBSETS_BINS (1): subset i = bins j of the flattened sinogram
                                 with j mod m == i (the equidistantly divided bins of the stability
                                 example of Sec. 1.3).  A bin subset touches every view, so its
                                 projection costs a full projection */
} spdhg_geometry;

enum { SPDHG_SUBSETS_VIEWS = 0, SPDHG_SUBSETS_BINS = 1 };

enum { SPDHG_PRIOR_NONE = 0, SPDHG_PRIOR_TV = 1, SPDHG_PRIOR_DTV = 2, SPDHG_PRIOR_ATV = 3,
       SPDHG_PRIOR_TGV = 4 };
enum { SPDHG_SAMPLING_BALANCED = 0, SPDHG_SAMPLING_UNIFORM = 1, SPDHG_SAMPLING_CUSTOM = 2 };

typedef struct {
  int prior;                  /* SPDHG_PRIOR_* */
  double alpha;               /* weight of TV (Eq. EQU:SETTING:TV), dTV, aTV */
  double alpha0, alpha1;      /* TGV: alpha0 ||grad u - w|| + alpha1 ||E w|| (Sec. 4.3) */
  double dtv_gamma;           /* dTV: D = I - dtv_gamma xi xi^T, 0 <= dtv_gamma < 1 */
  double dtv_eta_frac;        /* dTV: xi = grad v / sqrt(|grad v|^2 + eta^2), eta = frac*max|grad v| */
  int sampling;               /* SPDHG_SAMPLING_*: balanced = prior w.p. 1/2 (Sec. 4.2); custom =
                                 the probabilities in `probs` */
  int precond;                /* 1: Eq. EQU:STEPSIZE:PRECOND for data blocks; 0: scalar Eq.
                                 EQU:STEPSIZE:SCALAR with ||P_i|| by power iteration on P_i^T P_i
                                 from the constant vector, until the eigenvalue changes by less than
                                 1e-7 (relative) over 10 steps (at most 2000 steps) */
  double rho;                 /* < 1 (Theorem "Step Size Parameters"); 0.99 if <= 0 */
  double gamma;               /* > 0; 1 if <= 0 (Sec. 4: gamma = 1) */
  uint64_t seed;              /* sampler seed (spdhg_run) */
  int epochs;                 /* spdhg_run: number of epochs */
  int objective_every;        /* spdhg_run: evaluate Psi every k epochs (0: never) */
  int graph;                  /* spdhg_run: 1 = every epoch is one CUDA graph launch (the path of
                                 spdhg_run_batch); 0 = kernels launched one by one */
  double target_gap;          /* spdhg_run / spdhg_run_batch: > 0 stops the run at the first
                                 evaluated epoch whose relative objective
                                 (Psi(x^k) - psi_star) / (Psi(0) - psi_star) is <= target_gap (the
                                 measure of Sec. 4, normalised by the zero image for every start);
                                 the objective is then evaluated every objective_every epochs, or
                                 every epoch if objective_every is 0.  0: run all epochs */
  double psi_star;            /* Psi(x*) of an approximate minimiser, used by target_gap */
  const float* x_star;        /* NULL, or an approximate minimiser x* (N floats, device memory):
                                 the report then receives PSNR(x^k, x*) (Sec. 4) at every evaluated
                                 epoch */
  const double* probs;        /* SPDHG_SAMPLING_CUSTOM: p_i of the n blocks (data subsets, then
                                 the prior blocks), each > 0, summing to 1 (Remark "Sampling": any
                                 proper sampling converges; the step sizes T_i use these p_i).
                                 Read by spdhg_setup only */
} spdhg_params;

typedef struct {
  int epochs_done;
  int64_t iterations_done;
  double* objective;          /* caller array of epochs+1 doubles or NULL: Psi after each
                                 evaluated epoch (index 0 = start), NaN where not evaluated */
  double* epoch_ms;           /* caller array of `epochs` doubles or NULL: device time per epoch */
  double* psnr;               /* caller array of epochs+1 doubles or NULL: PSNR(x^k, x*) =
                                 20 log10(max|x*| / ||x^k - x*||_2) after each evaluated epoch
                                 (index 0 = start; needs params.x_star), NaN where not evaluated */
  int stop_epoch;             /* epochs after which the relative objective first reached
                                 params.target_gap (-1: not reached, or no target) */
  double ms_to_stop;          /* device time of the epochs up to stop_epoch (solver time only:
                                 objective evaluations excluded); NaN if not reached */
  double psi_zero;            /* Psi(0), the normaliser of the relative objective (NaN without a
                                 target) */
} spdhg_report;

/* Creates a context for a geometry on the current CUDA device (device tables, no data yet).
 * Fails with SPDHG_ERR_UNSUPPORTED when vx != vy, when a multi-plane segment's spacing differs
 * from vz, when radius <= max |s|, when an oblique LOR crosses more than 4 slices inside one
 * transaxial pixel, or when a segment has more than 32 components.  *out receives the context
 * (NULL on failure). */
int spdhg_create(const spdhg_geometry* geom, spdhg_ctx** out);
/* The same call under the name of the problem set-up's first step (the scanner geometry that
 * defines the projection P of Sec. 1.2). */
int spdhg_create_geometry(const spdhg_geometry* geom, spdhg_ctx** out);

/* Releases every device buffer of the context.  NULL is accepted. */
void spdhg_destroy(spdhg_ctx* ctx);

/* Message of the last failure on ctx (empty string if none); valid until the next call on ctx. */
const char* spdhg_last_error(const spdhg_ctx* ctx);

/* Sizes: voxels N, bins M, SPDHG blocks n for the current parameters (m before spdhg_setup). */
int spdhg_sizes(const spdhg_ctx* ctx, int64_t* n_voxels, int64_t* n_bins, int* n_blocks);

/* Copies the measured counts b (Sec. 1.2: b in N^M), the background r (scatter + randoms) and
 * the per-bin multipliers mult (attenuation x normalisation; NULL = all ones) into the context;
 * side is the anatomical side image of dTV (N voxels; NULL unless dTV is used).  where =
 * SPDHG_WHERE_HOST or SPDHG_WHERE_DEVICE for all four pointers.  Rejects (SPDHG_ERR_DATA)
 * non-finite values, b < 0, r < 0, mult <= 0. */
int spdhg_set_data(spdhg_ctx* ctx, const float* b, const float* r, const float* mult,
                   const float* side, int where);

/* y = P_i x on the bins of subset i (i = -1: all bins); bins of other subsets are not written.
 * x (N floats) and y (M floats) are device pointers in the documented layouts.  Uses mult of the
 * last spdhg_set_data (ones if none). */
int spdhg_project(spdhg_ctx* ctx, const float* x, float* y, int subset, void* stream);

/* x = P_i^T y restricted to the bins of subset i (i = -1: all bins); device pointers. */
int spdhg_backproject(spdhg_ctx* ctx, const float* y, float* x, int subset, void* stream);

/* Step sizes and initial state for `params`: sigma_j = gamma rho / (P_i 1)_j for every bin
 * (stored), T = min_i T_i with T_i = rho p_i / (gamma P_i^T 1) for data blocks and the
 * scalar form for prior blocks; T = 0 where no block sees a voxel.  x = max(x0, 0) (the first
 * primal step of Algorithm 2 with zbar = 0), y = 0, z = 0, prior duals 0.  x0 = NULL: zeros. */
int spdhg_setup(spdhg_ctx* ctx, const spdhg_params* params, const float* x0, int where,
                void* stream);

/* Runs n SPDHG iterations (Algorithm 2) on the block indices blocks[0..n-1] (host array).
 * Each iteration updates the selected dual block, z, and then takes the next primal step, so
 * after the call the context's x is the primal iterate that opens the following iteration. */
int spdhg_iterate(spdhg_ctx* ctx, const int32_t* blocks, int n, void* stream);

enum { SPDHG_STATE_X = 0, SPDHG_STATE_Z = 1, SPDHG_STATE_T = 2, SPDHG_STATE_Y = 3,
       SPDHG_STATE_Q = 4, SPDHG_STATE_SIGMA = 5, SPDHG_STATE_W = 6, SPDHG_STATE_ZW = 7,
       SPDHG_STATE_Q2 = 8 };
/* Copies a state array into dst (host or device per `where`): X, Z, T (N floats), Y, SIGMA
 * (M floats; SIGMA as stored by spdhg_setup), Q (3N: first prior dual, components x,y,z), and for
 * TGV W (3N), ZW (3N), Q2 (6N: xx,yy,zz,xy,xz,yz). */
int spdhg_get(spdhg_ctx* ctx, int what, void* dst, int where, void* stream);

/* Overwrites a state array from src (host or device per `where`), the counterpart of spdhg_get
 * for resuming a run or changing its iterate: X (N floats, stored as max(src, 0): the primal
 * iterate that opens the next iteration), Z, Y, Q and for TGV W, ZW, Q2.  T and SIGMA follow
 * from the data and are rejected (SPDHG_ERR_ARG).  A consistent SPDHG state keeps z = A^T y
 * (Algorithm 2); replacing X alone is always consistent, since any primal point may start the
 * iteration.  Requires spdhg_setup. */
int spdhg_set(spdhg_ctx* ctx, int what, const void* src, int where, void* stream);

/* Checkpoint files.  spdhg_save_state writes the iteration state (x, z, y, the prior duals and
 * for TGV w, zw and the second dual; not T or sigma, which follow from the data and parameters),
 * the problem sizes, the parameters that define the iteration and the iteration count.
 * spdhg_load_state reads such a file into a context that has the same data sizes and was set up
 * with the same parameters (run length, objective cadence, sampler seed and launch mode may
 * differ); it fails with SPDHG_ERR_STATE otherwise and SPDHG_ERR_DATA for a file that is not a
 * state file or is truncated (a truncated file may leave the state partly overwritten).  Both
 * synchronise the device. */
int spdhg_save_state(spdhg_ctx* ctx, const char* path);
int spdhg_load_state(spdhg_ctx* ctx, const char* path);

/* Psi(x) in FP64 (Problem "PET Reconstruction with Subsets"): out[0] = sum_j varphi_j((P x)_j)
 * (Eq. EQU:LOCALDISTANCE), out[1] = alpha R(x) for the prior of the last spdhg_setup (0 if none),
 * out[2] = out[0] + out[1].  x = NULL uses the context's current iterate (and w for TGV). */
int spdhg_objective(spdhg_ctx* ctx, const float* x, int where, double out[3], void* stream);

/* OSEM (Eq. EQU:OSEM) or, with mlem = 1, MLEM (Eq. EQU:MLEM) on the context's data: the
 * unregularised expectation-maximisation baselines the paper compares SPDHG with (Sec. 1.3).  One
 * epoch is m sub-iterations u <- u / (P_i^T 1) * P_i^T (b_i / (P_i u + r_i)), i = k mod m (one
 * iteration over all bins for MLEM); u = 0 where P_i^T 1 = 0.  The start image comes from x_inout
 * (host or device per `where`; NULL: ones) and the result is written back to it.  From `params`
 * only epochs, objective_every, target_gap / psi_star and x_star are used (as in spdhg_run; the
 * objective is the data term, no prior).  The sensitivity images P_i^T 1 are computed on the first
 * call after spdhg_set_data and kept (m x N floats for OSEM, N for MLEM).  The call replaces the
 * context's iterate: run spdhg_setup before further SPDHG iterations. */
int spdhg_osem(spdhg_ctx* ctx, const spdhg_params* params, int mlem, float* x_inout, int where,
               spdhg_report* report, void* stream);

/* PSNR(x, x*) = 20 log10(max|x*| / ||x - x*||_2) (Sec. 4; log base 10) in FP64 on the GPU.  x and
 * x_star are N floats in host or device memory per `where` (x = NULL: the context's current
 * iterate). */
int spdhg_psnr(spdhg_ctx* ctx, const float* x, const float* x_star, int where, double* out, void* stream);

/* Sampling probabilities p_i of the blocks for the current parameters (Sec. 4.2). */
int spdhg_probabilities(const spdhg_ctx* ctx, double* probs, int* n_blocks);

/* Block indices drawn with probabilities probs[0..n_blocks-1]: draw k uses the SplitMix64
 * output number offset+k of the stream seeded with `seed`, its top 53 bits as a uniform u in
 * [0,1), and the first block whose cumulative probability exceeds u (Remark "Sampling"). */
int spdhg_sample(uint64_t seed, uint64_t offset, int n, const double* probs, int n_blocks,
                 int32_t* out);

/* Full reconstruction: spdhg_setup(params, x_inout) then params->epochs epochs of
 * iterations_per_epoch draws each (2m for balanced sampling), evaluating Psi every
 * objective_every epochs (FP64 on the GPU); with params->target_gap > 0 the run stops after the
 * first evaluated epoch whose relative objective reaches the target (Sec. 4) and the report
 * gives that epoch and the solver time to it.  A non-finite objective ends the run with
 * SPDHG_ERR_DIVERGED.  The final iterate is written back to x_inout (host or device). */
int spdhg_run(spdhg_ctx* ctx, const spdhg_params* params, float* x_inout, int where,
              spdhg_report* report, void* stream);

/* The paper has no counterpart of this call.  y = P_i^T y for one subset (0 <= i < n_subsets),
 * like spdhg_backproject, but the call allocates no device memory: for callers that cannot let
 * a library call cudaMalloc (device memory owned by their own pool with a hard budget, or loops
 * where an allocation's device synchronisation is not acceptable).  Its scratch is a fixed
 * device array of 2^21 floats (8 MiB) inside the library, held by every device that loads the
 * library until the process exits; a subset with more bins is rejected with SPDHG_ERR_ARG.  Every
 * call looks up the array's device address (cudaGetSymbolAddress) with the context's device
 * current, so a reset of the device's primary context does not leave a stale address behind; the
 * first call on a device may also load the library's device code, so make that first call before
 * any stream capture.  All calls share the array and
 * every call overwrites the part it reads, so nothing has to be cleared between calls, but calls
 * whose work overlaps on the GPU (concurrent streams, several contexts) race on it.  x and y are
 * device pointers as in spdhg_backproject. */
int spdhg_backproject_noalloc(spdhg_ctx* ctx, const float* y, float* x, int subset, void* stream);

/* Launch-shape knobs of the iteration kernels (0 restores the built-in choice).  They change
 * only how work is split across threads and blocks, never the arithmetic. */
enum { SPDHG_TUNE_PRIOR_COLS = 0,   /* prior kernel: voxel columns per block, incl. one halo column
                                       (blocks of up to 32 warps) */
       SPDHG_TUNE_PRIOR_YCHUNK = 1, /* prior kernel: rows marched per block */
       SPDHG_TUNE_FWD_SPLIT = 2,    /* forward kernel: row parts of one LOR line (partial sums
                                       reduced in a fixed order) */
       SPDHG_TUNE_FWD_WARPS = 3,    /* forward kernel: warps per block (1, 2, 4, 8 or 16); a warp
                                       owns two runs of 32 planes, so a line's runs are spread
                                       over ceil(runs / (2 * warps)) blocks */
       SPDHG_TUNE_PRIOR_STAGES = 4, /* prior kernel: rows in its shared-memory pipeline (3 or 4) */
       SPDHG_TUNE_BWD_TABLE = 5,    /* backprojector of the iterations: 0 reads its (pixel, bin,
                                       segment) tap items from a table built by spdhg_setup when
                                       it fits in 40 % of the free device memory (about 7 GB at
                                       the mMR scale; same results bit for bit); 1 computes them in
                                       the kernel */
       SPDHG_TUNE_FWD_GROUPS = 6,   /* forward projector: warps that share each plane run, each
                                       taking every k-th pixel entry of the line (1 .. 8; their
                                       partial sums are added in a fixed order); 0 = enough for
                                       four warps per block when a line has few plane runs */
       SPDHG_TUNE_PRIOR_VZ = 7,     /* prior kernel: voxels per thread along z (1, 2 or 4;
                                       0 = 1) */
       SPDHG_TUNE_KNOBS = 8 };

/* Sets one launch-shape knob of the context (value 0: default).  Out-of-range values are rejected
 * with SPDHG_ERR_ARG. */
int spdhg_tune(spdhg_ctx* ctx, int knob, int value);

/* Device-memory limit of the context, in bytes (0: none, the default).  Every device allocation
 * of the context (data, state, scratch, the backprojector's item table) is charged to it; one
 * that would exceed it fails as the driver's own would: the call returns SPDHG_ERR_OOM, the
 * context stays valid and keeps what it already holds (the item table, an optional cache, is
 * skipped instead).  A limit below what the context already holds applies to later
 * allocations only.  *used (may be NULL) receives the bytes the context holds now. */
int spdhg_set_memory_limit(spdhg_ctx* ctx, uint64_t limit_bytes, uint64_t* used);

/* Picks the launch-shape knobs of the context by measurement: for each knob in turn, every
 * admissible value is timed (CUDA events on `stream`: best of three trials of `reps` launches,
 * 10 if reps <= 0, after one warm-up) on the kernel it shapes, with the current state and data but scratch outputs (the reconstruction
 * state is not changed), and the fastest value is kept.  Requires spdhg_setup.  chosen (NULL or
 * SPDHG_TUNE_KNOBS ints) receives the resulting knob values (0 = built-in choice kept). */
int spdhg_autotune(spdhg_ctx* ctx, int reps, int* chosen, void* stream);

/* Many reconstructions, one CUDA graph launch per epoch (no counterpart in the paper, which
 * reconstructs one data set at a time).  For each r < n: spdhg_setup(ctx[r], &params[r],
 * x_inout[r]) as spdhg_run does, then params[r].epochs epochs.  Every epoch of all contexts is
 * one graph: each context is an independent branch holding its iterations' kernels in order,
 * with the block sequence of the epoch (spdhg_sample with params[r].seed, as spdhg_run) written
 * into the branch before the launch; a context whose epochs are done idles.  Results are
 * bit-identical to spdhg_run of each context alone.  Contexts must be distinct and on the
 * current device; x_inout (NULL, or n pointers each NULL or N_r floats, host or device per
 * `where`) receives the final iterates; reports (NULL or n) as in spdhg_run, with epoch_ms the
 * device time of the whole batch epoch.  Errors are reported on the context concerned (the first
 * one for graph-wide failures). */
int spdhg_run_batch(spdhg_ctx* const* ctx, const spdhg_params* params, float* const* x_inout,
                    int where, int n, spdhg_report* reports, void* stream);

/* Kernel classes timed by the per-launch profiler. */
enum { SPDHG_KERNEL_FORWARD = 0,   /* subset projection fused with the KL dual prox */
       SPDHG_KERNEL_BACKWARD = 1,  /* subset backprojection fused with z and the primal step */
       SPDHG_KERNEL_PRIOR = 2,     /* TV / dTV / aTV dual step fused with z and the primal step */
       SPDHG_KERNEL_TGV = 3,       /* TGV dual steps */
       SPDHG_KERNEL_WSTEP = 4,     /* TGV primal step of w in data iterations */
       SPDHG_KERNEL_KINDS = 5 };

/* Enables (1) or disables (0) per-launch timing of the iteration kernels with CUDA events on the
 * launching stream, and clears the accumulated figures. */
int spdhg_profile(spdhg_ctx* ctx, int enable);

/* Synchronises the recorded events and returns, per kernel class k < n (n <= SPDHG_KERNEL_KINDS),
 * the summed device time ms[k] and the launch count launches[k] since the last spdhg_profile. */
int spdhg_profile_read(spdhg_ctx* ctx, double* ms, int64_t* launches, int n);

#ifdef __cplusplus
}
#endif
#endif /* SPDHG_H */
