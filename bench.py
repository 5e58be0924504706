#!/usr/bin/env python
"""Benchmark of the SPDHG+ hot path on the mMR-scale workload.

Workload (one "step" = one epoch = 2m = 504 SPDHG iterations, balanced sampling, seeded):
344x344x127 voxels (2.08 mm), span-11-like sinogram 252 views x 344 radial x 837 planes
(72,557,856 bins) with per-bin attenuation x normalisation, 4e8 counts + 10% background,
dTV prior with a synthetic anatomical side image, 252 view subsets, preconditioned steps.

Reported: epochs/s over the timed epochs (device time, CUDA events, max over ranks), the
roofline of the dominant kernel (algorithmic bytes / average launch time from per-launch CUDA
events recorded by the library during the timed region), an end-to-end figure through the
public API with host buffers, and the FP64 oracle timed on a bounded sample on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import glob
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to 1e-3 rel. objective gap vs plain SPDHG; epoch time; proj GB/s vs HBM peak"
WORKLOAD = "mmr-344x344x127-252v344r837p-dtv-252subsets"
SEED = 1808
ALPHA = 0.05
HBM_FALLBACK_GBS = 6800.0
GAP = 1e-3
REF_EPOCHS = 60       # Psi* of the mMR workload: Psi after this many epochs
MAX_GAP_EPOCHS = 40


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-time-to-gap", action="store_true")
    ap.add_argument("--ncu-case", action="store_true",
                    help="set up the workload, run one data and one prior iteration, exit (ncu captures)")
    ap.add_argument("--ncu-unet", action="store_true",
                    help="three U-Net training steps on a 128x128x64 volume, exit (ncu captures)")
    ap.add_argument("--workload", default="mmr", choices=["mmr", "batch16", "warmstart", "precond", "osem", "configs"],
                    help="mmr: the mMR-scale dTV reconstruction (default); batch16: 16 uneven "
                         "reconstructions, one CUDA graph launch per epoch; warmstart: the learned "
                         "warm start (U-Net trained on SPDHG+ solutions, 128x128x64 scanner)")
    ap.add_argument("--n-train", type=int, default=512)
    ap.add_argument("--n-test", type=int, default=64)
    ap.add_argument("--train-epochs", type=int, default=16)
    ap.add_argument("--k", type=int, default=2, help="warm start: SPDHG+ epochs before the network")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, device=None):
    """The largest `value` over all ranks of the default process group (the value itself when
    there is no group); the timing rule of the weak-scaling replicas."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def aggregate_rate(units_per_rank, ws, seconds):
    """Whole-job throughput of ws replicas that each processed units_per_rank units, timed by
    the slowest rank."""
    return ws * units_per_rank / seconds


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return

        def reader():
            for line in self.proc.stdout:
                self.lines.append(line.strip())

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def traffic_from_profiles(kernel_key):
    """DRAM bytes per launch of `kernel_key` from a committed ncu summary, provided the source
    file named there is unchanged since the capture (else None)."""
    import hashlib
    src = os.path.join(ROOT, "paper_1808_07150_gb300", "csrc")
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        txt = open(path).read()
        m = re.search(rf"^traffic\[{re.escape(kernel_key)}\]:\s*([0-9.eE+]+)\s+bytes per launch\s+"
                      rf"source_sha256\[([\w.]+)\]:\s*(\w+)", txt, re.M)
        if not m:
            continue
        f = os.path.join(src, m.group(2))
        if os.path.exists(f) and hashlib.sha256(open(f, "rb").read()).hexdigest()[:16] == m.group(3):
            return float(m.group(1))
    return None


def make_workload():
    import synth
    sc = synth.config_mmr()
    d = synth.make_problem(sc, SEED, counts=4e8, bg_frac=0.1, with_mult=True, with_side=True)
    return sc, d


def kernel_bytes(sc, kind):
    """Algorithmic bytes one launch must move (FP32): see the per-kernel accounting."""
    N = sc.n_voxels
    Mi = sc.n_radial * sc.n_planes * ((sc.n_views + sc.n_subsets - 1) // sc.n_subsets)
    return {
        "forward": 4 * N + 24 * Mi,    # read x; read b, r, mult, y; write y, mult*dy
        "backward": 20 * N + 4 * Mi,   # read mult*dy; read x, z, T; write x, z
        "prior": 48 * N,               # dTV: read x, q(3), z, T, v; write x, q(3), z
    }[kind]


# ------------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, one data and one prior iteration of the workload
# ------------------------------------------------------------------------------------------

def oracle_sample(sc, d, subset=5):
    """One data iteration on `subset` and one dTV prior iteration of the FP64 oracle, each from the
    setup state (x = max(x_true, 0), y = z = q = 0), timed on the host cores.  Returns the seconds
    of each, the thread count and the two states (the data iteration's y and z = P_i^T dy, the prior
    iteration's q and z = A_n^T dq) that the GPU's iterations are compared with.  The oracle's full T
    needs every subset's backprojection (minutes at this size), so the primal step here uses a
    stand-in T; the compared arrays do not depend on T."""
    import oracle
    from oracle import algorithms as O
    oracle.build()
    prob = O.Problem(sc, d["b"].astype(np.float64), d["r"].astype(np.float64), d["mult"].astype(np.float64))
    prior = O.Prior("dtv", alpha=ALPHA, side=d["side"].astype(np.float64))
    probs = O.probabilities(sc.n_subsets, prior)
    # the data block's sigma from its own projection of ones (Eq. EQU:STEPSIZE:PRECOND)
    a1 = O.project(sc, np.ones(sc.image_shape), subset, prob.mult)
    sigma = np.where(a1 > 0, 0.99 / np.where(a1 > 0, a1, 1.0), 0.0)
    gn = O.grad_norm((sc.nx, sc.ny, sc.nz))
    steps = dict(sigma=sigma, T=np.full(sc.image_shape, 0.99 * probs[-1] / gn), sigma_prior=[0.99 / gn])
    x0 = np.maximum(d["x_true"].astype(np.float32), 0).astype(np.float64)
    t0 = time.perf_counter()
    st_d, _ = O.spdhg(prob, prior, [subset], probs, steps=steps, x0=x0)
    t1 = time.perf_counter()
    st_p, _ = O.spdhg(prob, prior, [sc.n_subsets], probs, steps=steps, x0=x0)
    t2 = time.perf_counter()
    mask = O.subset_mask(sc, subset)
    states = {"data": {"y": st_d.y[mask], "z": st_d.z.ravel()}, "prior": {"q": st_p.q[0].ravel(), "z": st_p.z.ravel()}}
    return t1 - t0, t2 - t1, oracle.threads(), states


def cpu_baseline_entry(sc, td, tp, cores):
    m = sc.n_subsets
    epoch_s = m * td + m * tp  # 2m iterations, half data, half prior in expectation
    return {"value": 1.0 / epoch_s, "unit": "epoch/s", "cores": cores, "kind": "oracle",
            "sample": f"1 data + 1 dTV prior iteration of the mMR-scale workload (FP64 oracle), "
                      f"{td:.2f} s + {tp:.2f} s, extrapolated to one epoch of {m} + {m} iterations"}


def parity_entry(ctx, sc, d, params, states, subset=5):
    """The GPU's data and prior iterations from the same setup state as the oracle sample, compared
    array by array: relative L2 and max |gpu - oracle| / max |oracle| (the precision policy's
    error report: FP32 kernels against the FP64 oracle)."""
    import torch
    from oracle import algorithms as O
    dev = torch.device("cuda", torch.cuda.current_device())
    x0 = torch.from_numpy(np.maximum(d["x_true"].astype(np.float32), 0).ravel()).to(dev)
    out = {}
    mask = O.subset_mask(sc, subset).ravel()
    for name, blocks, keys in (("data_iteration", [subset], ("y", "z")), ("prior_iteration", [sc.n_subsets], ("q", "z"))):
        ctx.spdhg_setup(params, x0)
        ctx.spdhg_iterate(blocks)
        ref = states["data" if name == "data_iteration" else "prior"]
        res = {}
        for k in keys:
            n = {"y": sc.n_bins, "z": sc.n_voxels, "q": 3 * sc.n_voxels}[k]
            t = torch.zeros(n, device=dev)
            ctx.spdhg_get(k, t)
            g = t.cpu().numpy().astype(np.float64)
            if k == "y":
                g = g[mask]
            r = ref[k]
            res[k] = {"rel_l2": float(np.linalg.norm(g - r) / max(np.linalg.norm(r), 1e-300)),
                      "max_err": float(np.abs(g - r).max() / max(np.abs(r).max(), 1e-300)), "n": int(r.size)}
        out[name] = res
    out["what"] = (f"one data iteration (subset {subset}: y on its {int(mask.sum())} bins, z = P_i^T dy on all voxels) "
                   "and one dTV prior iteration (q, z on all voxels) from x = max(x_true, 0), GPU FP32 vs FP64 oracle")
    return out


# ------------------------------------------------------------------------------------------

def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    sc, d = make_workload()
    vals = []
    cores = 0
    for k in range(args.warmup + args.steps):
        td, tp, cores, _ = oracle_sample(sc, d)
        if k >= args.warmup:
            vals.append((td, tp))
    m = sc.n_subsets
    step_s = statistics.median([td + tp for td, tp in vals])
    epoch_s = m * step_s
    value = 1.0 / epoch_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "epoch/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * step_s,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": "1 data + 1 dTV prior iteration of the FP64 oracle (measured)"},
            "extrapolation": {"epoch_s": epoch_s, "iterations_per_epoch": 2 * m,
                              "what": f"value = 1 / ({m} x median step time): one epoch is {m} data + {m} prior "
                                      "iterations in expectation (balanced sampling); ms_per_step is the measured "
                                      "time of one step"},
            "cpu_baseline": {"value": value, "unit": "epoch/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} timed steps of 1 data + 1 dTV prior iteration of the mMR-scale "
                                       f"workload (after {args.warmup} untimed), extrapolated to {m} + {m} iterations"},
            "e2e": {"value": value, "unit": "epoch/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    import paper_1808_07150_gb300 as pkg
    from paper_1808_07150_gb300 import _build_ext

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    _build_ext.build()
    dev = torch.device("cuda", torch.cuda.current_device())

    sc, d = make_workload()
    N, M = sc.n_voxels, sc.n_bins
    params = pkg.make_params("dtv", alpha=ALPHA, dtv_gamma=0.995, dtv_eta_frac=0.01, seed=SEED)

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, np.float32).ravel()).to(dev)

    ctx = pkg.Context(sc)
    ctx.spdhg_set_data(to_dev(d["b"]), to_dev(d["r"]), to_dev(d["mult"]), to_dev(d["side"]))
    ctx.spdhg_setup(params)
    probs = ctx.spdhg_probabilities()
    m = sc.n_subsets
    ipe = int(round(m / probs[:m].sum()))
    seqs = [pkg.spdhg_sample(SEED, e * ipe, ipe, probs) for e in range(args.warmup + args.steps)]
    stream = torch.cuda.current_stream()

    for e in range(args.warmup):
        ctx.spdhg_iterate(seqs[e])
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    clocks = ClockSampler(torch.cuda.current_device())
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for e in range(args.warmup, args.warmup + args.steps):
        ctx.spdhg_iterate(seqs[e])
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    # the same epochs again with the library's per-launch events (an event between two launches
    # keeps the second from starting early, so the epoch time above is taken without them)
    ctx.spdhg_profile(True)
    for e in range(args.warmup, args.warmup + args.steps):
        ctx.spdhg_iterate(seqs[e])
    torch.cuda.synchronize()
    prof = ctx.spdhg_profile_read()
    ctx.spdhg_profile(False)
    ms = max_over_ranks(ms, dev)
    ms_per_epoch = ms / args.steps
    value = aggregate_rate(args.steps, ws, ms / 1e3)

    # roofline of the dominant kernel (per-launch CUDA events on the launching stream)
    dom = max(("forward", "backward", "prior"), key=lambda k: prof[k][0])
    dom_ms, dom_n = prof[dom]
    peak, peak_src = measured_peaks()
    per_launch = kernel_bytes(sc, dom)
    achieved = per_launch / (dom_ms / dom_n / 1e3) / 1e9
    epoch_bytes = sum(kernel_bytes(sc, k) * prof[k][1] for k in ("forward", "backward", "prior")) / args.steps
    launches = int(sum(v[1] for v in prof.values()))

    # end to end through the public API with host buffers: set_data + spdhg_run(K epochs) + x back
    pin = {k: torch.from_numpy(np.ascontiguousarray(d[k], np.float32).ravel()).pin_memory()
           for k in ("b", "r", "mult", "side")}
    x_host = torch.zeros(N, dtype=torch.float32).pin_memory()
    e2e_params = pkg.make_params("dtv", alpha=ALPHA, dtv_gamma=0.995, dtv_eta_frac=0.01, seed=SEED,
                                 epochs=args.steps)
    ctx2 = pkg.Context(sc)
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx2.spdhg_set_data(pin["b"], pin["r"], pin["mult"], pin["side"])
    ctx2.spdhg_run(e2e_params, x_host)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    barrier()
    e2e_s = max_over_ranks(e2e_s, dev)
    ctx2.close()
    h2d = (3 * M + 2 * N) * 4 / args.steps
    d2h = N * 4 / args.steps

    # time to a 1e-3 relative objective gap (Sec. 4), stop decided by the library: Psi* from a
    # longer run; SPDHG+ from zero with kernels launched one by one, and with epoch graphs
    ttg = None
    if not args.no_time_to_gap:
        ref = ctx.spdhg_run(pkg.make_params("dtv", alpha=ALPHA, dtv_gamma=0.995, dtv_eta_frac=0.01, seed=SEED,
                                            epochs=REF_EPOCHS, objective_every=REF_EPOCHS), None)
        psi_star = float(ref["objective"][-1])
        ttg = {"gap": GAP, "psi_star_epochs": REF_EPOCHS, "max_epochs": MAX_GAP_EPOCHS}
        for mode, graph in (("spdhg_plus_eager", False), ("spdhg_plus_graph", True)):
            rep = ctx.spdhg_run(pkg.make_params("dtv", alpha=ALPHA, dtv_gamma=0.995, dtv_eta_frac=0.01, seed=SEED,
                                                epochs=MAX_GAP_EPOCHS, graph=graph, target_gap=GAP,
                                                psi_star=psi_star), None)
            ttg[mode] = {"epochs": rep["stop_epoch"], "solver_s": rep["ms_to_stop"] / 1e3}
        ttg["what"] = ("solver device time from zero until (Psi - Psi*) / (Psi(0) - Psi*) <= 1e-3, checked by "
                       "spdhg_run after every epoch (objective evaluations excluded); Psi* = Psi after "
                       f"{REF_EPOCHS} epochs")

    cpu = None
    parity = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        td, tp, cores, states = oracle_sample(sc, d)
        cpu = cpu_baseline_entry(sc, td, tp, cores)
        parity = parity_entry(ctx, sc, d, params, states)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "epoch/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_epoch, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "step": f"one SPDHG+ epoch = {ipe} iterations (balanced sampling)",
                       "prior": f"dTV alpha={ALPHA}", "parallelism": f"replicas x{ws}",
                       "l2": "no flush: each iteration streams >= 0.36 GB (> 126 MB L2)"},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_source": f"{peak_src} hbm_gbs",
                         "traffic": traffic_from_profiles(dom), "algorithmic_bytes_per_launch": per_launch,
                         "avg_launch_ms": dom_ms / dom_n},
            "epoch_algorithmic_gbs": epoch_bytes / (ms_per_epoch / 1e3) / 1e9,
            "kernels": {k: {"ms_total": v[0], "launches": v[1]} for k, v in prof.items() if v[1]},
            "gpu_launches": launches,
            "e2e": {"value": aggregate_rate(args.steps, ws, e2e_s), "unit": "epoch/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h),
                    "what": "spdhg_set_data + spdhg_run(steps epochs) from pinned host buffers, x read back"},
            "clocks": clk,
        }
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if parity is not None:
            line["parity"] = parity
        if ttg is not None:
            line["time_to_gap"] = ttg
        print(json.dumps(line), flush=True)
    ctx.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------------------------------
# batched workload: 16 uneven reconstructions in one graph launch per epoch
# ------------------------------------------------------------------------------------------

BATCH_WORKLOAD = "batch16-uneven-96^3..200x200x100-120..252v-tv/tgv"


def make_batch():
    """16 seeded problems: sizes and views from synth.batch_geometries, counts log-uniform in
    [1e6, 5e8], TV (alpha 0.05) and TGV (alpha0 0.2, alpha1 0.1) alternating."""
    import synth
    gs = synth.batch_geometries(SEED, 16)
    rng = np.random.default_rng(SEED)
    counts = np.exp(rng.uniform(np.log(1e6), np.log(5e8), len(gs)))
    kinds = ["tv" if k % 2 == 0 else "tgv" for k in range(len(gs))]
    data = [synth.make_problem(sc, SEED + k, counts=float(counts[k]), bg_frac=0.1, with_mult=True,
                               with_side=False, n_ellipsoids=8) for k, sc in enumerate(gs)]
    return gs, kinds, counts, data


def run_batch(args):
    import torch

    import paper_1808_07150_gb300 as pkg
    from paper_1808_07150_gb300 import _build_ext
    torch.cuda.set_device(0)
    _build_ext.build()
    dev = torch.device("cuda", 0)
    gs, kinds, counts, data = make_batch()
    n = len(gs)

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, np.float32).ravel()).to(dev)

    ctxs = [pkg.Context(sc) for sc in gs]
    for c, d in zip(ctxs, data):
        c.spdhg_set_data(to_dev(d["b"]), to_dev(d["r"]), to_dev(d["mult"]))

    def params(k, epochs, graph, every=0):
        return pkg.make_params(kinds[k], alpha=ALPHA, alpha0=0.2, alpha1=0.1, seed=SEED + k, epochs=epochs,
                               objective_every=every, graph=graph)

    def zeros():
        return [torch.zeros(sc.n_voxels, device=dev) for sc in gs]

    # launch shapes per problem, measured on its own data
    tuned = []
    for k, c in enumerate(ctxs):
        c.spdhg_setup(params(k, 1, False))
        tuned.append(c.spdhg_autotune())

    # throughput: K epochs of all 16, device time of the epoch graphs (setup excluded)
    pkg.spdhg_run_batch(ctxs, [params(k, args.warmup, True) for k in range(n)], zeros())
    clocks = ClockSampler(0)
    torch.cuda.synchronize()
    clocks.start()
    t0 = time.perf_counter()
    reps = pkg.spdhg_run_batch(ctxs, [params(k, args.steps, True) for k in range(n)], zeros())
    torch.cuda.synchronize()
    wall_batch = time.perf_counter() - t0
    clk = clocks.stop()
    ms_batch = float(np.sum(reps[0]["epoch_ms"]))
    # the same epochs one problem at a time, kernels launched one by one
    t0 = time.perf_counter()
    ms_seq = 0.0
    for k, c in enumerate(ctxs):
        r = c.spdhg_run(params(k, args.steps, False), zeros()[k])
        ms_seq += float(np.sum(r["epoch_ms"]))
    torch.cuda.synchronize()
    wall_seq = time.perf_counter() - t0

    # per-kernel time of one eager epoch of every problem (library profiler)
    prof_tot = {}
    for k, c in enumerate(ctxs):
        c.spdhg_setup(params(k, 1, False))
        probs = c.spdhg_probabilities()
        m = gs[k].n_subsets
        ipe = int(round(m / probs[:m].sum()))
        c.spdhg_profile(True)
        c.spdhg_iterate(pkg.spdhg_sample(SEED + k, 0, ipe, probs))
        for kk, (ms, cnt) in c.spdhg_profile_read().items():
            a = prof_tot.setdefault(kk, [0.0, 0])
            a[0] += ms
            a[1] += cnt
        c.spdhg_profile(False)

    # time to a relative objective gap of 1e-3: Psi* from a long run, then the first epoch that
    # reaches the gap; then both ways timed on exactly those epochs, solver only
    long_epochs, max_epochs = 150, 60
    ref = pkg.spdhg_run_batch(ctxs, [params(k, long_epochs, True, every=long_epochs) for k in range(n)],
                              zeros())
    log = pkg.spdhg_run_batch(ctxs, [params(k, max_epochs, True, every=1) for k in range(n)], zeros())
    reach = []
    for k in range(n):
        o = log[k]["objective"]
        psi_star = min(float(np.nanmin(ref[k]["objective"])), float(np.nanmin(o)))
        gap = (o - psi_star) / (o[0] - psi_star)
        hit = np.nonzero(gap[1:] <= GAP)[0]
        reach.append(int(hit[0]) + 1 if hit.size else max_epochs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rb = pkg.spdhg_run_batch(ctxs, [params(k, reach[k], True) for k in range(n)], zeros())
    torch.cuda.synchronize()
    gap_wall_batch = time.perf_counter() - t0
    gap_ms_batch = float(max(np.sum(r["epoch_ms"]) for r in rb))
    t0 = time.perf_counter()
    gap_ms_seq = 0.0
    for k, c in enumerate(ctxs):
        r = c.spdhg_run(params(k, reach[k], False), zeros()[k])
        gap_ms_seq += float(np.sum(r["epoch_ms"]))
    torch.cuda.synchronize()
    gap_wall_seq = time.perf_counter() - t0

    value = n * args.steps / (ms_batch / 1e3)
    line = {
        "metric": METRIC, "value": value, "unit": "reconstruction-epoch/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_batch / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": BATCH_WORKLOAD, "step": "one epoch (2m iterations) of all 16 reconstructions",
                   "problems": [f"{sc.name} {kk} m={sc.n_subsets} counts={c:.3g}"
                                for sc, kk, c in zip(gs, kinds, counts)],
                   "l2": "no flush: the 16 problems hold 2.3 GB, far above L2, and run in turn within an epoch"},
        "sequential_eager": {"value": n * args.steps / (ms_seq / 1e3), "unit": "reconstruction-epoch/s",
                             "what": "the same epochs, one problem at a time, kernels launched one by one"},
        "wall_s": {"batch": wall_batch, "sequential_eager": wall_seq, "what": "incl. per-problem setup"},
        "time_to_gap": {"gap": GAP, "epochs": reach, "batch_graph_s": gap_ms_batch / 1e3,
                        "sequential_eager_s": gap_ms_seq / 1e3, "batch_wall_s": gap_wall_batch,
                        "sequential_wall_s": gap_wall_seq,
                        "what": "solver device time to bring every problem to (Psi - Psi*) / (Psi(0) - Psi*) <= 1e-3; "
                                "Psi* = min objective of a 150-epoch run; wall includes setup"},
        "kernels_one_epoch_each": {k: {"ms_total": v[0], "launches": v[1]} for k, v in prof_tot.items() if v[1]},
        "autotuned": tuned,
        "gpu_launches": int(sum(v[1] for v in prof_tot.values())) * args.steps,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    for c in ctxs:
        c.close()
    return 0


# ------------------------------------------------------------------------------------------
# learned warm start: U-Net on the 3-D scanner, time to a 1e-3 gap against SPDHG+ from zero
# ------------------------------------------------------------------------------------------

WS_WORKLOAD = "warmstart-cyl3d-oblique-128x128x64-180v128r64p-tv-21subsets-unet16-32-64-128"


def unet_flops_per_sample(shape, channels):
    """Multiply-adds x 2 of one training step (forward, data and weight gradients) of every
    convolution, with the true input channel count (1) of the first layer."""
    ny, nx, nz = shape
    L = len(channels)
    V = [ny * nx * nz // 8 ** l for l in range(L)]
    f = 0
    cin = 1
    for l in range(L):
        a = V[l] * 27 * cin * channels[l]
        b = V[l] * 27 * channels[l] * channels[l]
        f += a * (2 if l == 0 else 3) + 3 * b       # no data gradient into the input
        cin = channels[l]
    for l in range(L - 2, -1, -1):
        f += 3 * V[l + 1] * 8 * channels[l + 1] * channels[l]
        f += 3 * V[l] * 27 * 2 * channels[l] * channels[l] + 3 * V[l] * 27 * channels[l] * channels[l]
    return 2 * f


def run_warmstart(args):
    import torch

    import paper_1808_07150_gb300 as pkg
    import synth
    from paper_1808_07150_gb300 import _build_ext, learned, warmstart as W
    torch.cuda.set_device(0)
    _build_ext.build()
    sc = synth.config_3d_oblique()
    k, ref_epochs, max_epochs, group = args.k, 60, 30, 32
    channels = (16, 32, 64, 128)
    alpha = 0.05
    seeds_train = list(range(args.n_train))
    seeds_test = list(range(10000, 10000 + args.n_test))

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, np.float32).ravel()).cuda()

    def problem(seed):
        return synth.make_problem(sc, seed, counts=3e7, bg_frac=0.1, with_mult=True, with_side=False,
                                  n_ellipsoids=8)

    def params(seed, **kw):
        return pkg.make_params("tv", alpha=alpha, seed=SEED + seed, **kw)

    t_data = time.perf_counter()
    xk, xs, test_ctx, test_ref = [], [], [], []
    for start in range(0, len(seeds_train) + len(seeds_test), group):
        chunk = (seeds_train + seeds_test)[start:start + group]
        ctxs = []
        for s_ in chunk:
            d = problem(s_)
            c = pkg.Context(sc)
            c.spdhg_set_data(to_dev(d["b"]), to_dev(d["r"]), to_dev(d["mult"]))
            ctxs.append(c)
        a, b = W.pairs(ctxs, [params(s_) for s_ in chunk], k, ref_epochs)
        for c, s_, xa, xb in zip(ctxs, chunk, a, b):
            if s_ < 10000:
                xk.append(xa)
                xs.append(xb)
                c.close()
            else:
                test_ctx.append((c, s_, xa))
                test_ref.append(xb)
    t_data = time.perf_counter() - t_data

    # training on the tensor cores
    net = learned.UNet(sc.image_shape, channels)
    net.init(SEED)
    for _ in range(2):  # warm-up of every kernel
        net.forward(xk[0], 0.0)
        net.backward(xs[0], want_loss=False)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    losses = W.train(net, xk, xs, epochs=args.train_epochs, lr=1e-3, batch=4, seed=SEED)
    ev1.record()
    torch.cuda.synchronize()
    train_ms = ev0.elapsed_time(ev1)
    steps = args.train_epochs * len(xk)
    flops = unet_flops_per_sample(sc.image_shape, channels)
    achieved_tflops = flops * steps / (train_ms / 1e3) / 1e12
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except Exception:
        pass
    bf16_peak = peaks.get("bf16_tflops_sustained") or peaks.get("bf16_tflops") or 1700.0

    # evaluation: epochs and solver time to a relative objective gap of 1e-3
    res = {"plain": [], "continue": [], "restart": []}
    net_ms = []
    gap_xk, gap_x0, dist_ratio = [], [], []
    zero = torch.zeros(sc.n_voxels, device="cuda")
    for (ctx, s_, xa), xref in zip(test_ctx, test_ref):
        p = params(s_)
        ctx.spdhg_setup(p, None)
        psi0 = ctx.spdhg_objective(zero)[2]
        psi_star = ctx.spdhg_objective(xref)[2]
        obj, ms = W.run_epochs(ctx, p, max_epochs, 0)
        psi_star = min(psi_star, float(obj.min()))
        # checkpoints (cumulative solver ms, objective): after every epoch, and for the warm
        # starts also right after the network (the objective at x0)
        runs = {"plain": list(zip(np.cumsum(ms), obj[1:]))}
        for mode in ("continue", "restart"):
            ctx.spdhg_setup(p, None)
            ok_, msk = W.run_epochs(ctx, p, k, 0)
            x0 = torch.zeros(sc.n_voxels, device="cuda")
            xcur = torch.zeros(sc.n_voxels, device="cuda")
            ctx.spdhg_get("x", xcur)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            net.forward(xcur, 0.0, None, x0)
            b.record()
            torch.cuda.synchronize()
            t_net = a.elapsed_time(b)
            net_ms.append(t_net)
            if mode == "continue":
                gap_xk.append(float((ok_[-1] - psi_star) / (psi0 - psi_star)))
                gap_x0.append(float((ctx.spdhg_objective(torch.clamp(x0, min=0))[2] - psi_star) / (psi0 - psi_star)))
                dist_ratio.append(float(torch.linalg.vector_norm(torch.clamp(x0, min=0) - xref) /
                                        torch.linalg.vector_norm(xcur - xref)))
                W.continue_from(ctx, x0)
            else:
                W.restart_from(ctx, x0, "tv")
            ow, msw = W.run_epochs(ctx, p, max_epochs - k, k)
            psi_star = min(psi_star, float(ow.min()))
            t0 = float(np.sum(msk)) + t_net
            runs[mode] = (list(zip(np.cumsum(msk), ok_[1:])) + [(t0, ow[0])] +
                          list(zip(t0 + np.cumsum(msw), ow[1:])))
        for mode, chk in runs.items():
            hit = [(i, t) for i, (t, o) in enumerate(chk) if (o - psi_star) / (psi0 - psi_star) <= GAP]
            res[mode].append(hit[0] if hit else (None, None))
    assert learned.device_error() == 0

    def summary(v):
        hit = [x for x in v if x[0] is not None]
        return {"reached": len(hit), "of": len(v),
                "mean_checkpoint": float(np.mean([x[0] + 1 for x in hit])) if hit else None,
                "mean_ms": float(np.mean([x[1] for x in hit])) if hit else None}

    summ = {m: summary(v) for m, v in res.items()}
    best = min(("continue", "restart"), key=lambda m: summ[m]["mean_ms"] or 1e30)
    line = {
        "metric": METRIC, "value": summ[best]["mean_ms"], "unit": "ms to 1e-3 rel. objective gap (mean)",
        "n_gpus": 1, "steps": steps, "warmup": 2, "ms_per_step": train_ms / steps,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (U-Net) / f32 (SPDHG+)",
        "data": "synthetic",
        "config": {"workload": WS_WORKLOAD, "train_problems": len(xk), "test_problems": len(test_ctx),
                   "k_epochs_before_net": k, "reference_epochs": ref_epochs, "train_epochs": args.train_epochs,
                   "step": "value: mean solver time to gap 1e-3 with the learned warm start; ms_per_step: one "
                           "U-Net training step (forward + backward) on one 128x128x64 sample"},
        "time_to_gap": {"plain_zero_start": summ["plain"], "warm_continue": summ["continue"],
                        "warm_restart": summ["restart"], "best_warm": best,
                        "speedup_mean_ms": (summ["plain"]["mean_ms"] / summ[best]["mean_ms"])
                        if summ["plain"]["mean_ms"] and summ[best]["mean_ms"] else None,
                        "net_inference_ms": float(np.mean(net_ms)),
                        "median_gap_at_x_k": float(np.median(gap_xk)), "median_gap_at_x0": float(np.median(gap_x0)),
                        "mean_dist_x0_over_dist_x_k_to_x_star": float(np.mean(dist_ratio)),
                        "note": "gaps use the Psi* of each problem as finally estimated"},
        "training": {"loss_first_epoch": losses[0], "loss_last_epoch": losses[-1], "ms_total": train_ms,
                     "samples_per_s": steps / (train_ms / 1e3), "data_generation_s": t_data},
        "roofline": {"bound": "tensor", "kernel": "k_igemm (all U-Net convolution passes, one training step)",
                     "achieved": achieved_tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                     "frac": achieved_tflops / bf16_peak, "traffic": None,
                     "algorithmic_flops_per_step": flops,
                     "note": "whole training step (incl. pooling, head, loss, Adam) timed; of measured bf16 peak"},
    }
    print(json.dumps(line), flush=True)
    net.close()
    for c, _, _ in test_ctx:
        c.close()
    return 0


# ------------------------------------------------------------------------------------------
# the paper's comparison: SPDHG (scalar steps) against SPDHG+ (preconditioned), from zero
# ------------------------------------------------------------------------------------------

PRECOND_WORKLOAD = "precond-cyl3d-oblique-128x128x64-180v128r64p-tv-21subsets"


def run_precond(args):
    import torch

    import paper_1808_07150_gb300 as pkg
    import synth
    from paper_1808_07150_gb300 import _build_ext, warmstart as W
    torch.cuda.set_device(0)
    _build_ext.build()
    sc = synth.config_3d_oblique()
    n_prob, max_plus, max_plain, ref_epochs = 8, 30, 120, 120

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, np.float32).ravel()).cuda()

    out = {"spdhg_plus": [], "spdhg_scalar": []}
    setup_s = {"spdhg_plus": [], "spdhg_scalar": []}
    zero = torch.zeros(sc.n_voxels, device="cuda")
    for k in range(n_prob):
        d = synth.make_problem(sc, 20000 + k, counts=3e7, bg_frac=0.1, with_mult=True, with_side=False,
                               n_ellipsoids=8)
        with pkg.Context(sc) as ctx:
            ctx.spdhg_set_data(to_dev(d["b"]), to_dev(d["r"]), to_dev(d["mult"]))
            logs = {}
            for name, pre, ep in (("spdhg_plus", True, max_plus), ("spdhg_scalar", False, max_plain)):
                p = pkg.make_params("tv", alpha=ALPHA, seed=SEED + k, precond=pre)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ctx.spdhg_setup(p, None)
                torch.cuda.synchronize()
                setup_s[name].append(time.perf_counter() - t0)
                logs[name] = W.run_epochs(ctx, p, ep, 0)
            p = pkg.make_params("tv", alpha=ALPHA, seed=SEED + k, precond=True, epochs=ref_epochs,
                                objective_every=ref_epochs, graph=True)
            rep = ctx.spdhg_run(p, None)
            psi_star = min(float(np.nanmin(rep["objective"])), *(float(o.min()) for o, _ in logs.values()))
            psi0 = ctx.spdhg_objective(zero)[2]
            for name, (obj, ms) in logs.items():
                e = W.first_epoch_at(obj, psi0, psi_star, GAP)
                out[name].append((e, float(np.sum(ms[:e])) if e else None,
                                  float((obj[-1] - psi_star) / (psi0 - psi_star))))

    def summary(v, cap):
        hit = [x for x in v if x[0] is not None]
        return {"reached": len(hit), "of": len(v), "max_epochs": cap,
                "mean_epochs": float(np.mean([x[0] for x in hit])) if hit else None,
                "mean_ms": float(np.mean([x[1] for x in hit])) if hit else None,
                "median_final_gap": float(np.median([x[2] for x in v]))}

    plus, scal = summary(out["spdhg_plus"], max_plus), summary(out["spdhg_scalar"], max_plain)
    line = {
        "metric": METRIC, "value": plus["mean_ms"], "unit": "ms to 1e-3 rel. objective gap (mean, SPDHG+)",
        "n_gpus": 1, "steps": n_prob, "warmup": 0, "ms_per_step": plus["mean_ms"], "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": PRECOND_WORKLOAD, "problems": n_prob, "seeds": "20000..20007",
                   "step": "one seeded problem solved to a relative objective gap of 1e-3 from zero"},
        "spdhg_plus": plus, "spdhg_scalar": scal,
        "speedup_epochs": (scal["mean_epochs"] / plus["mean_epochs"]) if scal["mean_epochs"] and plus["mean_epochs"] else None,
        "setup_s": {k: float(np.mean(v)) for k, v in setup_s.items()},
        "note": "Psi* = minimum objective of a 120-epoch SPDHG+ run and of both logs; setup (step sizes, "
                "incl. the power iterations of the scalar form) excluded from the solver time",
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------------------------------
# the paper's OSEM comparison (Sec. 1.3): MLEM, OSEM and SPDHG+ without a prior on the 3-D scanner
# ------------------------------------------------------------------------------------------

OSEM_WORKLOAD = "osem-cyl3d-oblique-128x128x64-180v128r64p-ml-21subsets"


def run_osem(args):
    """Unregularised reconstruction (alpha = 0) of the 3-D scanner by MLEM (Eq. EQU:MLEM), OSEM
    (Eq. EQU:OSEM, 21 view subsets) and SPDHG+ (21 and 180 view subsets, uniform sampling), each
    logged by PSNR against x* = MLEM after many iterations (the reference of the paper's Fig. 3;
    PSNR as printed, with the 2-norm of the whole image, so its values are negative at this image
    size); then the stability example of Sec. 1.3: OSEM and SPDHG+ with 21 bin-interleaved
    subsets.  The headline value is the solver time SPDHG+ with 180 subsets needs to reach the
    PSNR that OSEM with 21 subsets has after 10 epochs (the paper's Fig. 4 comparison point)."""
    import torch

    import paper_1808_07150_gb300 as pkg
    import synth
    from paper_1808_07150_gb300 import _build_ext
    torch.cuda.set_device(0)
    _build_ext.build()
    sc = synth.config_3d_oblique()
    d = synth.make_problem(sc, SEED, counts=3e7, bg_frac=0.1, with_mult=True, with_side=False, n_ellipsoids=8)

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, np.float32).ravel()).cuda()

    ref_iters, epochs = 2000, 50
    out = {}
    runs_done = {}
    for name, m, kind in (("views21", 21, "views"), ("views180", 180, "views"), ("bins21", 21, "bins")):
        g = sc.with_subsets(m, kind)
        with pkg.Context(g) as ctx:
            ctx.spdhg_set_data(to_dev(d["b"]), to_dev(d["r"]), to_dev(d["mult"]))
            if "x_star" not in runs_done:
                x_star = torch.ones(sc.n_voxels, device="cuda")
                ctx.spdhg_osem(pkg.make_params("none", epochs=ref_iters), x_star, mlem=True)
                runs_done["x_star"] = x_star
                rep = ctx.spdhg_osem(pkg.make_params("none", epochs=epochs, x_star=x_star), None, mlem=True)
                out["mlem"] = rep
            x_star = runs_done["x_star"]
            p = pkg.make_params("none", seed=SEED, sampling="uniform", epochs=epochs, x_star=x_star)
            if name != "views180":
                out[f"osem_{name}"] = ctx.spdhg_osem(p, None)
            out[f"spdhg_plus_{name}"] = ctx.spdhg_run(p, None)
    target = float(out["osem_views21"]["psnr"][10])
    summ = {k: _psnr_summary(v, (target,)) for k, v in out.items()}
    best = summ["spdhg_plus_views180"]["ms_to_psnr"][str(target)]
    line = {
        "metric": METRIC, "value": best,
        "unit": "ms (SPDHG+, 180 subsets) to the PSNR of OSEM (21 subsets) after 10 epochs",
        "n_gpus": 1, "steps": epochs, "warmup": 0, "ms_per_step": summ["spdhg_plus_views180"]["ms_per_epoch"],
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": OSEM_WORKLOAD, "x_star": f"MLEM after {ref_iters} iterations",
                   "psnr_target_db": target,
                   "step": "one epoch: MLEM one iteration; OSEM and SPDHG+ one pass over their subsets"},
        "methods": summ,
        "note": "bin subsets: bin j in subset j mod 21 (every subset iteration is a full projection); "
                "PSNR = 20 log10(max|x*| / ||x - x*||_2) as printed in Sec. 4; solver device time "
                "(evaluations excluded)",
    }
    print(json.dumps(line), flush=True)
    return 0


def _psnr_summary(rep, thresholds):
    ps = rep["psnr"][1:]
    ms = np.cumsum(rep["epoch_ms"])
    res = {"final_psnr": float(ps[-1]), "psnr_every_5": [round(float(v), 3) for v in ps[4::5]],
           "ms_per_epoch": float(np.mean(rep["epoch_ms"])), "epochs_to_psnr": {}, "ms_to_psnr": {}}
    for t in thresholds:
        hit = np.nonzero(ps >= t)[0]
        res["epochs_to_psnr"][str(t)] = int(hit[0]) + 1 if hit.size else None
        res["ms_to_psnr"][str(t)] = float(ms[hit[0]]) if hit.size else None
    return res


# ------------------------------------------------------------------------------------------
# per-configuration figures: GPU ms per epoch and time to a 1e-3 gap, the oracle's time per epoch
# ------------------------------------------------------------------------------------------

CONFIGS_WORKLOAD = "configs-2d-64x64-10subsets-tv0.1/3d-oblique-128x128x64-21subsets-tv0.05"


def _oracle_epoch_seconds(cfg, n_iter):
    """Seconds per epoch of the FP64 oracle on `cfg` ("2d" / "3d"), from n_iter timed iterations
    (balanced sampling, in the seeded sequence's order), measured in this process."""
    import oracle
    import synth
    from oracle import algorithms as O
    oracle.build()
    sc = synth.config_2d() if cfg == "2d" else synth.config_3d_oblique()
    alpha = 0.1 if cfg == "2d" else 0.05
    d = synth.make_problem(sc, SEED, counts=1e5 if cfg == "2d" else 3e7, bg_frac=0.05 if cfg == "2d" else 0.1,
                           with_mult=False)
    prob = O.Problem(sc, d["b"].astype(np.float64), d["r"].astype(np.float64), None)
    prior = O.Prior("tv", alpha=alpha)
    probs = O.probabilities(sc.n_subsets, prior)
    ipe = O.iters_per_epoch(sc.n_subsets, probs)
    t0 = time.perf_counter()
    steps = O.step_sizes(sc, None, prior, probs)
    t_setup = time.perf_counter() - t0
    seq = O.sample(SEED, n_iter, probs)
    t0 = time.perf_counter()
    O.spdhg(prob, prior, seq, probs, steps=steps)
    t_it = (time.perf_counter() - t0) / n_iter
    return {"s_per_epoch": t_it * ipe, "setup_s": t_setup, "iterations_timed": n_iter, "threads": oracle.threads()}


def run_configs(args):
    """GPU ms per epoch (CUDA events, eager launches) and solver time to a 1e-3 relative objective
    gap (the library's stopping rule, Psi* from a 300-epoch run) on the 2-D and 3-D
    configurations, next to the FP64 oracle's seconds per epoch with all host cores and with one
    thread (each from a bounded number of iterations, extrapolated to an epoch)."""
    import torch

    import paper_1808_07150_gb300 as pkg
    import synth
    from paper_1808_07150_gb300 import _build_ext
    torch.cuda.set_device(0)
    _build_ext.build()
    res = {}
    for cfg, sc, alpha, counts, bg, n_or in (("2d", synth.config_2d(), 0.1, 1e5, 0.05, 200),
                                             ("3d", synth.config_3d_oblique(), 0.05, 3e7, 0.1, 8)):
        d = synth.make_problem(sc, SEED, counts=counts, bg_frac=bg, with_mult=False)
        with pkg.Context(sc) as ctx:
            ctx.spdhg_set_data(torch.from_numpy(d["b"].ravel()).cuda(), torch.from_numpy(d["r"].ravel()).cuda())
            rep = ctx.spdhg_run(pkg.make_params("tv", alpha=alpha, seed=SEED, epochs=20), None)
            ms = float(np.median(rep["epoch_ms"][3:]))
            ref = ctx.spdhg_run(pkg.make_params("tv", alpha=alpha, seed=SEED, epochs=300, objective_every=300), None)
            psi_star = float(ref["objective"][-1])
            gap = ctx.spdhg_run(pkg.make_params("tv", alpha=alpha, seed=SEED, epochs=200, target_gap=GAP,
                                                psi_star=psi_star), None)
        N, m = sc.n_voxels, sc.n_subsets
        Mi = sc.n_bins / m
        epoch_bytes = m * (24 * N + 24 * Mi) + m * 44 * N  # data + TV prior iterations (FP32 arrays)
        res[cfg] = {"scanner": sc.name, "gpu_ms_per_epoch": ms, "algorithmic_gbs": epoch_bytes / (ms / 1e3) / 1e9,
                    "time_to_gap": {"epochs": gap["stop_epoch"], "solver_ms": gap["ms_to_stop"]}}
        res[cfg]["oracle_all_cores"] = _oracle_epoch_seconds(cfg, n_or)
        one = subprocess.run([sys.executable, "-c", f"import bench, json; print(json.dumps(bench._oracle_epoch_seconds("
                              f"'{cfg}', {max(2, n_or // 4)})))"], cwd=ROOT, capture_output=True, text=True,
                             env=dict(os.environ, OMP_NUM_THREADS="1"))
        res[cfg]["oracle_one_thread"] = json.loads(one.stdout.strip().splitlines()[-1]) if one.returncode == 0 else None
    line = {"metric": METRIC, "value": res["3d"]["gpu_ms_per_epoch"], "unit": "ms per epoch (3-D configuration)",
            "n_gpus": 1, "steps": 17, "warmup": 3, "ms_per_step": res["3d"]["gpu_ms_per_epoch"],
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": CONFIGS_WORKLOAD, "nproc": os.cpu_count()},
            "configs": res,
            "note": "the 3-D arrays (4 MB) stay in L2, so its algorithmic GB/s can exceed HBM bandwidth"}
    print(json.dumps(line), flush=True)
    return 0


def run_ncu_case():
    """Few launches with the per-launch work of the full workload on a few GB of device memory:
    the mMR-scale image and geometry with 28 views in 28 subsets (one view per subset, as in the
    252-subset workload; the backprojector's item table 28/252 of its full size).  Setup (28
    sensitivity backprojections, one sigma projection), then one data iteration (k_forward,
    k_backward; subset 1, the view at 6.4 degrees) and one dTV prior iteration (k_prior)."""
    import dataclasses

    import torch

    import paper_1808_07150_gb300 as pkg
    import synth
    from paper_1808_07150_gb300 import _build_ext
    torch.cuda.set_device(0)
    _build_ext.build()
    sc = dataclasses.replace(synth.config_mmr(), n_views=28, n_subsets=28, name="mmr-28v")
    d = synth.make_problem(sc, SEED, counts=4e8 * 28 / 252, bg_frac=0.1, with_mult=True, with_side=True)
    dev = torch.device("cuda", 0)

    def to_dev(a):
        return torch.from_numpy(np.ascontiguousarray(a, np.float32).ravel()).to(dev)

    with pkg.Context(sc) as ctx:
        ctx.spdhg_set_data(to_dev(d["b"]), to_dev(d["r"]), to_dev(d["mult"]), to_dev(d["side"]))
        ctx.spdhg_setup(pkg.make_params("dtv", alpha=ALPHA, dtv_gamma=0.995, dtv_eta_frac=0.01, seed=SEED))
        ctx.spdhg_iterate([1, sc.n_subsets])
        torch.cuda.synchronize()
    print("ncu case done")
    return 0


def run_ncu_unet():
    """Three training steps (forward, backward, Adam) of the 16-32-64-128 U-Net on a 128x128x64
    volume of seeded random values: the launches ncu captures for the tensor-core kernels."""
    import torch

    from paper_1808_07150_gb300 import _build_ext, learned
    torch.cuda.set_device(0)
    _build_ext.build()
    shape = (128, 128, 64)
    r = np.random.default_rng(SEED)
    x = torch.from_numpy(r.random(shape).astype(np.float32).ravel()).cuda()
    t = torch.from_numpy(r.random(shape).astype(np.float32).ravel()).cuda()
    with learned.UNet(shape, (16, 32, 64, 128)) as net:
        net.init(SEED)
        for _ in range(3):
            net.forward(x, 0.0)
            net.backward(t, want_loss=False)
            net.adam_step(1e-3)
        torch.cuda.synchronize()
        assert learned.device_error() == 0
    print("ncu unet case done")
    return 0


def main():
    args = parse()
    if args.ncu_case:
        return run_ncu_case()
    if args.ncu_unet:
        return run_ncu_unet()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch16":
        return run_batch(args)
    if args.workload == "warmstart":
        return run_warmstart(args)
    if args.workload == "precond":
        return run_precond(args)
    if args.workload == "osem":
        return run_osem(args)
    if args.workload == "configs":
        return run_configs(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
