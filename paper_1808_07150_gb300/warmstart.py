"""Learned warm start workflow on the library's kernels (no counterpart in the paper).

A 3-D U-Net (learned.UNet) maps the iterate x_k after k SPDHG+ epochs to a starting point x0;
Algorithm 2 then runs from x0, so only the starting point changes and the MAP solution does not.

* training pairs: (x_k, x*) from SPDHG+ runs of many problems, all problems of a group advancing
  together, one CUDA graph launch per epoch (spdhg_run_batch);
* training: Adam on the mean squared error of (pred, x*/s), s = mean(x_k), gradients averaged
  over mini-batches;
* warm start, two ways: "restart" starts Algorithm 2 again at x0 with zero duals; "continue" keeps
  the duals of the k epochs and replaces only the primal iterate (spdhg_set), which keeps the
  SPDHG state consistent (z = A^T y).

Every arithmetic step runs in libspdhg.so; this module sequences the calls.
"""
from __future__ import annotations

import numpy as np

from . import _capi, spdhg_run_batch, spdhg_sample
from .learned import UNet


def _params_with(params, **kw):
    p = _capi.Params()
    for name, _ in _capi.Params._fields_:
        setattr(p, name, getattr(params, name))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def iterations_per_epoch(ctx):
    probs = ctx.spdhg_probabilities()
    m = ctx.scanner.n_subsets
    return int(round(m / probs[:m].sum())), probs


def pairs(contexts, params, k_epochs, ref_epochs, device="cuda"):
    """x_k and x* (device float32 tensors) of every context: two batched runs from zero."""
    import torch
    n = len(contexts)
    xk = [torch.zeros(c.n_voxels, device=device) for c in contexts]
    xs = [torch.zeros(c.n_voxels, device=device) for c in contexts]
    spdhg_run_batch(contexts, [_params_with(params[i], epochs=k_epochs, graph=1) for i in range(n)], xk)
    spdhg_run_batch(contexts, [_params_with(params[i], epochs=ref_epochs, graph=1) for i in range(n)], xs)
    return xk, xs


def train(net: UNet, inputs, targets, epochs, lr, batch=4, seed=0):
    """Adam over the pairs; returns the mean loss of every epoch."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(epochs):
        order = rng.permutation(len(inputs))
        tot, cnt = 0.0, 0
        for j, i in enumerate(order):
            net.forward(inputs[i], 0.0)
            tot += net.backward(targets[i], accumulate=(j % batch) != 0)
            cnt += 1
            if (j % batch) == batch - 1 or j == len(order) - 1:
                net.adam_step(lr)
        out.append(tot / cnt)
    return out


def run_epochs(ctx, params, epochs, first_epoch=0):
    """Epochs first_epoch .. first_epoch+epochs-1 of SPDHG+ on the context's current state (after
    spdhg_setup), with the objective after each.  Returns (objective[epochs+1], device ms per
    epoch); objective[0] is the value before the first of these epochs."""
    import torch
    ipe, probs = iterations_per_epoch(ctx)
    obj = [ctx.spdhg_objective()[2]]
    ms = []
    stream = torch.cuda.current_stream()
    for e in range(first_epoch, first_epoch + epochs):
        seq = spdhg_sample(params.seed, e * ipe, ipe, probs)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        ctx.spdhg_iterate(seq)
        b.record(stream)
        obj.append(ctx.spdhg_objective()[2])
        ms.append(a.elapsed_time(b))
    return np.array(obj), np.array(ms)


def continue_from(ctx, x0):
    """Keep the duals, replace the primal iterate (a consistent SPDHG state)."""
    ctx.spdhg_set("x", x0)


def restart_from(ctx, x0, prior):
    """Start Algorithm 2 again at x0 with zero duals and the step sizes already set up (equal to
    spdhg_setup(params, x0) without recomputing them)."""
    import torch
    N, M = ctx.n_voxels, ctx.n_bins
    z = torch.zeros(max(6 * N, M), device="cuda")
    ctx.spdhg_set("y", z[:M])
    ctx.spdhg_set("z", z[:N])
    if prior != "none":
        ctx.spdhg_set("q", z[:3 * N])
    if prior == "tgv":
        ctx.spdhg_set("w", z[:3 * N])
        ctx.spdhg_set("zw", z[:3 * N])
        ctx.spdhg_set("q2", z[:6 * N])
    ctx.spdhg_set("x", x0)


def first_epoch_at(obj, psi0, psi_star, gap):
    """First index e >= 1 with (obj[e] - psi*) / (psi0 - psi*) <= gap, or None."""
    rel = (np.asarray(obj) - psi_star) / (psi0 - psi_star)
    hit = np.nonzero(rel[1:] <= gap)[0]
    return int(hit[0]) + 1 if hit.size else None
