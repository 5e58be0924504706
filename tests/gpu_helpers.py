"""Shared helpers of the GPU parity tests (CUDA path through the C ABI vs the FP64 oracle)."""
import numpy as np

import synth
from oracle import algorithms as O


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32).ravel()).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def maxerr(a, b):
    """Elementwise bound: max |a - b| / max |b| (a few wrong entries cannot hide in the norm)."""
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    mb = float(np.abs(b).max()) if b.size else 0.0
    return float(np.abs(a - b).max() / (mb if mb > 0 else 1.0)) if a.size else 0.0


def wide_2d(n_subsets=3):
    """Tiny 2-D geometry whose outer radial bins miss the image (A_i 1 = 0 there)."""
    return synth.Scanner(nx=8, ny=8, nz=1, vx=1.0, vy=1.0, vz=1.0, n_radial=15, d_radial=1.0,
                         n_views=6, radius=20.0, seg_n=(1,), seg_zmid0=(0.0,), seg_dzmid=(1.0,),
                         seg_dz=(0.0,), n_subsets=n_subsets, name="wide2d")


def problem(sc, seed=3, counts=2e4, mult=True, side=False):
    d = synth.make_problem(sc, seed, counts=counts, bg_frac=0.1, with_mult=mult, with_side=side,
                           n_ellipsoids=4)
    prob = O.Problem(sc, d["b"].astype(np.float64), d["r"].astype(np.float64),
                     None if d["mult"] is None else d["mult"].astype(np.float64))
    return d, prob


def upload(ctx, d):
    ctx.spdhg_set_data(dev(d["b"]), dev(d["r"]), None if d["mult"] is None else dev(d["mult"]),
                       None if d.get("side") is None else dev(d["side"]))
