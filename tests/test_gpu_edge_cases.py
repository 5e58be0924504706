"""Degenerate and ragged inputs of the CUDA path against the FP64 oracle (40 SPDHG iterations,
relative L2 <= 1e-4 as in test_gpu_iterations).

* zero counts everywhere: the KL prox takes its b = 0 branch (y+ = min(w, 1));
* one subset (n = 2 blocks with a prior), and one view per subset (m = n_views);
* voxels that no LOR crosses: T = 0 there (no block bounds them), so they keep max(x0, 0);
* a non-square image (nx != ny) and an axial extent beyond 128 slices (the wider register
  paths of the backprojector and the prior kernel).
"""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import algorithms as O

from gpu_helpers import dev, host, problem, rel, upload

pytestmark = pytest.mark.gpu


def _run(sc, d, prob, kind, seed=99, n_iter=40, x0=None):
    import torch
    import paper_1808_07150_gb300 as pkg
    prior = None if kind == "none" else O.Prior(kind, alpha=0.08)
    probs = O.probabilities(sc.n_subsets, prior)
    seq = O.sample(seed, n_iter, probs)
    params = pkg.make_params(kind, alpha=0.08)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        ctx.spdhg_setup(params, None if x0 is None else dev(x0))
        ctx.spdhg_iterate(seq)
        out = {}
        for k, n in (("x", sc.n_voxels), ("y", sc.n_bins), ("T", sc.n_voxels)):
            t = torch.zeros(n, device="cuda")
            ctx.spdhg_get(k, t)
            out[k] = host(t)
    st, steps = O.spdhg(prob, prior, seq, probs,
                        x0=None if x0 is None else x0.reshape(sc.image_shape).astype(np.float64))
    return out, st, steps


def _check(out, st, steps):
    assert rel(out["x"], O.next_primal(st, steps)) < 1e-4
    assert rel(out["y"], st.y) < 1e-4


def test_zero_counts():
    sc = synth.tiny_3d(steep=True)
    d, _ = problem(sc)
    d = dict(d, b=np.zeros_like(d["b"]))
    prob = O.Problem(sc, d["b"].astype(np.float64), d["r"].astype(np.float64), d["mult"].astype(np.float64))
    out, st, steps = _run(sc, d, prob, "tv")
    _check(out, st, steps)


@pytest.mark.parametrize("m", [1, 4])
def test_one_subset_and_one_view_per_subset(m):
    sc = synth.tiny_3d(n_subsets=m, steep=True)
    d, prob = problem(sc)
    for kind in ("none", "tv"):
        out, st, steps = _run(sc, d, prob, kind)
        _check(out, st, steps)


def test_voxels_no_lor_crosses_keep_their_start():
    # every LOR is a chord of a cylinder of radius 4.1 (voxel units) through an 8 x 8 image: the
    # corner pixels, whose nearest point is 3 sqrt(2) = 4.24 from the centre, lie outside it
    sc = synth.Scanner(nx=8, ny=8, nz=1, vx=1.0, vy=1.0, vz=1.0, n_radial=5, d_radial=1.0,
                       n_views=6, radius=4.1, seg_n=(1,), seg_zmid0=(0.0,), seg_dzmid=(1.0,),
                       seg_dz=(0.0,), n_subsets=2, name="small-cylinder-2d")
    d, prob = problem(sc)
    x0 = (synth.random_image(sc, 4) + 0.5).astype(np.float32)
    out, st, steps = _run(sc, d, prob, "none", x0=x0)
    _check(out, st, steps)
    unseen = steps["T"].ravel() == 0
    assert unseen.sum() >= 4  # the four corners at least
    np.testing.assert_array_equal(out["T"][unseen], 0.0)
    np.testing.assert_array_equal(out["x"][unseen], np.maximum(x0.ravel()[unseen], 0))


def test_non_square_image():
    base = synth.tiny_3d()
    sc = dataclasses.replace(base, nx=9, ny=5, n_radial=13, name="tiny3d-9x5")
    d, prob = problem(sc)
    out, st, steps = _run(sc, d, prob, "tv")
    _check(out, st, steps)


def test_axial_extent_beyond_128_slices():
    nz = 150
    sc = synth.Scanner(nx=6, ny=6, nz=nz, vx=1.0, vy=1.0, vz=1.0, n_radial=9, d_radial=0.8,
                       n_views=4, radius=12.0, seg_n=(nz, nz - 4, nz - 4),
                       seg_zmid0=(-(nz - 1) / 2, -(nz - 1) / 2 + 2, -(nz - 1) / 2 + 2),
                       seg_dzmid=(1.0, 1.0, 1.0), seg_dz=(0.0, 3.0, -3.0), n_subsets=2, name="tall")
    d, prob = problem(sc)
    out, st, steps = _run(sc, d, prob, "tv")
    _check(out, st, steps)


def test_memory_limit_fails_as_out_of_memory_and_the_context_recovers():
    """An allocation past the context's memory limit fails with SPDHG_ERR_OOM, as a failed
    cudaMalloc would, without faulting anything: the context keeps what it holds, and once the
    limit is lifted the same calls succeed and give the bits of a context that never hit it."""
    import torch
    import paper_1808_07150_gb300 as pkg
    sc = synth.config_2d()
    d, _ = problem(sc)
    params = pkg.make_params("tv", alpha=0.1, seed=3)
    seq = O.sample(11, 20, O.probabilities(sc.n_subsets, O.Prior("tv", alpha=0.1)))

    def state(ctx):
        x = torch.zeros(sc.n_voxels, device="cuda")
        ctx.spdhg_get("x", x)
        torch.cuda.synchronize()
        return host(x)

    with pkg.Context(sc) as ref:
        upload(ref, d)
        ref.spdhg_setup(params)
        ref.spdhg_iterate(seq)
        x_ref = state(ref)
    with pkg.Context(sc) as ctx:
        held = ctx.spdhg_set_memory_limit(0)
        assert held > 0                      # the geometry tables
        ctx.spdhg_set_memory_limit(held + 1024)
        with pytest.raises(pkg.SpdhgError) as e:
            upload(ctx, d)
        assert e.value.code == -3            # SPDHG_ERR_OOM
        ctx.spdhg_set_memory_limit(0)
        upload(ctx, d)
        held = ctx.spdhg_set_memory_limit(0)
        ctx.spdhg_set_memory_limit(held + 4096)
        with pytest.raises(pkg.SpdhgError) as e:
            ctx.spdhg_setup(params)
        assert e.value.code == -3
        assert ctx.spdhg_set_memory_limit(0) >= held
        ctx.spdhg_setup(params)
        ctx.spdhg_iterate(seq)
        np.testing.assert_array_equal(state(ctx), x_ref)
