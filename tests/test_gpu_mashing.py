"""GPU parity of exact mashing (each bin the sum of its ring-pair LORs; span-11 compression of the
span-1 ring-pair data of Sec. 1) against the FP64 oracle, through the C ABI.

* Projection, backprojection and the step sizes on a tiny mashed scanner (range and parity rules)
  and on the 3-D scanner with its adjacent-oblique pairs summed into each plane.
* SPDHG+ iterations on both.
* The exact span-11 mMR-like scanner (121 components) in the launch configuration of the
  benchmark: sampled bins and voxels against the oracle's definition.
Tolerances as for the unmashed operators: 1e-5 relative L2 and elementwise against the largest
entry for single operators, 1e-4 for iteration sequences.
"""
import numpy as np
import pytest

import synth
from oracle import algorithms as O

from gpu_helpers import dev, host, maxerr, problem, rel, upload

pytestmark = pytest.mark.gpu

GEOMS = [synth.tiny_mashed(), synth.config_3d_oblique()]


@pytest.mark.parametrize("sc", GEOMS, ids=lambda s: s.name)
def test_mashed_project_and_backproject_match_oracle(sc):
    import paper_1808_07150_gb300 as pkg
    import torch
    mult = synth.smooth_multipliers(sc, 9)
    x = synth.random_image(sc, 1)
    yv = synth.random_sinogram(sc, 2)
    with pkg.Context(sc) as ctx:
        ones = np.ones(sc.sino_shape, np.float32)
        ctx.spdhg_set_data(dev(ones), dev(ones * 0.1), dev(mult))
        for subset in (-1, 0, sc.n_subsets - 1):
            y_gpu = torch.zeros(sc.n_bins, device="cuda")
            ctx.spdhg_project(dev(x), y_gpu, subset)
            bp = torch.zeros(sc.n_voxels, device="cuda")
            ctx.spdhg_backproject(dev(yv), bp, subset)
            torch.cuda.synchronize()
            mask = O.subset_mask(sc, subset).ravel()
            y_ref = O.project(sc, x.astype(np.float64), subset, mult.astype(np.float64)).ravel()
            assert rel(host(y_gpu)[mask], y_ref[mask]) < 1e-5
            assert maxerr(host(y_gpu)[mask], y_ref[mask]) < 1e-5
            bp_ref = O.backproject(sc, yv.astype(np.float64) * mask.reshape(sc.sino_shape), subset,
                                   mult.astype(np.float64))
            assert rel(host(bp), bp_ref) < 1e-5
            assert maxerr(host(bp), bp_ref) < 1e-5


@pytest.mark.parametrize("sc", GEOMS, ids=lambda s: s.name)
def test_mashed_steps_and_iterations_match_oracle(sc):
    import paper_1808_07150_gb300 as pkg
    import torch
    d, prob = problem(sc)
    prior = O.Prior("tv", alpha=0.08)
    probs = O.probabilities(sc.n_subsets, prior)
    steps = O.step_sizes(sc, prob.mult, prior, probs)
    seq = O.sample(31, 30, probs)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        ctx.spdhg_setup(pkg.make_params("tv", alpha=0.08))
        out = {}
        for k, n in (("sigma", sc.n_bins), ("T", sc.n_voxels)):
            t = torch.zeros(n, device="cuda")
            ctx.spdhg_get(k, t)
            out[k] = t
        ctx.spdhg_iterate(seq)
        for k, n in (("x", sc.n_voxels), ("y", sc.n_bins), ("z", sc.n_voxels)):
            t = torch.zeros(n, device="cuda")
            ctx.spdhg_get(k, t)
            out[k] = t
        torch.cuda.synchronize()
        g = {k: host(v) for k, v in out.items()}
    assert rel(g["sigma"], steps["sigma"]) < 1e-5
    assert rel(g["T"], steps["T"]) < 1e-5
    st, steps = O.spdhg(prob, prior, seq, probs, steps=steps)
    assert rel(g["x"], O.next_primal(st, steps)) < 1e-4
    assert rel(g["y"], st.y) < 1e-4
    assert rel(g["z"], st.z) < 1e-4


def test_exact_span11_mmr_operators_on_sampled_outputs():
    import paper_1808_07150_gb300 as pkg
    import torch
    sc = synth.config_mmr_exact()
    ells = synth.random_phantom(sc, 1808, n=10)
    x = synth.voxelize(sc, ells)
    rng = np.random.default_rng(0)
    with pkg.Context(sc) as ctx:
        ones = np.ones(sc.sino_shape, np.float32)
        ctx.spdhg_set_data(dev(ones), dev(ones * 0.1))
        for subset in (0, 126):
            y_gpu = torch.zeros(sc.n_bins, device="cuda")
            ctx.spdhg_project(dev(x), y_gpu, subset)
            torch.cuda.synchronize()
            bins = np.array([np.ravel_multi_index((subset, r, p), sc.sino_shape)
                             for r, p in zip(rng.integers(0, sc.n_radial, 800), rng.integers(0, sc.n_planes, 800))])
            ref = O.project_at_bins(sc, x.astype(np.float64), bins)
            assert rel(host(y_gpu)[bins], ref) < 1e-5
            assert maxerr(host(y_gpu)[bins], ref) < 1e-5
            yv = np.zeros(sc.sino_shape, np.float32)
            yv[subset] = rng.standard_normal(yv[subset].shape).astype(np.float32)
            bp = torch.zeros(sc.n_voxels, device="cuda")
            ctx.spdhg_backproject(dev(yv), bp, subset)
            torch.cuda.synchronize()
            vox = rng.integers(0, sc.n_voxels, 48)
            ref_bp = O.backproject_at_voxels(sc, yv.astype(np.float64), vox, subset)
            assert rel(host(bp)[vox], ref_bp) < 1e-5
            assert maxerr(host(bp)[vox], ref_bp) < 1e-5
