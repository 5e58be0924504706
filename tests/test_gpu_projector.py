"""GPU parity of the projector, backprojector and step sizes against the FP64 oracle.

Tolerance: per-operator relative L2 error <= 1e-5 in FP32 (the stated bar for single
operators), and elementwise max |gpu - ref| / max |ref| <= 1e-5 so that a few wrong bins or voxels
cannot hide under the norm.  The GPU adjoint pairing <P x, y> vs <x, P^T y> is held to 2e-6: both directions
use bit-identical lengths, so only the summation order differs.
"""
import numpy as np
import pytest

import synth
from oracle import _native
from oracle import algorithms as O

from gpu_helpers import dev, host, maxerr, problem, rel, upload, wide_2d

pytestmark = pytest.mark.gpu

GEOMS = [
    synth.tiny_2d(), synth.tiny_3d(), synth.tiny_3d(steep=True), wide_2d(),
    synth.config_2d(), synth.config_3d(),
]


def _ctx(sc, mult=None):
    import paper_1808_07150_gb300 as pkg
    ctx = pkg.Context(sc)
    b = np.ones(sc.sino_shape, np.float32)
    ctx.spdhg_set_data(dev(b), dev(b * 0.1), None if mult is None else dev(mult))
    return ctx


@pytest.mark.parametrize("sc", GEOMS, ids=lambda s: s.name)
def test_project_and_backproject_match_oracle(sc):
    import torch
    mult = synth.smooth_multipliers(sc, 9)
    x = synth.random_image(sc, 1)
    yv = synth.random_sinogram(sc, 2)
    with _ctx(sc, mult) as ctx:
        for subset in (-1, 0, sc.n_subsets - 1):
            y_gpu = torch.zeros(sc.n_bins, device="cuda")
            ctx.spdhg_project(dev(x), y_gpu, subset)
            bp_gpu = torch.zeros(sc.n_voxels, device="cuda")
            ctx.spdhg_backproject(dev(yv), bp_gpu, subset)
            torch.cuda.synchronize()
            mask = O.subset_mask(sc, subset)
            y_ref = O.project(sc, x.astype(np.float64), subset, mult.astype(np.float64))
            assert rel(host(y_gpu)[mask.ravel()], y_ref[mask]) < 1e-5
            assert maxerr(host(y_gpu)[mask.ravel()], y_ref[mask]) < 1e-5
            if subset >= 0:  # bins of other subsets are not written
                assert np.all(host(y_gpu)[~mask.ravel()] == 0.0)
            bp_ref = O.backproject(sc, yv.astype(np.float64) * mask, subset, mult.astype(np.float64))
            assert rel(host(bp_gpu), bp_ref) < 1e-5
            assert maxerr(host(bp_gpu), bp_ref) < 1e-5
            # adjoint pairing on the GPU results
            lhs = float(np.dot(host(y_gpu)[mask.ravel()], yv.astype(np.float64).ravel()[mask.ravel()]))
            rhs = float(np.dot(x.astype(np.float64).ravel(), host(bp_gpu)))
            assert abs(lhs - rhs) <= 2e-6 * abs(lhs)


@pytest.mark.parametrize("groups,split", [(1, 1), (2, 1), (4, 1), (8, 1), (3, 2), (4, 4)])
@pytest.mark.parametrize("sc", [synth.tiny_3d(steep=True), synth.config_2d(), synth.config_3d()],
                         ids=lambda s: s.name)
def test_forward_entry_groups_match_oracle(sc, groups, split):
    """The forward projector with several warps sharing each plane run (entry groups, alone and
    with row parts) against the oracle, on every plane of the first subset."""
    import torch
    mult = synth.smooth_multipliers(sc, 9)
    x = synth.random_image(sc, 1)
    with _ctx(sc, mult) as ctx:
        ctx.spdhg_tune("fwd_groups", groups)
        ctx.spdhg_tune("fwd_split", split)
        y_gpu = torch.zeros(sc.n_bins, device="cuda")
        ctx.spdhg_project(dev(x), y_gpu, 0)
        torch.cuda.synchronize()
    mask = O.subset_mask(sc, 0)
    y_ref = O.project(sc, x.astype(np.float64), 0, mult.astype(np.float64))
    assert rel(host(y_gpu)[mask.ravel()], y_ref[mask]) < 1e-5
    assert maxerr(host(y_gpu)[mask.ravel()], y_ref[mask]) < 1e-5
    assert np.all(host(y_gpu)[~mask.ravel()] == 0.0)


@pytest.mark.parametrize("sc", [synth.tiny_3d(steep=True), wide_2d(), synth.config_2d()], ids=lambda s: s.name)
def test_sigma_and_T_match_oracle(sc):
    import paper_1808_07150_gb300 as pkg
    import torch
    d, prob = problem(sc)
    prior = O.Prior("tv", alpha=0.1)
    probs = O.probabilities(sc.n_subsets, prior)
    st = O.step_sizes(sc, prob.mult, prior, probs)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        ctx.spdhg_setup(pkg.make_params("tv", alpha=0.1))
        assert np.allclose(ctx.spdhg_probabilities(), probs)
        sig = torch.zeros(sc.n_bins, device="cuda")
        T = torch.zeros(sc.n_voxels, device="cuda")
        ctx.spdhg_get("sigma", sig)
        ctx.spdhg_get("T", T)
        torch.cuda.synchronize()
    assert rel(host(sig), st["sigma"]) < 1e-5
    assert maxerr(host(sig), st["sigma"]) < 1e-5
    assert np.array_equal(host(sig) == 0, st["sigma"].ravel() == 0)
    assert rel(host(T), st["T"]) < 1e-5
    assert maxerr(host(T), st["T"]) < 1e-5


def test_mmr_scale_operators_on_sampled_outputs():
    """Full mMR-scale geometry (344x344x127, 252 views x 344 x 837, 252 subsets) in the launch
    configuration of the benchmark: sampled bins / voxels against the oracle's definitions."""
    import torch
    sc = synth.config_mmr()
    ells = synth.random_phantom(sc, 1808, n=10)
    x = synth.voxelize(sc, ells)
    mult = synth.smooth_multipliers(sc, 1811)
    rng = np.random.default_rng(0)
    with _ctx(sc, mult) as ctx:
        for subset in (0, 126, 251):
            y_gpu = torch.zeros(sc.n_bins, device="cuda")
            ctx.spdhg_project(dev(x), y_gpu, subset)
            torch.cuda.synchronize()
            bins = np.array([np.ravel_multi_index((subset, r, p), sc.sino_shape)
                             for r, p in zip(rng.integers(0, sc.n_radial, 1500), rng.integers(0, sc.n_planes, 1500))])
            ref = _native.line_integrals_at(sc, x.astype(np.float64), bins) * mult.ravel()[bins]
            assert rel(host(y_gpu)[bins], ref) < 1e-5
            assert maxerr(host(y_gpu)[bins], ref) < 1e-5
            yv = np.zeros(sc.sino_shape, np.float32)
            yv[subset] = rng.standard_normal(yv[subset].shape).astype(np.float32)
            bp = torch.zeros(sc.n_voxels, device="cuda")
            ctx.spdhg_backproject(dev(yv), bp, subset)
            torch.cuda.synchronize()
            vox = rng.integers(0, sc.n_voxels, 96)
            ref_bp = _native.adjoint_at_voxels(sc, yv.astype(np.float64) * mult, vox, subset)
            assert rel(host(bp)[vox], ref_bp) < 1e-5
            assert maxerr(host(bp)[vox], ref_bp) < 1e-5
