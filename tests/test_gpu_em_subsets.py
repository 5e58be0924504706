"""GPU parity of the OSEM / MLEM baselines (Eqs. EQU:OSEM, EQU:MLEM), of bin-interleaved subsets
(Sec. 1.3) and of user-given sampling probabilities (Remark "Sampling"), through the C ABI,
against the FP64 oracle.

Tolerances: single operators 1e-5 relative L2 (and elementwise against the largest entry); EM
iterations and SPDHG sequences compound FP32 rounding over their sub-iterations and are held to
1e-4, the bar of the other short iteration tests.
"""
import numpy as np
import pytest

import synth
from oracle import algorithms as O

from gpu_helpers import dev, host, maxerr, problem, rel, upload

pytestmark = pytest.mark.gpu

GEOMS = [synth.tiny_3d(steep=True), synth.config_2d(), synth.config_3d_small()]


@pytest.mark.parametrize("kind", ["views", "bins"])
@pytest.mark.parametrize("sc", GEOMS, ids=lambda s: s.name)
def test_osem_matches_oracle(sc, kind):
    import paper_1808_07150_gb300 as pkg
    sc = sc.with_subsets(sc.n_subsets, kind)
    d, prob = problem(sc)
    x = np.ones(sc.image_shape, np.float32)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        rep = ctx.spdhg_osem(pkg.make_params("none", epochs=3, objective_every=3), x)
    ref = O.osem(prob, 3)
    assert rel(x, ref) < 1e-4
    assert maxerr(x, ref) < 1e-4
    assert rep["epochs_done"] == 3 and rep["iterations_done"] == 3 * sc.n_subsets
    psi = O.objective(prob, None, ref)
    assert rep["objective"][3] == pytest.approx(psi, rel=1e-5)


@pytest.mark.parametrize("sc", GEOMS, ids=lambda s: s.name)
def test_mlem_matches_oracle(sc):
    import paper_1808_07150_gb300 as pkg
    d, prob = problem(sc)
    x0 = (0.5 + synth.random_image(sc, 3)).astype(np.float32)
    x = x0.copy()
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        rep = ctx.spdhg_osem(pkg.make_params("none", epochs=5), x, mlem=True)
    ref = O.mlem(prob, 5, x0=x0.astype(np.float64))
    assert rel(x, ref) < 1e-4
    assert rep["iterations_done"] == 5


@pytest.mark.parametrize("sc", [synth.tiny_3d(steep=True), synth.config_2d()], ids=lambda s: s.name)
def test_bin_subset_operators_match_oracle(sc):
    import paper_1808_07150_gb300 as pkg
    import torch
    sc = sc.with_subsets(4, "bins")
    mult = synth.smooth_multipliers(sc, 9)
    x = synth.random_image(sc, 1)
    yv = synth.random_sinogram(sc, 2)
    with pkg.Context(sc) as ctx:
        ones = np.ones(sc.sino_shape, np.float32)
        ctx.spdhg_set_data(dev(ones), dev(ones * 0.1), dev(mult))
        for subset in (0, 3):
            y_gpu = torch.zeros(sc.n_bins, device="cuda")
            ctx.spdhg_project(dev(x), y_gpu, subset)
            bp = torch.zeros(sc.n_voxels, device="cuda")
            ctx.spdhg_backproject(dev(yv), bp, subset)
            torch.cuda.synchronize()
            mask = O.subset_mask(sc, subset).ravel()
            y_ref = O.project(sc, x.astype(np.float64), subset, mult.astype(np.float64)).ravel()
            assert rel(host(y_gpu)[mask], y_ref[mask]) < 1e-5
            assert maxerr(host(y_gpu)[mask], y_ref[mask]) < 1e-5
            assert np.all(host(y_gpu)[~mask] == 0.0)
            bp_ref = O.backproject(sc, yv.astype(np.float64), subset, mult.astype(np.float64))
            assert rel(host(bp), bp_ref) < 1e-5
            assert maxerr(host(bp), bp_ref) < 1e-5


def _state(ctx, sc):
    import torch
    out = {}
    for k, n in (("x", sc.n_voxels), ("y", sc.n_bins), ("z", sc.n_voxels), ("T", sc.n_voxels)):
        t = torch.zeros(n, device="cuda")
        ctx.spdhg_get(k, t)
        out[k] = t
    torch.cuda.synchronize()
    return {k: host(v) for k, v in out.items()}


@pytest.mark.parametrize("precond", [True, False])
@pytest.mark.parametrize("sc", [synth.tiny_3d(steep=True), synth.config_2d()], ids=lambda s: s.name)
def test_spdhg_with_bin_subsets_matches_oracle(sc, precond):
    import paper_1808_07150_gb300 as pkg
    sc = sc.with_subsets(5, "bins")
    d, prob = problem(sc)
    prior = O.Prior("tv", alpha=0.08)
    probs = O.probabilities(sc.n_subsets, prior)
    seq = O.sample(99, 30, probs)
    norms = None
    if not precond:
        norms = []
        for i in range(sc.n_subsets):
            mask = O.subset_mask(sc, i)
            norms.append(O.operator_norm_power(lambda x: O.project(sc, x, i, prob.mult),
                                               lambda y: O.backproject(sc, y * mask, i, prob.mult),
                                               sc.image_shape, iters=3000))
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        ctx.spdhg_setup(pkg.make_params("tv", alpha=0.08, precond=precond))
        ctx.spdhg_iterate(seq)
        g = _state(ctx, sc)
    steps = O.step_sizes(sc, prob.mult, prior, probs, precond=precond, data_norms=norms)
    assert rel(g["T"], steps["T"]) < 1e-5
    st, steps = O.spdhg(prob, prior, seq, probs, steps=steps)
    assert rel(g["x"], O.next_primal(st, steps)) < 1e-4
    assert rel(g["y"], st.y) < 1e-4
    assert rel(g["z"], st.z) < 1e-4


def test_custom_probabilities_match_oracle():
    import paper_1808_07150_gb300 as pkg
    sc = synth.config_2d()
    d, prob = problem(sc)
    prior = O.Prior("tv", alpha=0.08)
    m = sc.n_subsets
    w = np.array([prob.b[O.subset_mask(sc, i)].sum() for i in range(m)])
    custom = np.concatenate([0.6 * w / w.sum(), [0.4]])
    probs = O.probabilities(m, prior, "custom", custom)
    seq = O.sample(5, 40, probs)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        ctx.spdhg_setup(pkg.make_params("tv", alpha=0.08, sampling="custom", probs=custom))
        np.testing.assert_allclose(ctx.spdhg_probabilities(), probs, rtol=0, atol=0)
        ctx.spdhg_iterate(seq)
        g = _state(ctx, sc)
        with pytest.raises(pkg.SpdhgError):
            ctx.spdhg_setup(pkg.make_params("tv", alpha=0.08, sampling="custom", probs=custom * 0.5))
    st, steps = O.spdhg(prob, prior, seq, probs)
    assert rel(g["T"], steps["T"]) < 1e-5
    assert rel(g["x"], O.next_primal(st, steps)) < 1e-4
    assert rel(g["z"], st.z) < 1e-4
