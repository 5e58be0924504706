"""GPU parity of SPDHG iterations (Algorithm 2) against the FP64 oracle on the same block sequence.

Tolerances: a short sequence (a few dozen iterations) agrees to relative L2 1e-4 in every state
array (FP32 rounding of single operators, <= 1e-5, compounded over the iterations); the final
image after a fixed seeded sequence of a full reconstruction agrees to 1e-3 (the stated bar).
"""
import numpy as np
import pytest

import synth
from oracle import algorithms as O

from gpu_helpers import dev, host, problem, rel, upload

pytestmark = pytest.mark.gpu


def _gpu_state(ctx, sc, keys):
    import torch
    out = {}
    sizes = {"x": sc.n_voxels, "z": sc.n_voxels, "T": sc.n_voxels, "y": sc.n_bins, "q": 3 * sc.n_voxels,
             "w": 3 * sc.n_voxels, "zw": 3 * sc.n_voxels, "q2": 6 * sc.n_voxels}
    for k in keys:
        t = torch.zeros(sizes[k], device="cuda")
        ctx.spdhg_get(k, t)
        out[k] = t
    torch.cuda.synchronize()
    return {k: host(v) for k, v in out.items()}


def _prior(kind, side):
    if kind == "none":
        return None
    if kind == "tgv":
        return O.Prior("tgv", alpha0=0.2, alpha1=0.1)
    return O.Prior(kind, alpha=0.08, side=None if side is None else side.astype(np.float64))


@pytest.mark.parametrize("kind", ["none", "tv", "dtv", "atv", "tgv"])
@pytest.mark.parametrize("sc", [synth.tiny_3d(steep=True), synth.config_2d()], ids=lambda s: s.name)
def test_iterations_match_oracle(sc, kind):
    import paper_1808_07150_gb300 as pkg
    d, prob = problem(sc, side=(kind == "dtv"))
    prior = _prior(kind, d["side"])
    probs = O.probabilities(sc.n_subsets, prior)
    seq = O.sample(1234, 40, probs)
    x0 = synth.random_image(sc, 17) * float(d["x_true"].max())
    params = pkg.make_params(kind, alpha=0.08, alpha0=0.2, alpha1=0.1)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        ctx.spdhg_setup(params, dev(x0))
        ctx.spdhg_iterate(seq)
        keys = ["x", "z", "y"] + (["q"] if kind != "none" else []) + (["w", "zw", "q2"] if kind == "tgv" else [])
        g = _gpu_state(ctx, sc, keys)
    st, steps = O.spdhg(prob, prior, seq, probs, x0=x0.astype(np.float64))
    assert rel(g["x"], O.next_primal(st, steps)) < 1e-4
    assert rel(g["z"], st.z) < 1e-4
    assert rel(g["y"], st.y) < 1e-4
    if kind != "none":
        assert rel(g["q"], st.q[0]) < 1e-4
    if kind == "tgv":
        Tu, Tw = steps["T"]
        assert rel(g["w"], st.w - Tw * st.zbar_w) < 1e-4
        assert rel(g["zw"], st.zw) < 1e-4
        assert rel(g["q2"], st.q[1]) < 1e-4


def test_full_reconstruction_2d_final_image():
    """2-D PET, 64x64, 90 views x 95 bins, TV beta = 0.1, 10 subsets, 50 epochs of SPDHG+."""
    import paper_1808_07150_gb300 as pkg
    sc = synth.config_2d()
    d, prob = problem(sc, seed=1808, counts=1e5, mult=False)
    prior = O.Prior("tv", alpha=0.1)
    probs = O.probabilities(sc.n_subsets, prior)
    ipe = O.iters_per_epoch(sc.n_subsets, probs)
    epochs = 50
    params = pkg.make_params("tv", alpha=0.1, seed=1810, epochs=epochs, objective_every=10)
    x_gpu = np.zeros(sc.image_shape, np.float32)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        rep = ctx.spdhg_run(params, x_gpu)
    seq = np.concatenate([O.sample(1810, ipe, probs, offset=e * ipe) for e in range(epochs)])
    st, steps = O.spdhg(prob, prior, seq, probs)
    x_ref = O.next_primal(st, steps)
    assert rep["epochs_done"] == epochs and rep["iterations_done"] == epochs * ipe
    assert rel(x_gpu, x_ref) < 1e-3
    psi_ref = O.objective(prob, prior, x_ref)
    assert rep["objective"][-1] == pytest.approx(psi_ref, rel=1e-5)
    # objective decreases over the logged epochs of this run
    logged = rep["objective"][~np.isnan(rep["objective"])]
    assert logged[-1] < logged[0]


def test_3d_one_epoch_matches_oracle():
    """3-D cylindrical scanner 128x128x64, 180 views (21 uneven subsets), TV beta = 0.05."""
    import paper_1808_07150_gb300 as pkg
    sc = synth.config_3d()
    d, prob = problem(sc, seed=1808, counts=3e7, mult=False)
    prior = O.Prior("tv", alpha=0.05)
    probs = O.probabilities(sc.n_subsets, prior)
    ipe = O.iters_per_epoch(sc.n_subsets, probs)
    seq = O.sample(1810, ipe, probs)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        ctx.spdhg_setup(pkg.make_params("tv", alpha=0.05))
        ctx.spdhg_iterate(seq)
        g = _gpu_state(ctx, sc, ["x", "z"])
    st, steps = O.spdhg(prob, prior, seq, probs)
    assert rel(g["x"], O.next_primal(st, steps)) < 1e-4
    assert rel(g["z"], st.z) < 1e-4


@pytest.mark.parametrize("kind", ["none", "tv", "dtv", "atv", "tgv"])
def test_objective_matches_oracle(kind):
    import paper_1808_07150_gb300 as pkg
    sc = synth.tiny_3d(steep=True)
    d, prob = problem(sc, side=(kind == "dtv"))
    prior = _prior(kind, d["side"])
    x = synth.random_image(sc, 5) * float(d["x_true"].max())
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        ctx.spdhg_setup(pkg.make_params(kind, alpha=0.08, alpha0=0.2, alpha1=0.1), dev(x))
        D, R, tot = ctx.spdhg_objective()
    xd = x.astype(np.float64)
    ref_D = O.data_fidelity(O.project(sc, xd, -1, prob.mult), prob.b, prob.r)
    w = np.zeros((3,) + sc.image_shape) if kind == "tgv" else None
    ref_R = O.prior_value(prior, xd, w) if prior is not None else 0.0
    scale = float((O.project(sc, xd, -1, prob.mult) + prob.r).sum())
    assert abs(D - ref_D) <= 1e-5 * scale
    assert R == pytest.approx(ref_R, rel=1e-5, abs=1e-9)
    assert tot == pytest.approx(D + R)


def test_invalid_inputs_are_rejected():
    import paper_1808_07150_gb300 as pkg
    sc = synth.tiny_2d()
    d, _ = problem(sc)
    with pkg.Context(sc) as ctx:
        bad = d["b"].copy()
        bad[0, 0, 0] = -1.0
        with pytest.raises(pkg.SpdhgError) as e:
            ctx.spdhg_set_data(dev(bad), dev(d["r"]))
        assert e.value.code == pkg._capi.ERR_DATA
        bad[0, 0, 0] = np.nan
        with pytest.raises(pkg.SpdhgError):
            ctx.spdhg_set_data(dev(bad), dev(d["r"]))
        with pytest.raises(pkg.SpdhgError) as e:  # iterate before setup
            ctx.spdhg_iterate([0])
        assert e.value.code == pkg._capi.ERR_STATE
        upload(ctx, d)
        ctx.spdhg_setup(pkg.make_params("tv"))
        with pytest.raises(pkg.SpdhgError) as e:
            ctx.spdhg_iterate([sc.n_subsets + 1])
        assert e.value.code == pkg._capi.ERR_ARG
        import torch
        with pytest.raises(pkg.SpdhgError):
            ctx.spdhg_project(torch.zeros(sc.n_voxels, device="cuda"), torch.zeros(sc.n_bins, device="cuda"), sc.n_subsets)


def test_non_finite_objective_is_reported_as_diverged():
    """A start image holding +Inf makes the FP64 objective non-finite after the first epoch:
    spdhg_run stops there with SPDHG_ERR_DIVERGED (the failure is made on the host; no kernel
    faults, the arithmetic just carries Inf / NaN)."""
    import paper_1808_07150_gb300 as pkg
    sc = synth.tiny_2d()
    d, _ = problem(sc)
    x = np.full(sc.image_shape, np.inf, np.float32)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        with pytest.raises(pkg.SpdhgError) as e:
            ctx.spdhg_run(pkg.make_params("tv", alpha=0.1, epochs=3, objective_every=1), x)
        assert e.value.code == pkg._capi.ERR_DIVERGED
        assert b"not finite" in pkg._capi.lib().spdhg_last_error(ctx.h)
        # the context stays usable: a finite start runs to the end
        x0 = np.zeros(sc.image_shape, np.float32)
        rep = ctx.spdhg_run(pkg.make_params("tv", alpha=0.1, epochs=2, objective_every=1), x0)
        assert rep["epochs_done"] == 2 and np.all(np.isfinite(rep["objective"]))


@pytest.mark.parametrize("sc", [synth.tiny_3d(steep=True), synth.config_2d()], ids=lambda s: s.name)
def test_scalar_step_sizes_and_iterations_match_oracle(sc):
    """precond = 0 (Eq. EQU:STEPSIZE:SCALAR): sigma_i = gamma rho / ||P_i|| on the bins of subset i,
    T = min_i rho p_i / (gamma ||P_i||) and the prior's scalar step.  The norms come from power
    iteration on both sides (the oracle runs 3000 steps); then 40 SPDHG iterations."""
    import torch
    import paper_1808_07150_gb300 as pkg
    d, prob = problem(sc)
    prior = _prior("tv", None)
    probs = O.probabilities(sc.n_subsets, prior)
    norms = []
    for i in range(sc.n_subsets):
        mask = O.subset_mask(sc, i)
        norms.append(O.operator_norm_power(lambda x: O.project(sc, x, i, prob.mult),
                                           lambda y: O.backproject(sc, y * mask, i, prob.mult),
                                           sc.image_shape, iters=3000))
    steps = O.step_sizes(sc, prob.mult, prior, probs, precond=False, data_norms=norms)
    seq = O.sample(4321, 40, probs)
    params = pkg.make_params("tv", alpha=0.08, precond=False)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        ctx.spdhg_setup(params, None)
        g = _gpu_state(ctx, sc, ["T"])
        sig = torch.zeros(sc.n_bins, device="cuda")
        ctx.spdhg_get("sigma", sig)
        assert rel(host(sig), steps["sigma"]) < 1e-5
        assert rel(g["T"], steps["T"]) < 1e-5
        ctx.spdhg_iterate(seq)
        g = _gpu_state(ctx, sc, ["x", "y"])
    st, steps_o = O.spdhg(prob, prior, seq, probs, steps=steps)
    assert rel(g["x"], O.next_primal(st, steps_o)) < 1e-4
    assert rel(g["y"], st.y) < 1e-4


@pytest.mark.slow
@pytest.mark.parametrize("sc,epochs", [(synth.config_3d(), 30), (synth.config_3d_oblique(), 6)],
                         ids=["direct-30", "oblique-6"])
def test_full_reconstruction_3d_final_image(sc, epochs):
    """3-D cylindrical scanner 128x128x64, 180 views (21 uneven subsets), TV beta = 0.05: 30 epochs
    of SPDHG+ from zero on a fixed seeded sequence with each plane's direct LOR, and 6 epochs with
    the adjacent-oblique pairs summed into the planes (three times the oracle's cost per epoch):
    final image within 1e-3 of the oracle, the FP64 objective within 1e-5."""
    import paper_1808_07150_gb300 as pkg
    d, prob = problem(sc, seed=1808, counts=3e7, mult=False)
    prior = O.Prior("tv", alpha=0.05)
    probs = O.probabilities(sc.n_subsets, prior)
    ipe = O.iters_per_epoch(sc.n_subsets, probs)
    params = pkg.make_params("tv", alpha=0.05, seed=1811, epochs=epochs, objective_every=epochs)
    x_gpu = np.zeros(sc.image_shape, np.float32)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        rep = ctx.spdhg_run(params, x_gpu)
    seq = np.concatenate([O.sample(1811, ipe, probs, offset=e * ipe) for e in range(epochs)])
    st, steps = O.spdhg(prob, prior, seq, probs)
    x_ref = O.next_primal(st, steps)
    assert rel(x_gpu, x_ref) < 1e-3
    assert rep["objective"][-1] == pytest.approx(O.objective(prob, prior, x_ref), rel=1e-5)
