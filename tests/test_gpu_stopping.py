"""The library's own stopping rule and quality log (Sec. 4: relative objective
(Psi(x^k) - Psi*) / (Psi(0) - Psi*) and PSNR(x^k, x*)), through the C ABI.

* Psi(0) is the FP64 oracle's objective of the zero image (to 1e-5 of the expected counts).
* spdhg_run with target_gap stops after the first epoch whose relative objective reaches the
  target: the same epoch a full run's objective log gives, with the same iterate (bit-identical:
  the same kernels on the same sequence), and its solver time is the sum of those epochs.
* PSNR(x, x*) equals the definition evaluated in FP64 on the host from the same two images.
* spdhg_run_batch stops every reconstruction at its own target, each as if run alone.
"""
import numpy as np
import pytest

import synth
from oracle import algorithms as O

from gpu_helpers import dev, host, problem, upload

pytestmark = pytest.mark.gpu


def _rel_gap(obj, psi0, psi_star):
    return (obj - psi_star) / (psi0 - psi_star)


def test_psi_zero_and_stop_epoch_match_the_full_log():
    import paper_1808_07150_gb300 as pkg
    sc = synth.config_2d()
    d, prob = problem(sc, seed=1808, counts=1e5, mult=True)
    epochs = 40
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        # full log, and Psi* from the last epochs of a longer run
        ref = ctx.spdhg_run(pkg.make_params("tv", alpha=0.1, seed=5, epochs=120, objective_every=40), None)
        psi_star = float(np.nanmin(ref["objective"]))
        x_full = np.zeros(sc.image_shape, np.float32)
        log = ctx.spdhg_run(pkg.make_params("tv", alpha=0.1, seed=5, epochs=epochs, objective_every=1,
                                            target_gap=1e-12, psi_star=psi_star - 1.0), x_full)
        assert log["stop_epoch"] == -1 and log["epochs_done"] == epochs
        psi0 = log["psi_zero"]
        psi0_ref = O.objective(prob, O.Prior("tv", alpha=0.1), np.zeros(sc.image_shape))
        scale = float(prob.r.sum() + prob.b.sum())
        assert abs(psi0 - psi0_ref) <= 1e-5 * scale
        gaps = _rel_gap(log["objective"][1:], psi0, psi_star)
        target = 1e-2
        expect = int(np.nonzero(gaps <= target)[0][0]) + 1
        assert 1 < expect < epochs
        x_stop = np.zeros(sc.image_shape, np.float32)
        rep = ctx.spdhg_run(pkg.make_params("tv", alpha=0.1, seed=5, epochs=epochs, target_gap=target,
                                            psi_star=psi_star), x_stop)
        assert rep["stop_epoch"] == expect and rep["epochs_done"] == expect
        assert rep["ms_to_stop"] == pytest.approx(float(np.sum(rep["epoch_ms"][:expect])), rel=1e-9)
        np.testing.assert_array_equal(rep["objective"][1:expect + 1], log["objective"][1:expect + 1])
        # the iterate at the stop is the full run's iterate after the same number of epochs
        x_part = np.zeros(sc.image_shape, np.float32)
        ctx.spdhg_run(pkg.make_params("tv", alpha=0.1, seed=5, epochs=expect), x_part)
        np.testing.assert_array_equal(x_stop, x_part)


def test_psnr_matches_definition_and_is_logged():
    import paper_1808_07150_gb300 as pkg
    import torch
    sc = synth.config_2d()
    d, prob = problem(sc, seed=1808, counts=1e5, mult=False)
    x_star = d["x_true"].astype(np.float32) * 1.1
    xs = dev(x_star)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        rep = ctx.spdhg_run(pkg.make_params("tv", alpha=0.1, seed=9, epochs=3, x_star=xs), None)
        x = torch.zeros(sc.n_voxels, device="cuda")
        ctx.spdhg_get("x", x)
        ref = O.psnr(host(x).reshape(sc.image_shape), x_star.astype(np.float64))
        assert rep["psnr"][3] == pytest.approx(ref, abs=1e-9)
        assert ctx.spdhg_psnr(xs) == pytest.approx(ref, abs=1e-9)
        assert ctx.spdhg_psnr(x_star, host(x).astype(np.float32)) == pytest.approx(ref, abs=1e-9)
        assert np.all(np.isfinite(rep["psnr"]))


def test_batch_stops_each_reconstruction_at_its_own_target():
    import paper_1808_07150_gb300 as pkg
    gs = [synth.config_2d(), synth.config_3d_small()]
    ds = [problem(sc, seed=11 + k, counts=1e5, mult=True)[0] for k, sc in enumerate(gs)]
    ctxs = [pkg.Context(sc) for sc in gs]
    try:
        for c, d in zip(ctxs, ds):
            upload(c, d)
        stars = []
        for k, c in enumerate(ctxs):
            r = c.spdhg_run(pkg.make_params("tv", alpha=0.1, seed=20 + k, epochs=80, objective_every=80), None)
            stars.append(float(np.nanmin(r["objective"])))
        targets = [3e-2, 1e-2]
        params = [pkg.make_params("tv", alpha=0.1, seed=20 + k, epochs=30, graph=True, target_gap=targets[k],
                                  psi_star=stars[k]) for k in range(2)]
        reps = pkg.spdhg_run_batch(ctxs, params)
        for k, c in enumerate(ctxs):
            solo = c.spdhg_run(pkg.make_params("tv", alpha=0.1, seed=20 + k, epochs=30, target_gap=targets[k],
                                               psi_star=stars[k]), None)
            assert reps[k]["stop_epoch"] == solo["stop_epoch"] > 0
            assert reps[k]["epochs_done"] == solo["stop_epoch"]
            np.testing.assert_array_equal(reps[k]["objective"], solo["objective"])
    finally:
        for c in ctxs:
            c.close()
