"""State setting / resume, and the learned warm start end to end (CUDA path, C ABI).

* spdhg_set is the inverse of spdhg_get (X is clamped to the non-negative orthant as the primal
  iterate opening the next iteration); a run checkpointed with spdhg_get and resumed in another
  context with spdhg_set continues bit-identically.
* Warm start: a U-Net trained (on the GPU, by the library's kernels) on pairs (x_2, x*) of seeded
  problems of one scanner maps the 2-epoch iterate of held-out problems closer to x* than the
  iterate itself, and SPDHG+ continued from it has a smaller relative objective gap than SPDHG+
  from zero after the same number of epochs.  Only the starting point changes: continued to the
  reference epoch count, the warm-started run reaches the zero start's objective (relative gap
  < 1e-3), and its image is as close (within 1.5x) to a zero-start run twice as long as the zero
  start's own image is.  (An image bar of 1e-3 between the two runs would need far more epochs
  than a test affords: TV images converge more slowly than the objective, and after 60 epochs
  the two runs still differ by about 2 %.)
"""
import numpy as np
import pytest

import synth

from gpu_helpers import dev, host, problem, rel, upload

pytestmark = pytest.mark.gpu


def _state(ctx, sc, keys):
    import torch
    n = {"x": sc.n_voxels, "z": sc.n_voxels, "y": sc.n_bins, "q": 3 * sc.n_voxels}
    out = {}
    for k in keys:
        t = torch.zeros(n[k], device="cuda")
        ctx.spdhg_get(k, t)
        out[k] = t
    return out


def test_set_round_trip_and_clamp():
    import torch
    import paper_1808_07150_gb300 as pkg
    sc = synth.tiny_3d(steep=True)
    d, _ = problem(sc)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        ctx.spdhg_setup(pkg.make_params("tv", alpha=0.1), None)
        r = np.random.default_rng(0)
        vals = {"x": r.standard_normal(sc.n_voxels), "z": r.standard_normal(sc.n_voxels),
                "y": r.standard_normal(sc.n_bins), "q": r.standard_normal(3 * sc.n_voxels)}
        for k, v in vals.items():
            ctx.spdhg_set(k, dev(v))
        got = {k: host(v) for k, v in _state(ctx, sc, vals).items()}
        np.testing.assert_array_equal(got["x"], np.maximum(vals["x"].astype(np.float32), 0))
        for k in ("z", "y", "q"):
            np.testing.assert_array_equal(got[k], vals[k].astype(np.float32))
        with pytest.raises(pkg.SpdhgError):
            pkg._capi.check(pkg._capi.lib().spdhg_set(ctx.h, pkg.STATE["T"], dev(vals["x"]).data_ptr(),
                                                      pkg._capi.WHERE_DEVICE, None), ctx.h)


def test_checkpoint_resume_is_bit_identical():
    import paper_1808_07150_gb300 as pkg
    from paper_1808_07150_gb300 import warmstart as W
    sc = synth.config_3d_small()
    d, _ = problem(sc, seed=21, counts=1e5)
    params = pkg.make_params("tv", alpha=0.05, seed=5)
    with pkg.Context(sc) as a, pkg.Context(sc) as b:
        for c in (a, b):
            upload(c, d)
            c.spdhg_setup(params, None)
        W.run_epochs(a, params, 2, 0)
        snap = _state(a, sc, ["x", "z", "y", "q"])
        for k, v in snap.items():
            b.spdhg_set(k, v)
        oa, _ = W.run_epochs(a, params, 2, 2)
        ob, _ = W.run_epochs(b, params, 2, 2)
        xa, xb = _state(a, sc, ["x"])["x"], _state(b, sc, ["x"])["x"]
    np.testing.assert_array_equal(oa, ob)
    np.testing.assert_array_equal(host(xa), host(xb))


def test_learned_warm_start_gains_over_zero_start():
    import torch
    import paper_1808_07150_gb300 as pkg
    from paper_1808_07150_gb300 import learned, warmstart as W
    sc = synth.config_3d_small()
    n_train, n_test, k, ref = 24, 3, 2, 60
    ctxs = []
    for s in range(n_train + n_test):
        d = synth.make_problem(sc, 300 + 7 * s, counts=3e5, bg_frac=0.1, with_mult=True, with_side=False,
                               n_ellipsoids=6)
        c = pkg.Context(sc)
        upload(c, d)
        ctxs.append(c)
    params = [pkg.make_params("tv", alpha=0.05, seed=40 + s) for s in range(len(ctxs))]
    try:
        xk, xs = W.pairs(ctxs, params, k, ref)
        with learned.UNet(sc.image_shape, (16, 32, 64)) as net:
            from oracle import unet as U
            spec = U.UNetSpec((16, 32, 64))
            init = np.concatenate([v.ravel() for v in U.init_params(spec, 1).values()])
            net.set_params(init)
            losses = W.train(net, xk[:n_train], xs[:n_train], epochs=40, lr=2e-3, batch=4)
            assert losses[-1] < 0.5 * losses[0]
            x0s = []
            for i in range(n_train, n_train + n_test):
                x0 = torch.zeros(sc.n_voxels, device="cuda")
                net.forward(xk[i], 0.0, None, x0)
                x0s.append(torch.clamp(x0, min=0))
            assert learned.device_error() == 0
        gains_img, gains_gap = [], []
        map_img = map_gap = None
        for j, i in enumerate(range(n_train, n_train + n_test)):
            ctx, p = ctxs[i], params[i]
            gains_img.append(rel(host(x0s[j]), host(xs[i])) / rel(host(xk[i]), host(xs[i])))
            ctx.spdhg_setup(p, None)
            ctx.spdhg_run(pkg.make_params("tv", alpha=0.05, seed=p.seed, epochs=ref, objective_every=ref), None)
            psi_star = ctx.spdhg_objective()[2]
            x_ref = torch.zeros(sc.n_voxels, device="cuda")
            ctx.spdhg_get("x", x_ref)
            ctx.spdhg_setup(p, None)
            psi0 = ctx.spdhg_objective(torch.zeros(sc.n_voxels, device="cuda"))[2]
            plain, _ = W.run_epochs(ctx, p, k + 2, 0)
            ctx.spdhg_setup(p, None)
            W.run_epochs(ctx, p, k, 0)
            W.continue_from(ctx, x0s[j])
            warm, _ = W.run_epochs(ctx, p, 2, k)
            gp = (plain[-1] - psi_star) / (psi0 - psi_star)
            gw = (warm[-1] - psi_star) / (psi0 - psi_star)
            gains_gap.append(gw / gp)
            if j == 0:
                # only the starting point changes: continued to the reference epoch count, the
                # warm-started run reaches the zero start's objective, and its image is as close
                # to a zero start run twice as long as the zero start's own image is
                tail, _ = W.run_epochs(ctx, p, ref - k - 2, k + 2)
                x_warm = torch.zeros(sc.n_voxels, device="cuda")
                ctx.spdhg_get("x", x_warm)
                map_gap = abs(tail[-1] - psi_star) / (psi0 - psi_star)
                ctx.spdhg_setup(p, None)
                ctx.spdhg_run(pkg.make_params("tv", alpha=0.05, seed=p.seed, epochs=2 * ref,
                                              objective_every=2 * ref), None)
                x_long = torch.zeros(sc.n_voxels, device="cuda")
                ctx.spdhg_get("x", x_long)
                map_img = (rel(host(x_warm), host(x_long)), rel(host(x_ref), host(x_long)))
    finally:
        for c in ctxs:
            c.close()
    assert np.mean(gains_img) < 0.8, gains_img      # x0 closer to x* than x_k
    assert np.mean(gains_gap) < 1.0, gains_gap      # smaller gap after the same epochs
    assert map_gap < 1e-3, map_gap                  # same objective
    assert map_img[0] <= 1.5 * map_img[1], map_img  # converging to the same image


@pytest.mark.parametrize("kind", ["tv", "tgv"])
def test_state_file_resume_is_bit_identical(tmp_path, kind):
    """spdhg_save_state after 2 epochs, spdhg_load_state into a fresh context set up alike: the
    next 2 epochs are bit-identical; a file written with other parameters is refused."""
    import paper_1808_07150_gb300 as pkg
    from paper_1808_07150_gb300 import warmstart as W
    sc = synth.config_3d_small()
    d, _ = problem(sc, seed=23, counts=1e5)
    params = pkg.make_params(kind, alpha=0.05, alpha0=0.2, alpha1=0.1, seed=7)
    path = tmp_path / "state.bin"
    with pkg.Context(sc) as a, pkg.Context(sc) as b:
        for c in (a, b):
            upload(c, d)
            c.spdhg_setup(params, None)
        W.run_epochs(a, params, 2, 0)
        a.spdhg_save_state(path)
        oa, _ = W.run_epochs(a, params, 2, 2)
        b.spdhg_load_state(path)
        ob, _ = W.run_epochs(b, params, 2, 2)
        xa, xb = _state(a, sc, ["x"])["x"], _state(b, sc, ["x"])["x"]
        b.spdhg_setup(pkg.make_params(kind, alpha=0.07, alpha0=0.3, alpha1=0.1, seed=7), None)
        with pytest.raises(pkg.SpdhgError):
            b.spdhg_load_state(path)
    np.testing.assert_array_equal(oa, ob)
    np.testing.assert_array_equal(host(xa), host(xb))
