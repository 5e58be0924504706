"""Epoch graphs, batched reconstructions and the launch-shape autotuner (CUDA path via the C ABI).

* A graph-mode run (one CUDA graph launch per epoch) executes the kernels, launch shapes and
  arguments of the eager path, so its iterate and objective log are bit-identical to
  spdhg_run without graphs; both match the FP64 oracle run on the same sampled sequence
  (Algorithm 2, seeded sampler) to relative L2 1e-4.
* spdhg_run_batch over uneven problems (image and sinogram sizes, subsets, TV and TGV, different
  epoch counts) gives every problem exactly its solo result.
* The autotuner changes no state array, keeps its choices within the documented ranges, and
  the tuned kernels keep parity with the oracle.
"""
import numpy as np
import pytest

import synth
from oracle import algorithms as O

from gpu_helpers import dev, host, problem, rel, upload

pytestmark = pytest.mark.gpu


def _prior(kind):
    if kind == "tgv":
        return O.Prior("tgv", alpha0=0.2, alpha1=0.1)
    return O.Prior(kind, alpha=0.08)


def _params(pkg, kind, epochs, graph, seed=1808, every=1):
    return pkg.make_params(kind, alpha=0.08, alpha0=0.2, alpha1=0.1, seed=seed, epochs=epochs,
                           objective_every=every, graph=graph)


def _oracle_run(sc, prob, kind, epochs, seed, x0):
    prior = _prior(kind)
    probs = O.probabilities(sc.n_subsets, prior)
    ipe = O.iters_per_epoch(sc.n_subsets, probs)
    # the oracle's own sampler (pinned bit-equal to the library's elsewhere): nothing of the
    # oracle's input comes from the product
    seq = np.concatenate([O.sample(seed, ipe, probs, offset=e * ipe) for e in range(epochs)])
    st, steps = O.spdhg(prob, prior, seq, probs, x0=x0.reshape(sc.image_shape).astype(np.float64))
    return O.next_primal(st, steps)


@pytest.mark.parametrize("kind", ["tv", "tgv"])
@pytest.mark.parametrize("sc", [synth.tiny_3d(steep=True), synth.config_2d()], ids=lambda s: s.name)
def test_graph_run_is_bit_identical_to_eager_and_matches_oracle(sc, kind):
    import paper_1808_07150_gb300 as pkg
    d, prob = problem(sc)
    x0 = (synth.random_image(sc, 5) * float(d["x_true"].max())).astype(np.float32)
    out = {}
    for graph in (False, True):
        x = x0.copy()
        with pkg.Context(sc) as ctx:
            upload(ctx, d)
            rep = ctx.spdhg_run(_params(pkg, kind, 2, graph), x)
        out[graph] = (x, rep)
    np.testing.assert_array_equal(out[True][0], out[False][0])
    np.testing.assert_array_equal(out[True][1]["objective"], out[False][1]["objective"])
    assert out[True][1]["epochs_done"] == 2
    assert np.all(out[True][1]["epoch_ms"] > 0)
    ref = _oracle_run(sc, prob, kind, 2, 1808, x0)
    assert rel(out[True][0], ref) < 1e-4


def test_graph_run_repeated_calls_and_device_buffers():
    """Templates survive a second run with the same parameters and are rebuilt for new ones."""
    import paper_1808_07150_gb300 as pkg
    import torch
    sc = synth.tiny_3d(steep=True)
    d, _ = problem(sc)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        xs = []
        for alpha in (0.08, 0.08, 0.2):
            x = torch.zeros(sc.n_voxels, device="cuda")
            p = pkg.make_params("tv", alpha=alpha, seed=9, epochs=3, graph=True)
            ctx.spdhg_run(p, x)
            xs.append(host(x))
        xe = np.zeros(sc.n_voxels, np.float32)
        ctx.spdhg_run(pkg.make_params("tv", alpha=0.2, seed=9, epochs=3), xe)
    np.testing.assert_array_equal(xs[0], xs[1])
    np.testing.assert_array_equal(xs[2], xe.astype(np.float64))
    assert rel(xs[0], xs[2]) > 0


def _uneven_batch():
    scs = synth.batch_geometries(7, 4, small=True) + [synth.config_2d(), synth.tiny_3d(steep=True)]
    kinds = ["tv", "tgv", "tv", "tgv", "tv", "tgv"]
    epochs = [3, 2, 1, 2, 2, 0]
    return scs, kinds, epochs


def test_batch_equals_solo_runs_and_oracle():
    import paper_1808_07150_gb300 as pkg
    scs, kinds, epochs = _uneven_batch()
    data = [problem(sc, seed=11 + k, counts=[1e4, 3e5, 5e4, 2e6, 1e5, 2e4][k]) for k, sc in enumerate(scs)]
    x0s = [np.zeros(sc.n_voxels, np.float32) for sc in scs]
    ctxs = [pkg.Context(sc) for sc in scs]
    try:
        for ctx, (d, _) in zip(ctxs, data):
            upload(ctx, d)
        params = [_params(pkg, kind, ep, True, seed=100 + k) for k, (kind, ep) in enumerate(zip(kinds, epochs))]
        xb = [x.copy() for x in x0s]
        reps = pkg.spdhg_run_batch(ctxs, params, xb)
        for k, ctx in enumerate(ctxs):
            xs = x0s[k].copy()
            rs = ctx.spdhg_run(_params(pkg, kinds[k], epochs[k], False, seed=100 + k), xs)
            np.testing.assert_array_equal(xb[k], xs, err_msg=scs[k].name)
            np.testing.assert_array_equal(reps[k]["objective"], rs["objective"], err_msg=scs[k].name)
            assert reps[k]["epochs_done"] == epochs[k]
        # again, on the captured iterations cached by the first batch, after the solo runs of
        # differently sized contexts have launched the same kernels with other shapes
        xb2 = [x.copy() for x in x0s]
        pkg.spdhg_run_batch(ctxs, params, xb2)
        for k in range(len(ctxs)):
            np.testing.assert_array_equal(xb2[k], xb[k], err_msg=scs[k].name)
    finally:
        for c in ctxs:
            c.close()
    # one member (2-D, TV, 2 epochs from zero) against the oracle
    k = 4
    ref = _oracle_run(scs[k], data[k][1], kinds[k], epochs[k], 100 + k, x0s[k])
    assert rel(xb[k], ref) < 1e-4


def test_batch_rejects_duplicates():
    import paper_1808_07150_gb300 as pkg
    sc = synth.tiny_3d()
    d, _ = problem(sc)
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        p = _params(pkg, "tv", 1, True)
        with pytest.raises(pkg.SpdhgError):
            pkg.spdhg_run_batch([ctx, ctx], [p, p])


@pytest.mark.parametrize("kind", ["dtv", "tgv"])
def test_autotune_keeps_state_and_parity(kind):
    import paper_1808_07150_gb300 as pkg
    import torch
    sc = synth.batch_geometries(3, 1, small=True)[0]
    d, prob = problem(sc, side=(kind == "dtv"))
    prior = O.Prior("tgv", alpha0=0.2, alpha1=0.1) if kind == "tgv" else \
        O.Prior("dtv", alpha=0.08, side=d["side"].astype(np.float64))
    probs = O.probabilities(sc.n_subsets, prior)
    seq = O.sample(77, 30, probs)
    params = pkg.make_params(kind, alpha=0.08, alpha0=0.2, alpha1=0.1)
    keys = {"x": sc.n_voxels, "z": sc.n_voxels, "y": sc.n_bins, "q": 3 * sc.n_voxels, "T": sc.n_voxels}
    with pkg.Context(sc) as ctx:
        upload(ctx, d)
        ctx.spdhg_setup(params, None)
        ctx.spdhg_iterate(seq[:10])

        def state():
            out = {}
            for k, n in keys.items():
                t = torch.zeros(n, device="cuda")
                ctx.spdhg_get(k, t)
                out[k] = host(t)
            return out

        before = state()
        chosen = ctx.spdhg_autotune(reps=2)
        after = state()
        for k in keys:
            np.testing.assert_array_equal(after[k], before[k], err_msg=k)
        assert chosen["fwd_warps"] in (0, 2, 4, 8, 16)
        assert chosen["fwd_split"] in (0, 1, 2, 4, 8)
        assert chosen["fwd_groups"] in (0, 1, 2, 4, 8)
        if kind == "dtv":  # 0: the built-in choice was the fastest
            assert chosen["prior_cols"] == 0 or 2 <= chosen["prior_cols"] <= 32
            assert chosen["prior_ychunk"] in (0, 16, 32, 64, 128, 256)
            assert chosen["prior_stages"] in (0, 3, 4) and chosen["prior_vz"] in (0, 1, 2, 4)
        ctx.spdhg_iterate(seq[10:])
        x = torch.zeros(sc.n_voxels, device="cuda")
        ctx.spdhg_get("x", x)
        xg = host(x)
    st, steps = O.spdhg(prob, prior, seq, probs)
    assert rel(xg, O.next_primal(st, steps)) < 1e-4


@pytest.mark.parametrize("sc", [synth.tiny_3d(steep=True), synth.config_2d(), synth.config_3d_small(),
                                synth.tiny_mashed(), synth.config_3d_oblique()], ids=lambda s: s.name)
def test_backprojector_item_table_is_bit_identical(sc):
    """The backprojector's tap items read from the table spdhg_setup builds give the same bits as
    the items the kernel computes itself (knob bwd_table = 1)."""
    import paper_1808_07150_gb300 as pkg
    import torch
    d, prob = problem(sc)
    probs = O.probabilities(sc.n_subsets, _prior("tv"))
    seq = O.sample(77, 40, probs)
    out = []
    for knobs in ({"bwd_table": 1}, {}):
        with pkg.Context(sc) as ctx:
            upload(ctx, d)
            for k, v in knobs.items():
                ctx.spdhg_tune(k, v)
            ctx.spdhg_setup(_params(pkg, "tv", 1, False))
            ctx.spdhg_iterate(seq)
            st = {}
            for k, n in (("x", sc.n_voxels), ("z", sc.n_voxels), ("y", sc.n_bins), ("T", sc.n_voxels)):
                t = torch.zeros(n, device="cuda")
                ctx.spdhg_get(k, t)
                st[k] = t
            torch.cuda.synchronize()
            out.append({k: host(v) for k, v in st.items()})
    for other in out[1:]:
        for k in out[0]:
            np.testing.assert_array_equal(out[0][k], other[k], err_msg=k)

