"""Full-size (mMR-scale) parity of one data iteration and one dTV prior iteration, in the launch
configuration the benchmark times: 344x344x127 voxels, 252 views x 344 x 837 planes, 252 subsets,
per-bin multipliers, dTV with a side image.

Both iterations start from the setup state (x = max(x0, 0), y = 0, z = 0, q = 0).  Compared:
the dual y of the subset's 287,928 bins and the prior dual q and dz on all voxels (relative L2
<= 1e-5, and elementwise max |gpu - ref| / max |ref| <= 1e-5), and z, x at sampled voxels where the oracle evaluates T by its definition
(min over the 252 subsets of rho p_i / (P_i^T 1), and the prior's scalar step).
"""
import numpy as np
import pytest

import synth
from oracle import _native
from oracle import algorithms as O

from gpu_helpers import dev, host, maxerr, rel

pytestmark = pytest.mark.gpu

ALPHA = 0.05
SUBSET = 5


@pytest.fixture(scope="module")
def mmr():
    sc = synth.config_mmr()
    d = synth.make_problem(sc, 1808, counts=4e8, bg_frac=0.1, with_mult=True, with_side=True)
    x0 = np.maximum(d["x_true"], 0).astype(np.float32)
    rng = np.random.default_rng(7)
    # voxels inside the field of view (radius < 330 mm) plus a few near the edges
    cand = rng.integers(0, sc.n_voxels, 4000)
    iy, ix, iz = np.unravel_index(cand, sc.image_shape)
    rr = np.hypot((ix + 0.5 - sc.nx / 2) * sc.vx, (iy + 0.5 - sc.ny / 2) * sc.vy)
    vox = np.concatenate([cand[rr < 330][:20], cand[rr >= 330][:4]]).astype(np.int64)
    S = _native.subset_adjoints_at_voxels(sc, d["mult"].astype(np.float64), vox)
    m = sc.n_subsets
    prior = O.Prior("dtv", alpha=ALPHA, side=d["side"].astype(np.float64))
    probs = O.probabilities(m, prior)
    gn = O.grad_norm((sc.nx, sc.ny, sc.nz))
    with np.errstate(divide="ignore"):
        Td = np.where(S > 0, 0.99 * probs[:m][None, :] / np.where(S > 0, S, 1.0), np.inf).min(axis=1)
    T = np.minimum(Td, 0.99 * probs[m] / gn)
    T = np.where(np.isinf(T), 0.0, T)
    return sc, d, x0, vox, T, probs, prior


def _run(sc, d, x0, blocks, keys):
    import paper_1808_07150_gb300 as pkg
    import torch
    sizes = {"x": sc.n_voxels, "z": sc.n_voxels, "T": sc.n_voxels, "y": sc.n_bins, "q": 3 * sc.n_voxels}
    with pkg.Context(sc) as ctx:
        ctx.spdhg_set_data(dev(d["b"]), dev(d["r"]), dev(d["mult"]), dev(d["side"]))
        ctx.spdhg_setup(pkg.make_params("dtv", alpha=ALPHA, dtv_gamma=0.995, dtv_eta_frac=0.01), dev(x0))
        ctx.spdhg_iterate(blocks)
        out = {}
        for k in keys:
            t = torch.zeros(sizes[k], device="cuda")
            ctx.spdhg_get(k, t)
            out[k] = t
        torch.cuda.synchronize()
    return {k: host(v) for k, v in out.items()}


def test_mmr_step_sizes_at_sampled_voxels(mmr):
    sc, d, x0, vox, T, probs, prior = mmr
    g = _run(sc, d, x0, [], ["T"])
    assert rel(g["T"][vox], T) < 1e-5
    assert maxerr(g["T"][vox], T) < 1e-5


def test_mmr_data_iteration(mmr):
    sc, d, x0, vox, T, probs, prior = mmr
    g = _run(sc, d, x0, [SUBSET], ["y", "z", "x"])
    mult = d["mult"].astype(np.float64)
    xd = x0.astype(np.float64)
    mask = O.subset_mask(sc, SUBSET)
    ax = O.project(sc, xd, SUBSET, mult)[mask]
    a1 = O.project(sc, np.ones(sc.image_shape), SUBSET, mult)[mask]
    sigma = np.where(a1 > 0, 0.99 / np.where(a1 > 0, a1, 1.0), 0.0)
    y_new = O.kl_prox(sigma * ax, sigma, d["b"].astype(np.float64)[mask], d["r"].astype(np.float64)[mask])
    assert rel(g["y"].reshape(sc.sino_shape)[mask], y_new) < 1e-5
    assert maxerr(g["y"].reshape(sc.sino_shape)[mask], y_new) < 1e-5
    dy = np.zeros(sc.sino_shape)
    dy[mask] = y_new
    dz = _native.adjoint_at_voxels(sc, dy * mult, vox, SUBSET)
    assert rel(g["z"][vox], dz) < 1e-5
    assert maxerr(g["z"][vox], dz) < 1e-5
    x_ref = np.maximum(xd.ravel()[vox] - T * (dz + dz / probs[SUBSET]), 0.0)
    assert rel(g["x"][vox], x_ref) < 1e-5
    assert maxerr(g["x"][vox], x_ref) < 1e-5


def test_mmr_dtv_prior_iteration(mmr):
    sc, d, x0, vox, T, probs, prior = mmr
    m = sc.n_subsets
    g = _run(sc, d, x0, [m], ["q", "z", "x"])
    xd = x0.astype(np.float64)
    xi = O.dtv_field(prior.side, prior.eta_frac)
    sig = 0.99 / O.grad_norm((sc.nx, sc.ny, sc.nz))
    q_new = O.proj_l2(sig * O.dtv_apply(xi, O.grad(xd), prior.gamma_d), ALPHA)
    dz = O.grad_adj(O.dtv_apply(xi, q_new, prior.gamma_d))
    assert rel(g["q"], q_new) < 1e-5
    assert maxerr(g["q"], q_new) < 1e-5
    assert rel(g["z"], dz) < 1e-5
    assert maxerr(g["z"], dz) < 1e-5
    x_ref = np.maximum(xd.ravel()[vox] - T * (dz.ravel()[vox] * (1 + 1 / probs[m])), 0.0)
    assert rel(g["x"][vox], x_ref) < 1e-5
    assert maxerr(g["x"][vox], x_ref) < 1e-5
