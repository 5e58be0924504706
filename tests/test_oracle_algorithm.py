"""Pins of the oracle's step sizes, sampler and iterations.

* Step sizes: the convergence condition ||S_i^1/2 A_i T^1/2||^2 < p_i (Eq. EQU:STEPSIZE) on
  dense blocks, computed with numpy's SVD (independent of the oracle's operators).
* PDHG (Algorithm 1) and SPDHG (Algorithm 2) coincide for one block with p = 1 (Remark after
  Theorem "Step Size Parameters").
* Unregularised problem: long SPDHG runs satisfy the ML optimality (KKT) conditions and reach
  the objective of MLEM (Eq. EQU:MLEM), an independent algorithm for the same minimiser.
* TV problem: SPDHG+ and PDHG reach the same objective value.
* Sampler: frequencies match p_i (balanced and uniform sampling, Sec. 4.2).
"""
import math

import numpy as np
import pytest

import synth
from oracle import _native
from oracle import algorithms as O


def _problem(sc, seed=3, counts=2e4, with_mult=True):
    d = synth.make_problem(sc, seed, counts=counts, bg_frac=0.1, with_mult=with_mult, n_ellipsoids=4)
    return O.Problem(sc, d["b"].astype(np.float64), d["r"].astype(np.float64),
                     None if d["mult"] is None else d["mult"].astype(np.float64))


@pytest.mark.parametrize("precond", [True, False])
def test_step_size_condition_on_dense_blocks(precond):
    sc = synth.tiny_3d(n_subsets=2)
    prob = _problem(sc)
    prior = O.Prior("tv", alpha=0.1)
    probs = O.probabilities(sc.n_subsets, prior, "balanced")
    A = _native.dense_by_clipping(sc) * prob.mult.reshape(-1, 1)
    norms = None
    if not precond:
        norms = []
        for i in range(sc.n_subsets):
            rows = O.subset_mask(sc, i).ravel()
            norms.append(np.linalg.norm(A[rows], 2))
    st = O.step_sizes(sc, prob.mult, prior, probs, precond=precond, data_norms=norms)
    sqT = np.sqrt(st["T"].ravel())
    worst = 0.0
    for i in range(sc.n_subsets):
        rows = O.subset_mask(sc, i).ravel()
        M = np.sqrt(st["sigma"].ravel()[rows])[:, None] * A[rows] * sqT[None, :]
        assert np.linalg.norm(M, 2) ** 2 < probs[i]
        worst = max(worst, np.linalg.norm(M, 2) ** 2 / probs[i])
    # the steps are not needlessly small: some data block is close to its bound rho^2 p_i
    assert worst > 0.5 * 0.99 ** 2
    # prior block: scalar sigma_n on A_n = grad
    N = sc.n_voxels
    G = np.stack([O.grad(np.eye(N)[k].reshape(sc.image_shape)).ravel() for k in range(N)], 1)
    M = math.sqrt(st["sigma_prior"][0]) * G * sqT[None, :]
    assert np.linalg.norm(M, 2) ** 2 < probs[sc.n_subsets]


def test_pdhg_equals_spdhg_for_one_block():
    sc = synth.tiny_2d(n_subsets=1)
    prob = _problem(sc)
    probs = O.probabilities(1, None)
    assert probs.tolist() == [1.0]
    s1, steps = O.spdhg(prob, None, [0] * 25, probs)
    s2, _ = O.pdhg(prob, None, 25, steps=steps)
    np.testing.assert_array_equal(s1.x, s2.x)
    np.testing.assert_array_equal(s1.y, s2.y)
    np.testing.assert_array_equal(s1.zbar, s2.zbar)


def _ml_kkt(prob, x):
    sc = prob.sc
    ax = O.project(sc, x, -1, prob.mult)
    g = O.backproject(sc, 1.0 - prob.b / (ax + prob.r), -1, prob.mult)
    scale = O.backproject(sc, np.ones(sc.sino_shape), -1, prob.mult)
    return g, scale


def test_unregularised_spdhg_reaches_ml_optimum_and_mlem():
    sc = synth.tiny_2d(n_subsets=3)
    prob = _problem(sc, counts=5e3)
    probs = O.probabilities(sc.n_subsets, None)
    seq = O.sample(7, 40000, probs)
    st, steps = O.spdhg(prob, None, seq, probs)
    x = O.next_primal(st, steps)
    g, scale = _ml_kkt(prob, x)
    seen = scale > 0
    assert np.all(x >= 0)
    # stationarity on the support, non-negative gradient on the active set
    assert np.max(np.abs(g[seen & (x > 1e-3 * x.max())]) / scale[seen & (x > 1e-3 * x.max())]) < 2e-3
    assert np.min(g[seen] / scale[seen]) > -2e-3
    u = O.mlem(prob, 20000)
    psi_spdhg = O.objective(prob, None, x)
    psi_mlem = O.objective(prob, None, u)
    assert psi_spdhg == pytest.approx(psi_mlem, rel=1e-6, abs=1e-6)


def test_tv_spdhg_plus_and_pdhg_agree():
    sc = synth.tiny_2d(n_subsets=3)
    prob = _problem(sc, counts=5e3)
    prior = O.Prior("tv", alpha=0.5)
    probs = O.probabilities(sc.n_subsets, prior, "balanced")
    seq = O.sample(11, 40000, probs)
    st, steps = O.spdhg(prob, prior, seq, probs)
    x1 = O.next_primal(st, steps)
    s2, st2 = O.pdhg(prob, prior, 8000)
    x2 = O.next_primal(s2, st2)
    p1, p2 = O.objective(prob, prior, x1), O.objective(prob, prior, x2)
    assert p1 == pytest.approx(p2, rel=1e-5)
    assert np.linalg.norm(x1 - x2) / np.linalg.norm(x2) < 1e-2


@pytest.mark.parametrize("kind,m", [("balanced", 10), ("uniform", 10), ("tgv", 6)])
def test_sampler_frequencies(kind, m):
    prior = O.Prior("tgv") if kind == "tgv" else O.Prior("tv")
    probs = O.probabilities(m, prior, "uniform" if kind == "uniform" else "balanced")
    assert probs.sum() == pytest.approx(1.0)
    n = 60000
    seq = O.sample(1808, n, probs)
    counts = np.bincount(seq, minlength=len(probs))
    chi2 = float((((counts - n * probs) ** 2) / (n * probs)).sum())
    # chi-square with len(p)-1 dof: mean dof, sd sqrt(2 dof); 6 sd is far out in the tail
    dof = len(probs) - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)
    assert O.iters_per_epoch(m, probs) == (2 * m if kind != "uniform" else m + 1)


def test_splitmix_uniforms_are_uniform():
    u = np.array([(O.splitmix64(42, k) >> 11) / 2.0 ** 53 for k in range(50000)])
    assert u.min() >= 0 and u.max() < 1
    assert abs(u.mean() - 0.5) < 0.01
    assert abs(u.var() - 1 / 12) < 0.005
    # lag-1 correlation of a good generator is ~0
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.02
