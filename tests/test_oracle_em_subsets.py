"""Pins of the oracle's OSEM / MLEM baselines (Eqs. EQU:OSEM, EQU:MLEM), of bin-interleaved
subsets (the stability example of Sec. 1.3 divides the bins equidistantly) and of user-given
sampling probabilities (Remark "Sampling").

* An (OS)EM update on subset i with zero background keeps the subset's counts:
  sum_{j in S_i} (P_i u+)_j = sum_{j in S_i} b_j, by the algebra of the update (independent of
  how the oracle evaluates it).
* OSEM with one subset is MLEM (two separately written functions).
* Bin-interleaved subset masks partition the sinogram, bin j in subset j mod m.
* SPDHG converges to the same minimiser for any proper sampling (Theorem "Convergence"): with
  bin subsets the unregularised problem reaches MLEM's objective, and TV with user-given
  probabilities reaches PDHG's objective.
"""
import numpy as np
import pytest

import synth
from oracle import algorithms as O


def _problem(sc, seed=3, counts=5e3, bg=0.1):
    d = synth.make_problem(sc, seed, counts=counts, bg_frac=bg, with_mult=True, n_ellipsoids=4)
    return O.Problem(sc, d["b"].astype(np.float64), d["r"].astype(np.float64), d["mult"].astype(np.float64))


@pytest.mark.parametrize("kind", ["views", "bins"])
@pytest.mark.parametrize("epochs", [1, 3])
def test_osem_keeps_the_last_subsets_counts_without_background(kind, epochs):
    sc = synth.tiny_2d(n_subsets=3).with_subsets(3, kind)
    prob = _problem(sc, bg=0.0)
    assert np.all(prob.r == 0)
    u = O.osem(prob, epochs)
    last = O.subset_mask(sc, sc.n_subsets - 1)
    proj = O.project(sc, u, sc.n_subsets - 1, prob.mult)
    assert float(proj[last].sum()) == pytest.approx(float(prob.b[last].sum()), rel=1e-12)


def test_osem_with_one_subset_is_mlem():
    sc = synth.tiny_3d(n_subsets=1)
    prob = _problem(sc)
    np.testing.assert_allclose(O.osem(prob, 7), O.mlem(prob, 7), rtol=1e-12, atol=1e-14)


def test_bin_subsets_partition_the_sinogram():
    sc = synth.tiny_3d(n_subsets=5).with_subsets(5, "bins")
    masks = np.stack([O.subset_mask(sc, i).ravel() for i in range(5)])
    assert np.all(masks.sum(0) == 1)
    for i in range(5):
        assert np.array_equal(np.nonzero(masks[i])[0], np.arange(i, sc.n_bins, 5))
    # the projection of a subset is the full projection on its bins, zero elsewhere
    x = synth.random_image(sc, 1).astype(np.float64)
    full = O.project(sc, x)
    for i in range(5):
        np.testing.assert_allclose(O.project(sc, x, i), np.where(masks[i].reshape(sc.sino_shape), full, 0.0))


def test_spdhg_with_bin_subsets_reaches_mlem_objective():
    sc = synth.tiny_2d(n_subsets=3).with_subsets(3, "bins")
    prob = _problem(sc)
    probs = O.probabilities(sc.n_subsets, None)
    st, steps = O.spdhg(prob, None, O.sample(7, 40000, probs), probs)
    x = O.next_primal(st, steps)
    u = O.mlem(prob, 20000)
    assert O.objective(prob, None, x) == pytest.approx(O.objective(prob, None, u), rel=1e-6, abs=1e-6)


def test_tv_spdhg_with_custom_probabilities_reaches_pdhg_objective():
    sc = synth.tiny_2d(n_subsets=3)
    prob = _problem(sc)
    prior = O.Prior("tv", alpha=0.5)
    # data blocks weighted by their counts, the prior drawn with probability 0.4
    w = np.array([prob.b[O.subset_mask(sc, i)].sum() for i in range(3)])
    probs = np.concatenate([0.6 * w / w.sum(), [0.4]])
    p = O.probabilities(3, prior, "custom", probs)
    st, steps = O.spdhg(prob, prior, O.sample(11, 40000, p), p)
    x1 = O.next_primal(st, steps)
    s2, st2 = O.pdhg(prob, prior, 8000)
    x2 = O.next_primal(s2, st2)
    assert O.objective(prob, prior, x1) == pytest.approx(O.objective(prob, prior, x2), rel=1e-5)
    with pytest.raises(ValueError):
        O.probabilities(3, prior, "custom", [0.5, 0.5, 0.0, 0.0])
