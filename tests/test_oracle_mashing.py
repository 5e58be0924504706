"""Pins of exact mashing (each bin the sum of the LORs of the ring pairs it collects; the paper's
data are span-1 ring-pair LORs, Sec. 1, and compressed data sum them).

* The mashed projection equals, bin by bin, the sum of single-LOR line integrals computed by the
  brute-force box-clipping matrix of one-plane scanners built here from the mashing rule (not from
  the helper the oracle uses).
* The exact span-11 rule of the mMR-like scanner collects every ring pair of 64 rings with ring
  difference up to 60 exactly once (4084 LORs per view and radial bin), enumerated over all pairs.
* The mashed operators are adjoint.
"""
import dataclasses

import numpy as np
import pytest

import synth
from oracle import _native
from oracle import algorithms as O


def _single_lor_row(sc, z_mid, dz):
    """Dense rows (views x radial, voxels) of the one-plane scanner with the given LOR."""
    one = dataclasses.replace(sc, seg_n=(1,), seg_zmid0=(z_mid,), seg_dzmid=(sc.vz,), seg_dz=(dz,), components=())
    return _native.dense_by_clipping(one).reshape(sc.n_views, sc.n_radial, sc.n_voxels)


@pytest.mark.parametrize("sc", [synth.tiny_mashed()], ids=lambda s: s.name)
def test_mashed_projection_is_sum_of_single_lor_integrals(sc):
    x = synth.random_image(sc, 4).astype(np.float64).ravel()
    got = O.project(sc, x.reshape(sc.image_shape))
    expect = np.zeros(sc.sino_shape)
    p0 = 0
    for g, n in enumerate(sc.seg_n):
        for q in range(n):
            z_mid = sc.seg_zmid0[g] + q * sc.seg_dzmid[g]
            for dz, qlo, qhi, step in sc.components[g]:
                if qlo <= q < qhi and (q - qlo) % step == 0:
                    expect[:, :, p0 + q] += _single_lor_row(sc, z_mid, dz) @ x
        p0 += n
    np.testing.assert_allclose(got, expect, rtol=1e-12, atol=1e-12)


def test_mashed_operators_are_adjoint():
    sc = synth.tiny_mashed()
    x = synth.random_image(sc, 1).astype(np.float64)
    y = synth.random_sinogram(sc, 2).astype(np.float64)
    for subset in (-1, 0, 1):
        lhs = float((O.project(sc, x, subset) * y).sum())
        rhs = float((x * O.backproject(sc, y * O.subset_mask(sc, subset), subset)).sum())
        assert lhs == pytest.approx(rhs, rel=1e-12)


def test_exact_span11_rule_collects_every_ring_pair_once():
    sc = synth.config_mmr_exact()
    rings, max_diff = 64, 60
    count = {}
    p0 = 0
    firsts = [f for f, _, _ in synth.MMR_SPAN11_SEGMENTS]
    for g, n in enumerate(sc.seg_n):
        for q in range(n):
            for dz, qlo, qhi, step in sc.components[g]:
                if qlo <= q < qhi and (q - qlo) % step == 0:
                    d = int(round(dz / (2 * sc.vz)))
                    s_ = firsts[g] + q
                    key = ((s_ + d) // 2, (s_ - d) // 2)
                    assert (s_ + d) % 2 == 0
                    count[key] = count.get(key, 0) + 1
        p0 += n
    pairs = {(r1, r2) for r1 in range(rings) for r2 in range(rings) if abs(r1 - r2) <= max_diff}
    assert set(count) == pairs
    assert all(v == 1 for v in count.values())
    assert len(pairs) == 4084
    # every plane's mid-point is the mean ring position of its pairs: ring sum s at z = (s - 63) vz
    for g, (f, n, _) in enumerate(synth.MMR_SPAN11_SEGMENTS):
        assert sc.seg_zmid0[g] == pytest.approx((f - 63) * sc.vz)


def test_oblique_3d_planes():
    sc = synth.config_3d_oblique()
    (c,) = sc.components
    assert c[0] == (0.0, 0, 64, 1)
    # the two oblique pairs (p-1, p+1), (p+1, p-1) exist for the inner planes only
    assert {c[1][1:], c[2][1:]} == {(1, 63, 1)}
    assert abs(c[1][0]) == abs(c[2][0]) == 4.0


def test_sampled_mashed_operators_equal_full_ones():
    sc = synth.tiny_mashed()
    x = synth.random_image(sc, 3).astype(np.float64)
    y = synth.random_sinogram(sc, 4).astype(np.float64)
    np.testing.assert_allclose(O.project_at_bins(sc, x, np.arange(sc.n_bins)), O.project(sc, x).ravel(),
                               rtol=1e-13, atol=1e-13)
    for subset in (-1, 1):
        np.testing.assert_allclose(O.backproject_at_voxels(sc, y, np.arange(sc.n_voxels), subset),
                                   O.backproject(sc, y * O.subset_mask(sc, subset), subset).ravel(),
                                   rtol=1e-12, atol=1e-12)
