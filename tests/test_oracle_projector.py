"""Pins of the oracle's projector against what geometry fixes independently of it.

The projector's definition (exact line integral of the piecewise-constant image along the
LOR segment, the projection model of Sec. 1.2) is checked against: an independent dense
matrix by per-voxel slab clipping, exact lengths through axis-aligned boxes of voxels (a
numpy slab clip of one box, no per-voxel code), analytic disk chords, and the adjoint identity.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import _native


def _lor_numpy(sc, v, r, p):
    phi = math.pi * v / sc.n_views
    c, s_ = math.cos(phi), math.sin(phi)
    c = 0.0 if abs(c) < 1e-12 else c
    s_ = 0.0 if abs(s_) < 1e-12 else s_
    s = (r - (sc.n_radial - 1) / 2.0) * sc.d_radial
    zm, dz = sc.plane_table()
    h = math.sqrt(sc.radius ** 2 - s ** 2)
    return np.array([s * c, s * s_, zm[p]]), np.array([-s_, c, dz[p] / (2 * h)]), h


def _box_len(o, d, h, lo, hi):
    """Length of {o + t d : t in [-h, h]} inside the box [lo, hi) (half-open for d_a = 0)."""
    t0, t1 = -h, h
    for a in range(3):
        if d[a] == 0.0:
            if not (lo[a] <= o[a] < hi[a]):
                return 0.0
        else:
            ta, tb = (lo[a] - o[a]) / d[a], (hi[a] - o[a]) / d[a]
            t0, t1 = max(t0, min(ta, tb)), min(t1, max(ta, tb))
    return max(0.0, t1 - t0) * float(np.linalg.norm(d))


GEOMS = [synth.tiny_2d(), synth.tiny_3d(), synth.tiny_3d(steep=True)]


@pytest.mark.parametrize("sc", GEOMS, ids=lambda s: s.name)
def test_siddon_equals_dense_slab_clipping(sc):
    A = _native.dense_by_clipping(sc)
    x = synth.random_image(sc, 11).astype(np.float64)
    y = synth.random_sinogram(sc, 12).astype(np.float64)
    np.testing.assert_allclose(_native.line_integrals(sc, x).ravel(), A @ x.ravel(), rtol=0, atol=1e-12)
    np.testing.assert_allclose(_native.line_integrals_adjoint(sc, y).ravel(), A.T @ y.ravel(), rtol=0, atol=1e-12)


@pytest.mark.parametrize("sc", GEOMS + [synth.config_2d()], ids=lambda s: s.name)
def test_line_integral_through_voxel_box_is_exact(sc):
    rng = np.random.default_rng(5)
    for _ in range(3):
        i0 = [int(rng.integers(0, n)) for n in (sc.nx, sc.ny, sc.nz)]
        i1 = [int(rng.integers(a + 1, n + 1)) for a, n in zip(i0, (sc.nx, sc.ny, sc.nz))]
        x = np.zeros(sc.image_shape)
        x[i0[1]:i1[1], i0[0]:i1[0], i0[2]:i1[2]] = 1.0
        y = _native.line_integrals(sc, x)
        lo = [-n * v / 2 + i * v for n, v, i in zip((sc.nx, sc.ny, sc.nz), (sc.vx, sc.vy, sc.vz), i0)]
        hi = [-n * v / 2 + i * v for n, v, i in zip((sc.nx, sc.ny, sc.nz), (sc.vx, sc.vy, sc.vz), i1)]
        for v in range(sc.n_views):
            for r in range(sc.n_radial):
                for p in range(sc.n_planes):
                    o, d, h = _lor_numpy(sc, v, r, p)
                    assert abs(y[v, r, p] - _box_len(o, d, h, lo, hi) / sc.vx) < 1e-10


def test_chord_through_image_box_mmr_sample():
    sc = synth.config_mmr()
    rng = np.random.default_rng(1)
    bins = rng.integers(0, sc.n_bins, size=300)
    got = _native.line_integrals_at(sc, np.ones(sc.image_shape), bins)
    lo = [-sc.nx * sc.vx / 2, -sc.ny * sc.vy / 2, -sc.nz * sc.vz / 2]
    hi = [-a for a in lo]
    for k, j in enumerate(bins):
        v, r, p = np.unravel_index(j, sc.sino_shape)
        o, d, h = _lor_numpy(sc, v, r, p)
        assert abs(got[k] - _box_len(o, d, h, lo, hi) / sc.vx) < 1e-9 * max(1.0, got[k])


def test_disk_chords_within_pixelisation_bound():
    n, vpix, R = 256, 0.5, 40.0
    sc = synth.Scanner(nx=n, ny=n, nz=1, vx=vpix, vy=vpix, vz=1.0, n_radial=61, d_radial=1.25,
                       n_views=7, radius=200.0, seg_n=(1,), seg_zmid0=(0.0,), seg_dzmid=(1.0,),
                       seg_dz=(0.0,), n_subsets=1)
    c = -n * vpix / 2 + (np.arange(n) + 0.5) * vpix
    Y, X = np.meshgrid(c, c, indexing="ij")
    x = ((X ** 2 + Y ** 2) <= R ** 2).astype(np.float64)[:, :, None]
    y = _native.line_integrals(sc, x)[:, :, 0] * vpix  # back to mm
    s = (np.arange(sc.n_radial) - 30) * sc.d_radial
    delta = math.sqrt(2) * vpix / 2  # a pixel whose centre is inside lies within R + delta
    for r, sv in enumerate(s):
        exact = 2 * math.sqrt(max(R * R - sv * sv, 0.0))
        outer = 2 * math.sqrt(max((R + delta) ** 2 - sv * sv, 0.0))
        inner = 2 * math.sqrt(max((R - delta) ** 2 - sv * sv, 0.0))
        bound = max(outer - exact, exact - inner) + 1e-9
        assert np.all(np.abs(y[:, r] - exact) <= bound), (r, y[:, r], exact, bound)


def test_axis_aligned_rays_follow_half_open_rule():
    sc = synth.config_2d()  # view 0 rays (phi = 0) lie on pixel boundaries x = s
    x = np.zeros(sc.image_shape)
    x[:, 32, 0] = 1.0  # column ix = 32: x in [0, 2) mm
    y = _native.line_integrals(sc, x)
    r0 = 47  # s = 0
    assert y[0, r0, 0] == pytest.approx(64.0)  # 128 mm / 2 mm voxels
    assert y[0, r0 + 1, 0] == 0.0  # s = 2 mm belongs to column 33
    x[:] = 0.0
    x[:, 31, 0] = 1.0
    assert _native.line_integrals(sc, x)[0, r0, 0] == 0.0


@pytest.mark.parametrize("sc", [synth.config_2d(), synth.tiny_3d(steep=True)], ids=lambda s: s.name)
def test_adjoint_identity_and_definition_backprojection(sc):
    x = synth.random_image(sc, 3).astype(np.float64)
    y = synth.random_sinogram(sc, 4).astype(np.float64)
    for i in (-1, 1):
        Ax = oracle.project(sc, x, i)
        Aty = oracle.backproject(sc, y * oracle.subset_mask(sc, i), i)
        lhs, rhs = float((Ax * y).sum()), float((x * Aty).sum())
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
        vox = np.arange(0, sc.n_voxels, max(1, sc.n_voxels // 97), dtype=np.int64)
        by_def = _native.adjoint_at_voxels(sc, y, vox, i)
        np.testing.assert_allclose(by_def, Aty.ravel()[vox], rtol=1e-12, atol=1e-12)


def test_project_bins_matches_full_projection():
    sc = synth.tiny_3d()
    x = synth.random_image(sc, 8).astype(np.float64)
    full = _native.line_integrals(sc, x).ravel()
    bins = np.arange(0, sc.n_bins, 7, dtype=np.int64)
    np.testing.assert_array_equal(_native.line_integrals_at(sc, x, bins), full[bins])


def test_subset_adjoints_at_voxels_match_per_subset_backprojection():
    sc = synth.tiny_3d(n_subsets=2, steep=True)
    w = synth.random_sinogram(sc, 6).astype(np.float64)
    vox = np.arange(0, sc.n_voxels, 7, dtype=np.int64)
    got = _native.subset_adjoints_at_voxels(sc, w, vox)
    for i in range(sc.n_subsets):
        ref = oracle.backproject(sc, w * oracle.subset_mask(sc, i), i).ravel()[vox]
        np.testing.assert_allclose(got[:, i], ref, rtol=1e-12, atol=1e-12)
