"""Host-side launch bounds of the backprojector, checked by brute force on the CPU.

k_backward stages, per view, the radial rows that a 4 x 4 tile of voxel columns can touch; the
launcher sizes that staging buffer as floor(4 sqrt(2) vx / d_radial) + 4 rows (the projection of
the tile's pixel centres spans 3 (|cos| + |sin|) pixels, a footprint |cos| + |sin| more, at most
4 sqrt(2); the kernel's rounding ceil - 1 .. floor + 1 adds three rows).  A bound that is too
small would drop (pixel, bin) pairs silently, so it is checked here against the row range the
kernel computes (same FP32 formulas) for every view and tile of the test and benchmark
geometries.
"""
import math

import numpy as np
import pytest

import synth

TILE = 4


def rows_needed(sc):
    f = np.float32
    inv = f(sc.vx / sc.d_radial)
    half_r = f(0.5 * (sc.n_radial - 1))
    worst = 0
    tx = np.arange(0, sc.nx, TILE)
    ty = np.arange(0, sc.ny, TILE)
    X0 = (tx.astype(f) + f(0.5) - f(0.5) * f(sc.nx)).astype(f)
    Y0 = (ty.astype(f) + f(0.5) - f(0.5) * f(sc.ny)).astype(f)
    X0, Y0 = np.meshgrid(X0, Y0, indexing="ij")
    X1, Y1 = (X0 + f(TILE - 1)).astype(f), (Y0 + f(TILE - 1)).astype(f)
    for v in range(sc.n_views):
        c, s = math.cos(math.pi * v / sc.n_views), math.sin(math.pi * v / sc.n_views)
        c, s = f(0.0 if abs(c) < 1e-12 else c), f(0.0 if abs(s) < 1e-12 else s)
        hw = f(f(0.5) * (abs(c) + abs(s)))
        corners = [(X * c + Y * s).astype(f) for X in (X0, X1) for Y in (Y0, Y1)]
        smin = np.minimum(np.minimum(corners[0], corners[1]), np.minimum(corners[2], corners[3]))
        smax = np.maximum(np.maximum(corners[0], corners[1]), np.maximum(corners[2], corners[3]))
        r_min = np.ceil(((smin - hw) * inv + half_r).astype(f)).astype(np.int64) - 1
        r_max = np.floor(((smax + hw) * inv + half_r).astype(f)).astype(np.int64) + 1
        worst = max(worst, int((r_max - r_min + 1).max()))
    return worst


def staged_rows(sc):
    return int(math.floor(np.float32(TILE * 1.4143) * np.float32(sc.vx / sc.d_radial))) + 4


GEOMS = [synth.tiny_2d(), synth.tiny_3d(), synth.config_2d(), synth.config_3d_small(),
         synth.batch_geometries(7, 3, small=True)[0], synth.batch_geometries(1808, 4)[3]]


@pytest.mark.parametrize("sc", GEOMS, ids=lambda s: s.name)
def test_staged_rows_cover_every_tile_footprint(sc):
    assert rows_needed(sc) <= staged_rows(sc)


def test_staged_rows_at_mmr_scale():
    sc = synth.config_mmr()
    need = rows_needed(sc)
    assert need <= staged_rows(sc) == 9
    assert need >= 8  # the bound is tight within one row here
