"""Seeded synthetic inputs shared by the CUDA path, the oracle, the tests and the bench.

This module describes *inputs* only: scanner geometries, phantoms, side images, per-bin
multipliers and Poisson data.  It contains none of the reconstruction method's arithmetic
(no discrete projector, no proximal operator, no step sizes, no sampler): the measured data
are drawn from the *analytic* line integrals of continuous ellipsoid phantoms, so neither the
oracle nor the CUDA path is needed (or used) to make them.

Conventions (the same ones the C ABI documents):

* image ``x[iy][ix][iz]`` (z fastest), voxel ``(ix, iy, iz)`` occupies
  ``[X_ix, X_ix+1) x [Y_iy, Y_iy+1) x [Z_iz, Z_iz+1)`` with ``X_i = -nx*vx/2 + i*vx`` etc.;
* sinogram ``y[view][radial][plane]`` (plane fastest); view ``v`` has angle ``phi = v*pi/V``,
  radial bin ``r`` sits at ``s = (r - (R-1)/2) * d_radial``;
* planes are grouped in segments (a michelogram segment: a fixed axial LOR tilt).  Plane ``q``
  of segment ``g`` has its LOR mid-point at ``z_mid = seg_zmid0[g] + q*seg_dzmid[g]`` and its
  two detector ends ``seg_dz[g]`` apart axially;
* LOR ``(v, r, p)`` is the segment between two points of a cylinder of radius ``radius``:
  ``P(t) = (s cos phi - t sin phi, s sin phi + t cos phi, z_mid + t * dz / (2h))`` for
  ``t in [-h, h]``, ``h = sqrt(radius^2 - s^2)``;
* lengths are measured in units of the transaxial voxel size ``vx``.
"""
from __future__ import annotations

import dataclasses
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np

__all__ = [
    "Scanner", "config_2d", "config_3d", "config_3d_oblique", "config_3d_small", "config_mmr", "config_mmr_exact",
    "tiny_2d", "tiny_3d", "tiny_mashed", "batch_geometries", "component_scanners",
    "Ellipsoid", "random_phantom", "voxelize", "analytic_projection", "smooth_multipliers",
    "side_image", "make_problem", "random_image", "random_sinogram", "subset_views",
]


@dataclasses.dataclass(frozen=True)
class Scanner:
    """Image grid + cylindrical-scanner sinogram description (input data, no method)."""
    nx: int
    ny: int
    nz: int
    vx: float
    vy: float
    vz: float
    n_radial: int
    d_radial: float
    n_views: int
    radius: float
    seg_n: tuple
    seg_zmid0: tuple
    seg_dzmid: tuple
    seg_dz: tuple
    n_subsets: int
    name: str = ""
    subset_kind: str = "views"  # "views": view-interleaved subsets; "bins": bin j in subset j mod m
    # Exact mashing: per segment, the LOR components summed into its bins, each (dz_mm, q_lo,
    # q_hi, step): plane q of the segment includes the component's LOR (axial separation dz_mm,
    # the plane's mid-point) when q_lo <= q < q_hi and (q - q_lo) % step == 0.  Empty: every bin
    # is the single LOR of its segment's seg_dz.
    components: tuple = ()

    @property
    def n_planes(self) -> int:
        return int(sum(self.seg_n))

    @property
    def n_bins(self) -> int:
        return self.n_views * self.n_radial * self.n_planes

    @property
    def n_voxels(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def image_shape(self):
        return (self.ny, self.nx, self.nz)

    @property
    def sino_shape(self):
        return (self.n_views, self.n_radial, self.n_planes)

    def with_subsets(self, m: int, kind: str = None) -> "Scanner":
        return dataclasses.replace(self, n_subsets=m, subset_kind=self.subset_kind if kind is None else kind)

    def plane_table(self):
        """Per-plane (z_mid, dz) in plane order (segment-major)."""
        zm, dz = [], []
        for n, z0, dzm, d in zip(self.seg_n, self.seg_zmid0, self.seg_dzmid, self.seg_dz):
            for q in range(n):
                zm.append(z0 + q * dzm)
                dz.append(d)
        return np.asarray(zm, np.float64), np.asarray(dz, np.float64)

    def as_dict(self):
        return dataclasses.asdict(self)


def component_scanners(g: Scanner):
    """The LOR families of a scanner with mashed bins: one single-segment scanner per component
    (its planes at the component's spacing and axial separation) with the sinogram planes it
    adds to.  None when the bins are not mashed."""
    if not g.components:
        return None
    out = []
    p0 = 0
    for gi, (n, z0, dzm) in enumerate(zip(g.seg_n, g.seg_zmid0, g.seg_dzmid)):
        for dz, qlo, qhi, step in g.components[gi]:
            qs = list(range(int(qlo), int(qhi), int(step)))
            if qs:
                vs = dataclasses.replace(g, seg_n=(len(qs),), seg_zmid0=(z0 + qlo * dzm,), seg_dzmid=(step * dzm,),
                                         seg_dz=(float(dz),), components=(), name=f"{g.name}-comp")
                out.append((vs, np.asarray([p0 + q for q in qs], np.int64)))
        p0 += n
    return out


def subset_views(g: Scanner, i: int):
    """Views of the view-interleaved subset i (evenly spaced view angles)."""
    return list(range(i, g.n_views, g.n_subsets))


# --------------------------------------------------------------------------------------
# geometries of the synthetic workloads
# --------------------------------------------------------------------------------------

def config_2d(n_subsets: int = 10) -> Scanner:
    """2-D PET: 64x64 image at 2 mm, parallel sinogram 90 views x 95 radial bins at 2 mm."""
    return Scanner(nx=64, ny=64, nz=1, vx=2.0, vy=2.0, vz=2.0, n_radial=95, d_radial=2.0,
                   n_views=90, radius=200.0, seg_n=(1,), seg_zmid0=(0.0,), seg_dzmid=(2.0,),
                   seg_dz=(0.0,), n_subsets=n_subsets, name="pet2d-64x64-90v95r")


def config_3d(n_subsets: int = 21) -> Scanner:
    """3-D cylindrical scanner: 128x128x64 voxels at 2 mm, 128 radial x 180 views x 64 planes.

    Each of the 64 planes is the direct plane of one ring; the adjacent-oblique pairs that
    share its axial centre have a mean ring difference of zero, so the representative LOR of
    the plane is the direct one (axial position = slice centre).
    """
    return Scanner(nx=128, ny=128, nz=64, vx=2.0, vy=2.0, vz=2.0, n_radial=128, d_radial=2.0,
                   n_views=180, radius=300.0, seg_n=(64,), seg_zmid0=(-63.0,), seg_dzmid=(2.0,),
                   seg_dz=(0.0,), n_subsets=n_subsets, name="cyl3d-128x128x64-180v128r64p")


def config_3d_oblique(n_subsets: int = 21) -> Scanner:
    """The 3-D configuration with its adjacent-oblique planes summed exactly: plane p is the direct
    LOR of ring p plus the two LORs of rings (p-1, p+1) and (p+1, p-1), which share its axial
    centre (ring difference +-2, i.e. +-4 mm with 2 mm rings; only the direct LOR at the two edge
    planes)."""
    g = config_3d(n_subsets)
    ring = 2.0
    comps = ((0.0, 0, 64, 1), (2 * ring, 1, 63, 1), (-2 * ring, 1, 63, 1))
    return dataclasses.replace(g, components=(comps,), name="cyl3d-oblique-128x128x64-180v128r64p")


def tiny_mashed(n_subsets: int = 2) -> Scanner:
    """The steep tiny scanner with mashed bins: each plane of the direct segment sums its direct
    LOR and, on its three inner planes, two LORs tilted by +-1 mm; the oblique segments hold
    LORs of two tilts on alternating planes (the range and parity rules of exact mashing)."""
    g = tiny_3d(n_subsets, steep=True)
    c0 = ((0.0, 0, 5, 1), (1.0, 1, 4, 1), (-1.0, 1, 4, 1))
    c1 = ((8.0, 0, 4, 2), (6.0, 1, 4, 2))
    c2 = ((-8.0, 0, 4, 2), (-6.0, 1, 4, 2))
    return dataclasses.replace(g, components=(c0, c1, c2), name="tiny3d-mashed")


MMR_SPAN11_DIFFS = ((-5, 5), (6, 16), (-16, -6), (17, 27), (-27, -17), (28, 38), (-38, -28), (39, 49),
                    (-49, -39), (50, 60), (-60, -50))


def config_mmr_exact(n_subsets: int = 252) -> Scanner:
    """The mMR-like scanner with exact span-11 mashing: a bin of segment g at ring sum s sums the
    LORs of every ring pair (r1, r2) with r1 + r2 = s and r1 - r2 in the segment's ring-difference
    range (64 rings; ring difference d has ring sums |d| .. 126 - |d| of d's parity)."""
    g = config_mmr(n_subsets)
    ring_pitch = 2.0 * g.vz
    comps = []
    for (first, n, _), (d_lo, d_hi) in zip(MMR_SPAN11_SEGMENTS, MMR_SPAN11_DIFFS):
        cs = []
        for d in range(d_lo, d_hi + 1):
            s_lo, s_hi = abs(d), 126 - abs(d)          # ring sums of the pairs with this difference
            q_lo, q_hi = s_lo - first, s_hi - first + 1
            q_lo, q_hi = max(q_lo, 0), min(q_hi, n)
            if q_lo < q_hi:
                cs.append((d * ring_pitch, q_lo, q_hi, 2))
        comps.append(tuple(cs))
    return dataclasses.replace(g, components=tuple(comps), name="mmr-exact-span11-344x344x127-252v344r837p")


def config_3d_small(n_subsets: int = 8) -> Scanner:
    """The 3-D configuration's scanner at test size: 32x32x16 voxels at 2 mm, 48 views x 32 radial
    x 16 direct planes, R = 60 mm."""
    return Scanner(nx=32, ny=32, nz=16, vx=2.0, vy=2.0, vz=2.0, n_radial=32, d_radial=2.0,
                   n_views=48, radius=60.0, seg_n=(16,), seg_zmid0=(-15.0,), seg_dzmid=(2.0,),
                   seg_dz=(0.0,), n_subsets=n_subsets, name="cyl3d-small-32x32x16-48v32r16p")


MMR_SPAN11_SEGMENTS = (  # (first ring-sum, planes, nominal ring difference)
    (0, 127, 0), (6, 115, 11), (6, 115, -11), (17, 93, 22), (17, 93, -22),
    (28, 71, 33), (28, 71, -33), (39, 49, 44), (39, 49, -44), (50, 27, 55), (50, 27, -55),
)


def config_mmr(n_subsets: int = 252) -> Scanner:
    """mMR-like scale: 344x344x127 voxels at 2.08 mm, span-11-like 344 radial x 252 views x 837 planes.

    64 rings at a pitch of two slices.  Segment g collects the ring pairs whose ring
    difference lies in its span-11 range; plane k of the segment has ring sum
    ``first_sum + k`` (axial mid-point on a slice centre) and every LOR of the segment uses
    the segment's nominal ring difference (0, +-11, ..., +-55 rings).
    """
    vz = 2.08
    ring_pitch = 2.0 * vz
    seg_n, seg_z0, seg_dzm, seg_dz = [], [], [], []
    for first, n, rd in MMR_SPAN11_SEGMENTS:
        seg_n.append(n)
        seg_z0.append((first - 63) * vz)
        seg_dzm.append(vz)
        seg_dz.append(rd * ring_pitch)
    return Scanner(nx=344, ny=344, nz=127, vx=2.08, vy=2.08, vz=vz, n_radial=344,
                   d_radial=2.08, n_views=252, radius=380.0, seg_n=tuple(seg_n),
                   seg_zmid0=tuple(seg_z0), seg_dzmid=tuple(seg_dzm), seg_dz=tuple(seg_dz),
                   n_subsets=n_subsets, name="mmr-344x344x127-252v344r837p")


def tiny_2d(n_subsets: int = 3) -> Scanner:
    """8x8 pixels, 6 views x 11 radial bins; bins at pixel boundaries and centres."""
    return Scanner(nx=8, ny=8, nz=1, vx=1.0, vy=1.0, vz=1.0, n_radial=11, d_radial=0.75,
                   n_views=6, radius=20.0, seg_n=(1,), seg_zmid0=(0.0,), seg_dzmid=(1.0,),
                   seg_dz=(0.0,), n_subsets=n_subsets, name="tiny2d")


def tiny_3d(n_subsets: int = 2, steep: bool = False) -> Scanner:
    """6x6x5 voxels with a direct segment and two oblique segments.

    ``steep`` shrinks the scanner so that an oblique LOR can cross three slices inside one
    transaxial pixel.
    """
    radius = 5.0 if steep else 12.0
    dz = 8.0 if steep else 3.0
    return Scanner(nx=6, ny=6, nz=5, vx=1.0, vy=1.0, vz=1.0, n_radial=9, d_radial=0.8,
                   n_views=4, radius=radius, seg_n=(5, 4, 4), seg_zmid0=(-2.0, -1.75, -1.75),
                   seg_dzmid=(1.0, 1.0, 1.0), seg_dz=(0.0, dz, -dz), n_subsets=n_subsets,
                   name="tiny3d-steep" if steep else "tiny3d")


def batch_geometries(seed: int, count: int = 16, small: bool = False):
    """Uneven 3-D problems: 96^3 .. 200x200x100 voxels, 120-252 views (direct + 2 oblique segments).

    small=True draws the same kind of scanner at test size: 24..48 pixels across, 10..16 slices,
    24..40 views.
    """
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        if small:
            nxy = int(rng.integers(24, 49))
            nz = int(rng.integers(10, 17))
            views = int(rng.integers(24, 41))
        else:
            nxy = int(rng.integers(96, 201))
            nz = int(rng.integers(96 if nxy < 100 else 64, 101))
            views = int(rng.integers(120, 253))
        v = 2.0
        half = nxy * v / 2
        nr = nxy
        radius = math.ceil(math.hypot(half, half)) + 10.0
        # one direct segment and a +-tilted pair, planes on slice centres
        off = 2 if small else 4  # oblique planes start `off` slices in from either end
        n_ob = max(nz - 2 * off, 1)
        z0 = -(nz - 1) * v / 2
        out.append(Scanner(nx=nxy, ny=nxy, nz=nz, vx=v, vy=v, vz=v, n_radial=nr, d_radial=v,
                           n_views=views, radius=radius, seg_n=(nz, n_ob, n_ob),
                           seg_zmid0=(z0, z0 + off * v, z0 + off * v), seg_dzmid=(v, v, v),
                           seg_dz=(0.0, 6 * v, -6 * v),
                           n_subsets=max(views // (4 if small else 12), 1),
                           name=f"batch{k}-{nxy}x{nxy}x{nz}-{views}v"))
    return out


# --------------------------------------------------------------------------------------
# phantoms
# --------------------------------------------------------------------------------------

@dataclasses.dataclass(frozen=True)
class Ellipsoid:
    cx: float
    cy: float
    cz: float
    ax: float
    ay: float
    az: float
    theta: float  # rotation about z
    value: float


def _extent(g: Scanner):
    return g.nx * g.vx / 2.0, g.ny * g.vy / 2.0, g.nz * g.vz / 2.0


def random_phantom(g: Scanner, seed: int, n: int = 10):
    """A body ellipsoid plus n-1 random inner ellipsoids with values in [0, 1] (additive)."""
    rng = np.random.default_rng(seed)
    hx, hy, hz = _extent(g)
    fov = min(hx, hy, math.sqrt(max(g.radius ** 2 - (g.n_radial * g.d_radial / 2) ** 2, 0.0)) + 1e9)
    rt = 0.8 * min(hx, hy, fov)
    flat = g.nz == 1
    body_z = 1e9 if flat else 0.85 * hz
    ells = [Ellipsoid(0.0, 0.0, 0.0, 0.85 * rt, 0.75 * rt, body_z, 0.0, float(rng.uniform(0.15, 0.3)))]
    for _ in range(n - 1):
        ax, ay = rng.uniform(0.06, 0.3, size=2) * rt
        az = 1e9 if flat else float(rng.uniform(0.1, 0.4) * hz)
        rho = rng.uniform(0.0, 0.5) * rt
        ang = rng.uniform(0, 2 * np.pi)
        cz = 0.0 if flat else float(rng.uniform(-0.5, 0.5) * hz)
        ells.append(Ellipsoid(float(rho * np.cos(ang)), float(rho * np.sin(ang)), cz, float(ax), float(ay),
                              az, float(rng.uniform(0, np.pi)), float(rng.uniform(0.0, 1.0))))
    return ells


def _voxel_centres(g: Scanner):
    xs = -g.nx * g.vx / 2 + (np.arange(g.nx) + 0.5) * g.vx
    ys = -g.ny * g.vy / 2 + (np.arange(g.ny) + 0.5) * g.vy
    zs = -g.nz * g.vz / 2 + (np.arange(g.nz) + 0.5) * g.vz
    return xs, ys, zs


def voxelize(g: Scanner, ells, dtype=np.float32):
    """Sample the additive ellipsoid phantom at voxel centres; layout [iy][ix][iz]."""
    xs, ys, zs = _voxel_centres(g)
    out = np.zeros(g.image_shape, np.float64)
    Y, X = np.meshgrid(ys, xs, indexing="ij")  # (ny, nx)
    for e in ells:
        ct, st = math.cos(e.theta), math.sin(e.theta)
        dx, dy = X - e.cx, Y - e.cy
        u = (ct * dx + st * dy) / e.ax
        w = (-st * dx + ct * dy) / e.ay
        q2 = u * u + w * w  # (ny, nx)
        zt = ((zs - e.cz) / e.az) ** 2  # (nz,)
        inside = (q2[:, :, None] + zt[None, None, :]) <= 1.0
        out += e.value * inside
    return out.astype(dtype)


def _view_lors(g: Scanner, v: int):
    """o, d (each (3, R, P)) and h (R,) of every LOR of view v (float64)."""
    phi = math.pi * v / g.n_views
    c, sn = math.cos(phi), math.sin(phi)
    if abs(c) < 1e-12:
        c = 0.0
    if abs(sn) < 1e-12:
        sn = 0.0
    s = (np.arange(g.n_radial) - (g.n_radial - 1) / 2.0) * g.d_radial
    h = np.sqrt(g.radius ** 2 - s ** 2)
    zm, dz = g.plane_table()
    R, P = g.n_radial, g.n_planes
    o = np.empty((3, R, P))
    d = np.empty((3, R, P))
    o[0] = (s * c)[:, None]
    o[1] = (s * sn)[:, None]
    o[2] = zm[None, :]
    d[0] = -sn
    d[1] = c
    d[2] = dz[None, :] / (2.0 * h[:, None])
    return o, d, h


def _project_views(g: Scanner, ells, v0: int, v1: int):
    """Exact chords of views v0..v1-1 (the same elementwise arithmetic for every bin as one view
    at a time, so the result does not depend on the grouping)."""
    parts = [_view_lors(g, v) for v in range(v0, v1)]
    o = np.stack([q[0] for q in parts], axis=1)              # (3, G, R, P)
    d = np.stack([q[1] for q in parts], axis=1)
    hh = parts[0][2][None, :, None]                          # h depends on the radial bin only
    dnorm = np.sqrt((d * d).sum(0))
    acc = np.zeros(o.shape[1:])
    for e in ells:
        ct, st = math.cos(e.theta), math.sin(e.theta)
        # rotate into the ellipsoid frame and scale to the unit sphere
        px, py, pz = o[0] - e.cx, o[1] - e.cy, o[2] - e.cz
        p0 = np.stack([(ct * px + st * py) / e.ax, (-st * px + ct * py) / e.ay, pz / e.az])
        d0 = np.stack([(ct * d[0] + st * d[1]) / e.ax, (-st * d[0] + ct * d[1]) / e.ay, d[2] / e.az])
        A = (d0 * d0).sum(0)
        B = (p0 * d0).sum(0)
        C = (p0 * p0).sum(0) - 1.0
        disc = B * B - A * C
        ok = disc > 0
        sq = np.sqrt(np.where(ok, disc, 0.0))
        t1 = (-B - sq) / A
        t2 = (-B + sq) / A
        seg = np.clip(np.minimum(t2, hh) - np.maximum(t1, -hh), 0.0, None)
        acc += e.value * np.where(ok, seg, 0.0)
    return acc * dnorm / g.vx


def analytic_projection(g: Scanner, ells, threads: int = 0):
    """Exact line integrals of the continuous phantom along every LOR (voxel-size units); a
    mashed bin holds the sum over its LOR components."""
    comps = component_scanners(g)
    if comps is not None:
        out = np.zeros(g.sino_shape, np.float64)
        for vs, planes in comps:
            out[:, :, planes] += analytic_projection(vs, ells, threads)
        return out
    out = np.empty(g.sino_shape, np.float64)
    workers = threads or min(32, max(1, (__import__("os").cpu_count() or 1)))
    group = max(1, min(g.n_views, (1 << 18) // max(1, g.n_radial * g.n_planes)))
    starts = list(range(0, g.n_views, group))

    def work(v0):
        v1 = min(g.n_views, v0 + group)
        out[v0:v1] = _project_views(g, ells, v0, v1)

    with ThreadPoolExecutor(workers) as ex:
        list(ex.map(work, starts))
    return out


def smooth_multipliers(g: Scanner, seed: int):
    """Attenuation x normalisation per bin: norm in [0.8, 1.2] (low-order cosines),
    attenuation exp(-a) with a smooth a in [0, 2]."""
    rng = np.random.default_rng(seed)
    ph = rng.uniform(0, 2 * np.pi, size=4)
    R, P, V = g.n_radial, g.n_planes, g.n_views
    r = np.arange(R)[:, None]
    p = np.arange(P)[None, :]
    norm_rp = 1.0 + 0.1 * np.cos(2 * np.pi * 3 * r / R + ph[0]) + 0.1 * np.cos(2 * np.pi * 2 * p / P + ph[1])
    s = (np.arange(R) - (R - 1) / 2.0) * g.d_radial
    smax = 0.8 * np.abs(s).max()
    prof = np.clip(1.0 - (s / smax) ** 2, 0.0, None)  # (R,)
    out = np.empty(g.sino_shape, np.float32)
    for v in range(V):
        phi = math.pi * v / V
        a = 2.0 * prof * (0.9 + 0.1 * math.cos(2 * phi + ph[2]))
        out[v] = (norm_rp * np.exp(-a)[:, None]).astype(np.float32)
    return out


def side_image(g: Scanner, phantom_ells, seed: int):
    """Anatomical side image: half of the phantom's ellipsoids (new values) plus extra edges."""
    rng = np.random.default_rng(seed)
    keep = [dataclasses.replace(e, value=float(rng.uniform(0.2, 1.0))) for e in phantom_ells[::2]]
    extra = random_phantom(g, seed + 7919, n=4)[1:]
    return voxelize(g, keep + extra)


def make_problem(g: Scanner, seed: int, counts: float, bg_frac: float, with_mult: bool = False,
                 with_side: bool = False, n_ellipsoids: int = 10, threads: int = 0):
    """Seeded PET problem: b ~ Poisson(mult * kappa * L_analytic + r).

    ``counts`` is the expected total of the trues ``sum(mult * kappa * L_analytic)``,
    ``r`` is a constant background equal to ``bg_frac`` times the mean of the trues.
    Returns a dict with float32 arrays b, r, mult (or None), side (or None), x_true (scaled so
    that it is in the same units as the reconstruction).
    Seeds: phantom ``seed``, noise ``seed + 1``, multipliers ``seed + 3``, side image ``seed + 4``.
    """
    ells = random_phantom(g, seed, n=n_ellipsoids)
    proj = analytic_projection(g, ells, threads=threads)
    mult = smooth_multipliers(g, seed + 3) if with_mult else None
    trues = proj if mult is None else proj * mult
    kappa = counts / trues.sum()
    trues = trues * kappa
    r_val = bg_frac * trues.mean()
    lam = trues + r_val
    b = np.empty(g.sino_shape, np.float32)

    def noise(v):
        b[v] = np.random.default_rng([seed + 1, v]).poisson(lam[v]).astype(np.float32)

    with ThreadPoolExecutor(min(32, (__import__("os").cpu_count() or 1))) as ex:
        list(ex.map(noise, range(g.n_views)))
    return dict(
        b=b,
        r=np.full(g.sino_shape, r_val, np.float32),
        mult=mult,
        side=side_image(g, ells, seed + 4) if with_side else None,
        x_true=(voxelize(g, ells) * kappa).astype(np.float32),
        ellipsoids=ells,
        kappa=kappa,
    )


def random_image(g: Scanner, seed: int, nonneg: bool = True, dtype=np.float32):
    rng = np.random.default_rng(seed)
    x = rng.random(g.image_shape) if nonneg else rng.standard_normal(g.image_shape)
    return x.astype(dtype)


def random_sinogram(g: Scanner, seed: int, nonneg: bool = False, dtype=np.float32):
    rng = np.random.default_rng(seed)
    y = rng.random(g.sino_shape) if nonneg else rng.standard_normal(g.sino_shape)
    return y.astype(dtype)
