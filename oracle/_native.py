"""Build and ctypes binding of the oracle's FP64 projector (siddon.c).

Test infrastructure only.  Compiled with plain gcc; OpenMP is used when the compiler
supports it (the forward projection and the per-voxel definition loop are parallel over
independent outputs, so the result does not depend on the thread count).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "siddon.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile siddon.c into oracle/_build/liboracle.so (skipped when up to date)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


class _Geom(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("vx", ctypes.c_double), ("vy", ctypes.c_double), ("vz", ctypes.c_double),
        ("n_radial", ctypes.c_int), ("d_radial", ctypes.c_double),
        ("n_views", ctypes.c_int), ("radius", ctypes.c_double),
        ("n_seg", ctypes.c_int),
        ("seg_n", ctypes.POINTER(ctypes.c_int)),
        ("seg_zmid0", ctypes.POINTER(ctypes.c_double)),
        ("seg_dzmid", ctypes.POINTER(ctypes.c_double)),
        ("seg_dz", ctypes.POINTER(ctypes.c_double)),
        ("n_subsets", ctypes.c_int),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        P = ctypes.POINTER
        dp = P(ctypes.c_double)
        lp = P(ctypes.c_long)
        gp = P(_Geom)
        L.og_project.argtypes = [gp, dp, dp, ctypes.c_int]
        L.og_backproject.argtypes = [gp, dp, dp, ctypes.c_int]
        L.og_project_bins.argtypes = [gp, dp, ctypes.c_long, lp, dp]
        L.og_backproject_voxels.argtypes = [gp, dp, ctypes.c_int, ctypes.c_long, lp, dp]
        L.og_dense_clip.argtypes = [gp, dp]
        L.og_subset_sums_at_voxels.argtypes = [gp, dp, ctypes.c_long, lp, dp]
        L.og_threads.restype = ctypes.c_int
        _lib = L
    return _lib


class CGeom:
    """Keeps the ctypes geometry struct and its arrays alive."""

    def __init__(self, sc):
        self.sc = sc
        n = len(sc.seg_n)
        self._n = (ctypes.c_int * n)(*sc.seg_n)
        self._z0 = (ctypes.c_double * n)(*sc.seg_zmid0)
        self._dzm = (ctypes.c_double * n)(*sc.seg_dzmid)
        self._dz = (ctypes.c_double * n)(*sc.seg_dz)
        self.s = _Geom(sc.nx, sc.ny, sc.nz, sc.vx, sc.vy, sc.vz, sc.n_radial, sc.d_radial,
                       sc.n_views, sc.radius, n, self._n, self._z0, self._dzm, self._dz,
                       sc.n_subsets)

    @property
    def ref(self):
        return ctypes.byref(self.s)


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_long))


def line_integrals(sc, x, subset=-1):
    """L x over the subset's bins (float64, full sinogram shape, other bins 0)."""
    x = np.ascontiguousarray(x, np.float64)
    y = np.zeros(sc.sino_shape, np.float64)
    lib().og_project(CGeom(sc).ref, _dptr(x), _dptr(y), int(subset))
    return y


def line_integrals_adjoint(sc, y, subset=-1):
    """L_subset^T y (float64 image)."""
    y = np.ascontiguousarray(y, np.float64)
    x = np.zeros(sc.image_shape, np.float64)
    lib().og_backproject(CGeom(sc).ref, _dptr(y), _dptr(x), int(subset))
    return x


def line_integrals_at(sc, x, bins):
    x = np.ascontiguousarray(x, np.float64)
    bins = np.ascontiguousarray(bins, np.int64)
    out = np.zeros(len(bins), np.float64)
    lib().og_project_bins(CGeom(sc).ref, _dptr(x), len(bins), _lptr(bins), _dptr(out))
    return out


def adjoint_at_voxels(sc, y, voxels, subset=-1):
    y = np.ascontiguousarray(y, np.float64)
    voxels = np.ascontiguousarray(voxels, np.int64)
    out = np.zeros(len(voxels), np.float64)
    lib().og_backproject_voxels(CGeom(sc).ref, _dptr(y), int(subset), len(voxels), _lptr(voxels), _dptr(out))
    return out


def subset_adjoints_at_voxels(sc, w, voxels):
    """(len(voxels), n_subsets): (L_i^T w) at each voxel for every subset i, by the definition."""
    w = np.ascontiguousarray(w, np.float64)
    voxels = np.ascontiguousarray(voxels, np.int64)
    out = np.zeros((len(voxels), sc.n_subsets), np.float64)
    lib().og_subset_sums_at_voxels(CGeom(sc).ref, _dptr(w), len(voxels), _lptr(voxels), _dptr(out))
    return out


def dense_by_clipping(sc):
    A = np.zeros((sc.n_bins, sc.n_voxels), np.float64)
    lib().og_dense_clip(CGeom(sc).ref, _dptr(A))
    return A


def threads() -> int:
    return int(lib().og_threads())
