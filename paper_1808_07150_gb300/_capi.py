"""ctypes binding of include/spdhg.h (argument marshalling only).

Every function here forwards to the CUDA library libspdhg.so; nothing is computed in Python.
If the library has not been built (``__graft_entry__.build()`` or
``python -m paper_1808_07150_gb300._build_ext``) loading fails loudly: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import _build_ext

OK = 0
ERR_ARG, ERR_CUDA, ERR_OOM, ERR_DATA, ERR_TIMEOUT, ERR_DIVERGED, ERR_STATE, ERR_UNSUPPORTED = range(-1, -9, -1)
WHERE_HOST, WHERE_DEVICE = 0, 1
PRIOR = {"none": 0, "tv": 1, "dtv": 2, "atv": 3, "tgv": 4}
SAMPLING = {"balanced": 0, "uniform": 1, "custom": 2}
SUBSETS = {"views": 0, "bins": 1}
STATE = {"x": 0, "z": 1, "T": 2, "y": 3, "q": 4, "sigma": 5, "w": 6, "zw": 7, "q2": 8}

_EXPORTS = [
    "spdhg_create", "spdhg_create_geometry", "spdhg_destroy", "spdhg_last_error", "spdhg_sizes", "spdhg_set_data",
    "spdhg_project", "spdhg_backproject", "spdhg_setup", "spdhg_iterate", "spdhg_get",
    "spdhg_objective", "spdhg_probabilities", "spdhg_sample", "spdhg_run", "spdhg_profile",
    "spdhg_profile_read", "spdhg_backproject_noalloc", "spdhg_tune", "spdhg_autotune",
    "spdhg_run_batch", "spdhg_set", "spdhg_save_state", "spdhg_load_state", "spdhg_psnr", "spdhg_osem",
    "spdhg_set_memory_limit",
    "unet_gemm", "unet_device_error", "unet_create", "unet_destroy", "unet_last_error", "unet_num_params",
    "unet_set_params", "unet_init", "unet_get_params", "unet_get_grads", "unet_forward", "unet_backward", "unet_adam_step",
]
TUNE = {"prior_cols": 0, "prior_ychunk": 1, "fwd_split": 2, "fwd_warps": 3, "prior_stages": 4, "bwd_table": 5,
        "fwd_groups": 6, "prior_vz": 7}
TUNE_KNOBS = 8
KERNELS = ["forward", "backward", "prior", "tgv", "w_step"]


class SpdhgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"spdhg error {code}: {msg}")
        self.code = code


class Geometry(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int),
        ("vx", ctypes.c_double), ("vy", ctypes.c_double), ("vz", ctypes.c_double),
        ("n_radial", ctypes.c_int), ("d_radial", ctypes.c_double), ("n_views", ctypes.c_int),
        ("radius", ctypes.c_double), ("n_segments", ctypes.c_int),
        ("seg_n", ctypes.POINTER(ctypes.c_int)), ("seg_zmid0", ctypes.POINTER(ctypes.c_double)),
        ("seg_dzmid", ctypes.POINTER(ctypes.c_double)), ("seg_dz", ctypes.POINTER(ctypes.c_double)),
        ("n_subsets", ctypes.c_int), ("n_components", ctypes.c_int),
        ("comp_seg", ctypes.POINTER(ctypes.c_int)), ("comp_dz", ctypes.POINTER(ctypes.c_double)),
        ("comp_qlo", ctypes.POINTER(ctypes.c_int)), ("comp_qhi", ctypes.POINTER(ctypes.c_int)),
        ("comp_step", ctypes.POINTER(ctypes.c_int)), ("subset_kind", ctypes.c_int),
    ]


class Params(ctypes.Structure):
    _fields_ = [
        ("prior", ctypes.c_int), ("alpha", ctypes.c_double), ("alpha0", ctypes.c_double),
        ("alpha1", ctypes.c_double), ("dtv_gamma", ctypes.c_double), ("dtv_eta_frac", ctypes.c_double),
        ("sampling", ctypes.c_int), ("precond", ctypes.c_int), ("rho", ctypes.c_double),
        ("gamma", ctypes.c_double), ("seed", ctypes.c_uint64), ("epochs", ctypes.c_int),
        ("objective_every", ctypes.c_int), ("graph", ctypes.c_int),
        ("target_gap", ctypes.c_double), ("psi_star", ctypes.c_double), ("x_star", ctypes.c_void_p),
        ("probs", ctypes.POINTER(ctypes.c_double)),
    ]


class Report(ctypes.Structure):
    _fields_ = [
        ("epochs_done", ctypes.c_int), ("iterations_done", ctypes.c_int64),
        ("objective", ctypes.POINTER(ctypes.c_double)), ("epoch_ms", ctypes.POINTER(ctypes.c_double)),
        ("psnr", ctypes.POINTER(ctypes.c_double)), ("stop_epoch", ctypes.c_int), ("ms_to_stop", ctypes.c_double),
        ("psi_zero", ctypes.c_double),
    ]


_lib = None


def library_path() -> str:
    return _build_ext.LIB


def lib():
    """The loaded libspdhg.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        path = _build_ext.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libspdhg.so not built ({path}); run __graft_entry__.build() first")
        L = ctypes.CDLL(path)
        vp, i32, i64, u64, dp = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        P = ctypes.POINTER
        sig = {
            "spdhg_create": ([P(Geometry), P(vp)], i32),
            "spdhg_create_geometry": ([P(Geometry), P(vp)], i32),
            "spdhg_destroy": ([vp], None),
            "spdhg_last_error": ([vp], ctypes.c_char_p),
            "spdhg_sizes": ([vp, P(i64), P(i64), P(i32)], i32),
            "spdhg_set_data": ([vp, vp, vp, vp, vp, i32], i32),
            "spdhg_project": ([vp, vp, vp, i32, vp], i32),
            "spdhg_backproject": ([vp, vp, vp, i32, vp], i32),
            "spdhg_setup": ([vp, P(Params), vp, i32, vp], i32),
            "spdhg_iterate": ([vp, P(ctypes.c_int32), i32, vp], i32),
            "spdhg_get": ([vp, i32, vp, i32, vp], i32),
            "spdhg_set": ([vp, i32, vp, i32, vp], i32),
            "spdhg_save_state": ([vp, ctypes.c_char_p], i32),
            "spdhg_load_state": ([vp, ctypes.c_char_p], i32),
            "spdhg_objective": ([vp, vp, i32, P(dp), vp], i32),
            "spdhg_probabilities": ([vp, P(dp), P(i32)], i32),
            "spdhg_sample": ([u64, u64, i32, P(dp), i32, P(ctypes.c_int32)], i32),
            "spdhg_run": ([vp, P(Params), vp, i32, P(Report), vp], i32),
            "spdhg_profile": ([vp, i32], i32),
            "spdhg_profile_read": ([vp, P(dp), P(i64), i32], i32),
            "spdhg_backproject_noalloc": ([vp, vp, vp, i32, vp], i32),
            "spdhg_tune": ([vp, i32, i32], i32),
            "spdhg_set_memory_limit": ([vp, u64, P(u64)], i32),
            "spdhg_autotune": ([vp, i32, P(i32), vp], i32),
            "spdhg_run_batch": ([P(vp), P(Params), P(vp), i32, i32, P(Report), vp], i32),
            "spdhg_psnr": ([vp, vp, vp, i32, P(dp), vp], i32),
            "spdhg_osem": ([vp, P(Params), i32, vp, i32, P(Report), vp], i32),
            "unet_gemm": ([vp, vp, vp, i32, i32, i32, i32, vp], i32),
            "unet_device_error": ([vp], i32),
            "unet_create": ([i32, P(i32), i32, i32, i32, P(vp)], i32),
            "unet_destroy": ([vp], None),
            "unet_last_error": ([vp], ctypes.c_char_p),
            "unet_num_params": ([vp], i64),
            "unet_set_params": ([vp, P(ctypes.c_float), i64], i32),
            "unet_get_params": ([vp, P(ctypes.c_float), i64], i32),
            "unet_init": ([vp, u64], i32),
            "unet_get_grads": ([vp, P(ctypes.c_float), i64], i32),
            "unet_forward": ([vp, vp, ctypes.c_float, vp, vp, vp], i32),
            "unet_backward": ([vp, vp, vp, i32, P(dp), vp], i32),
            "unet_adam_step": ([vp, ctypes.c_float, vp], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return list(_EXPORTS)


def check(code, ctx=None):
    if code != OK:
        msg = lib().spdhg_last_error(ctx).decode() if ctx else ""
        raise SpdhgError(code, msg)


def make_geometry(sc):
    """ctypes Geometry from any object with the Scanner fields; returns (struct, keepalive)."""
    n = len(sc.seg_n)
    keep = [(ctypes.c_int * n)(*sc.seg_n), (ctypes.c_double * n)(*sc.seg_zmid0),
            (ctypes.c_double * n)(*sc.seg_dzmid), (ctypes.c_double * n)(*sc.seg_dz)]
    comps = [(k, c) for k, cs in enumerate(getattr(sc, "components", ()) or ()) for c in cs]
    nc = len(comps)
    ck = [(ctypes.c_int * max(nc, 1))(*[k for k, _ in comps]),
          (ctypes.c_double * max(nc, 1))(*[float(c[0]) for _, c in comps]),
          (ctypes.c_int * max(nc, 1))(*[int(c[1]) for _, c in comps]),
          (ctypes.c_int * max(nc, 1))(*[int(c[2]) for _, c in comps]),
          (ctypes.c_int * max(nc, 1))(*[int(c[3]) for _, c in comps])]
    keep += ck
    g = Geometry(sc.nx, sc.ny, sc.nz, sc.vx, sc.vy, sc.vz, sc.n_radial, sc.d_radial, sc.n_views,
                 sc.radius, n, keep[0], keep[1], keep[2], keep[3], sc.n_subsets, nc,
                 ck[0], ck[1], ck[2], ck[3], ck[4], SUBSETS[getattr(sc, "subset_kind", "views")])
    return g, keep


def make_params(prior="tv", alpha=0.1, alpha0=0.2, alpha1=0.1, dtv_gamma=0.995, dtv_eta_frac=0.01,
                sampling="balanced", precond=True, rho=0.99, gamma=1.0, seed=1808, epochs=1,
                objective_every=0, graph=False, target_gap=0.0, psi_star=0.0, x_star=None, probs=None):
    """spdhg_params; x_star (an approximate minimiser for the PSNR log) is a device tensor, kept
    alive by the caller for as long as the parameters are used; probs (sampling="custom") are the
    block probabilities, kept alive with the returned structure."""
    xs = None if x_star is None else ctypes.c_void_p(x_star.data_ptr())
    pp = None
    if probs is not None:
        arr = np.ascontiguousarray(probs, np.float64)
        pp = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    p = Params(PRIOR[prior], alpha, alpha0, alpha1, dtv_gamma, dtv_eta_frac, SAMPLING[sampling],
               int(bool(precond)), rho, gamma, seed, epochs, objective_every, int(bool(graph)),
               float(target_gap), float(psi_star), xs, pp)
    if probs is not None:
        p._probs_keep = arr
    return p


def pointer(a, numel=None, dtype=np.float32):
    """(address, where) of a torch tensor or numpy array; None -> (None, WHERE_HOST)."""
    if a is None:
        return None, WHERE_HOST
    try:
        import torch
        if isinstance(a, torch.Tensor):
            if a.dtype != {np.float32: torch.float32, np.int32: torch.int32}[dtype]:
                raise TypeError(f"expected {dtype.__name__} tensor, got {a.dtype}")
            if not a.is_contiguous():
                raise ValueError("tensor must be contiguous")
            if numel is not None and a.numel() != numel:
                raise ValueError(f"expected {numel} elements, got {a.numel()}")
            return a.data_ptr(), (WHERE_DEVICE if a.is_cuda else WHERE_HOST)
    except ImportError:  # pragma: no cover
        pass
    if not isinstance(a, np.ndarray) or a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
        raise TypeError(f"expected a C-contiguous {np.dtype(dtype).name} numpy array or tensor")
    if numel is not None and a.size != numel:
        raise ValueError(f"expected {numel} elements, got {a.size}")
    return a.ctypes.data, WHERE_HOST
