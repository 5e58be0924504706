"""GB300 SPDHG+ PET reconstruction: thin Python binding of libspdhg (include/spdhg.h).

Method: Ehrhardt, Markiewicz, Schoenlieb, "Faster PET reconstruction with non-smooth priors by
randomization and preconditioning" -- stochastic primal-dual hybrid gradient (Algorithm 2) with
subset-wise preconditioning (Eq. EQU:STEPSIZE:PRECOND) and balanced sampling (Sec. 4.2).

Every step runs in the library's CUDA kernels; this module only marshals arguments (torch CUDA
tensors are passed as device pointers, numpy arrays / CPU tensors as host pointers).  Function
names are those of the C ABI.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi
from ._capi import PRIOR, SAMPLING, STATE, SpdhgError, make_params  # noqa: F401

__all__ = ["Context", "spdhg_sample", "spdhg_run_batch", "make_params", "SpdhgError", "build", "library_path"]


def build(force: bool = False) -> str:
    from . import _build_ext
    return _build_ext.build(force=force)


def library_path() -> str:
    return _capi.library_path()


def _stream(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except ImportError:  # pragma: no cover
            pass
        return None
    return getattr(stream, "cuda_stream", stream)


def _same_where(*pw):
    wh = {w for p, w in pw if p is not None}
    if len(wh) > 1:
        raise ValueError("all arrays of one call must be on the host or all on the device")
    return wh.pop() if wh else _capi.WHERE_HOST


class Context:
    """One reconstruction problem (geometry + data + SPDHG state) on the current CUDA device."""

    def __init__(self, scanner):
        self.scanner = scanner
        g, self._keep = _capi.make_geometry(scanner)
        h = ctypes.c_void_p()
        code = _capi.lib().spdhg_create(ctypes.byref(g), ctypes.byref(h))
        if code != _capi.OK:
            raise SpdhgError(code, f"spdhg_create rejected geometry {getattr(scanner, 'name', '')}")
        self.h = h
        n, m, b = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int()
        _capi.check(_capi.lib().spdhg_sizes(self.h, ctypes.byref(n), ctypes.byref(m), ctypes.byref(b)), self.h)
        self.n_voxels, self.n_bins = n.value, m.value

    # -- lifetime -----------------------------------------------------------------------
    def close(self):
        if getattr(self, "h", None):
            _capi.lib().spdhg_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def _check(self, code):
        _capi.check(code, self.h)

    # -- C ABI ----------------------------------------------------------------------------
    def spdhg_set_data(self, b, r, mult=None, side=None):
        pb = _capi.pointer(b, self.n_bins)
        pr = _capi.pointer(r, self.n_bins)
        pm = _capi.pointer(mult, self.n_bins)
        ps = _capi.pointer(side, self.n_voxels)
        where = _same_where(pb, pr, pm, ps)
        self._check(_capi.lib().spdhg_set_data(self.h, pb[0], pr[0], pm[0], ps[0], where))

    def spdhg_project(self, x, y, subset=-1, stream=None):
        px = _capi.pointer(x, self.n_voxels)
        py = _capi.pointer(y, self.n_bins)
        if px[1] != _capi.WHERE_DEVICE or py[1] != _capi.WHERE_DEVICE:
            raise ValueError("spdhg_project takes device arrays")
        self._check(_capi.lib().spdhg_project(self.h, px[0], py[0], int(subset), _stream(stream)))

    def spdhg_backproject(self, y, x, subset=-1, stream=None):
        px = _capi.pointer(x, self.n_voxels)
        py = _capi.pointer(y, self.n_bins)
        if px[1] != _capi.WHERE_DEVICE or py[1] != _capi.WHERE_DEVICE:
            raise ValueError("spdhg_backproject takes device arrays")
        self._check(_capi.lib().spdhg_backproject(self.h, py[0], px[0], int(subset), _stream(stream)))

    def spdhg_setup(self, params, x0=None, stream=None):
        p0 = _capi.pointer(x0, self.n_voxels)
        self._check(_capi.lib().spdhg_setup(self.h, ctypes.byref(params), p0[0], p0[1], _stream(stream)))

    def spdhg_iterate(self, blocks, stream=None):
        blocks = np.ascontiguousarray(blocks, np.int32)
        ptr = blocks.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        self._check(_capi.lib().spdhg_iterate(self.h, ptr, int(blocks.size), _stream(stream)))

    def spdhg_get(self, what, dst, stream=None):
        code = STATE[what] if isinstance(what, str) else int(what)
        N, M = self.n_voxels, self.n_bins
        numel = {0: N, 1: N, 2: N, 3: M, 4: 3 * N, 5: M, 6: 3 * N, 7: 3 * N, 8: 6 * N}.get(code)
        if numel is None:
            raise ValueError(f"unknown state array {what!r}")
        pd = _capi.pointer(dst, numel)
        self._check(_capi.lib().spdhg_get(self.h, code, pd[0], pd[1], _stream(stream)))
        return dst

    def spdhg_set(self, what, src, stream=None):
        code = STATE[what] if isinstance(what, str) else int(what)
        N, M = self.n_voxels, self.n_bins
        numel = {0: N, 1: N, 3: M, 4: 3 * N, 6: 3 * N, 7: 3 * N, 8: 6 * N}.get(code)
        if numel is None:
            raise ValueError(f"state array {what!r} cannot be set")
        ps = _capi.pointer(src, numel)
        self._check(_capi.lib().spdhg_set(self.h, code, ps[0], ps[1], _stream(stream)))

    def spdhg_save_state(self, path):
        self._check(_capi.lib().spdhg_save_state(self.h, str(path).encode()))

    def spdhg_load_state(self, path):
        self._check(_capi.lib().spdhg_load_state(self.h, str(path).encode()))

    def spdhg_objective(self, x=None, stream=None):
        px = _capi.pointer(x, self.n_voxels)
        out = (ctypes.c_double * 3)()
        self._check(_capi.lib().spdhg_objective(self.h, px[0], px[1], out, _stream(stream)))
        return out[0], out[1], out[2]

    def spdhg_psnr(self, x_star, x=None, stream=None):
        """PSNR(x, x*) in dB (x = None: the current iterate)."""
        ps = _capi.pointer(x_star, self.n_voxels)
        px = _capi.pointer(x, self.n_voxels)
        where = _same_where(ps, px)
        out = ctypes.c_double()
        self._check(_capi.lib().spdhg_psnr(self.h, px[0], ps[0], where, ctypes.byref(out), _stream(stream)))
        return out.value

    def spdhg_probabilities(self):
        n = ctypes.c_int()
        self._check(_capi.lib().spdhg_probabilities(self.h, None, ctypes.byref(n)))
        arr = (ctypes.c_double * n.value)()
        self._check(_capi.lib().spdhg_probabilities(self.h, arr, ctypes.byref(n)))
        return np.array(arr[:], np.float64)

    def spdhg_run(self, params, x, stream=None):
        px = _capi.pointer(x, self.n_voxels)
        rep, keep = _report(params)
        self._check(_capi.lib().spdhg_run(self.h, ctypes.byref(params), px[0], px[1], ctypes.byref(rep),
                                          _stream(stream)))
        return _report_dict(rep, keep, params)

    def spdhg_osem(self, params, x=None, mlem=False, stream=None):
        """OSEM (or MLEM with mlem=True) for params.epochs epochs from x (None: ones); x receives
        the result.  Returns the report dict as spdhg_run does."""
        px = _capi.pointer(x, self.n_voxels)
        rep, keep = _report(params)
        self._check(_capi.lib().spdhg_osem(self.h, ctypes.byref(params), int(bool(mlem)), px[0], px[1],
                                           ctypes.byref(rep), _stream(stream)))
        return _report_dict(rep, keep, params)

    def spdhg_autotune(self, reps=10, stream=None):
        """Measures and sets the launch-shape knobs; returns {knob: value} (0 = built-in)."""
        out = (ctypes.c_int * _capi.TUNE_KNOBS)()
        self._check(_capi.lib().spdhg_autotune(self.h, int(reps), out, _stream(stream)))
        return {k: out[i] for k, i in _capi.TUNE.items()}

    def spdhg_tune(self, knob, value):
        """Sets a launch-shape knob ('prior_cols', 'prior_ychunk', 'fwd_split', 'fwd_warps', 'prior_stages',
        'bwd_table', 'fwd_groups', 'prior_vz'); 0 = default."""
        code = _capi.TUNE[knob] if isinstance(knob, str) else int(knob)
        self._check(_capi.lib().spdhg_tune(self.h, code, int(value)))

    def spdhg_set_memory_limit(self, limit_bytes):
        """Device-memory limit of the context in bytes (0: none); returns the bytes it holds now."""
        used = ctypes.c_uint64(0)
        self._check(_capi.lib().spdhg_set_memory_limit(self.h, int(limit_bytes), ctypes.byref(used)))
        return int(used.value)

    def spdhg_profile(self, enable=True):
        self._check(_capi.lib().spdhg_profile(self.h, int(bool(enable))))

    def spdhg_profile_read(self):
        """{kernel class: (total ms, launches)} since the last spdhg_profile()."""
        n = len(_capi.KERNELS)
        ms = (ctypes.c_double * n)()
        cnt = (ctypes.c_int64 * n)()
        self._check(_capi.lib().spdhg_profile_read(self.h, ms, cnt, n))
        return {k: (ms[i], cnt[i]) for i, k in enumerate(_capi.KERNELS)}


def _report(params):
    obj = np.full(params.epochs + 1, np.nan)
    ms = np.zeros(max(params.epochs, 1))
    psnr = np.full(params.epochs + 1, np.nan)
    dp = ctypes.POINTER(ctypes.c_double)
    rep = _capi.Report(0, 0, obj.ctypes.data_as(dp), ms.ctypes.data_as(dp), psnr.ctypes.data_as(dp), -1, np.nan,
                       np.nan)
    return rep, (obj, ms, psnr)


def _report_dict(rep, keep, params):
    obj, ms, psnr = keep
    return dict(epochs_done=rep.epochs_done, iterations_done=rep.iterations_done, objective=obj,
                epoch_ms=ms[:params.epochs], psnr=psnr, stop_epoch=rep.stop_epoch, ms_to_stop=rep.ms_to_stop,
                psi_zero=rep.psi_zero)


def spdhg_run_batch(contexts, params, xs=None, stream=None):
    """One CUDA graph launch per epoch for all contexts (spdhg_run_batch); returns their reports."""
    n = len(contexts)
    if len(params) != n or (xs is not None and len(xs) != n):
        raise ValueError("one params (and x) per context")
    hs = (ctypes.c_void_p * n)(*[c.h for c in contexts])
    ps = (_capi.Params * n)(*params)
    reps = (_capi.Report * n)()
    keeps = []
    for r in range(n):
        rep, keep = _report(params[r])
        reps[r] = rep
        keeps.append(keep)
    xp = None
    where = _capi.WHERE_DEVICE
    if xs is not None:
        pts = [_capi.pointer(x, c.n_voxels) for x, c in zip(xs, contexts)]
        where = _same_where(*pts)
        xp = (ctypes.c_void_p * n)(*[p for p, _ in pts])
    code = _capi.lib().spdhg_run_batch(hs, ps, xp, where, n, reps, _stream(stream))
    if code != _capi.OK:
        msgs = "; ".join(_capi.lib().spdhg_last_error(c.h).decode() for c in contexts)
        raise SpdhgError(code, msgs)
    return [_report_dict(reps[r], keeps[r], params[r]) for r in range(n)]


def spdhg_sample(seed, offset, n, probs):
    probs = np.ascontiguousarray(probs, np.float64)
    out = np.empty(int(n), np.int32)
    code = _capi.lib().spdhg_sample(int(seed), int(offset), int(n),
                                    probs.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), int(probs.size),
                                    out.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
    _capi.check(code)
    return out
