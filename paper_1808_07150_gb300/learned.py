"""Binding of the learned warm start (include/unet.h): a 3-D U-Net on the library's tensor-core
kernels.  Argument marshalling only; the network runs in libspdhg.so.

The network maps an early SPDHG iterate x_k (scaled by s = mean(x_k)) to a starting point
x0 = s * pred for Algorithm 2; only the starting point changes, never the iteration.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _capi


def _stream(stream):
    from . import _stream as st
    return st(stream)


class UNet:
    def __init__(self, shape, channels=(16, 32, 64, 128)):
        ny, nx, nz = shape
        ch = (ctypes.c_int * len(channels))(*channels)
        h = ctypes.c_void_p()
        code = _capi.lib().unet_create(len(channels), ch, ny, nx, nz, ctypes.byref(h))
        if code != _capi.OK:
            raise _capi.SpdhgError(code, f"unet_create rejected {shape} {channels}")
        self.h = h
        self.shape = tuple(shape)
        self.channels = tuple(channels)
        self.n_params = int(_capi.lib().unet_num_params(self.h))

    def close(self):
        if getattr(self, "h", None):
            _capi.lib().unet_destroy(self.h)
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
        if code != _capi.OK:
            raise _capi.SpdhgError(code, _capi.lib().unet_last_error(self.h).decode())

    def set_params(self, vec):
        vec = np.ascontiguousarray(vec, np.float32)
        if vec.size != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {vec.size}")
        self._check(_capi.lib().unet_set_params(self.h, vec.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), vec.size))

    def init(self, seed):
        """He-normal weights, zero biases and head (the untrained network is the identity)."""
        self._check(_capi.lib().unet_init(self.h, int(seed)))

    def get_params(self):
        out = np.empty(self.n_params, np.float32)
        self._check(_capi.lib().unet_get_params(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size))
        return out

    def get_grads(self):
        out = np.empty(self.n_params, np.float32)
        self._check(_capi.lib().unet_get_grads(self.h, out.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), out.size))
        return out

    def forward(self, x, scale, pred=None, x0=None, stream=None):
        """x, pred, x0: float32 CUDA tensors of the volume's voxel count (pred / x0 may be None)."""
        n = int(np.prod(self.shape))
        px = _capi.pointer(x, n)[0]
        pp = _capi.pointer(pred, n)[0] if pred is not None else None
        p0 = _capi.pointer(x0, n)[0] if x0 is not None else None
        self._check(_capi.lib().unet_forward(self.h, px, float(scale), pp, p0, _stream(stream)))

    def backward(self, target=None, gpred=None, accumulate=False, want_loss=True, stream=None):
        n = int(np.prod(self.shape))
        pt = _capi.pointer(target, n)[0] if target is not None else None
        pg = _capi.pointer(gpred, n)[0] if gpred is not None else None
        loss = ctypes.c_double(np.nan)
        self._check(_capi.lib().unet_backward(self.h, pt, pg, int(bool(accumulate)),
                                              ctypes.byref(loss) if want_loss else None, _stream(stream)))
        return loss.value

    def adam_step(self, lr, stream=None):
        self._check(_capi.lib().unet_adam_step(self.h, float(lr), _stream(stream)))


def gemm(a, b, d, flags=0, stream=None):
    """D = A B^T on the tensor cores (unet_gemm); a, b bfloat16 CUDA tensors, d float32."""
    M, N = d.shape
    K = a.shape[1] if not flags & 1 else a.shape[0]
    code = _capi.lib().unet_gemm(a.data_ptr(), b.data_ptr(), d.data_ptr(), M, N, K, int(flags), _stream(stream))
    if code != _capi.OK:
        raise _capi.SpdhgError(code, "unet_gemm")


def device_error(stream=None):
    return int(_capi.lib().unet_device_error(_stream(stream)))
