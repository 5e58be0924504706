"""Host-side checks of the C ABI that need no GPU: the library loads, exports every function the
header declares, validates geometries before touching the device, and its sampler draws the same
block sequence as the oracle (Sec. 4.2 sampling, SplitMix64 stream)."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth
from oracle import algorithms as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def capi():
    from paper_1808_07150_gb300 import _build_ext, _capi
    _build_ext.build()
    return _capi


def _declared():
    names = set()
    for h in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not h.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", h)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"\b((?:spdhg|unet)_[a-z_0-9]+)\s*\(", src))
    return sorted(names)


def test_every_declared_function_is_exported(capi):
    names = _declared()
    assert len(names) >= 30
    assert "unet_forward" in names and "spdhg_run_batch" in names
    lib = ctypes.CDLL(capi.library_path())
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(capi.exported_symbols()) | {n for n in names if hasattr(lib, n)}


@pytest.mark.parametrize("seed,offset,probs", [
    (1808, 0, [0.05] * 10 + [0.5]),
    (7, 1000, [1 / 11] * 11),
    (2 ** 63 + 5, 3, [0.1, 0.2, 0.3, 0.15, 0.25]),
    (0, 0, [1.0]),
])
def test_sampler_matches_oracle(capi, seed, offset, probs):
    import paper_1808_07150_gb300 as pkg
    got = pkg.spdhg_sample(seed, offset, 500, probs)
    ref = O.sample(seed, 500, np.array(probs), offset=offset)
    np.testing.assert_array_equal(got, ref)


def _create(capi, sc):
    g, keep = capi.make_geometry(sc)
    h = ctypes.c_void_p()
    code = capi.lib().spdhg_create(ctypes.byref(g), ctypes.byref(h))
    if h.value:
        capi.lib().spdhg_destroy(h)
    return code


def test_unsupported_geometries_are_rejected_before_device_use(capi):
    import dataclasses
    base = synth.tiny_3d()
    assert _create(capi, dataclasses.replace(base, vy=1.5)) == capi.ERR_UNSUPPORTED
    assert _create(capi, dataclasses.replace(base, radius=3.0)) == capi.ERR_UNSUPPORTED
    assert _create(capi, dataclasses.replace(base, seg_dzmid=(1.0, 0.5, 1.0))) == capi.ERR_UNSUPPORTED
    assert _create(capi, dataclasses.replace(base, radius=4.0, seg_dz=(0.0, 60.0, -60.0))) == capi.ERR_UNSUPPORTED
    assert _create(capi, dataclasses.replace(base, n_subsets=base.n_views + 1)) == capi.ERR_ARG
    assert _create(capi, dataclasses.replace(base, nx=0)) == capi.ERR_ARG


def test_without_a_device_calls_fail_with_a_status(capi):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    assert _create(capi, synth.tiny_2d()) in (capi.ERR_CUDA, capi.ERR_OOM)


def test_library_loading_fails_loudly_when_missing(tmp_path, monkeypatch):
    from paper_1808_07150_gb300 import _build_ext, _capi
    monkeypatch.setattr(_build_ext, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_capi, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        _capi.lib()


def test_unet_rejects_bad_shapes_before_touching_the_device(capi):
    lib = capi.lib()
    h = ctypes.c_void_p()
    ch = (ctypes.c_int * 4)(16, 32, 64, 128)
    assert lib.unet_create(1, ch, 16, 16, 16, ctypes.byref(h)) == capi.ERR_ARG       # one level
    assert lib.unet_create(4, ch, 20, 16, 16, ctypes.byref(h)) == capi.ERR_ARG       # 20 % 8 != 0
    bad = (ctypes.c_int * 2)(16, 48)                                                 # 48: not a power of two
    assert lib.unet_create(2, bad, 16, 16, 16, ctypes.byref(h)) == capi.ERR_ARG
    assert h.value is None
    assert lib.unet_num_params(None) == -1
    # GEMM sizes the tensor-core tile cannot take
    p = ctypes.c_void_p(16)
    assert lib.unet_gemm(p, p, p, 128, 24, 64, 0, None) == capi.ERR_ARG             # N % 16 != 0
    assert lib.unet_gemm(p, p, p, 128, 16, 12, 0, None) == capi.ERR_ARG             # K % 8 != 0
    assert lib.unet_gemm(p, p, p, 128, 512, 64, 0, None) == capi.ERR_ARG            # N > 256
