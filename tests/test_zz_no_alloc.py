"""The allocation-free subset backprojection (spdhg_backproject_noalloc), called through the C ABI.

This entry point exists for callers that cannot let the library call cudaMalloc (memory owned by
their own pool, or loops that must not synchronise on an allocation).  It must return what
spdhg_backproject returns, on consecutive calls that reuse its fixed scratch array, and reject
subsets larger than that array.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import synth

from gpu_helpers import dev, host

pytestmark = pytest.mark.gpu


def _call_noalloc(ctx, y, x, subset):
    from paper_1808_07150_gb300 import _capi
    import torch
    return _capi.lib().spdhg_backproject_noalloc(ctx.h, y.data_ptr(), x.data_ptr(), int(subset),
                                                 torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("sc", [synth.config_3d(), synth.config_mmr()], ids=lambda s: s.name)
def test_noalloc_backprojection_matches_backproject_twice(sc):
    import paper_1808_07150_gb300 as pkg
    import torch
    mult = synth.smooth_multipliers(sc, 21)
    ones = np.ones(sc.sino_shape, np.float32)
    with pkg.Context(sc) as ctx:
        ctx.spdhg_set_data(dev(ones), dev(ones * 0.1), dev(mult))
        for call, subset in enumerate((sc.n_subsets - 1, 0)):  # two calls in a row, different sizes
            y = dev(synth.random_sinogram(sc, 100 + call))
            ref = torch.zeros(sc.n_voxels, device="cuda")
            got = torch.full((sc.n_voxels,), float("nan"), device="cuda")
            ctx.spdhg_backproject(y, ref, subset)
            assert _call_noalloc(ctx, y, got, subset) == 0, pkg._capi.lib().spdhg_last_error(ctx.h)
            torch.cuda.synchronize()
            # the same gather and backprojection kernels on the same inputs: identical bits
            np.testing.assert_array_equal(host(got), host(ref))


def test_noalloc_rejects_subsets_beyond_its_scratch():
    import paper_1808_07150_gb300 as pkg
    import torch
    sc = synth.config_mmr(n_subsets=1)  # 72.6 M bins in the single subset
    with pkg.Context(sc) as ctx:
        y = torch.zeros(1, device="cuda")
        x = torch.zeros(1, device="cuda")
        code = _call_noalloc(ctx, y, x, 0)
        assert code == pkg._capi.ERR_ARG
        assert b"scratch" in pkg._capi.lib().spdhg_last_error(ctx.h)
        assert _call_noalloc(ctx, y, x, 1) == pkg._capi.ERR_ARG
