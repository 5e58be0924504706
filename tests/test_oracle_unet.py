"""Pins of the U-Net oracle (oracle/unet.py) against what does not depend on it.

* conv3 against scipy.ndimage.correlate (zero boundary) and against a loop over the definition;
* tconv2 against a loop over its definition;
* every hand-written backward against the adjoint identity <A x, g> = <x, A^T g> (in the input
  and in the weights);
* pool2's gradient and the whole network's gradient (weights, biases, head, input) against
  central finite differences of the loss.
"""
import numpy as np
import pytest
import scipy.ndimage as ndi

from oracle import unet as U


def _rng(s):
    return np.random.default_rng(s)


def test_conv3_single_channel_is_scipy_correlate():
    r = _rng(0)
    x = r.standard_normal((1, 7, 6, 5))
    W = r.standard_normal((1, 1, 3, 3, 3))
    got = U.conv3(x, W, np.zeros(1))[0]
    ref = ndi.correlate(x[0], W[0, 0], mode="constant", cval=0.0)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_conv3_multichannel_by_definition():
    r = _rng(1)
    x = r.standard_normal((3, 4, 5, 3))
    W = r.standard_normal((2, 3, 3, 3, 3))
    b = r.standard_normal(2)
    got = U.conv3(x, W, b)
    C, Y, X, Z = x.shape
    ref = np.zeros((2, Y, X, Z))
    for o in range(2):
        for y in range(Y):
            for xx in range(X):
                for z in range(Z):
                    acc = b[o]
                    for i in range(C):
                        for ty in range(3):
                            for tx in range(3):
                                for tz in range(3):
                                    yy, xq, zz = y + ty - 1, xx + tx - 1, z + tz - 1
                                    if 0 <= yy < Y and 0 <= xq < X and 0 <= zz < Z:
                                        acc += W[o, i, ty, tx, tz] * x[i, yy, xq, zz]
                    ref[o, y, xx, z] = acc
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_tconv2_by_definition():
    r = _rng(2)
    x = r.standard_normal((3, 2, 3, 2))
    W = r.standard_normal((3, 2, 2, 2, 2))
    b = r.standard_normal(2)
    got = U.tconv2(x, W, b)
    ref = np.zeros((2, 4, 6, 4)) + b[:, None, None, None]
    for i in range(3):
        for y in range(2):
            for xx in range(3):
                for z in range(2):
                    for ty in range(2):
                        for tx in range(2):
                            for tz in range(2):
                                ref[:, 2 * y + ty, 2 * xx + tx, 2 * z + tz] += W[i, :, ty, tx, tz] * x[i, y, xx, z]
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("op", ["conv3", "tconv2"])
def test_backward_is_the_adjoint(op):
    r = _rng(3)
    if op == "conv3":
        x = r.standard_normal((3, 5, 4, 6))
        W = r.standard_normal((4, 3, 3, 3, 3))
        f, fb = U.conv3, U.conv3_backward
    else:
        x = r.standard_normal((3, 2, 3, 2))
        W = r.standard_normal((3, 4, 2, 2, 2))
        f, fb = U.tconv2, U.tconv2_backward
    zero_b = np.zeros(4)
    y = f(x, W, zero_b)
    g = r.standard_normal(y.shape)
    gx, gW, gb = fb(x, W, g)
    lhs = float((y * g).sum())
    assert abs(lhs - float((x * gx).sum())) <= 1e-10 * max(1.0, abs(lhs))   # linear in x
    assert abs(lhs - float((W * gW).sum())) <= 1e-10 * max(1.0, abs(lhs))  # linear in W
    np.testing.assert_allclose(gb, g.sum(axis=(1, 2, 3)), rtol=1e-12)


def test_pool2_gradient_by_finite_differences():
    r = _rng(4)
    x = r.standard_normal((2, 4, 4, 2))  # distinct values: no ties
    out, arg = U.pool2(x)
    g = r.standard_normal(out.shape)
    gx = U.pool2_backward(arg, g, x.shape)
    eps = 1e-7
    for idx in [(0, 0, 0, 0), (1, 3, 2, 1), (0, 2, 1, 0), (1, 1, 3, 1)]:
        xp = x.copy()
        xp[idx] += eps
        xm = x.copy()
        xm[idx] -= eps
        fd = ((U.pool2(xp)[0] * g).sum() - (U.pool2(xm)[0] * g).sum()) / (2 * eps)
        assert abs(fd - gx[idx]) < 1e-6


def test_pool2_ties_go_to_the_first_maximum():
    x = np.zeros((1, 2, 2, 2))
    out, arg = U.pool2(x)
    assert arg.ravel()[0] == 0
    gx = U.pool2_backward(arg, np.ones_like(out), x.shape)
    assert gx[0, 0, 0, 0] == 1.0 and gx.sum() == 1.0


def test_network_gradient_by_finite_differences():
    spec = U.UNetSpec((2, 3, 4))
    r = _rng(5)
    p = {k: v + 0.3 * r.standard_normal(v.shape) for k, v in U.init_params(spec, 6).items()}
    xn = r.random((8, 8, 4)) + 0.1
    target = r.random((8, 8, 4))

    def loss(pp, xx):
        pred, _ = U.forward(spec, pp, xx)
        return U.mse_loss(pred, target)[0]

    pred, cache = U.forward(spec, p, xn)
    _, gpred = U.mse_loss(pred, target)
    g, gxn = U.backward(spec, p, cache, gpred)
    eps = 1e-6
    checked = 0
    for name in sorted(p):
        flat = p[name].ravel()
        for j in r.choice(flat.size, size=min(3, flat.size), replace=False):
            pp = {k: v.copy() for k, v in p.items()}
            pp[name].ravel()[j] += eps
            lp = loss(pp, xn)
            pp[name].ravel()[j] -= 2 * eps
            lm = loss(pp, xn)
            fd = (lp - lm) / (2 * eps)
            an = g[name].ravel()[j]
            assert abs(fd - an) <= 1e-6 + 1e-4 * abs(an), (name, j, fd, an)
            checked += 1
    for idx in [(0, 0, 0), (3, 5, 2), (7, 7, 3), (4, 1, 1)]:
        xp = xn.copy()
        xp[idx] += eps
        xm = xn.copy()
        xm[idx] -= eps
        fd = (loss(p, xp) - loss(p, xm)) / (2 * eps)
        assert abs(fd - gxn[idx]) <= 1e-6 + 1e-4 * abs(gxn[idx])
    assert checked >= 40


def test_untrained_network_is_the_identity():
    spec = U.UNetSpec((2, 3, 4))
    xn = _rng(7).random((8, 8, 4))
    pred, _ = U.forward(spec, U.init_params(spec, 1), xn)
    np.testing.assert_array_equal(pred, xn)
