"""FP64 oracle of the learned warm start: a 3-D U-Net and its exact gradients (numpy, CPU).

Test infrastructure only (imported by tests/, never by the library).  The paper has no network:
the learned part only replaces the starting point x0 of Algorithm 2 ("Initialize x^0"), so the
converged solution is unchanged.  Everything here is written from the plain definitions:

* conv3(x, W, b):  out[o, p] = b[o] + sum_{i, t} W[o, i, t] x[i, p + t - 1]   (t in {0,1,2}^3,
  zero outside the volume; cross-correlation, "same" size);
* tconv2(x, W, b): out[o, 2p + t] = b[o] + sum_i W[i, o, t] x[i, p]          (t in {0,1}^3,
  stride 2: the transposed 2x2x2 convolution, doubles every dimension);
* pool2(x):        out[c, p] = max_{t in {0,1}^3} x[c, 2p + t]; its gradient goes to the first
  maximum in scan order (ty, tx, tz);
* relu, channel concatenation, a 1x1x1 head and a residual connection.

Arrays are channel-first (C, Y, X, Z), matching the image layout x[iy][ix][iz] per channel.

Network (levels L, channels c_0 < ... < c_{L-1}):
  encoder level l: conv3 + relu, conv3 + relu  (c_{l-1} -> c_l -> c_l; c_{-1} = 1 input channel),
  pooled (pool2) before every level but the first;
  decoder level l = L-2 .. 0: u = tconv2(h, c_{l+1} -> c_l), h = relu(conv3(relu(conv3([u, s_l]))))
  with s_l the encoder output of level l;  head: pred = x_n + sum_c w_c h_c + b_h  (x_n the input).
Warm start: x_n = x_k / s, s = mean(x_k) (+ 1e-12), target x*/s; x0 = s * pred.

Pins (tests/test_oracle_unet.py): conv3 and tconv2 against scipy.ndimage.correlate / a loop over
the definition, adjoint identities of every linear map and its hand-written backward, finite
differences of the whole network's loss with respect to weights and input, pool2 gradients by
brute force.
"""
from __future__ import annotations

import dataclasses

import numpy as np

OFFS3 = [(ty, tx, tz) for ty in range(3) for tx in range(3) for tz in range(3)]  # tap order t
OFFS2 = [(ty, tx, tz) for ty in range(2) for tx in range(2) for tz in range(2)]


def _shift(x, t):
    """x[:, p + t - 1] on the grid of x (zero outside), for a 3x3x3 tap t."""
    C, Y, X, Z = x.shape
    out = np.zeros_like(x)
    dy, dx, dz = t[0] - 1, t[1] - 1, t[2] - 1
    ys, yd = (slice(dy, Y), slice(0, Y - dy)) if dy >= 0 else (slice(0, Y + dy), slice(-dy, Y))
    xs, xd = (slice(dx, X), slice(0, X - dx)) if dx >= 0 else (slice(0, X + dx), slice(-dx, X))
    zs, zd = (slice(dz, Z), slice(0, Z - dz)) if dz >= 0 else (slice(0, Z + dz), slice(-dz, Z))
    out[:, yd, xd, zd] = x[:, ys, xs, zs]
    return out


def _unshift(g, t):
    """Adjoint of _shift: the value at p + t - 1 receives g[:, p]."""
    return _shift(g, (2 - t[0], 2 - t[1], 2 - t[2]))


def conv3(x, W, b):
    """W: (Cout, Cin, 3, 3, 3), b: (Cout,), x: (Cin, Y, X, Z)."""
    out = np.zeros((W.shape[0],) + x.shape[1:])
    for t in OFFS3:
        out += np.einsum("oi,iyxz->oyxz", W[:, :, t[0], t[1], t[2]], _shift(x, t))
    return out + b[:, None, None, None]


def conv3_backward(x, W, g):
    """Gradients of sum(g * conv3(x, W, b)) with respect to x, W, b."""
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for t in OFFS3:
        Wt = W[:, :, t[0], t[1], t[2]]
        gx += _unshift(np.einsum("oi,oyxz->iyxz", Wt, g), t)
        gW[:, :, t[0], t[1], t[2]] = np.einsum("oyxz,iyxz->oi", g, _shift(x, t))
    return gx, gW, g.sum(axis=(1, 2, 3))


def tconv2(x, W, b):
    """W: (Cin, Cout, 2, 2, 2), b: (Cout,), x: (Cin, Y, X, Z) -> (Cout, 2Y, 2X, 2Z)."""
    C, Y, X, Z = x.shape
    out = np.zeros((W.shape[1], 2 * Y, 2 * X, 2 * Z))
    for t in OFFS2:
        out[:, t[0]::2, t[1]::2, t[2]::2] = np.einsum("io,iyxz->oyxz", W[:, :, t[0], t[1], t[2]], x)
    return out + b[:, None, None, None]


def tconv2_backward(x, W, g):
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    for t in OFFS2:
        gt = g[:, t[0]::2, t[1]::2, t[2]::2]
        gx += np.einsum("io,oyxz->iyxz", W[:, :, t[0], t[1], t[2]], gt)
        gW[:, :, t[0], t[1], t[2]] = np.einsum("iyxz,oyxz->io", x, gt)
    return gx, gW, g.sum(axis=(1, 2, 3))


def pool2(x):
    C, Y, X, Z = x.shape
    v = np.stack([x[:, t[0]::2, t[1]::2, t[2]::2] for t in OFFS2])  # (8, C, Y/2, X/2, Z/2)
    return v.max(axis=0), v.argmax(axis=0)  # argmax: first maximum in tap order


def pool2_backward(arg, g, shape):
    gx = np.zeros(shape)
    for k, t in enumerate(OFFS2):
        gx[:, t[0]::2, t[1]::2, t[2]::2] = np.where(arg == k, g, 0.0)
    return gx


def relu(x):
    return np.maximum(x, 0.0)


# ------------------------------------------------------------------------------------------
# the network
# ------------------------------------------------------------------------------------------

@dataclasses.dataclass
class UNetSpec:
    channels: tuple = (16, 32, 64, 128)


def layer_shapes(spec):
    """Ordered (name, shape) of every parameter."""
    ch = spec.channels
    L = len(ch)
    out = []
    cin = 1
    for l in range(L):
        out += [(f"enc{l}a.W", (ch[l], cin, 3, 3, 3)), (f"enc{l}a.b", (ch[l],)),
                (f"enc{l}b.W", (ch[l], ch[l], 3, 3, 3)), (f"enc{l}b.b", (ch[l],))]
        cin = ch[l]
    for l in range(L - 2, -1, -1):
        out += [(f"up{l}.W", (ch[l + 1], ch[l], 2, 2, 2)), (f"up{l}.b", (ch[l],)),
                (f"dec{l}a.W", (ch[l], 2 * ch[l], 3, 3, 3)), (f"dec{l}a.b", (ch[l],)),
                (f"dec{l}b.W", (ch[l], ch[l], 3, 3, 3)), (f"dec{l}b.b", (ch[l],))]
    out += [("head.W", (1, ch[0], 1, 1, 1)), ("head.b", (1,))]
    return out


def init_params(spec, seed):
    """He-normal weights (std sqrt(2 / fan_in)), zero biases, zero head (the untrained net is the
    identity warm start x0 = x_k)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in layer_shapes(spec):
        if name.endswith(".b") or name.startswith("head"):
            p[name] = np.zeros(shape)
        else:
            fan_in = int(np.prod(shape[1:])) if not name.startswith("up") else shape[0] * 8
            p[name] = rng.normal(0.0, np.sqrt(2.0 / fan_in), shape)
    return p


def forward(spec, p, xn):
    """xn: (Y, X, Z) normalised input -> pred (Y, X, Z), cache."""
    L = len(spec.channels)
    cache = {}
    h = xn[None]
    skips = []
    for l in range(L):
        if l > 0:
            cache[f"pool{l}.in"] = h
            h, cache[f"pool{l}.arg"] = pool2(h)
        cache[f"enc{l}a.in"] = h
        h = relu(conv3(h, p[f"enc{l}a.W"], p[f"enc{l}a.b"]))
        cache[f"enc{l}b.in"] = h
        h = relu(conv3(h, p[f"enc{l}b.W"], p[f"enc{l}b.b"]))
        cache[f"enc{l}b.out"] = h
        skips.append(h)
    for l in range(L - 2, -1, -1):
        cache[f"up{l}.in"] = h
        u = tconv2(h, p[f"up{l}.W"], p[f"up{l}.b"])
        cat = np.concatenate([u, skips[l]], axis=0)
        cache[f"dec{l}a.in"] = cat
        h = relu(conv3(cat, p[f"dec{l}a.W"], p[f"dec{l}a.b"]))
        cache[f"dec{l}b.in"] = h
        h = relu(conv3(h, p[f"dec{l}b.W"], p[f"dec{l}b.b"]))
        cache[f"dec{l}b.out"] = h
    cache["head.in"] = h
    pred = xn + np.einsum("c,cyxz->yxz", p["head.W"][0, :, 0, 0, 0], h) + p["head.b"][0]
    return pred, cache


def backward(spec, p, cache, gpred):
    """Gradients of sum(gpred * pred) with respect to every parameter and to the input xn:
    the decoder levels 0..L-2 (the reverse of their forward order), then the encoder from the
    bottom level up, each skip gradient joining its encoder output."""
    L = len(spec.channels)
    ch = spec.channels
    g = {}
    h = cache["head.in"]
    g["head.W"] = np.einsum("yxz,cyxz->c", gpred, h)[None, :, None, None, None]
    g["head.b"] = np.array([gpred.sum()])
    gh = np.einsum("c,yxz->cyxz", p["head.W"][0, :, 0, 0, 0], gpred)
    gskip = [None] * L
    for l in range(0, L - 1):
        gh = gh * (cache[f"dec{l}b.out"] > 0)
        gx, g[f"dec{l}b.W"], g[f"dec{l}b.b"] = conv3_backward(cache[f"dec{l}b.in"], p[f"dec{l}b.W"], gh)
        gx = gx * (cache[f"dec{l}b.in"] > 0)
        gcat, g[f"dec{l}a.W"], g[f"dec{l}a.b"] = conv3_backward(cache[f"dec{l}a.in"], p[f"dec{l}a.W"], gx)
        gskip[l] = gcat[ch[l]:]
        gh, g[f"up{l}.W"], g[f"up{l}.b"] = tconv2_backward(cache[f"up{l}.in"], p[f"up{l}.W"], gcat[:ch[l]])
    # gh: gradient at the bottom encoder output (level L-1); encoder levels top-down in reverse
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            gh = gh + gskip[l]
        gh = gh * (cache[f"enc{l}b.out"] > 0)
        gx, g[f"enc{l}b.W"], g[f"enc{l}b.b"] = conv3_backward(cache[f"enc{l}b.in"], p[f"enc{l}b.W"], gh)
        gx = gx * (cache[f"enc{l}b.in"] > 0)
        gh, g[f"enc{l}a.W"], g[f"enc{l}a.b"] = conv3_backward(cache[f"enc{l}a.in"], p[f"enc{l}a.W"], gx)
        if l > 0:
            gh = pool2_backward(cache[f"pool{l}.arg"], gh, cache[f"pool{l}.in"].shape)
    gxn = gpred + gh[0]
    return g, gxn


def mse_loss(pred, target):
    """L = mean((pred - target)^2) and dL/dpred."""
    d = pred - target
    return float(np.mean(d * d)), 2.0 * d / d.size
