"""Pins of the oracle's data term, KL prox and prior operators.

Closed forms are checked against brute force (numeric supremum / 1-D minimisation), special
cases that reduce to textbook formulas, and dense-matrix norms.
"""
import math

import numpy as np
import pytest
from scipy.optimize import minimize_scalar

import oracle
from oracle import algorithms as O

CASES = [  # (y, sigma, b, r)
    (0.3, 0.7, 4.0, 0.5), (-2.0, 0.05, 12.0, 1.5), (0.99, 3.0, 1.0, 0.1), (5.0, 0.2, 0.0, 0.3),
    (-0.5, 1.0, 0.0, 2.0), (0.0, 10.0, 30.0, 0.01), (0.8, 1e-3, 2.0, 1.0), (-40.0, 0.5, 7.0, 3.0),
]


@pytest.mark.parametrize("y,sigma,b,r", CASES)
def test_kl_conjugate_is_numeric_supremum(y, sigma, b, r):
    if y >= 1:
        return
    # sup_x { x y - phi(x) } over x > -r
    f = lambda x: -(x * y - float(O.phi(x, b, r)))  # noqa: E731
    res = minimize_scalar(f, bounds=(-r + 1e-12, 1e6), method="bounded",
                          options=dict(xatol=1e-12, maxiter=10000))
    # refine near the stationary point x = b / (1 - y) - r
    xs = b / (1 - y) - r if b > 0 else -r
    best = max(-res.fun, xs * y - float(O.phi(xs, b, r)))
    assert float(O.phi_conj(y, b, r)) == pytest.approx(best, rel=1e-9, abs=1e-9)


@pytest.mark.parametrize("y,sigma,b,r", CASES)
def test_kl_prox_is_brute_force_minimiser(y, sigma, b, r):
    z = float(O.kl_prox(np.float64(y), sigma, b, r))
    # prox_{sigma phi*}(y) = argmin_z 1/2 (z - y)^2 / sigma + phi*(z)
    f = lambda t: 0.5 * (t - y) ** 2 / sigma + float(O.phi_conj(t, b, r))  # noqa: E731
    hi = 1.0 - 1e-15 if b > 0 else 1.0
    lo = min(y, z) - 10.0
    res = minimize_scalar(f, bounds=(lo, hi), method="bounded", options=dict(xatol=1e-13, maxiter=20000))
    assert f(z) <= f(res.x) + 1e-10
    assert z == pytest.approx(res.x, abs=1e-5)
    # optimality (z - w)(1 - z) + sigma b = 0 with w = y + sigma r
    w = y + sigma * r
    if b > 0:
        assert abs((z - w) * (1 - z) + sigma * b) < 1e-9 * max(1.0, abs(w), sigma * b)
        assert z < 1


def test_kl_prox_b_zero_is_clip_at_one():
    w = np.linspace(-5, 5, 101)
    z = O.kl_prox(w, 0.7, 0.0, 0.0)
    np.testing.assert_allclose(z, np.minimum(w, 1.0), atol=1e-15)


def test_fenchel_young_equality():
    rng = np.random.default_rng(0)
    b = rng.uniform(0.5, 20, 50)
    r = rng.uniform(0.1, 2, 50)
    x = rng.uniform(0.0, 30, 50)
    y = 1 - b / (x + r)  # y = phi'(x)
    np.testing.assert_allclose(O.phi(x, b, r) + O.phi_conj(y, b, r), x * y, rtol=1e-10, atol=1e-10)


def test_data_fidelity_zero_iff_fit():
    rng = np.random.default_rng(1)
    r = rng.uniform(0.1, 1, 40)
    y = rng.uniform(0, 10, 40)
    b = y + r
    assert O.data_fidelity(y, b, r) == pytest.approx(0.0, abs=1e-10)
    assert O.data_fidelity(y * 1.1, b, r) > 0
    assert O.data_fidelity(-r - 1.0, b, r) == math.inf


def _dense(op, shape):
    n = int(np.prod(shape))
    cols = []
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        cols.append(np.asarray(op(e.reshape(shape))).ravel())
    return np.stack(cols, 1)


def test_gradient_on_ramps():
    ny, nx, nz = 5, 6, 4
    iy, ix, iz = np.meshgrid(np.arange(ny), np.arange(nx), np.arange(nz), indexing="ij")
    u = 2.0 * ix - 3.0 * iy + 0.5 * iz
    g = O.grad(u)
    np.testing.assert_allclose(g[0][:, :-1, :], 2.0)
    np.testing.assert_allclose(g[0][:, -1, :], 0.0)
    np.testing.assert_allclose(g[1][:-1], -3.0)
    np.testing.assert_allclose(g[1][-1], 0.0)
    np.testing.assert_allclose(g[2][:, :, :-1], 0.5)
    np.testing.assert_allclose(g[2][:, :, -1], 0.0)


def test_gradient_adjoint_and_norm():
    shape = (5, 7, 4)  # (ny, nx, nz)
    rng = np.random.default_rng(2)
    u = rng.standard_normal(shape)
    p = rng.standard_normal((3,) + shape)
    assert float((O.grad(u) * p).sum()) == pytest.approx(float((u * O.grad_adj(p)).sum()), rel=1e-12)
    G = _dense(O.grad, shape)
    nrm = np.linalg.norm(G, 2)
    assert O.grad_norm((7, 5, 4)) == pytest.approx(nrm, rel=1e-10)
    assert O.grad_norm((7, 5, 4)) < math.sqrt(12)
    pw = O.operator_norm_power(O.grad, O.grad_adj, shape, iters=3000)
    assert pw == pytest.approx(nrm, rel=1e-4)


def test_symmetrised_gradient_linear_field_adjoint_and_norm():
    shape = (6, 5, 4)
    iy, ix, iz = np.meshgrid(np.arange(shape[0]), np.arange(shape[1]), np.arange(shape[2]), indexing="ij")
    M = np.array([[1.0, 2.0, -1.0], [0.5, -3.0, 4.0], [2.0, 1.0, 0.25]])  # w_a = sum_b M[a,b] coord_b
    coords = [ix, iy, iz]
    w = np.stack([sum(M[a, b] * coords[b] for b in range(3)) for a in range(3)]).astype(np.float64)
    e = O.sym_grad(w)
    inner = (slice(1, -1), slice(1, -1), slice(1, -1))
    S = 0.5 * (M + M.T)  # d_b w_a = M[a, b]
    for k, (a, b) in enumerate([(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]):
        np.testing.assert_allclose(e[k][inner], S[a, b], atol=1e-12)
    rng = np.random.default_rng(3)
    w = rng.standard_normal((3,) + shape)
    q = rng.standard_normal((6,) + shape)
    lhs = float((O.sym_grad(w)[:3] * q[:3]).sum() + 2 * (O.sym_grad(w)[3:] * q[3:]).sum())
    assert lhs == pytest.approx(float((w * O.sym_grad_adj(q)).sum()), rel=1e-12)
    small = (4, 3, 3)
    E = _dense(lambda f: O.sym_grad(f) * np.array([1, 1, 1, math.sqrt(2), math.sqrt(2), math.sqrt(2)])[:, None, None, None],
               (3,) + small)
    assert np.linalg.norm(E, 2) <= O.grad_norm((3, 4, 3)) + 1e-12


def test_dtv_special_cases():
    rng = np.random.default_rng(4)
    shape = (6, 6, 5)
    p = rng.standard_normal((3,) + shape)
    xi0 = O.dtv_field(np.ones(shape))
    np.testing.assert_allclose(xi0, 0.0)
    np.testing.assert_allclose(O.dtv_apply(xi0, p, 0.995), p)
    v = rng.standard_normal(shape)
    xi = O.dtv_field(v, 0.01)
    assert float(np.sqrt((xi ** 2).sum(0)).max()) < 1.0
    g = 0.995
    d_xi = O.dtv_apply(xi, xi, g)
    np.testing.assert_allclose(d_xi, (1 - g * (xi ** 2).sum(0)) * xi, atol=1e-12)
    # a vector orthogonal to xi is left unchanged
    perp = np.cross(xi, rng.standard_normal((3,) + shape), axis=0)
    np.testing.assert_allclose(O.dtv_apply(xi, perp, g), perp, atol=1e-12)


def test_dual_ball_projections_are_conjugate_proxes():
    rng = np.random.default_rng(5)
    q = rng.standard_normal((3, 4, 4, 3)) * 2
    a = 0.7
    pq = O.proj_l2(q, a)
    assert float(np.sqrt((pq ** 2).sum(0)).max()) <= a + 1e-12
    # Moreau: q - proj(q) = shrinkage of q (prox of a |.|_2)
    nrm = np.sqrt((q ** 2).sum(0))
    shrink = q * np.maximum(0.0, 1 - a / nrm)
    np.testing.assert_allclose(q - pq, shrink, atol=1e-12)
    pc = O.proj_linf(q, a)
    np.testing.assert_allclose(q - pc, np.sign(q) * np.maximum(np.abs(q) - a, 0.0), atol=1e-12)


def test_dtv_field_on_ramp_and_tv_value():
    ny, nx, nz = 6, 7, 5
    iy, ix, iz = np.meshgrid(np.arange(ny), np.arange(nx), np.arange(nz), indexing="ij")
    g = np.array([1.5, -2.0, 0.5])  # (d/dx, d/dy, d/dz)
    v = g[0] * ix + g[1] * iy + g[2] * iz
    xi = O.dtv_field(v, 0.2)
    inner = (slice(0, -1), slice(0, -1), slice(0, -1))
    expect = g / (np.linalg.norm(g) * math.sqrt(1 + 0.2 ** 2))
    for c in range(3):
        np.testing.assert_allclose(xi[c][inner], expect[c], rtol=1e-12)
    # TV of the ramp: |g| on the (n-1)^3 interior voxels plus the partial faces
    tv = O.prior_value(O.Prior("tv", alpha=1.0), v)
    gx = np.where(ix < nx - 1, g[0], 0.0)
    gy = np.where(iy < ny - 1, g[1], 0.0)
    gz = np.where(iz < nz - 1, g[2], 0.0)
    assert tv == pytest.approx(float(np.sqrt(gx ** 2 + gy ** 2 + gz ** 2).sum()), rel=1e-12)
    atv = O.prior_value(O.Prior("atv", alpha=2.0), v)
    assert atv == pytest.approx(2.0 * float((np.abs(gx) + np.abs(gy) + np.abs(gz)).sum()), rel=1e-12)


def test_metrics():
    xs = np.array([1.0, 2.0])
    assert O.psnr(np.array([1.0, 1.0]), xs) == pytest.approx(20 * math.log10(2.0))
    assert O.relative_objective(3.0, 1.0, 5.0) == pytest.approx(0.5)
