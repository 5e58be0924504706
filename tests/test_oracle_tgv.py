"""Pins of the oracle's TGV parts (Sec. 4.3: A_{n-1} = (grad, -I), A_n = (0, E)).

* The dual ball projection of the second block, ``proj_sym_l2``, against a brute-force
  constrained minimisation over full 3x3 matrices with numpy's Frobenius norm (so the weight
  two of the off-diagonal entries is checked, not assumed), and the Moreau identity with the
  shrinkage of alpha1 ||.||_F found by brute-force minimisation.
* ``prior_value`` for TGV on fields whose value follows by hand from the discretisation
  (forward differences with a zero last row, backward differences = their negative adjoint).
* TGV SPDHG+ (Algorithm 2, balanced sampling with two prior blocks) reaches the minimiser that
  an unrelated method finds: scipy's L-BFGS-B on a smoothed TGV objective (continuation in the
  smoothing) with the system matrix built by brute-force box clipping.  A wrong sign or step in
  the w update, or a wrong metric in the dual projection, moves the SPDHG+ limit away from it.
"""
import numpy as np
import pytest
from scipy.optimize import minimize

import synth
from oracle import _native
from oracle import algorithms as O

# 6-component layout of the symmetric fields: (xx, yy, zz, xy, xz, yz)
_PAIRS = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]


def _full(e6):
    """3x3 symmetric matrix from the 6 unique components."""
    m = np.zeros((3, 3))
    for k, (a, b) in enumerate(_PAIRS):
        m[a, b] = e6[k]
        m[b, a] = e6[k]
    return m


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
def test_sym_ball_projection_is_brute_force_frobenius_projection(seed):
    rng = np.random.default_rng(seed)
    alpha = 0.3
    q6 = rng.standard_normal(6) * (0.05 if seed == 0 else 1.0)  # seed 0: inside the ball
    Q = _full(q6)
    # argmin ||E - Q||_F^2 over all 3x3 matrices with ||E||_F <= alpha (9 free entries)
    cons = {"type": "ineq", "fun": lambda v: alpha ** 2 - float((v ** 2).sum())}
    res = minimize(lambda v: float(((v - Q.ravel()) ** 2).sum()), np.zeros(9), method="SLSQP",
                   constraints=[cons], options={"ftol": 1e-14, "maxiter": 500})
    E = res.x.reshape(3, 3)
    got = O.proj_sym_l2(q6.reshape(6, 1, 1, 1), alpha)[:, 0, 0, 0]
    np.testing.assert_allclose(_full(got), E, atol=1e-6)
    assert np.linalg.norm(_full(got), "fro") <= alpha * (1 + 1e-12)
    np.testing.assert_allclose(O.sym_norm2(q6.reshape(6, 1)), np.linalg.norm(Q, "fro") ** 2, rtol=1e-12)


def test_sym_ball_projection_moreau_identity():
    rng = np.random.default_rng(7)
    alpha = 0.4
    for _ in range(3):
        q6 = rng.standard_normal(6)
        Q = _full(q6)
        # prox of alpha ||.||_F at Q by brute force (symmetric 6-parameter search, Frobenius norm)
        res = minimize(lambda v: alpha * np.linalg.norm(_full(v), "fro") + 0.5 * np.linalg.norm(_full(v) - Q, "fro") ** 2,
                       q6, method="Nelder-Mead", options={"xatol": 1e-11, "fatol": 1e-14, "maxiter": 40000})
        shrink = _full(res.x)
        proj = _full(O.proj_sym_l2(q6.reshape(6, 1, 1, 1), alpha)[:, 0, 0, 0])
        np.testing.assert_allclose(proj + shrink, Q, atol=1e-6)


def test_tgv_value_quadratic_u_zero_w():
    ny, nx, nz = 5, 6, 4
    a = 0.7
    iy, ix, iz = np.meshgrid(np.arange(ny), np.arange(nx), np.arange(nz), indexing="ij")
    u = a * ix.astype(np.float64) ** 2
    w = np.zeros((3, ny, nx, nz))
    prior = O.Prior("tgv", alpha0=0.3, alpha1=0.9)
    # forward difference along x: a((ix+1)^2 - ix^2) = a(2 ix + 1) below the last column, 0 there
    expect = 0.3 * sum(abs(a * (2 * k + 1)) for k in range(nx - 1)) * ny * nz
    assert O.prior_value(prior, u, w) == pytest.approx(expect, rel=1e-12)


@pytest.mark.parametrize("shape", [(5, 6, 4), (4, 3, 1)])
def test_tgv_value_zero_u_constant_w(shape):
    ny, nx, nz = shape
    c = -1.3
    iy, ix, iz = np.meshgrid(np.arange(ny), np.arange(nx), np.arange(nz), indexing="ij")
    u = np.zeros(shape)
    w = np.zeros((3,) + shape)
    w[0] = c
    prior = O.Prior("tgv", alpha0=0.25, alpha1=0.6)
    # grad u - w = -w: |c| per voxel.  E w for a constant x component: the backward difference
    # (negative adjoint of the Neumann forward difference) of a constant is c at index 0, -c at
    # the last index and 0 between (0 when the axis has one point); only the x row/column of E w
    # is non-zero: [[d_x, d_y/2, d_z/2], [d_y/2, 0, 0], [d_z/2, 0, 0]].
    def edge(i, n):
        return c * ((i == 0).astype(float) - (i == n - 1).astype(float))
    dx, dy, dz = edge(ix, nx), edge(iy, ny), edge(iz, nz)
    fro = np.sqrt(dx ** 2 + 2 * (dy / 2) ** 2 + 2 * (dz / 2) ** 2)
    expect = 0.25 * abs(c) * ny * nx * nz + 0.6 * float(fro.sum())
    assert O.prior_value(prior, u, w) == pytest.approx(expect, rel=1e-12)


def _tiny_tgv_problem():
    sc = synth.tiny_2d(n_subsets=3)
    d = synth.make_problem(sc, 3, counts=5e3, bg_frac=0.1, with_mult=True, n_ellipsoids=4)
    prob = O.Problem(sc, d["b"].astype(np.float64), d["r"].astype(np.float64), d["mult"].astype(np.float64))
    return sc, prob, O.Prior("tgv", alpha0=0.4, alpha1=0.2)


def _lbfgs_tgv_minimiser(sc, prob, prior):
    """min_{u >= 0, w} D(P u) + alpha0 sum |grad u - w|_eps + alpha1 sum |E w|_eps, with
    |v|_eps = sqrt(|v|^2 + eps^2) and eps -> 1e-8, by L-BFGS-B; P from brute-force box clipping."""
    shp, N = sc.image_shape, sc.n_voxels
    Am = _native.dense_by_clipping(sc) * prob.mult.reshape(-1, 1)
    b, r = prob.b.ravel(), prob.r.ravel()

    def f(v, eps):
        u = v[:N].reshape(shp)
        w = v[N:].reshape((3,) + shp)
        ax = Am @ v[:N]
        s = ax + r
        D = float((ax + r - b + O.xlogy(b, b) - O.xlogy(b, s)).sum())
        g0 = O.grad(u) - w
        n0 = np.sqrt((g0 ** 2).sum(0) + eps ** 2)
        e = O.sym_grad(w)
        n1 = np.sqrt(O.sym_norm2(e) + eps ** 2)
        val = D + prior.alpha0 * float(n0.sum()) + prior.alpha1 * float(n1.sum())
        gu = (Am.T @ (1 - b / s)).reshape(shp) + prior.alpha0 * O.grad_adj(g0 / n0)
        gw = -prior.alpha0 * (g0 / n0) + prior.alpha1 * O.sym_grad_adj(e / n1)
        return val, np.concatenate([gu.ravel(), gw.ravel()])

    v = np.concatenate([np.full(N, 0.1), np.zeros(3 * N)])
    bounds = [(0, None)] * N + [(None, None)] * (3 * N)
    for eps in (1e-2, 1e-4, 1e-6, 1e-8):
        v = minimize(f, v, args=(eps,), jac=True, method="L-BFGS-B", bounds=bounds,
                     options=dict(maxiter=20000, maxfun=40000, ftol=1e-15, gtol=1e-12)).x
    return v[:N].reshape(shp), v[N:].reshape((3,) + shp)


def test_tgv_spdhg_plus_reaches_independent_minimiser():
    sc, prob, prior = _tiny_tgv_problem()
    u_ref, w_ref = _lbfgs_tgv_minimiser(sc, prob, prior)
    psi_ref = O.objective(prob, prior, u_ref, w_ref)
    probs = O.probabilities(sc.n_subsets, prior, "balanced")
    assert probs.tolist()[-2:] == [0.25, 0.25]
    seq = O.sample(11, 60000, probs)
    st, steps = O.spdhg(prob, prior, seq, probs)
    u = O.next_primal(st, steps)
    w = st.w - steps["T"][1] * st.zbar_w
    psi = O.objective(prob, prior, u, w)
    assert psi == pytest.approx(psi_ref, rel=1e-8)
    assert np.linalg.norm(u - u_ref) / np.linalg.norm(u_ref) < 1e-3
    # the duals are feasible in the norms the prior is defined with (full-matrix Frobenius)
    q0, q1 = st.q
    assert float(np.sqrt((q0 ** 2).sum(0)).max()) <= prior.alpha0 * (1 + 1e-12)
    fro = max(np.linalg.norm(_full(q1[(slice(None),) + idx]), "fro") for idx in np.ndindex(q1.shape[1:]))
    assert fro <= prior.alpha1 * (1 + 1e-12)
