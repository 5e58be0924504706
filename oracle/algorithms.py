"""FP64 oracle of SPDHG for PET with non-smooth priors (test infrastructure only).

Every function follows the paper (Ehrhardt, Markiewicz, Schoenlieb, "Faster PET
reconstruction with non-smooth priors by randomization and preconditioning") step by step
in plain numpy, in the paper's notation.  Nothing here is blocked, fused or reordered; the
CUDA library shares no code with it.  Readings of passages the paper leaves open are listed
next to the function that takes them.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import _native

# ----------------------------------------------------------------------------------------
# projection operator P = diag(mult) L  (Sec. 1.2: the projection model carries the geometric,
# attenuation and normalisation factors, here the per-bin multiplier); A_i = P_i for the data
# blocks (Eq. EQU:SETTING:TV).  Subset i = views v with v mod m == i (Sec. 4: subsets are formed
# from evenly spaced view angles).
# ----------------------------------------------------------------------------------------


def bin_subsets(sc):
    """True when the subsets interleave single bins (bin j of the flattened sinogram belongs to
    subset j mod m: the paper's stability example of Sec. 1.3 divides the bins equidistantly),
    False for view-interleaved subsets."""
    return getattr(sc, "subset_kind", "views") == "bins"


def subset_mask(sc, i):
    """Boolean sinogram mask of the bins of subset i (i < 0: all bins)."""
    m = np.zeros(sc.sino_shape, bool)
    if i < 0:
        m[:] = True
    elif bin_subsets(sc):
        m.ravel()[i::sc.n_subsets] = True
    else:
        m[i::sc.n_subsets] = True
    return m


def _line_integrals(sc, x, subset):
    """L x on the view subset (subset < 0: all views).  A mashed bin is the sum of the line
    integrals of its LOR components (exact mashing): each component family is projected as a
    scanner of its own and added into the planes it belongs to."""
    comps = synth_components(sc)
    if comps is None:
        return _native.line_integrals(sc, x, subset)
    y = np.zeros(sc.sino_shape)
    for vs, planes in comps:
        y[:, :, planes] += _native.line_integrals(vs, x, subset)
    return y


def _line_integrals_adjoint(sc, y, subset):
    comps = synth_components(sc)
    if comps is None:
        return _native.line_integrals_adjoint(sc, y, subset)
    out = np.zeros(sc.image_shape)
    for vs, planes in comps:
        out += _native.line_integrals_adjoint(vs, np.ascontiguousarray(y[:, :, planes]), subset)
    return out


def synth_components(sc):
    """The component families of a mashed scanner (None when bins are single LORs)."""
    if not getattr(sc, "components", ()):
        return None
    import synth  # the family geometry is input description, shared by both sides
    return synth.component_scanners(sc)


def project_at_bins(sc, x, bins):
    """(L x) at the given flattened bin indices (no multiplier), by the definition: for a mashed
    scanner the sum over the LOR components each bin's plane includes."""
    bins = np.asarray(bins, np.int64)
    comps = synth_components(sc)
    if comps is None:
        return _native.line_integrals_at(sc, x, bins)
    V, R, P = sc.sino_shape
    v, r, p = np.unravel_index(bins, (V, R, P))
    out = np.zeros(len(bins))
    for vs, planes in comps:
        where = {int(pl): k for k, pl in enumerate(planes)}
        sel = np.nonzero(np.isin(p, planes))[0]
        if sel.size:
            vb = np.ravel_multi_index((v[sel], r[sel], np.array([where[int(q)] for q in p[sel]])), vs.sino_shape)
            out[sel] += _native.line_integrals_at(vs, x, vb)
    return out


def backproject_at_voxels(sc, y, voxels, subset=-1):
    """(L_subset^T y) at the given flattened voxel indices (no multiplier), by the definition."""
    comps = synth_components(sc)
    if comps is None:
        return _native.adjoint_at_voxels(sc, y, voxels, subset)
    out = np.zeros(len(voxels))
    for vs, planes in comps:
        out += _native.adjoint_at_voxels(vs, np.ascontiguousarray(np.asarray(y)[:, :, planes]), voxels, subset)
    return out


def project(sc, x, subset=-1, mult=None):
    """P_i x (float64, full sinogram shape; bins outside subset i are 0)."""
    if subset >= 0 and bin_subsets(sc):
        y = _line_integrals(sc, x, -1) * subset_mask(sc, subset)
    else:
        y = _line_integrals(sc, x, subset)
    if mult is not None:
        y *= mult
    return y


def backproject(sc, y, subset=-1, mult=None):
    """P_i^T y."""
    y = np.asarray(y, np.float64)
    if mult is not None:
        y = y * mult
    if subset >= 0 and bin_subsets(sc):
        return _line_integrals_adjoint(sc, y * subset_mask(sc, subset), -1)
    return _line_integrals_adjoint(sc, y, subset)


# ----------------------------------------------------------------------------------------
# data fidelity (Sec. 2.1, Eqs. EQU:DATATERM, EQU:LOCALDISTANCE) and its conjugate
# (Example, Eq. EQU:PET:CVX)
# ----------------------------------------------------------------------------------------


def xlogy(b, v):
    """b log v with the convention 0 log 0 = 0 (Sec. 2.1)."""
    b = np.asarray(b, np.float64)
    v = np.asarray(v, np.float64)
    out = np.zeros(np.broadcast(b, v).shape)
    nz = np.broadcast_to(b != 0, out.shape)
    out[nz] = np.broadcast_to(b, out.shape)[nz] * np.log(np.broadcast_to(v, out.shape)[nz])
    return out


def phi(y, b, r):
    """varphi(y) = y + r - b log(y + r) - b + b log b  if y + r >= 0, else +inf."""
    y = np.asarray(y, np.float64)
    e = y + r
    with np.errstate(divide="ignore", invalid="ignore"):
        val = e - xlogy(b, np.where(e > 0, e, 1.0)) - b + xlogy(b, b)
    val = np.where(e < 0, np.inf, val)
    # y + r = 0 with b > 0: -log 0 = +inf
    val = np.where((e == 0) & (np.asarray(b) > 0), np.inf, val)
    return val


def data_fidelity(y, b, r):
    """D(y) = sum_j varphi_j(y_j)."""
    return float(np.sum(phi(y, b, r)))


def phi_conj(y, b, r):
    """varphi*(y) = -y r - b log(1 - y) for y <= 1, +inf otherwise (Eq. EQU:PET:CVX)."""
    y = np.asarray(y, np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        val = -y * r - xlogy(b, np.where(y < 1, 1.0 - y, 1.0))
    val = np.where(y > 1, np.inf, val)
    val = np.where((y == 1) & (np.asarray(b) > 0), np.inf, val)
    return val


def kl_prox(y, sigma, b, r):
    """prox of sigma * varphi* at y (Example after Def. "Proximal Operator"):
    1/2 [w + 1 - sqrt((w - 1)^2 + 4 sigma b)],  w = y + sigma r.

    Reading: the weighted prox is argmin_z 1/2 ||z - x||^2_S + f(z); the closed form printed
    by the paper follows from this convention (the factor 1/2 is missing in the definition).
    """
    w = y + sigma * r
    return 0.5 * (w + 1.0 - np.sqrt((w - 1.0) ** 2 + 4.0 * sigma * b))


# ----------------------------------------------------------------------------------------
# priors (Sec. 2.1 TV / dTV; Sec. 4.3 aTV, TGV)
# ----------------------------------------------------------------------------------------

# image layout [iy][ix][iz]; gradient components ordered (d/dx, d/dy, d/dz); array axes of
# the physical directions:
_AXIS = (1, 0, 2)


def grad(u):
    """Forward differences with a zero difference at the last index (Chambolle-Pock 2011
    discretisation cited in Sec. 2.1), unit spacing.  Returns (3, ny, nx, nz)."""
    u = np.asarray(u, np.float64)
    g = np.zeros((3,) + u.shape)
    for c, ax in enumerate(_AXIS):
        sl_hi = [slice(None)] * 3
        sl_lo = [slice(None)] * 3
        sl_hi[ax] = slice(1, None)
        sl_lo[ax] = slice(0, -1)
        g[c][tuple(sl_lo)] = u[tuple(sl_hi)] - u[tuple(sl_lo)]
    return g


def grad_adj(p):
    """grad^T p = -div p: per component, p[k-1] - p[k] with p[-1] = 0 and the last row of the
    forward difference being zero."""
    p = np.asarray(p, np.float64)
    out = np.zeros(p.shape[1:])
    for c, ax in enumerate(_AXIS):
        pc = p[c]
        n = pc.shape[ax]
        first = [slice(None)] * 3
        mid = [slice(None)] * 3
        prev = [slice(None)] * 3
        # -p[k] for k < n-1
        sl = [slice(None)] * 3
        sl[ax] = slice(0, n - 1)
        out[tuple(sl)] -= pc[tuple(sl)]
        # + p[k-1] for k >= 1 (only rows k-1 < n-1 are live)
        mid[ax] = slice(1, n)
        prev[ax] = slice(0, n - 1)
        out[tuple(mid)] += pc[tuple(prev)]
        del first
    return out


def grad_norm(shape):
    """||grad|| for the forward-difference gradient with Neumann rows: the largest eigenvalue of
    the Neumann Laplacian of n points is 4 sin^2(pi (n-1) / (2n)); the axes add."""
    return math.sqrt(sum(4.0 * math.sin(math.pi * (n - 1) / (2.0 * n)) ** 2 for n in shape))


def sym_grad(w):
    """Symmetrised gradient E w of a vector field w (3, ...) with backward differences
    d-_a = -D_a^T (the negative adjoint of the forward difference).  Returns the 6 unique
    components (xx, yy, zz, xy, xz, yz); off-diagonal entries count twice in the norm."""
    w = np.asarray(w, np.float64)

    def dm(f, c):  # backward difference along physical direction c
        ax = _AXIS[c]
        n = f.shape[ax]
        out = np.zeros_like(f)
        sl = [slice(None)] * 3
        sl[ax] = slice(0, n - 1)
        out[tuple(sl)] += f[tuple(sl)]
        sl2 = [slice(None)] * 3
        sl3 = [slice(None)] * 3
        sl2[ax] = slice(1, n)
        sl3[ax] = slice(0, n - 1)
        out[tuple(sl2)] -= f[tuple(sl3)]
        return out

    e = np.zeros((6,) + w.shape[1:])
    e[0] = dm(w[0], 0)
    e[1] = dm(w[1], 1)
    e[2] = dm(w[2], 2)
    e[3] = 0.5 * (dm(w[1], 0) + dm(w[0], 1))
    e[4] = 0.5 * (dm(w[2], 0) + dm(w[0], 2))
    e[5] = 0.5 * (dm(w[2], 1) + dm(w[1], 2))
    return e


def sym_grad_adj(e):
    """Adjoint of sym_grad w.r.t. the inner product sum(xx*xx' + yy*yy' + zz*zz' + 2 xy*xy' + ...)."""
    e = np.asarray(e, np.float64)

    def dm_adj(f, c):  # (d-_c)^T = (-D_c^T)^T = -D_c (minus the forward difference, Neumann)
        ax = _AXIS[c]
        n = f.shape[ax]
        out = np.zeros_like(f)
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[ax] = slice(0, n - 1)
        hi[ax] = slice(1, n)
        out[tuple(lo)] = f[tuple(lo)] - f[tuple(hi)]
        return out

    w = np.zeros((3,) + e.shape[1:])
    w[0] += dm_adj(e[0], 0)
    w[1] += dm_adj(e[1], 1)
    w[2] += dm_adj(e[2], 2)
    # off-diagonals weighted 2 in the inner product, times the 1/2 of the definition
    w[1] += dm_adj(e[3], 0)
    w[0] += dm_adj(e[3], 1)
    w[2] += dm_adj(e[4], 0)
    w[0] += dm_adj(e[4], 2)
    w[2] += dm_adj(e[5], 1)
    w[1] += dm_adj(e[5], 2)
    return w


def sym_norm2(e):
    """Pointwise squared Frobenius norm of the symmetric field (off-diagonals twice)."""
    return e[0] ** 2 + e[1] ** 2 + e[2] ** 2 + 2.0 * (e[3] ** 2 + e[4] ** 2 + e[5] ** 2)


def dtv_field(v, eta_frac=0.01):
    """xi = grad v / sqrt(|grad v|^2 + eta^2), eta = eta_frac * max |grad v|.

    Reading: the paper defers the definition of the dTV matrix D to its references (Sec. 2.1,
    Sec. 4.3); this oracle takes D = I - gamma xi xi^T with this xi."""
    gv = grad(v)
    nrm = np.sqrt((gv ** 2).sum(0))
    eta = eta_frac * float(nrm.max()) if nrm.max() > 0 else 1.0
    return gv / np.sqrt(nrm ** 2 + eta ** 2)


def dtv_apply(xi, p, gamma):
    """D p = p - gamma xi (xi . p), pointwise (D is symmetric, so this is also D^T)."""
    return p - gamma * xi * (xi * p).sum(0)


def proj_l2(q, alpha):
    """Projection onto {|q_k|_2 <= alpha} pointwise: prox of the conjugate of alpha||.||_{2,1}."""
    nrm = np.sqrt((q ** 2).sum(0))
    return q / np.maximum(1.0, nrm / alpha)


def proj_sym_l2(e, alpha):
    nrm = np.sqrt(sym_norm2(e))
    return e / np.maximum(1.0, nrm / alpha)


def proj_linf(q, alpha):
    """Projection onto {|q_kc| <= alpha}: prox of the conjugate of alpha||.||_{1,1} (aTV)."""
    return np.clip(q, -alpha, alpha)


@dataclasses.dataclass
class Prior:
    """kind in {'none', 'tv', 'dtv', 'atv', 'tgv'}; alpha for tv/dtv/atv; alpha0 on
    ||grad u - w|| and alpha1 on ||E w|| for TGV (the paper's Sec. 4.3 formula)."""
    kind: str = "tv"
    alpha: float = 0.1
    alpha0: float = 0.2
    alpha1: float = 0.1
    side: np.ndarray = None
    gamma_d: float = 0.995
    eta_frac: float = 0.01

    @property
    def n_blocks(self):
        return {"none": 0, "tv": 1, "dtv": 1, "atv": 1, "tgv": 2}[self.kind]


# ----------------------------------------------------------------------------------------
# sampling (Sec. 4.2 "Sampling"): uniform p_i = 1/n, or balanced: prior with probability 1/2,
# otherwise a data subset uniformly, p_i = 1/(2m).  Reading for TGV's two prior blocks: 1/4
# each.  Draws: SplitMix64 (Steele, Lea & Flood 2014) counter-based stream, 53-bit uniform,
# inverse CDF over the cumulative probabilities.
# ----------------------------------------------------------------------------------------

_MASK = (1 << 64) - 1


def splitmix64(seed, k):
    """k-th output (k >= 0) of the SplitMix64 stream started at state `seed`."""
    z = (seed + (k + 1) * 0x9E3779B97F4A7C15) & _MASK
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK
    return z ^ (z >> 31)


def probabilities(m, prior, sampling="balanced", custom=None):
    """p_i of the m data blocks followed by the prior blocks.  sampling = "custom" takes the
    given positive p (Remark "Sampling": any independent draws with p_i > 0 keep the convergence
    of Theorem "Convergence"; the Discussion leaves choosing them to future work)."""
    nb = prior.n_blocks if prior is not None else 0
    n = m + nb
    if sampling == "custom":
        p = np.asarray(custom, np.float64)
        if p.shape != (n,) or np.any(p <= 0) or abs(p.sum() - 1.0) > 1e-12:
            raise ValueError("custom probabilities: n positive values summing to one")
        return p.copy()
    if nb == 0 or sampling == "uniform":
        return np.full(n, 1.0 / n)
    p = np.empty(n)
    p[:m] = 1.0 / (2 * m)
    p[m:] = 0.5 / nb
    return p


def sample(seed, n, probs, offset=0):
    cum = []
    acc = 0.0
    for p in probs:
        acc += float(p)
        cum.append(acc)
    out = np.empty(n, np.int32)
    for k in range(n):
        u = (splitmix64(seed, offset + k) >> 11) * (1.0 / 9007199254740992.0)
        i = 0
        while i < len(cum) - 1 and not (u < cum[i]):
            i += 1
        out[k] = i
    return out


def iters_per_epoch(m, probs):
    """Iterations whose expected data use equals one full projection (Sec. 4 "epoch")."""
    return int(round(m / float(np.sum(probs[:m]))))


# ----------------------------------------------------------------------------------------
# step sizes (Theorem "Step Size Parameters", Eqs. EQU:STEPSIZE:SCALAR and EQU:STEPSIZE:PRECOND;
# Theorem "Convergence": T = min_i T_i).  Readings: rho = 0.99, gamma = 1 (Sec. 4); sigma_j = 0
# where A_i 1 = 0; T_i = +inf where A_i^T 1 = 0 (drops out of the min), T = 0 where every
# T_i is +inf; prior blocks (which have negative entries) use the scalar form; a block's T_i
# covers only the variables it acts on (TGV: data blocks do not bound the step of w).
# ----------------------------------------------------------------------------------------


def operator_norm_power(apply, apply_adj, shape, iters=200, seed=0):
    """||A|| by power iteration on A^T A (used for scalar data steps and as a test pin)."""
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(shape)
    x /= np.linalg.norm(x)
    lam = 0.0
    for _ in range(iters):
        y = apply_adj(apply(x))
        lam = float(np.linalg.norm(y))
        x = y / lam
    return math.sqrt(lam)


def prior_norms(sc, prior):
    """Operator norms of the prior blocks (closed form / bounds, see grad_norm)."""
    gn = grad_norm((sc.nx, sc.ny, sc.nz))
    if prior.kind == "tgv":
        # ||(grad, -I)||^2 = ||grad||^2 + 1;  ||E|| <= ||grad|| (Frobenius / Jensen bound)
        return [math.sqrt(gn ** 2 + 1.0), gn]
    if prior.kind in ("tv", "dtv", "atv"):
        # dTV: ||D grad|| <= ||D|| ||grad|| <= ||grad|| since ||D|| = 1 for 0 <= gamma < 1
        return [gn]
    return []


def step_sizes(sc, mult, prior, probs, rho=0.99, gamma=1.0, precond=True, data_norms=None):
    """Returns dict(sigma=(sino), T=(image) or (u, w) tuple, sigma_prior=[...])."""
    m = sc.n_subsets
    N = sc.image_shape
    Tu = np.full(N, np.inf)
    sigma = np.zeros(sc.sino_shape)
    for i in range(m):
        mask = subset_mask(sc, i)
        if precond:
            a1 = project(sc, np.ones(N), i, mult)  # A_i 1
            with np.errstate(divide="ignore"):
                sigma[mask] = np.where(a1[mask] > 0, gamma * rho / a1[mask], 0.0)
            at1 = backproject(sc, mask.astype(np.float64), i, mult)  # A_i^T 1
            with np.errstate(divide="ignore"):
                Ti = np.where(at1 > 0, rho * probs[i] / (gamma * at1), np.inf)
        else:
            nrm = data_norms[i]
            sigma[mask] = gamma * rho / nrm
            Ti = np.full(N, rho * probs[i] / (gamma * nrm))
        Tu = np.minimum(Tu, Ti)
    sig_p = []
    norms = prior_norms(sc, prior) if prior is not None else []
    if prior is not None and prior.kind == "tgv":
        n0, n1 = norms
        T0 = rho * probs[m] / (gamma * n0)
        T1 = rho * probs[m + 1] / (gamma * n1)
        Tu = np.minimum(Tu, T0)
        Tw = np.full((3,) + N, min(T0, T1))
        sig_p = [gamma * rho / n0, gamma * rho / n1]
        Tu = np.where(np.isinf(Tu), 0.0, Tu)
        return dict(sigma=sigma, T=(Tu, Tw), sigma_prior=sig_p)
    for k, nrm in enumerate(norms):
        Tu = np.minimum(Tu, rho * probs[m + k] / (gamma * nrm))
        sig_p.append(gamma * rho / nrm)
    Tu = np.where(np.isinf(Tu), 0.0, Tu)
    return dict(sigma=sigma, T=Tu, sigma_prior=sig_p)


# ----------------------------------------------------------------------------------------
# the algorithms
# ----------------------------------------------------------------------------------------


@dataclasses.dataclass
class Problem:
    sc: object
    b: np.ndarray
    r: np.ndarray
    mult: np.ndarray = None


def _prior_forward(prior, xi, u, w, k):
    """A_n x for prior block k (0 or 1)."""
    if prior.kind == "tgv":
        return grad(u) - w if k == 0 else sym_grad(w)
    g = grad(u)
    return dtv_apply(xi, g, prior.gamma_d) if prior.kind == "dtv" else g


def _prior_adjoint(prior, xi, dq, k):
    """A_n^T dq -> (du, dw)."""
    if prior.kind == "tgv":
        if k == 0:
            return grad_adj(dq), -dq
        return None, sym_grad_adj(dq)
    if prior.kind == "dtv":
        return grad_adj(dtv_apply(xi, dq, prior.gamma_d)), None
    return grad_adj(dq), None


def _prior_prox(prior, q, k):
    if prior.kind == "atv":
        return proj_linf(q, prior.alpha)
    if prior.kind == "tgv":
        return proj_l2(q, prior.alpha0) if k == 0 else proj_sym_l2(q, prior.alpha1)
    return proj_l2(q, prior.alpha)


def prior_value(prior, u, w=None):
    """alpha R(x): the prior part of Psi."""
    if prior is None or prior.kind == "none":
        return 0.0
    if prior.kind == "tgv":
        a = grad(u) - w
        return prior.alpha0 * float(np.sqrt((a ** 2).sum(0)).sum()) + \
            prior.alpha1 * float(np.sqrt(sym_norm2(sym_grad(w))).sum())
    g = grad(u)
    if prior.kind == "atv":
        return prior.alpha * float(np.abs(g).sum())
    if prior.kind == "dtv":
        g = dtv_apply(dtv_field(prior.side, prior.eta_frac), g, prior.gamma_d)
    return prior.alpha * float(np.sqrt((g ** 2).sum(0)).sum())


def objective(prob, prior, u, w=None):
    """Psi(x) = sum_i D_i(P_i u) + alpha R(u) + i_+(u)  (Problem "PET Reconstruction with Subsets")."""
    if np.any(u < 0):
        return math.inf
    y = project(prob.sc, u, -1, prob.mult)
    return data_fidelity(y, prob.b, prob.r) + prior_value(prior, u, w)


@dataclasses.dataclass
class State:
    x: np.ndarray          # primal u
    w: np.ndarray          # TGV vector field (None otherwise)
    y: np.ndarray          # data duals (full sinogram)
    q: list                # prior duals
    z: np.ndarray          # z = A^T y for u
    zw: np.ndarray         # z for w (TGV)
    zbar: np.ndarray
    zbar_w: np.ndarray


def spdhg(prob, prior, seq, probs, steps=None, x0=None, rho=0.99, gamma=1.0, precond=True,
          data_norms=None, state=None):
    """Algorithm 2 (SPDHG), run for the given block sequence `seq`.

    Returns (state, steps).  state.x is the primal iterate after the last iteration (Alg. 2
    line x = prox(x - T zbar) of that iteration); next_primal(state, steps) is the primal
    step of the following iteration.
    """
    sc = prob.sc
    m = sc.n_subsets
    if steps is None:
        steps = step_sizes(sc, prob.mult, prior, probs, rho, gamma, precond, data_norms)
    tgv = prior is not None and prior.kind == "tgv"
    xi = dtv_field(prior.side, prior.eta_frac) if (prior is not None and prior.kind == "dtv") else None
    T = steps["T"]
    Tu, Tw = (T if tgv else (T, None))
    if state is None:
        u = np.zeros(sc.image_shape) if x0 is None else np.array(x0, np.float64)
        w = np.zeros((3,) + sc.image_shape) if tgv else None
        nq = prior.n_blocks if prior is not None else 0
        qs = []
        for k in range(nq):
            qs.append(np.zeros((6 if (tgv and k == 1) else 3,) + sc.image_shape))
        # zbar = z = A^T y (= 0)  (Alg. 2, line 1)
        state = State(x=u, w=w, y=np.zeros(sc.sino_shape), q=qs, z=np.zeros(sc.image_shape),
                      zw=np.zeros((3,) + sc.image_shape) if tgv else None,
                      zbar=np.zeros(sc.image_shape), zbar_w=np.zeros((3,) + sc.image_shape) if tgv else None)
    s = state
    for i in seq:
        i = int(i)
        # x = prox_g^T (x - T zbar), g = i_+ on u (w unconstrained)
        s.x = np.maximum(s.x - Tu * s.zbar, 0.0)
        if tgv:
            s.w = s.w - Tw * s.zbar_w
        # the selected block i (drawn beforehand with probability p_i)
        dzw = None
        if i < m:
            mask = subset_mask(sc, i)
            ax = project(sc, s.x, i, prob.mult)
            y_arg = s.y + steps["sigma"] * ax
            y_new = kl_prox(y_arg[mask], steps["sigma"][mask], prob.b[mask], prob.r[mask])
            dy = np.zeros(sc.sino_shape)
            dy[mask] = y_new - s.y[mask]
            dz = backproject(sc, dy, i, prob.mult)
            s.y[mask] = y_new
        else:
            k = i - m
            q_arg = s.q[k] + steps["sigma_prior"][k] * _prior_forward(prior, xi, s.x, s.w, k)
            q_new = _prior_prox(prior, q_arg, k)
            du, dzw = _prior_adjoint(prior, xi, q_new - s.q[k], k)
            dz = du if du is not None else np.zeros(sc.image_shape)
            s.q[k] = q_new
        # z = z + dz ; zbar = z + dz / p_i
        s.z = s.z + dz
        s.zbar = s.z + dz / probs[i]
        if tgv:
            dzw = dzw if dzw is not None else np.zeros_like(s.zw)
            s.zw = s.zw + dzw
            s.zbar_w = s.zw + dzw / probs[i]
    return s, steps


def next_primal(state, steps):
    """The primal step x = max(x - T zbar, 0) that opens the next iteration."""
    T = steps["T"]
    Tu = T[0] if isinstance(T, tuple) else T
    return np.maximum(state.x - Tu * state.zbar, 0.0)


def pdhg(prob, prior, n_iter, x0=None, rho=0.99, gamma=1.0, precond=True, state=None, steps=None):
    """Algorithm 1 (PDHG): every dual block updated in each iteration, zbar = z + dz.

    Step sizes: the SPDHG step sizes of the same blocks with weights p_i that sum to one
    (data blocks share 1/2, prior blocks share 1/2; data only: 1/m each); since each block
    satisfies ||S_i^1/2 A_i T^1/2||^2 < p_i, the stacked operator satisfies ||S^1/2 A T^1/2|| < 1.
    """
    sc = prob.sc
    m = sc.n_subsets
    probs = probabilities(m, prior, "balanced")
    if steps is None:
        steps = step_sizes(sc, prob.mult, prior, probs, rho, gamma, precond)
    tgv = prior is not None and prior.kind == "tgv"
    xi = dtv_field(prior.side, prior.eta_frac) if (prior is not None and prior.kind == "dtv") else None
    T = steps["T"]
    Tu, Tw = (T if tgv else (T, None))
    nb = prior.n_blocks if prior is not None else 0
    if state is None:
        state = State(x=np.zeros(sc.image_shape) if x0 is None else np.array(x0, np.float64),
                      w=np.zeros((3,) + sc.image_shape) if tgv else None,
                      y=np.zeros(sc.sino_shape),
                      q=[np.zeros((6 if (tgv and k == 1) else 3,) + sc.image_shape) for k in range(nb)],
                      z=np.zeros(sc.image_shape), zw=np.zeros((3,) + sc.image_shape) if tgv else None,
                      zbar=np.zeros(sc.image_shape), zbar_w=np.zeros((3,) + sc.image_shape) if tgv else None)
    s = state
    for _ in range(n_iter):
        s.x = np.maximum(s.x - Tu * s.zbar, 0.0)
        if tgv:
            s.w = s.w - Tw * s.zbar_w
        ax = project(sc, s.x, -1, prob.mult)
        y_new = kl_prox(s.y + steps["sigma"] * ax, steps["sigma"], prob.b, prob.r)
        dz = backproject(sc, y_new - s.y, -1, prob.mult)
        dzw = np.zeros_like(s.zw) if tgv else None
        s.y = y_new
        for k in range(nb):
            q_arg = s.q[k] + steps["sigma_prior"][k] * _prior_forward(prior, xi, s.x, s.w, k)
            q_new = _prior_prox(prior, q_arg, k)
            du, dw = _prior_adjoint(prior, xi, q_new - s.q[k], k)
            if du is not None:
                dz = dz + du
            if dw is not None:
                dzw = dzw + dw
            s.q[k] = q_new
        s.z = s.z + dz
        s.zbar = s.z + dz
        if tgv:
            s.zw = s.zw + dzw
            s.zbar_w = s.zw + dzw
    return s, steps


def mlem(prob, n_iter, x0=None):
    """MLEM (Eq. EQU:MLEM): u <- u / (P^T 1) * P^T (b / (P u + r))."""
    sc = prob.sc
    sens = backproject(sc, np.ones(sc.sino_shape), -1, prob.mult)
    u = np.ones(sc.image_shape) if x0 is None else np.array(x0, np.float64)
    for _ in range(n_iter):
        ratio = prob.b / (project(sc, u, -1, prob.mult) + prob.r)
        with np.errstate(divide="ignore", invalid="ignore"):
            u = np.where(sens > 0, u / sens * backproject(sc, ratio, -1, prob.mult), 0.0)
    return u


def osem(prob, n_epochs, x0=None, order=None):
    """OSEM (Eq. EQU:OSEM): sub-iteration k uses subset i = order[k mod m] (default i = k mod m)
    and sets u <- u / (P_i^T 1) * P_i^T (b_i / (P_i u + r_i)); u = 0 where P_i^T 1 = 0.  One epoch
    is m sub-iterations."""
    sc = prob.sc
    m = sc.n_subsets
    order = list(range(m)) if order is None else [int(i) for i in order]
    sens = [backproject(sc, np.ones(sc.sino_shape), i, prob.mult) for i in range(m)]
    u = np.ones(sc.image_shape) if x0 is None else np.array(x0, np.float64)
    for _ in range(n_epochs):
        for k in range(m):
            i = order[k % len(order)]
            mask = subset_mask(sc, i)
            with np.errstate(divide="ignore", invalid="ignore"):
                ratio = np.where(mask, prob.b / (project(sc, u, i, prob.mult) + prob.r), 0.0)
                u = np.where(sens[i] > 0, u / sens[i] * backproject(sc, ratio, i, prob.mult), 0.0)
    return u


def psnr(x, x_star):
    """PSNR(x, x*) = 20 log10(||x*||_inf / ||x - x*||_2)  (Sec. 4; log base read as 10)."""
    return 20.0 * math.log10(float(np.abs(x_star).max()) / float(np.linalg.norm(x - x_star)))


def relative_objective(psi, psi_star, psi0):
    """(Psi(x^k) - Psi(x*)) / (Psi(x^0) - Psi(x*)); x^0 = 0 for every run (reading)."""
    return (psi - psi_star) / (psi0 - psi_star)
