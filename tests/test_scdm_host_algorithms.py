"""Host check of the pivoting algorithm the GPU's SCDM QR runs (column-pivoted
Gram-Schmidt applied twice, residual norms downdated by the new coefficients,
the first projection from the stored coefficients R[l][p]) against the
oracle's Householder QR with column pivoting: the same pivots on random,
orbital-derived and nearly dependent matrices.  (The kernels' own parity is
tested on the GPU; this pins the algorithmic choice on the CPU.)"""
import numpy as np
import pytest

import gen
import oracle
from oracle import scdm as oscdm


def gs_pivots(A, k):
    """The GPU's steps, restated in numpy (double)."""
    n, m = A.shape
    nu = (A * A).sum(0)
    nu0 = nu.max()
    Q = np.zeros((k, n))
    R = np.zeros((k, m))
    piv = []
    chosen = np.zeros(m, dtype=bool)
    for s in range(k):
        cand = np.where(chosen, -1.0, nu)
        p = int(np.argmax(cand))  # the first of equal maxima
        if not cand[p] > 1e-10 * nu0:
            raise ValueError("rank deficient")
        piv.append(p)
        chosen[p] = True
        r = A[:, p] - R[:s, p] @ Q[:s]       # first pass from the stored coefficients
        r = r - (Q[:s] @ r) @ Q[:s]          # second pass
        Q[s] = r / np.linalg.norm(r)
        R[s] = Q[s] @ A
        nu = np.maximum(nu - R[s] ** 2, 0.0)
    return np.array(piv)


@pytest.mark.parametrize("shape,seed", [((16, 500), 1), ((40, 300), 2), ((8, 8), 3)])
def test_gram_schmidt_pivots_match_householder_on_random_matrices(shape, seed):
    A = np.random.default_rng(seed).standard_normal(shape)
    k = min(shape)
    assert np.array_equal(gs_pivots(A, k), oscdm.qrcp_pivots(A, k))


def test_gram_schmidt_pivots_match_on_orbital_values():
    """The pre-selected orbital values of the 8-orbital 32^3 case, as SCDM
    uses them."""
    s = gen.config_small()
    rho, grad = oscdm.density_and_gradient(s["psi"], s["cell"], s["grid"], s["ecut"])
    cand = oscdm.preselect(rho, grad)
    A = oracle.to_real(s["psi"], s["cell"], s["grid"], s["ecut"]).reshape(8, -1)[:, cand]
    assert np.array_equal(gs_pivots(A, 8), oscdm.qrcp_pivots(A, 8))


def test_gram_schmidt_pivots_match_on_nearly_dependent_columns():
    """Columns that are small perturbations of a few directions: the late
    residuals are ~1e-3 of the column norms (the cancellation the second
    pass is there for)."""
    rng = np.random.default_rng(7)
    base = rng.standard_normal((12, 4))
    A = base @ rng.standard_normal((4, 400)) + 1e-3 * rng.standard_normal((12, 400))
    assert np.array_equal(gs_pivots(A, 12), oscdm.qrcp_pivots(A, 12))


def test_rank_threshold_is_the_same_on_both_sides():
    """Perturbations of 1e-6 leave residual norms^2 near 1e-12 of the columns':
    below the 1e-10 threshold, both the GPU's algorithm and the oracle stop."""
    rng = np.random.default_rng(7)
    base = rng.standard_normal((12, 4))
    A = base @ rng.standard_normal((4, 400)) + 1e-6 * rng.standard_normal((12, 400))
    with pytest.raises(ValueError):
        gs_pivots(A, 12)
    with pytest.raises(ValueError):
        oscdm.qrcp_pivots(A, 12)
    assert np.array_equal(gs_pivots(A, 4), oscdm.qrcp_pivots(A, 4))


def scaled_newton_schulz(V, l0, tol=1e-10, max_it=100):
    """The library's polar iteration, restated: X0 = V / |V|_F, then
    X <- 1.5 a X - 0.5 a^3 (X X^T) X with a = sqrt(3 / (1 + l + l^2)) and
    l <- min(1, 0.5 a l (3 - a^2 l^2)), until max |X X^T - I| < tol was seen
    before a step (that step included)."""
    X = V / np.linalg.norm(V)
    l = l0
    for it in range(max_it):
        a = np.sqrt(3.0 / (1.0 + l + l * l))
        T = X @ X.T
        err = np.abs(T - np.eye(len(V))).max()
        X = 1.5 * a * X - 0.5 * a ** 3 * (T @ X)
        l = min(1.0, 0.5 * a * l * (3.0 - a * a * l * l))
        if err < tol:
            return X, it + 1
    raise RuntimeError("no convergence")


@pytest.mark.parametrize("cond,seed", [(10.0, 1), (1e4, 2), (1e7, 3)])
def test_scaled_newton_schulz_gives_the_polar_factor(cond, seed):
    """V = U diag(s) W^T with singular values spread over `cond`; the start
    estimate l0 = min_k R_kk / |V|_F from the pivoted QR of V^T (as the
    library takes it from its own QR) over-estimates sigma_min: the iteration
    still converges to scipy's polar factor, in few steps."""
    import scipy.linalg
    rng = np.random.default_rng(seed)
    n = 24
    U, _ = np.linalg.qr(rng.standard_normal((n, n)))
    W, _ = np.linalg.qr(rng.standard_normal((n, n)))
    s = np.geomspace(1.0, 1.0 / cond, n)
    V = (U * s) @ W.T
    _, Rq, _ = scipy.linalg.qr(V.T, pivoting=True)
    l0 = np.abs(np.diag(Rq)).min() / np.linalg.norm(V)
    assert l0 >= s.min() / np.linalg.norm(V) * 0.999  # an over-estimate (or equal)
    X, its = scaled_newton_schulz(V, l0)
    P, _ = scipy.linalg.polar(V)
    assert np.abs(X - P).max() < 1e-14 * max(cond, 10.0)  # the polar factor's own conditioning
    assert its <= 10 + int(np.ceil(np.log(cond) / np.log(2.5)))
    # the plain iteration (l0 = 1: no scaling) needs more steps
    _, its_plain = scaled_newton_schulz(V, 1.0)
    assert its_plain >= its
