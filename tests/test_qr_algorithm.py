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
