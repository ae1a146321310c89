"""Pins of the SCDM oracle (Sections 2.4-2.5) against things other than itself:
closed forms of the density and its gradient evaluated directly at the grid
points, LAPACK's pivoted QR, and invariants of the selected-columns
construction."""
import numpy as np
import pytest
import scipy.linalg

import gen
import oracle
from oracle import scdm as oscdm


def _cos_orbital(miller, mode):
    c = np.zeros(len(miller), dtype=complex)
    m = np.array(mode)
    hit = np.nonzero((miller == m).all(1))[0]
    if len(hit) == 0:
        hit = np.nonzero((miller == -m).all(1))[0]
    c[hit[0]] = 1 / np.sqrt(2)
    return c


def _grid_points(cell, grid):
    """r(i0, i1, i2) = sum_d (i_d / n_d) a_d in box order, [N][3]."""
    a = np.asarray(cell).reshape(3, 3)
    idx = np.stack(np.meshgrid(*[np.arange(g) / g for g in grid], indexing="ij"), -1).reshape(-1, 3)
    return idx @ a


def test_density_gradient_of_two_cosines_closed_form():
    """psi_k = sqrt(2/Omega) cos(G_k.r): rho = (2/Omega)(cos^2 t1 + cos^2 t2),
    grad rho = -(2/Omega)(sin 2t1 G1 + sin 2t2 G2), t_k = G_k.r, evaluated at
    the grid points directly."""
    L, ecut, grid = 9.0, 20.0, (18, 20, 16)
    cell = np.diag([L, 1.1 * L, 0.9 * L])
    m = oracle.half_sphere(cell, ecut)
    modes = [np.array((1, 2, 0)), np.array((0, -1, 2))]
    psi = np.array([_cos_orbital(m, g) for g in modes])
    rho, grad = oscdm.density_and_gradient(psi, cell, grid, ecut)
    B = oscdm.reciprocal_rows(cell)
    r = _grid_points(cell, grid)
    om = abs(np.linalg.det(cell))
    Gs = [g @ B for g in modes]
    th = [r @ G for G in Gs]
    rho_x = (2 / om) * sum(np.cos(t) ** 2 for t in th)
    grad_x = -(2 / om) * sum(np.sin(2 * t)[None, :] * G[:, None] for t, G in zip(th, Gs))
    assert np.abs(rho - rho_x).max() < 1e-13 * rho_x.max()
    assert np.abs(grad - grad_x).max() < 1e-13 * np.abs(grad_x).max()
    # the reciprocal rows satisfy a_i . b_j = 2 pi delta_ij
    assert np.allclose(cell @ B.T, 2 * np.pi * np.eye(3), atol=1e-14)


def test_preselection_of_one_cosine():
    """rho > <rho> where cos 2t > 0; |grad rho| < <|grad rho|> where
    |sin 2t| is below its grid mean (points within rounding of either
    threshold excluded from the comparison)."""
    L, ecut, grid = 10.0, 30.0, (18, 18, 18)
    cell = gen.cubic_cell(L)
    m = oracle.half_sphere(cell, ecut)
    psi = _cos_orbital(m, (1, 2, 0))[None, :]
    rho, grad = oscdm.density_and_gradient(psi, cell, grid, ecut)
    sel = oscdm.preselect(rho, grad)
    t = _grid_points(cell, grid) @ (np.array((1, 2, 0)) @ oscdm.reciprocal_rows(cell))
    c2, s2 = np.cos(2 * t), np.abs(np.sin(2 * t))
    want = (c2 > 0) & (s2 < s2.mean())
    clear = (np.abs(c2) > 1e-9) & (np.abs(s2 - s2.mean()) > 1e-9)
    got = np.zeros(len(rho), dtype=bool)
    got[sel] = True
    assert np.array_equal(got[clear], want[clear])
    assert 0 < len(sel) < len(rho) and np.all(np.diff(sel) > 0)


@pytest.mark.parametrize("shape,seed", [((12, 300), 1), ((8, 50), 2), ((20, 20), 3)])
def test_qrcp_pivots_match_lapack(shape, seed):
    A = np.random.default_rng(seed).standard_normal(shape)
    k = min(shape)
    _, _, perm = scipy.linalg.qr(A, pivoting=True, mode="economic")
    assert np.array_equal(oscdm.qrcp_pivots(A, k), perm[:k])


def test_qrcp_orthogonal_columns_pivot_by_norm():
    """Orthogonal columns with distinct norms are chosen by decreasing norm."""
    rng = np.random.default_rng(4)
    Q, _ = np.linalg.qr(rng.standard_normal((6, 6)))
    norms = np.array([0.5, 3.0, 1.0, 2.5, 0.1, 1.7])
    piv = oscdm.qrcp_pivots(Q * norms[None, :], 6)
    assert np.array_equal(piv, np.argsort(-norms))
    with pytest.raises(ValueError):
        oscdm.qrcp_pivots(np.ones((3, 5)), 2)  # rank one


@pytest.fixture(scope="module")
def small():
    s = gen.config_small()
    return dict(s, psi=s["psi"][:6])


@pytest.mark.parametrize("pre", [True, False])
def test_scdm_orthonormal_same_span(small, pre):
    s = small
    r = oscdm.scdm(s["psi"], s["cell"], s["grid"], s["ecut"], use_preselect=pre)
    m = oracle.half_sphere(s["cell"], s["ecut"])
    n = len(s["psi"])
    assert np.abs(r["O"] @ r["O"].T - np.eye(n)).max() < 1e-12
    assert np.abs(oracle.gamma_gram(r["phi_G"], r["phi_G"], m) - np.eye(n)).max() < 1e-12
    # span: the projector onto the orbitals is unchanged
    S = oracle.gamma_gram(s["psi"], r["phi_G"], m)
    assert np.abs(S @ S.T - np.eye(n)).max() < 1e-12
    assert np.abs(r["phi_G"][:, 0].imag).max() < 1e-14
    assert len(set(r["pivots"].tolist())) == n and np.all(np.isin(r["pivots"], r["candidates"]))
    if pre:
        assert len(r["candidates"]) < np.prod(s["grid"])


def test_scdm_invariant_under_rotation_of_the_orbitals(small):
    """Gamma = Psi Psi^* does not change when Psi is rotated, nor do the
    pivots (QRCP of U^T A pivots as QRCP of A), so neither does Phi."""
    s = small
    n = len(s["psi"])
    U, _ = np.linalg.qr(np.random.default_rng(5).standard_normal((n, n)))
    a = oscdm.scdm(s["psi"], s["cell"], s["grid"], s["ecut"])
    b = oscdm.scdm(U @ s["psi"], s["cell"], s["grid"], s["ecut"])
    assert np.array_equal(a["pivots"], b["pivots"])
    assert np.abs(a["phi_G"] - b["phi_G"]).max() < 1e-10


def test_scdm_recovers_separated_gaussians():
    """Four normalised Gaussians 8 bohr apart (overlaps ~1e-8), mixed by a random
    rotation: the localised orbitals are the Gaussians again, up to order and
    sign, and each pivot sits at its Gaussian's centre."""
    L, ecut, grid = 16.0, 25.0, (32, 32, 32)
    cell = gen.cubic_cell(L)
    m = oracle.half_sphere(cell, ecut)
    centres = [np.array(c) for c in ((2.0, 2.0, 2.0), (10.0, 2.0, 2.0), (2.0, 10.0, 10.0), (10.0, 10.0, 2.0))]
    g = np.array([gen.gaussian_sum_coefficients(cell, m, [c], [0.9], [1.0]) for c in centres])
    S = oracle.gamma_gram(g, g, m)
    assert np.abs(S - np.eye(4)).max() < 1e-7
    U, _ = np.linalg.qr(np.random.default_rng(6).standard_normal((4, 4)))
    r = oscdm.scdm(U @ g, cell, grid, ecut)
    C = oracle.gamma_gram(g, r["phi_G"], m)
    assert np.abs(np.abs(C) - np.eye(4)[:, np.argmax(np.abs(C), 0)]).max() < 1e-5
    assert sorted(np.argmax(np.abs(C), 0).tolist()) == [0, 1, 2, 3]
    for p in _grid_points(cell, grid)[r["pivots"]]:
        assert min(np.linalg.norm(p - c) for c in centres) < 0.5 * L / grid[0] * np.sqrt(3) + 1e-9


def test_scdm_keeps_exchange_energy(small):
    """E_x is invariant under the rotation SCDM applies (unscreened)."""
    s = small
    r = oscdm.scdm(s["psi"], s["cell"], s["grid"], s["ecut"])
    _, E0 = oracle.exchange(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    _, E1 = oracle.exchange(r["phi_G"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    assert abs(E0 - E1) < 1e-12 * abs(E0)


def test_scdm_without_preselection_matches_lapack_and_polar():
    """Every grid point a candidate: the pivots are LAPACK's pivoted-QR pivots
    of the n x N matrix of orbital values, and O is the orthogonal polar factor
    of V (scipy.linalg.polar: V = O P, and also (V V^T)^{1/2} O)."""
    s = gen.config_small()
    psi = s["psi"][:5]
    r = oscdm.scdm(psi, s["cell"], s["grid"], s["ecut"], use_preselect=False)
    A = oracle.to_real(psi, s["cell"], s["grid"], s["ecut"]).reshape(len(psi), -1)
    _, _, perm = scipy.linalg.qr(A, pivoting=True, mode="economic")
    assert np.array_equal(r["pivots"], perm[:len(psi)])
    V = A[:, r["pivots"]].T
    U, _ = scipy.linalg.polar(V)
    assert np.abs(r["O"] - U).max() < 1e-12
    assert np.abs(r["phi_G"] - U @ psi).max() < 1e-12


def test_scdm_single_orbital():
    """One orbital: the pivot is the candidate where psi^2 is largest and the
    localised orbital is psi itself, with the sign of psi there."""
    s = gen.config_small()
    psi = s["psi"][:1]
    r = oscdm.scdm(psi, s["cell"], s["grid"], s["ecut"])
    phi = oracle.to_real(psi, s["cell"], s["grid"], s["ecut"]).reshape(-1)
    c = r["candidates"]
    p = c[np.argmax(phi[c] ** 2)]
    assert r["pivots"][0] == p
    assert np.abs(r["phi_G"] - np.sign(phi[p]) * psi).max() < 1e-14
