"""Pins of the FP64 oracle against things other than itself (CPU only).

* its FFT against a brute-force direct DFT and Parseval's identity;
* its cutoff sphere against Table 1 of arXiv:2110.07670;
* its Coulomb pair energies and exchange potentials against closed forms
  (plane waves, a normalised Gaussian with the Madelung term);
* its exchange operator against invariants of Eq. 1-4 (Hermiticity, v_ij
  symmetry, negative semidefiniteness, scaling with the cell);
* its ACE construction (Section 2.2) against exactness on span(Phi), the
  trace identity E_x = tr(M), unitary invariance and an LU route.
"""
import os

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------ FFT

def _direct_dft3(a, sign):
    """Brute force: X[k] = sum_j a[j] exp(sign 2 pi i sum_d j_d k_d / n_d)."""
    out = np.zeros_like(a, dtype=np.complex128)
    n = a.shape
    js = np.indices(n).reshape(3, -1).T
    flat = a.reshape(-1)
    for k in np.ndindex(*n):
        ph = sum(js[:, d] * k[d] / n[d] for d in range(3))
        out[k] = (flat * np.exp(sign * 2j * np.pi * ph)).sum()
    return out


@pytest.mark.parametrize("shape", [(2, 2, 2), (3, 3, 3), (4, 4, 4), (5, 5, 5), (6, 6, 6), (7, 7, 7), (8, 8, 8),
                                   (9, 9, 9), (10, 10, 10), (12, 12, 12), (4, 6, 10), (16, 15, 2),
                                   (1, 18, 1), (20, 1, 1), (1, 1, 24), (30, 1, 1)])
@pytest.mark.parametrize("sign", [-1, +1])
def test_fft_matches_direct_dft(shape, sign):
    rng = np.random.default_rng(hash(shape) % 1000)
    a = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
    ref = _direct_dft3(a, sign)
    got = oracle.fft3d(a, sign)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max() * max(1, np.log2(a.size))


def test_fft_parseval_and_roundtrip():
    rng = np.random.default_rng(3)
    a = rng.standard_normal((12, 10, 18)) + 1j * rng.standard_normal((12, 10, 18))
    A = oracle.fft3d(a, -1)
    assert abs((abs(A) ** 2).sum() / a.size - (abs(a) ** 2).sum()) < 1e-12 * (abs(a) ** 2).sum()
    back = oracle.fft3d(A, +1) / a.size
    assert np.abs(back - a).max() < 1e-13


def test_fft_single_mode():
    """A single plane wave transforms to one nonzero entry of height N."""
    n = (8, 6, 10)
    k0 = (3, 5, 7)
    idx = np.indices(n)
    a = np.exp(2j * np.pi * sum(idx[d] * k0[d] / n[d] for d in range(3)))
    A = oracle.fft3d(a, -1)
    expect = np.zeros(n, dtype=complex)
    expect[k0] = np.prod(n)
    assert np.abs(A - expect).max() < 1e-10


# --------------------------------------------------------------- cutoff

def test_table1_plane_wave_counts():
    for edge, n_wave, n_dens in _golden("table1_pw_counts.txt"):
        cell = gen.cubic_cell(float(edge) * gen.BOHR_PER_ANGSTROM)
        assert len(oracle.half_sphere(cell, 80.0)) == int(n_wave)
        assert len(oracle.half_sphere(cell, 320.0)) == int(n_dens)


@pytest.mark.parametrize("L,ecut", [(10.0, 30.0), (18.6, 80.0), (9.3, 55.5)])
def test_half_sphere_order_matches_generator(L, ecut):
    cell = gen.cubic_cell(L)
    a = oracle.half_sphere(cell, ecut)
    b = gen.half_sphere(cell, ecut)
    assert np.array_equal(a, b)
    assert tuple(a[0]) == (0, 0, 0)


def test_half_sphere_non_cubic_cell():
    cell = np.array([[8.0, 0.0, 0.0], [1.0, 9.0, 0.0], [0.5, -0.7, 10.0]])
    a = oracle.half_sphere(cell, 25.0)
    assert np.array_equal(a, gen.half_sphere(cell, 25.0))
    # every +-G pair represented exactly once
    s = {tuple(m) for m in a}
    assert all(tuple(-m) not in s for m in a if any(m))


# --------------------------------------------------------- closed forms

def _cos_orbital(miller, mode):
    """Coefficients of sqrt(2/Omega) cos(G.r) for G = mode (or -mode)."""
    c = np.zeros(len(miller), dtype=complex)
    m = np.array(mode)
    hit = np.nonzero((miller == m).all(1))[0]
    if len(hit) == 0:
        hit = np.nonzero((miller == -m).all(1))[0]
    c[hit[0]] = 1 / np.sqrt(2)
    return c


def test_plane_wave_self_energy():
    L, ecut, grid = 10.0, 30.0, (18, 18, 18)
    cell = gen.cubic_cell(L)
    m = oracle.half_sphere(cell, ecut)
    c = _cos_orbital(m, (1, 2, 0))
    e = oracle.pair_energy(c, c, cell, grid, ecut)
    G2 = (2 * np.pi / L) ** 2 * 5
    expect = np.pi / (2 * L ** 3 * G2)
    assert abs(e - expect) < 1e-15
    golden = dict((k, float(v)) for k, v in _golden("closed_forms.txt"))
    assert abs(e - golden["plane_wave_L10_G120"]) < 1e-16


def test_plane_wave_pair_energy():
    L, ecut, grid = 10.0, 30.0, (18, 18, 18)
    cell = gen.cubic_cell(L)
    m = oracle.half_sphere(cell, ecut)
    g1, g2 = np.array((1, 2, 0)), np.array((0, -1, 3))
    ca, cb = _cos_orbital(m, g1), _cos_orbital(m, g2)
    e = oracle.pair_energy(ca, cb, cell, grid, ecut)
    f = (2 * np.pi / L) ** 2
    expect = 2 * np.pi / L ** 3 * (1 / (f * ((g1 - g2) ** 2).sum()) + 1 / (f * ((g1 + g2) ** 2).sum()))
    assert abs(e - expect) < 1e-15
    assert abs(oracle.pair_energy(cb, ca, cell, grid, ecut) - e) < 1e-18


def test_plane_wave_exchange_potential():
    """One cosine orbital: V_X phi = -alpha v phi; its G-component is
    -alpha pi/(2 Omega |G|^2) c(G) (the 3G harmonic lies outside the sphere)."""
    L, ecut, grid, alpha = 10.0, 5.0, (16, 16, 16), 0.25
    cell = gen.cubic_cell(L)
    m = oracle.half_sphere(cell, ecut)
    mode = np.array((1, 1, 0))
    c = _cos_orbital(m, mode)[None, :]
    W, E = oracle.exchange(c, cell, grid, ecut, alpha)
    G2 = (2 * np.pi / L) ** 2 * 2
    expect = -alpha * np.pi / (2 * L ** 3 * G2) * c
    assert np.abs(W - expect).max() < 1e-16
    assert abs(E - (-alpha * np.pi / (2 * L ** 3 * G2))) < 1e-16


@pytest.mark.parametrize("sigma,L,n", [(1.0, 20.0, 96), (0.8, 14.0, 64)])
def test_gaussian_self_energy_madelung(sigma, L, n):
    ecut = 80.0
    cell = gen.cubic_cell(L)
    m = oracle.half_sphere(cell, ecut)
    c = gen.gaussian_sum_coefficients(cell, m, [np.array([3.0, 4.0, 5.0])], [sigma], [1.0])
    assert abs(2 * (abs(c) ** 2).sum() - abs(c[0]) ** 2 - 1) < 1e-12
    e = oracle.pair_energy(c, c, cell, (n, n, n), ecut)
    xi_m = 2.83729747948
    expect = np.sqrt(2 / np.pi) / sigma - xi_m / L + 2 * np.pi * sigma ** 2 / L ** 3
    assert abs(e - expect) < 1e-10
    if (sigma, L) == (1.0, 20.0):
        golden = dict((k, float(v)) for k, v in _golden("closed_forms.txt"))
        assert abs(e - golden["gaussian_sigma1_L20"]) < 1e-11


# ------------------------------------ truncated Coulomb (alternative G = 0)

def _k_trunc(q2, rc):
    """Transform of 1/r cut off at r = rc, written from the radial integral
    4 pi int_0^rc sin(q r) / q dr (q > 0) and 4 pi int_0^rc r dr (q = 0)."""
    if q2 == 0:
        return 2 * np.pi * rc ** 2
    q = np.sqrt(q2)
    return 4 * np.pi / q * (1 - np.cos(q * rc)) / q


@pytest.mark.parametrize("rc", [3.0, 6.2035049089940])
def test_truncated_plane_wave_self_energy(rc):
    """rho = (1 + cos 2G.r) / Omega: the G = 0 term K(0) / Omega and the 2G
    harmonic K(2G) / (2 Omega)."""
    L, ecut, grid = 10.0, 30.0, (18, 18, 18)
    cell = gen.cubic_cell(L)
    m = oracle.half_sphere(cell, ecut)
    c = _cos_orbital(m, (1, 2, 0))
    with oracle.coulomb_cutoff(rc):
        e = oracle.pair_energy(c, c, cell, grid, ecut)
    G2 = (2 * np.pi / L) ** 2 * 5
    expect = _k_trunc(0.0, rc) / L ** 3 + _k_trunc(4 * G2, rc) / (2 * L ** 3)
    assert abs(e - expect) < 5e-14 * abs(expect)
    # the context restores the dropped G = 0 term
    assert abs(oracle.pair_energy(c, c, cell, grid, ecut) - np.pi / (2 * L ** 3 * G2)) < 1e-15


def test_truncated_plane_wave_pair_energy():
    L, ecut, grid, rc = 10.0, 30.0, (18, 18, 18), 4.5
    cell = gen.cubic_cell(L)
    m = oracle.half_sphere(cell, ecut)
    g1, g2 = np.array((1, 2, 0)), np.array((0, -1, 3))
    ca, cb = _cos_orbital(m, g1), _cos_orbital(m, g2)
    with oracle.coulomb_cutoff(rc):
        e = oracle.pair_energy(ca, cb, cell, grid, ecut)
    f = (2 * np.pi / L) ** 2
    expect = (_k_trunc(f * ((g1 - g2) ** 2).sum(), rc) + _k_trunc(f * ((g1 + g2) ** 2).sum(), rc)) / (2 * L ** 3)
    assert abs(e - expect) < 5e-14 * abs(expect)


@pytest.mark.parametrize("sigma,L,n,rc", [(1.0, 20.0, 96, None), (0.8, 14.0, 64, 6.0)])
def test_truncated_gaussian_self_energy(sigma, L, n, rc):
    """A normalised Gaussian's density interacting through 1/r cut off at rc
    (no periodic image reaches the sphere): its self-convolution is a Gaussian
    of exponent 1 / (2 sigma^2), so e = sqrt(2/pi)/sigma (1 - exp(-rc^2 / (2 sigma^2)))
    exactly, with no Madelung term."""
    ecut = 80.0
    cell = gen.cubic_cell(L)
    if rc is None:
        rc = oracle.sphere_radius(cell)
        assert abs(rc - L * (3 / (4 * np.pi)) ** (1 / 3)) < 1e-12
    m = oracle.half_sphere(cell, ecut)
    c = gen.gaussian_sum_coefficients(cell, m, [np.array([3.0, 4.0, 5.0])], [sigma], [1.0])
    with oracle.coulomb_cutoff(rc):
        e = oracle.pair_energy(c, c, cell, (n, n, n), ecut)
    expect = np.sqrt(2 / np.pi) / sigma * (1 - np.exp(-rc ** 2 / (2 * sigma ** 2)))
    assert abs(e - expect) < 1e-10
    if (sigma, L) == (1.0, 20.0):
        golden = dict((k, float(v)) for k, v in _golden("closed_forms.txt"))
        assert abs(e - golden["gaussian_sigma1_L20_cutoff_sphere"]) < 1e-10


def test_truncated_exchange_invariants():
    """With the cut-off interaction V_X stays Hermitian and negative, and the
    ACE operator stays exact on span(Phi) with E_x = tr(M)."""
    cell = gen.cubic_cell(7.0)
    ecut, grid, alpha = 14.0, (16, 16, 16), 0.25
    psi = gen.random_orbitals(cell, ecut, 5, seed=11)
    trials = gen.random_trials(cell, ecut, 3, seed=12)
    m = oracle.half_sphere(cell, ecut)
    rc = oracle.sphere_radius(cell)
    with oracle.coulomb_cutoff(rc):
        V = oracle.vx_apply(psi, trials, cell, grid, ecut, alpha)
        ref = oracle.ace_build(psi, cell, grid, ecut, alpha)
        Kphi = oracle.ace_apply(ref["xi"], psi, m)
    A = oracle.gamma_gram(trials, V, m)
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).max() < 1e-14
    assert abs(ref["E_x"] - np.trace(ref["M"])) < 1e-13 * abs(ref["E_x"])
    assert np.abs(Kphi - ref["W_G"]).max() < 1e-12 * np.abs(ref["W_G"]).max()
    # the G = 0 term alone shifts every diagonal pair energy by K(0) / Omega
    ref0 = oracle.ace_build(psi, cell, grid, ecut, alpha)
    assert abs(ref["E_x"] - ref0["E_x"]) > 1e-6


# --------------------- auxiliary-function G = 0 term (Gygi-Baldereschi)

@pytest.mark.parametrize("L", [20.0, 13.0])
def test_auxiliary_function_k0_is_the_madelung_term(L):
    """For a cubic cell K(0) / Omega = xi_M / L, the simple-cubic Madelung
    constant xi_M = 2.83729747948 (independent of the cell size)."""
    k0 = oracle.auxiliary_function_k0(gen.cubic_cell(L))
    assert abs(k0 / L ** 2 - 2.83729747948) < 1e-10


def test_auxiliary_function_k0_independent_of_alpha():
    cell = np.array([[9.0, 0.0, 0.0], [1.5, 10.0, 0.0], [0.3, 0.7, 11.0]])
    k = [oracle.auxiliary_function_k0(cell, alpha=a) for a in (None, 0.3, 0.6)]
    assert max(k) - min(k) < 1e-12 * abs(k[0])


@pytest.mark.parametrize("sigma,L,n", [(1.0, 20.0, 96), (0.8, 14.0, 64)])
def test_gaussian_self_energy_with_auxiliary_g0(sigma, L, n):
    """With K(0) = 4 pi chi the Madelung term of the dropped-G = 0 self-energy
    cancels: e = sqrt(2/pi)/sigma + 2 pi sigma^2 / L^3."""
    ecut = 80.0
    cell = gen.cubic_cell(L)
    m = oracle.half_sphere(cell, ecut)
    c = gen.gaussian_sum_coefficients(cell, m, [np.array([3.0, 4.0, 5.0])], [sigma], [1.0])
    with oracle.coulomb_g0(oracle.auxiliary_function_k0(cell)):
        e = oracle.pair_energy(c, c, cell, (n, n, n), ecut)
    assert abs(e - (np.sqrt(2 / np.pi) / sigma + 2 * np.pi * sigma ** 2 / L ** 3)) < 1e-10
    if (sigma, L) == (1.0, 20.0):
        golden = dict((k, float(v)) for k, v in _golden("closed_forms.txt"))
        assert abs(e - golden["gaussian_sigma1_L20_auxiliary_g0"]) < 1e-10
    # and the context restores the dropped term
    e0 = oracle.pair_energy(c, c, cell, (n, n, n), ecut)
    assert abs(e0 - (np.sqrt(2 / np.pi) / sigma - 2.83729747948 / L + 2 * np.pi * sigma ** 2 / L ** 3)) < 1e-10


def test_auxiliary_g0_exchange_invariants():
    cell = gen.cubic_cell(7.0)
    ecut, grid, alpha = 14.0, (16, 16, 16), 0.25
    psi = gen.random_orbitals(cell, ecut, 5, seed=11)
    trials = gen.random_trials(cell, ecut, 3, seed=12)
    m = oracle.half_sphere(cell, ecut)
    with oracle.coulomb_g0(oracle.auxiliary_function_k0(cell)):
        V = oracle.vx_apply(psi, trials, cell, grid, ecut, alpha)
        ref = oracle.ace_build(psi, cell, grid, ecut, alpha)
        Kphi = oracle.ace_apply(ref["xi"], psi, m)
    A = oracle.gamma_gram(trials, V, m)
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).max() < 1e-14
    assert abs(ref["E_x"] - np.trace(ref["M"])) < 1e-13 * abs(ref["E_x"])
    assert np.abs(Kphi - ref["W_G"]).max() < 1e-12 * np.abs(ref["W_G"]).max()
    # each orbital's own pair density has mean 1 / Omega: the G = 0 term adds
    # -alpha K(0) / Omega per orbital to E_x
    E0 = oracle.ace_build(psi, cell, grid, ecut, alpha)["E_x"]
    k0 = oracle.auxiliary_function_k0(cell)
    assert abs((ref["E_x"] - E0) - (-alpha * k0 / 7.0 ** 3 * 5)) < 1e-12 * abs(E0)


# ------------------------------------------------------------ invariants

@pytest.fixture(scope="module")
def small():
    cell = gen.cubic_cell(7.0)
    ecut, grid = 14.0, (16, 16, 16)
    psi = gen.random_orbitals(cell, ecut, 5, seed=11)
    trials = gen.random_trials(cell, ecut, 3, seed=12)
    return dict(cell=cell, ecut=ecut, grid=grid, alpha=0.25, psi=psi, trials=trials,
                m=oracle.half_sphere(cell, ecut))


def test_vx_hermitian_and_negative(small):
    s = small
    V = oracle.vx_apply(s["psi"], s["trials"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    A = oracle.gamma_gram(s["trials"], V, s["m"])  # <t_a | V_X t_b>
    assert np.abs(A - A.T).max() < 1e-15
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).max() < 1e-14


def test_pair_symmetry(small):
    s = small
    p = s["psi"]
    for a, b in [(0, 1), (2, 4), (3, 3)]:
        e1 = oracle.pair_energy(p[a], p[b], s["cell"], s["grid"], s["ecut"])
        e2 = oracle.pair_energy(p[b], p[a], s["cell"], s["grid"], s["ecut"])
        assert abs(e1 - e2) < 1e-16 + 1e-13 * abs(e1)
        assert e1 >= -1e-16 if a == b else True


def test_symmetric_and_one_sided_paths_agree(small):
    s = small
    W, E = oracle.exchange(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    V = oracle.vx_apply(s["psi"], s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    assert np.abs(W - V).max() < 1e-15
    # E_x = -alpha sum_ij e_ij from pair energies
    n = len(s["psi"])
    e = sum(oracle.pair_energy(s["psi"][i], s["psi"][j], s["cell"], s["grid"], s["ecut"])
            for i in range(n) for j in range(n))
    assert abs(E + s["alpha"] * e) < 1e-14


def test_ace_exactness_trace_and_lu(small):
    s = small
    r = oracle.ace_build(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    # K phi_i = W_i on span(Phi)
    K = oracle.ace_apply(r["xi"], s["psi"], s["m"])
    assert np.abs(K - r["W_G"]).max() < 1e-15
    # E_x = tr(M)
    assert abs(np.trace(r["M"]) - r["E_x"]) < 1e-14
    # M symmetric negative definite
    assert np.abs(r["M"] - r["M"].T).max() < 1e-15
    assert np.linalg.eigvalsh(r["M"]).max() < 0
    # an independent route: W M^-1 W^T psi
    K1 = oracle.ace_apply(r["xi"], s["trials"], s["m"])
    K2 = oracle.ace_apply_lu(r["W_G"], r["M"], s["trials"], s["m"])
    assert np.abs(K1 - K2).max() < 1e-14 * np.abs(K1).max() + 1e-18


def test_cholesky_against_numpy():
    rng = np.random.default_rng(0)
    B = rng.standard_normal((9, 9))
    A = B @ B.T + 9 * np.eye(9)
    assert np.abs(oracle.cholesky(A) - np.linalg.cholesky(A)).max() < 1e-13
    with pytest.raises(RuntimeError):
        oracle.cholesky(-A)


def test_unitary_invariance(small):
    s = small
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.standard_normal((5, 5)))
    r1 = oracle.ace_build(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    r2 = oracle.ace_build(U.T @ s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    assert abs(r1["E_x"] - r2["E_x"]) < 1e-14
    K1 = oracle.ace_apply(r1["xi"], s["trials"], s["m"])
    K2 = oracle.ace_apply(r2["xi"], s["trials"], s["m"])
    assert np.abs(K1 - K2).max() < 1e-13 * np.abs(K1).max()


def test_exact_cell_scaling(small):
    """Same coefficients and grid, cell scaled by s: every Coulomb energy scales as 1/s."""
    s = small
    r1 = oracle.ace_build(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    sc = 1.7
    r2 = oracle.ace_build(s["psi"], s["cell"] * sc, s["grid"], s["ecut"] / sc ** 2, s["alpha"])
    assert abs(r2["E_x"] - r1["E_x"] / sc) < 1e-14
    assert np.abs(r2["W_G"] - r1["W_G"] / sc).max() < 1e-15


def test_screened_lists(small):
    s = small
    n = len(s["psi"])
    full = gen.all_pairs_csr(n)
    r0 = oracle.exchange(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    r1 = oracle.exchange(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"], pairs=full)
    assert np.abs(r0[0] - r1[0]).max() < 1e-16 and abs(r0[1] - r1[1]) < 1e-15
    diag = (np.arange(n + 1, dtype=np.int32), np.arange(n, dtype=np.int32))
    W, E = oracle.exchange(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"], pairs=diag)
    e = sum(oracle.pair_energy(p, p, s["cell"], s["grid"], s["ecut"]) for p in s["psi"])
    assert abs(E + s["alpha"] * e) < 1e-15


def test_grid_too_small_rejected():
    cell = gen.cubic_cell(10.0)
    psi = gen.random_orbitals(cell, 30.0, 2, seed=1)
    with pytest.raises(RuntimeError):
        oracle.exchange(psi, cell, (12, 12, 12), 30.0, 0.25)


def test_exchange_rows_match_full_exchange(small):
    s = small
    n = len(s["psi"])
    W, _ = oracle.exchange(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    Wr = oracle.exchange_rows(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"], [3, 0])
    assert np.abs(Wr - W[[3, 0]]).max() < 1e-16
    rng = np.random.default_rng(8)
    row_ptr, cols = [0], []
    for i in range(n):
        cols += [j for j in range(i, n) if j == i or rng.random() < 0.5]
        row_ptr.append(len(cols))
    pairs = (np.array(row_ptr, dtype=np.int32), np.array(cols, dtype=np.int32))
    Ws, _ = oracle.exchange(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"], pairs=pairs)
    Wr = oracle.exchange_rows(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"], [1, 4, 2], pairs=pairs)
    assert np.abs(Wr - Ws[[1, 4, 2]]).max() < 1e-16


# ---------------------------------------------------------------- s-MTACE overlap (Section 2.4)

def test_overlap_diagonal_symmetry_and_bounds():
    """Orthonormal orbitals: S_ii = <phi_i|phi_i> = 1 (the grid sum of phi^2 is
    the inner product), S symmetric, 0 <= S_ij <= 1 (Cauchy-Schwarz)."""
    cfg = gen.config_small()
    S = oracle.overlap(cfg["psi"], cfg["cell"], cfg["grid"], cfg["ecut"])
    assert np.allclose(np.diag(S), 1.0, atol=1e-12)
    assert np.array_equal(S, S.T)
    assert S.min() >= 0 and S.max() <= 1 + 1e-12


def test_overlap_of_two_cosines_is_separable():
    """phi_1 = sqrt(2/Omega) cos(2 pi x / L), phi_2 = sqrt(2/Omega) cos(2 pi y / L):
    the grid integral of |phi_1 phi_2| factorises into 1-D sums,
    S_12 = 2 A^2 with A = (1/n) sum_x |cos(2 pi x / n)|."""
    L, ecut, n = 10.0, 5.0, 18
    cell = gen.cubic_cell(L)
    m = gen.half_sphere(cell, ecut)
    psi = np.zeros((2, len(m)), dtype=np.complex128)
    for row, target in ((0, (1, 0, 0)), (1, (0, 1, 0))):
        k = np.where((m == target).all(1))[0][0]
        psi[row, k] = 1 / np.sqrt(2)
    S = oracle.overlap(psi, cell, (n, n, n), ecut)
    A = np.abs(np.cos(2 * np.pi * np.arange(n) / n)).mean()
    assert abs(S[0, 1] - 2 * A * A) < 1e-13
    assert np.allclose(np.diag(S), 1.0, atol=1e-13)


@pytest.mark.parametrize("d", [0.0, 1.0, 2.5, 4.0])
def test_overlap_of_two_gaussians_closed_form(d):
    """Two normalised Gaussians g_sigma at distance d (positive functions):
    integral g_1 g_2 = exp(-d^2 / (4 sigma^2)).  The product is band-limited
    below the grid's Nyquist frequency, so the grid sum is exact; the
    truncation of the coefficient sphere and the periodic images are below
    1e-12 at these sizes."""
    L, ecut, sigma, n = 20.0, 80.0, 1.0, 64
    cell = gen.cubic_cell(L)
    m = gen.half_sphere(cell, ecut)
    R1 = np.array([10.0, 10.0, 10.0])
    R2 = R1 + np.array([d, 0.0, 0.0])
    psi = np.stack([gen.gaussian_sum_coefficients(cell, m, [R], [sigma], [1.0]) for R in (R1, R2)])
    S = oracle.overlap(psi, cell, (n, n, n), ecut)
    assert abs(S[0, 1] - np.exp(-d * d / (4 * sigma * sigma))) < 1e-10
    assert abs(S[0, 0] - 1.0) < 1e-10


def test_overlap_brute_force_on_a_tiny_grid():
    """phi(r) by direct summation over the plane waves (no FFT), S by direct
    sums, against the oracle's FFT route."""
    cell = gen.cubic_cell(6.0)
    ecut, n = 6.0, 8
    psi = gen.random_orbitals(cell, ecut, 3, seed=4)
    m = gen.half_sphere(cell, ecut)
    G = gen.gvectors(cell, m)
    omega = abs(np.linalg.det(cell))
    ax = np.arange(n) / n
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    r = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1) @ cell  # fractional -> cartesian
    ph = np.exp(1j * (r @ G.T))  # [N][n_pw_half]
    f = []
    for c in psi:
        full = ph @ c + np.conj(ph[:, 1:]) @ np.conj(c[1:])  # c(-G) = c(G)*
        f.append(full.real / np.sqrt(omega))
    f = np.array(f)
    S_ref = np.abs(f[:, None, :] * f[None, :, :]).sum(-1) * omega / n ** 3
    S = oracle.overlap(psi, cell, (n, n, n), ecut)
    assert np.max(np.abs(S - S_ref)) < 1e-12


def test_screened_pairs_rule():
    S = np.array([[1.0, 0.3, 0.01], [0.3, 1.0, 0.02], [0.01, 0.02, 1.0]])
    rp, col = oracle.screened_pairs(S, 0.02)
    assert rp.tolist() == [0, 2, 4, 5] and col.tolist() == [0, 1, 1, 2, 2]
    rp, col = oracle.screened_pairs(S, 2.0)  # the diagonal is always kept
    assert rp.tolist() == [0, 1, 2, 3] and col.tolist() == [0, 1, 2]


def test_mts_drift_keeps_orthonormal_gamma_orbitals():
    """The harness's drifted orbitals stay Gamma-symmetric and orthonormal."""
    from paper_2110_07670_gb300 import mts
    cfg = gen.config_small()
    D = gen.random_orbitals(cfg["cell"], cfg["ecut"], 8, seed=33)
    for k in (0, 1, 5):
        c = mts.drifted_orbitals(cfg["psi"], D, 0.02, k)
        assert np.all(c[:, 0].imag == 0)
        assert np.allclose(gen.gamma_overlap(c, c), np.eye(8), atol=1e-12)
    assert np.allclose(mts.drifted_orbitals(cfg["psi"], D, 0.02, 0), cfg["psi"], atol=1e-12)
