"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only draws inputs: plane-wave coefficient sets of real (Gamma-point)
orbitals, trial vectors and screened pair lists.  It holds none of the exchange
arithmetic (no FFT, no Poisson solve, no ACE step), so that the oracle and the
CUDA path, which both read these arrays, stay independent of one another.

Conventions (the input format of the library):

* cell: 3x3 array whose ROWS are the lattice vectors a1, a2, a3 in bohr.
* Plane waves: G = h b1 + k b2 + l b3 with b = 2 pi inv(A)^T, kept when
  |G|^2 <= ecut (Ry, so |G|^2 in bohr^-2 equals the kinetic energy in Ry).
  The wave-function count this gives reproduces Table 1 of arXiv:2110.07670.
* Half sphere (one of each +-G pair): {h>0} U {h=0,k>0} U {h=k=0,l>=0}, in
  lexicographic (h, k, l) order, so G=0 is entry 0.
* Orbital psi(r) = Omega^-1/2 sum_G c(G) e^{iG.r} over the full sphere with
  c(-G) = c(G)^*; only the half sphere is stored.  Normalisation: the full-sphere
  sum of |c|^2 is 1.
"""
import numpy as np

BOHR_PER_ANGSTROM = 1.0 / 0.52917721


def cubic_cell(L):
    return np.eye(3) * float(L)


def reciprocal(cell):
    """Rows are b1, b2, b3 with a_i . b_j = 2 pi delta_ij."""
    return 2.0 * np.pi * np.linalg.inv(np.asarray(cell, dtype=np.float64)).T


def half_sphere(cell, ecut_ry):
    """Miller indices [n_pw_half, 3] (int32) of the half sphere, canonical order."""
    cell = np.asarray(cell, dtype=np.float64)
    b = reciprocal(cell)
    gmax = np.sqrt(ecut_ry)
    # |h| <= |G| |a1| / (2 pi), likewise for k, l.
    lim = [int(np.floor(gmax * np.linalg.norm(cell[i]) / (2 * np.pi))) + 1 for i in range(3)]
    h = np.arange(0, lim[0] + 1)
    k = np.arange(-lim[1], lim[1] + 1)
    l = np.arange(-lim[2], lim[2] + 1)
    H, K, L = np.meshgrid(h, k, l, indexing="ij")
    H, K, L = H.ravel(), K.ravel(), L.ravel()
    G = np.stack([H, K, L], 1) @ b
    inside = (G * G).sum(1) <= ecut_ry
    half = (H > 0) | ((H == 0) & (K > 0)) | ((H == 0) & (K == 0) & (L >= 0))
    m = np.stack([H, K, L], 1)[inside & half]
    return np.ascontiguousarray(m.astype(np.int32))  # meshgrid 'ij' order is lexicographic


def gvectors(cell, miller):
    return miller.astype(np.float64) @ reciprocal(cell)


def gamma_overlap(a, b):
    """Real overlap matrix S_ij = <a_i|b_j> of Gamma-point functions stored on
    the half sphere (G=0 first): 2 Re sum_half conj(a) b - conj(a0) b0."""
    a = np.asarray(a)
    b = np.asarray(b)
    s = 2.0 * (a.conj() @ b.T).real
    s -= np.outer(a[:, 0].conj(), b[:, 0]).real
    return s


def lowdin(c):
    """Loewdin-orthonormalise the rows of c (Gamma inner product): S^-1/2 c."""
    s = gamma_overlap(c, c)
    w, v = np.linalg.eigh(s)
    if w.min() <= 0:
        raise ValueError("orbitals are linearly dependent")
    return (v @ np.diag(w ** -0.5) @ v.T) @ c


def _gamma_fix(c):
    c = np.array(c, dtype=np.complex128)
    c[:, 0] = c[:, 0].real
    return c


def random_orbitals(cell, ecut_ry, n, seed):
    """Complex-normal coefficients inside the cutoff sphere, Gamma-symmetric
    (c(0) real), Loewdin-orthonormalised."""
    rng = np.random.default_rng(seed)
    npw = len(half_sphere(cell, ecut_ry))
    c = rng.standard_normal((n, npw)) + 1j * rng.standard_normal((n, npw))
    return lowdin(_gamma_fix(c))


def random_trials(cell, ecut_ry, T, seed):
    """Random Gamma-symmetric trial vectors, each normalised to 1."""
    rng = np.random.default_rng(seed)
    npw = len(half_sphere(cell, ecut_ry))
    c = _gamma_fix(rng.standard_normal((T, npw)) + 1j * rng.standard_normal((T, npw)))
    nrm = np.sqrt(np.einsum("ii->i", gamma_overlap(c, c)))
    return c / nrm[:, None]


def _min_image(d, L):
    return d - L * np.round(d / L)


def water_sites(L, n_mol, rng, min_dist=1.5):
    """n_mol * 3 random O/H-like sites in a cubic box, min-image spacing >= min_dist."""
    sites = []
    while len(sites) < 3 * n_mol:
        p = rng.uniform(0.0, L, 3)
        if all(np.linalg.norm(_min_image(p - q, L)) >= min_dist for q in sites):
            sites.append(p)
    return np.array(sites)


def gaussian_sum_coefficients(cell, miller, centres, widths, weights):
    """Plane-wave coefficients of phi(r) = sum_s w_s g_{sigma_s}(r - R_s), with
    the normalised Gaussian g_sigma = (pi sigma^2)^-3/4 exp(-r^2 / 2 sigma^2);
    its transform is (4 pi sigma^2)^3/4 exp(-sigma^2 G^2 / 2) e^{-iG.R} / sqrt(Omega)."""
    G = gvectors(cell, miller)
    G2 = (G * G).sum(1)
    omega = abs(np.linalg.det(cell))
    c = np.zeros(len(miller), dtype=np.complex128)
    for R, s, w in zip(centres, widths, weights):
        c += w * (4 * np.pi * s * s) ** 0.75 * np.exp(-0.5 * s * s * G2) * np.exp(-1j * (G @ R))
    return c / np.sqrt(omega)


def water_orbitals(L, ecut_ry, n_occ, seed):
    """Water-box-shaped orbitals: n_occ/4 molecules (3 sites each); orbital k is
    a Gaussian sum over molecule k//4's sites with N(0,1) weights and widths
    U[0.6, 1.2] bohr; Loewdin-orthonormalised."""
    rng = np.random.default_rng(seed)
    cell = cubic_cell(L)
    miller = half_sphere(cell, ecut_ry)
    n_mol = n_occ // 4
    sites = water_sites(L, n_mol, rng)
    c = np.empty((n_occ, len(miller)), dtype=np.complex128)
    for k in range(n_occ):
        m = k // 4
        R = sites[3 * m:3 * m + 3]
        c[k] = gaussian_sum_coefficients(cell, miller, R, rng.uniform(0.6, 1.2, 3), rng.standard_normal(3))
    return lowdin(_gamma_fix(c)), sites


def localized_orbitals(L, ecut_ry, n_occ, seed):
    """One random centre per orbital; three sites jittered by at most 1 bohr
    around it; Gaussian widths U[0.6, 1.2]; Loewdin-orthonormalised.
    Returns (coefficients, centres)."""
    rng = np.random.default_rng(seed)
    cell = cubic_cell(L)
    miller = half_sphere(cell, ecut_ry)
    centres = rng.uniform(0.0, L, (n_occ, 3))
    c = np.empty((n_occ, len(miller)), dtype=np.complex128)
    for k in range(n_occ):
        d = rng.standard_normal((3, 3))
        d *= (rng.uniform(0.0, 1.0, (3, 1)) / np.linalg.norm(d, axis=1, keepdims=True))
        c[k] = gaussian_sum_coefficients(cell, miller, centres[k] + d, rng.uniform(0.6, 1.2, 3),
                                         rng.standard_normal(3))
    return lowdin(_gamma_fix(c)), centres


def all_pairs_csr(n):
    """CSR of every pair i <= j: row_ptr[n+1], col[] (int32)."""
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    cols = []
    for i in range(n):
        cols.extend(range(i, n))
        row_ptr[i + 1] = len(cols)
    return row_ptr, np.array(cols, dtype=np.int32)


def distance_pairs_csr(centres, L, rcut):
    """CSR of pairs i <= j whose centres are closer than rcut (minimum image);
    the diagonal is always kept."""
    n = len(centres)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    cols = []
    for i in range(n):
        d = np.linalg.norm(_min_image(centres[i:] - centres[i], L), axis=1)
        js = i + np.nonzero(d < rcut)[0]
        cols.extend(js.tolist())
        row_ptr[i + 1] = len(cols)
    return row_ptr, np.array(cols, dtype=np.int32)


def fft_size(x):
    """Smallest even 2^a 3^b 5^c >= x."""
    n = max(2, int(np.ceil(x)))
    while True:
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        if m == 1 and n % 2 == 0:
            return n
        n += 1


# ---------------------------------------------------------------- workloads
# Each returns a dict with: cell (3x3), grid (3,), ecut, alpha, psi (n_occ x
# n_pw_half complex128), and optionally trials, pairs (row_ptr, col).

def config_small(seed=1):
    """8 random orbitals, 32^3 grid, 10-bohr cubic cell, 30 Ry (36 pairs)."""
    cell = cubic_cell(10.0)
    return dict(name="8orb-32^3-L10-30Ry", cell=cell, grid=(32, 32, 32), ecut=30.0, alpha=0.25,
                psi=random_orbitals(cell, 30.0, 8, seed), n_atom=6)


def config_water32(seed=2):
    """128 orbitals of 32 water-like molecules, 96^3 grid, 18.6-bohr cell, 80 Ry (8256 pairs)."""
    psi, _ = water_orbitals(18.6, 80.0, 128, seed)
    return dict(name="water32-128orb-96^3-L18.6-80Ry", cell=cubic_cell(18.6), grid=(96, 96, 96),
                ecut=80.0, alpha=0.25, psi=psi, n_atom=96)


def config_water64(seed=3, n_trial_sets=10, T=256):
    """256 orbitals of 64 water-like molecules, 120^3 grid, 23.5-bohr cell, 80 Ry,
    plus n_trial_sets x T random trial vectors (inner MTS steps)."""
    psi, _ = water_orbitals(23.5, 80.0, 256, seed)
    cell = cubic_cell(23.5)
    trials = [random_trials(cell, 80.0, T, seed * 1000 + s) for s in range(n_trial_sets)]
    return dict(name="water64-256orb-120^3-L23.5-80Ry", cell=cell, grid=(120, 120, 120), ecut=80.0,
                alpha=0.25, psi=psi, trials=trials, n_atom=192)


def batched_systems(seed=4, n_sys=16):
    """Independent cubic cells: n_occ from {32,...,256}, L ~ U[9, 23.5] bohr,
    grid = clamp(fft_size(5.16 L), 48, 120), 80 Ry."""
    rng = np.random.default_rng(seed)
    out = []
    for s in range(n_sys):
        n_occ = int(rng.choice([32, 64, 96, 128, 192, 256]))
        L = float(rng.uniform(9.0, 23.5))
        n = min(120, max(48, fft_size(5.16 * L)))
        psi, _ = water_orbitals(L, 80.0, n_occ, seed * 100 + s)
        out.append(dict(name=f"sys{s}-{n_occ}orb-{n}^3-L{L:.2f}", cell=cubic_cell(L), grid=(n, n, n),
                        ecut=80.0, alpha=0.25, psi=psi, n_atom=3 * n_occ // 4))
    return out


def config_localized(seed=5, n_occ=512, L=29.6, n=160, rcut=8.0):
    """512 localised orbitals, 160^3 grid, 29.6-bohr cell, 80 Ry, pairs with
    centre distance < 8 bohr."""
    psi, centres = localized_orbitals(L, 80.0, n_occ, seed)
    return dict(name=f"localized-{n_occ}orb-{n}^3-L{L}-80Ry-r{rcut}", cell=cubic_cell(L), grid=(n, n, n),
                ecut=80.0, alpha=0.25, psi=psi, pairs=distance_pairs_csr(centres, L, rcut),
                n_atom=3 * n_occ // 4)
