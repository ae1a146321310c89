"""FP64 CPU oracle (test infrastructure only).

Python access to ace_oracle.c, a plain double-precision restatement of the
exchange operator and its ACE compression (arXiv:2110.07670 Sections 2.1-2.2,
Eq. 1-5).  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline
leg may import this package; the GPU library never does, and this package
never imports the GPU library.

Array conventions follow gen/: coefficients are complex128 [n][n_pw_half] on
the half sphere in canonical order; cells have the lattice vectors as rows.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ace_oracle.c")
_LIB = os.path.join(_HERE, "libace_oracle.so")
_lib = None

ERRORS = {-1: "invalid argument", -2: "grid too small for the cutoff sphere", -3: "-M not positive definite",
          -4: "out of memory", -5: "singular matrix"}


def build(force=False):
    """Compile the oracle with gcc (plain C99, pthreads)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i32, f64 = ctypes.c_int, ctypes.c_double
        sig = {
            "orc_half_sphere": [P, f64, i32, P, P],
            "orc_fft3d": [P, P, i32],
            "orc_exchange": [P, i32, i32, P, P, P, f64, P, P, i32, P, P],
            "orc_exchange_timed": [P, i32, i32, P, P, P, f64, P, P, i32, P, P, P],
            "orc_vx_apply": [P, i32, P, i32, i32, P, P, P, f64, i32, P],
            "orc_exchange_rows": [P, i32, i32, P, P, P, f64, P, P, i32, P, i32, P],
            "orc_pair_energy": [P, P, i32, P, P, P, P],
            "orc_to_real": [P, i32, i32, P, P, P, P],
            "orc_overlap": [P, i32, i32, P, P, P, P],
            "orc_gamma_gram": [P, i32, P, i32, i32, P, P],
            "orc_cholesky": [P, i32, P],
            "orc_ace_build": [P, i32, i32, P, P, P, f64, P, P, i32, P, P, P, P],
            "orc_ace_apply": [P, i32, P, i32, i32, P, P],
            "orc_ace_apply_lu": [P, P, i32, P, i32, i32, P, P],
        }
        for name, args in sig.items():
            fn = getattr(lib, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int if name != "orc_fft3d" else None
        lib.orc_set_coulomb_cutoff.argtypes = [f64]
        lib.orc_set_coulomb_cutoff.restype = None
        lib.orc_set_coulomb_g0.argtypes = [f64]
        lib.orc_set_coulomb_g0.restype = None
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _check(st):
    if st != 0:
        raise RuntimeError(f"oracle error {st}: {ERRORS.get(st, '?')}")


def _c128(a):
    return np.ascontiguousarray(a, dtype=np.complex128)


def _cell(cell):
    return np.ascontiguousarray(np.asarray(cell, dtype=np.float64).reshape(9))


def _grid(grid):
    return np.ascontiguousarray(np.asarray(grid, dtype=np.int32).reshape(3))


def half_sphere(cell, ecut):
    lib = _load()
    n = ctypes.c_int(0)
    c = _cell(cell)
    _check(lib.orc_half_sphere(_p(c), float(ecut), 0, None, ctypes.byref(n)))
    m = np.zeros((n.value, 3), dtype=np.int32)
    _check(lib.orc_half_sphere(_p(c), float(ecut), n.value, _p(m), ctypes.byref(n)))
    return m


def fft3d(a, sign):
    """Unnormalised 3D DFT with kernel exp(sign 2 pi i j.k / n) of a complex array."""
    a = _c128(a).copy()
    n = np.array(a.shape, dtype=np.int32)
    _load().orc_fft3d(_p(a), _p(n), int(sign))
    return a


def _csr(pairs):
    if pairs is None:
        return None, None
    rp, col = pairs
    return np.ascontiguousarray(rp, dtype=np.int32), np.ascontiguousarray(col, dtype=np.int32)


class coulomb_cutoff:
    """Context in which every oracle call uses the Coulomb interaction cut off
    at r = rc (bohr): K(G) = 4 pi (1 - cos(|G| rc)) / |G|^2, K(0) = 2 pi rc^2
    (Spencer & Alavi, Phys. Rev. B 77, 193110 (2008)); rc = 0 restores 4 pi / |G|^2
    with G = 0 dropped."""

    def __init__(self, rc):
        self.rc = float(rc)

    def __enter__(self):
        _load().orc_set_coulomb_cutoff(ctypes.c_double(self.rc))
        return self

    def __exit__(self, *exc):
        _load().orc_set_coulomb_cutoff(ctypes.c_double(0.0))
        return False


class coulomb_g0:
    """Context in which the bare kernel 4 pi / |G|^2 keeps the value k0 at
    G = 0 instead of dropping it (k0 = auxiliary_function_k0(cell): the
    Gygi-Baldereschi correction)."""

    def __init__(self, k0):
        self.k0 = float(k0)

    def __enter__(self):
        _load().orc_set_coulomb_g0(ctypes.c_double(self.k0))
        return self

    def __exit__(self, *exc):
        _load().orc_set_coulomb_g0(ctypes.c_double(0.0))
        return False


def auxiliary_function_k0(cell, alpha=None):
    """K(0) = 4 pi chi of the auxiliary-function treatment of the G = 0
    divergence for Gamma-only sampling (Gygi & Baldereschi, Phys. Rev. B 34,
    4405 (1986)), with F(q) = exp(-alpha q^2) / q^2:
        chi = Omega / (2 pi)^3 int F d^3q - [sum_{G != 0} F(G) + lim_{q->0} (F(q) - 1/q^2)]
            = Omega / (2 pi)^3 * 2 pi^(3/2) / sqrt(alpha) - sum_{G != 0} F(G) + alpha,
    the sum over the whole reciprocal lattice (Gaussian-damped); the G = 0
    value of F's regular part (-alpha) belongs to the lattice sum, and with it
    chi does not depend on alpha while the real-space images of F are below
    double-precision resolution.  alpha defaults to (L_min / 12)^2 (L_min:
    the shortest lattice vector).  For a cubic cell 4 pi chi / L^3 is the
    Madelung term xi_M / L that dropping G = 0 leaves in a localised charge's
    self-energy."""
    a = np.asarray(cell, dtype=np.float64).reshape(3, 3)
    omega = abs(np.linalg.det(a))
    b = 2.0 * np.pi * np.linalg.inv(a).T
    if alpha is None:
        alpha = (np.linalg.norm(a, axis=1).min() / 12.0) ** 2
    gmax = np.sqrt(50.0 / alpha)  # exp(-alpha G^2) < 2e-22 beyond
    lim = [int(np.ceil(gmax * np.linalg.norm(a[i]) / (2 * np.pi))) + 1 for i in range(3)]
    h, k, l = np.meshgrid(*[np.arange(-m, m + 1) for m in lim], indexing="ij")
    G = np.stack([h.ravel(), k.ravel(), l.ravel()], 1) @ b
    g2 = (G * G).sum(1)
    g2 = g2[g2 > 0]
    lattice = float(np.sum(np.exp(-alpha * g2) / g2))
    integral = omega / (2 * np.pi) ** 3 * 2.0 * np.pi ** 1.5 / np.sqrt(alpha)
    return 4.0 * np.pi * (integral - lattice + alpha)


def sphere_radius(cell):
    """(3 Omega / 4 pi)^(1/3): the radius of the sphere of the cell's volume,
    the usual cutoff of the truncated interaction."""
    return float((3.0 * abs(np.linalg.det(np.asarray(cell, dtype=np.float64).reshape(3, 3))) / (4.0 * np.pi)) ** (1.0 / 3.0))


def exchange(psi, cell, grid, ecut, alpha, pairs=None, nthreads=0, times=False):
    """(W_G, E_x): W_G[i] = alpha-scaled V_X phi_i on the half sphere, E_x = -alpha sum (ij|ji).
    times=True adds the wall seconds (orbital transforms, pair solves, back transforms)."""
    psi = _c128(psi)
    m = half_sphere(cell, ecut)
    n, npw = psi.shape
    assert npw == len(m)
    W = np.zeros_like(psi)
    E = ctypes.c_double(0)
    t = np.zeros(3)
    rp, col = _csr(pairs)
    _check(_load().orc_exchange_timed(_p(psi), n, npw, _p(m), _p(_grid(grid)), _p(_cell(cell)), float(alpha),
                                      _p(rp), _p(col), int(nthreads), _p(W), ctypes.byref(E), _p(t)))
    return (W, E.value, t) if times else (W, E.value)


def exchange_rows(psi, cell, grid, ecut, alpha, rows, pairs=None, nthreads=0):
    """Rows of W_G (alpha-scaled V_X phi_i restricted to the listed pairs) for
    the requested orbitals only; equals exchange(...)[0][rows]."""
    psi = _c128(psi)
    m = half_sphere(cell, ecut)
    n, npw = psi.shape
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    out = np.zeros((len(rows), npw), dtype=np.complex128)
    rp, col = _csr(pairs)
    _check(_load().orc_exchange_rows(_p(psi), n, npw, _p(m), _p(_grid(grid)), _p(_cell(cell)), float(alpha),
                                     _p(rp), _p(col), len(rows), _p(rows), int(nthreads), _p(out)))
    return out


def vx_apply(psi_occ, trials, cell, grid, ecut, alpha, nthreads=0):
    psi_occ, trials = _c128(psi_occ), _c128(trials)
    m = half_sphere(cell, ecut)
    out = np.zeros_like(trials)
    _check(_load().orc_vx_apply(_p(psi_occ), psi_occ.shape[0], _p(trials), trials.shape[0], len(m), _p(m),
                                _p(_grid(grid)), _p(_cell(cell)), float(alpha), int(nthreads), _p(out)))
    return out


def pair_energy(c_a, c_b, cell, grid, ecut):
    m = half_sphere(cell, ecut)
    e = ctypes.c_double(0)
    _check(_load().orc_pair_energy(_p(_c128(c_a)), _p(_c128(c_b)), len(m), _p(m), _p(_grid(grid)),
                                   _p(_cell(cell)), ctypes.byref(e)))
    return e.value


def to_real(psi, cell, grid, ecut):
    psi = _c128(np.atleast_2d(psi))
    m = half_sphere(cell, ecut)
    out = np.zeros((psi.shape[0],) + tuple(int(g) for g in grid))
    _check(_load().orc_to_real(_p(psi), psi.shape[0], len(m), _p(m), _p(_grid(grid)), _p(_cell(cell)), _p(out)))
    return out


def overlap(psi, cell, grid, ecut):
    """S_ij = integral |phi_i phi_j| dr (the s-MTACE screening overlap, Section 2.4), FP64."""
    psi = _c128(np.atleast_2d(psi))
    m = half_sphere(cell, ecut)
    n = psi.shape[0]
    S = np.zeros((n, n))
    _check(_load().orc_overlap(_p(psi), n, len(m), _p(m), _p(_grid(grid)), _p(_cell(cell)), _p(S)))
    return S


def screened_pairs(S, rho_cut):
    """CSR (row_ptr, col) of the pairs i <= j kept by the s-MTACE criterion
    S_ij >= rho_cut, with the diagonal always kept."""
    n = S.shape[0]
    rp = np.zeros(n + 1, dtype=np.int32)
    cols = []
    for i in range(n):
        for j in range(i, n):
            if i == j or S[i, j] >= rho_cut:
                cols.append(j)
        rp[i + 1] = len(cols)
    return rp, np.array(cols, dtype=np.int32)


def gamma_gram(a, b, miller):
    a, b = _c128(np.atleast_2d(a)), _c128(np.atleast_2d(b))
    out = np.zeros((a.shape[0], b.shape[0]))
    _check(_load().orc_gamma_gram(_p(a), a.shape[0], _p(b), b.shape[0], a.shape[1],
                                  _p(np.ascontiguousarray(miller, dtype=np.int32)), _p(out)))
    return out


def cholesky(A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    L = np.zeros_like(A)
    _check(_load().orc_cholesky(_p(A), A.shape[0], _p(L)))
    return L


def ace_build(psi, cell, grid, ecut, alpha, pairs=None, nthreads=0):
    """dict(xi, E_x, W_G, M) of the ACE construction."""
    psi = _c128(psi)
    m = half_sphere(cell, ecut)
    n, npw = psi.shape
    xi = np.zeros_like(psi)
    W = np.zeros_like(psi)
    M = np.zeros((n, n))
    E = ctypes.c_double(0)
    rp, col = _csr(pairs)
    _check(_load().orc_ace_build(_p(psi), n, npw, _p(m), _p(_grid(grid)), _p(_cell(cell)), float(alpha),
                                 _p(rp), _p(col), int(nthreads), _p(xi), ctypes.byref(E), _p(W), _p(M)))
    return dict(xi=xi, E_x=E.value, W_G=W, M=M, miller=m)


def ace_apply(xi, trials, miller):
    xi, trials = _c128(xi), _c128(np.atleast_2d(trials))
    out = np.zeros_like(trials)
    _check(_load().orc_ace_apply(_p(xi), xi.shape[0], _p(trials), trials.shape[0], xi.shape[1],
                                 _p(np.ascontiguousarray(miller, dtype=np.int32)), _p(out)))
    return out


def ace_apply_lu(W_G, M, trials, miller):
    W_G, trials = _c128(W_G), _c128(np.atleast_2d(trials))
    out = np.zeros_like(trials)
    _check(_load().orc_ace_apply_lu(_p(W_G), _p(np.ascontiguousarray(M, dtype=np.float64)), W_G.shape[0],
                                    _p(trials), trials.shape[0], W_G.shape[1],
                                    _p(np.ascontiguousarray(miller, dtype=np.int32)), _p(out)))
    return out
