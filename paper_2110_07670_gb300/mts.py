"""The multiple-time-step use of the ACE operator (Section 2.3, Eq. 6-7).

At an outer step the ACE operator K_0 is built from the occupied orbitals
Phi_0; the inner steps use it unchanged on the orbitals Phi_k they reach, and
the difference to the exact exchange -- the slow part of the split, which the
paper evaluates every n steps -- is computed only there.  With no ions or
forces here, the exchange energy plays the role of the force:

    E_ACE(k)   = sum_i <phi_k,i | K_0 phi_k,i>      (fast: the apply's Gram, -sum C^2)
    E_exact(k) = E_x[Phi_k]                          (slow: a full build on Phi_k)
    dE(k)      = E_exact(k) - E_ACE(k)               (the slow correction)

K_0 equals alpha V_X on span(Phi_0), so dE(0) = 0, and dE grows with the
orbitals' drift.  With rho_cut set, the outer step is the s'-MTACE one
(Sections 2.4-2.5): SCDM localisation of Phi_0 with the density / gradient
pre-selection, the overlap screen S_ij >= rho_cut on the localised orbitals,
and K_0 built from the screened pairs only; dE(0) is then the screening
error.  Every step runs through the library's C ABI.
"""
import time

import numpy as np


def run(plan, phi0, alpha, orbitals_at, n_inner, every=1, rho_cut=None):
    """Outer build on phi0, then inner steps k = 1..n_inner on orbitals_at(k)
    (host arrays [n_occ][n_pw_half], Gamma-symmetric, orthonormal).  Returns a
    list of per-step records: k, E_ACE, and every `every` steps E_exact and dE,
    with the device time of each part.  rho_cut: build K_0 the s'-MTACE way
    (record 0 then also carries the SCDM pivots and the kept pair list)."""
    import torch

    import paper_2110_07670_gb300 as ace

    dt = np.complex64 if plan.prec == ace.ACE_MIXED else np.complex128
    d0 = torch.from_numpy(np.ascontiguousarray(phi0.astype(dt))).cuda()
    t0 = time.perf_counter()
    if rho_cut is None:
        xi, E0 = ace.ace_build(plan, d0, alpha)
        torch.cuda.synchronize()
        out = [{"k": 0, "E_ACE": E0, "E_exact": E0, "dE": 0.0, "build_s": time.perf_counter() - t0}]
    else:
        loc, piv, _, _ = ace.ace_scdm(plan, d0)
        pairs, _ = ace.ace_overlap_screen(plan, loc, rho_cut)
        xi, _ = ace.ace_build(plan, loc, alpha, pairs=pairs)
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        E0 = ace.ace_apply_energy(plan, xi, d0)
        _, E_ex = ace.ace_build(plan, d0, alpha, xi=torch.empty_like(d0))
        torch.cuda.synchronize()
        out = [{"k": 0, "E_ACE": E0, "E_exact": E_ex, "dE": E_ex - E0, "build_s": t_build, "pivots": piv,
                "pairs": pairs}]
    W = torch.empty_like(d0)
    for k in range(1, n_inner + 1):
        phik = orbitals_at(k)
        dk = torch.from_numpy(np.ascontiguousarray(phik.astype(dt))).cuda()
        t0 = time.perf_counter()
        E_ace = ace.ace_apply_energy(plan, xi, dk)
        rec = {"k": k, "apply_s": time.perf_counter() - t0, "E_ACE": E_ace}
        if k % every == 0:
            t0 = time.perf_counter()
            _, Ek = ace.ace_build(plan, dk, alpha, xi=W)
            torch.cuda.synchronize()
            rec.update(E_exact=Ek, dE=Ek - rec["E_ACE"], exact_s=time.perf_counter() - t0)
        out.append(rec)
    return out


def drifted_orbitals(phi0, direction, eps, k):
    """Phi_k = Loewdin(Phi_0 + k eps D): a smooth drift of the occupied set,
    re-orthonormalised with the Gamma-point overlap (Gamma symmetry kept:
    G = 0 coefficients real)."""
    c = phi0 + (k * eps) * direction
    c = np.array(c, dtype=np.complex128)
    c[:, 0] = c[:, 0].real
    s = 2.0 * np.real(np.conj(c) @ c.T) - np.outer(c[:, 0].real, c[:, 0].real)
    w, v = np.linalg.eigh(s)
    return (v @ np.diag(w ** -0.5) @ v.T) @ c
