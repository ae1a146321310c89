"""GPU parity of SCDM localisation with the s'-MTACE pre-selection (Sections
2.4-2.5) against the FP64 oracle, through the C ABI.

Integer results (candidate grid points, pivots) are decided in double on both
sides; the mixed form's real-space orbitals are single precision, so a grid
point whose rho or |grad rho| lies within a relative 1e-5 of the average, or a
pivot whose residual ties within 1e-6 of the best, may differ -- everything
else must match exactly.  The orbitals phi = O psi: 1e-10 (fp64) and 1e-5
(mixed: the FP32 values psi_i(r_C) enter the rotation, amplified by the
condition of V) relative to their maximum.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
from oracle import scdm as oscdm
import paper_2110_07670_gb300 as ace

pytestmark = pytest.mark.gpu


def _tr_gamma(a, b):
    """sum_i <a_i|b_i> with the Gamma-point inner product (host arrays)."""
    return float(np.trace(gen.gamma_overlap(a, b)))

TOL = {"fp64": dict(band=1e-10, tie=1e-12, phi=1e-10), "mixed": dict(band=1e-5, tie=1e-6, phi=1e-5)}


def dev(a, plan):
    dt = np.complex64 if plan.prec == ace.ACE_MIXED else np.complex128
    return torch.from_numpy(np.ascontiguousarray(a.astype(dt))).cuda()


def host(t):
    return t.cpu().numpy().astype(np.complex128)


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2110_07670_gb300 import build
    build.build_library()
    ace.load()


def _valid_pivots(phi_real, cand, piv, tie):
    """Each GPU pivot's residual norm, given the GPU's earlier pivots, is the
    largest over the oracle's candidates up to a relative `tie`."""
    A = phi_real[:, cand]
    col = {int(c): k for k, c in enumerate(cand)}
    Q = np.zeros((A.shape[0], 0))
    for p in piv:
        R = A - Q @ (Q.T @ A)
        nu = (R * R).sum(0)
        assert int(p) in col, "pivot outside the candidate set"
        assert nu[col[int(p)]] >= (1 - tie) * nu.max()
        r = R[:, col[int(p)]]
        Q = np.concatenate([Q, (r / np.linalg.norm(r))[:, None]], 1)


def _check_scdm(s, prec, pre):
    tol = TOL[prec]
    n = len(s["psi"])
    ref = oscdm.scdm(s["psi"], s["cell"], s["grid"], s["ecut"], use_preselect=pre)
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], n, prec)
    phi, piv, O, nc = ace.ace_scdm(plan, dev(s["psi"], plan), preselect=pre)
    N = int(np.prod(s["grid"]))
    if pre:
        rho, grad = oscdm.density_and_gradient(s["psi"], s["cell"], s["grid"], s["ecut"])
        gn = np.sqrt((grad * grad).sum(0))
        near = (np.abs(rho - rho.mean()) <= tol["band"] * rho.mean()) | \
               (np.abs(gn - gn.mean()) <= tol["band"] * gn.mean())
        assert abs(nc - len(ref["candidates"])) <= int(near.sum())
    else:
        assert nc == N
    assert np.abs(O @ O.T - np.eye(n)).max() < 1e-12
    phi_real = oracle.to_real(s["psi"], s["cell"], s["grid"], s["ecut"]).reshape(n, -1)
    _valid_pivots(phi_real, ref["candidates"], piv, tol["tie"])
    if np.array_equal(piv, ref["pivots"]):
        P = host(phi)
        assert np.abs(P - ref["phi_G"]).max() <= tol["phi"] * np.abs(ref["phi_G"]).max()
        assert np.abs(O - ref["O"]).max() <= tol["phi"]
    plan.close()
    return piv, ref


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("pre", [True, False])
def test_scdm_matches_oracle_small(prec, pre):
    """8 orbitals on the 32^3 cube."""
    s = gen.config_small()
    piv, ref = _check_scdm(s, prec, pre)
    if prec == "fp64":
        assert np.array_equal(piv, ref["pivots"])


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_scdm_odd_count_noncubic(prec):
    """5 orbitals on a 16 x 18 x 20 box of a non-cubic cell (generic passes)."""
    cell = np.array([[7.0, 0.0, 0.0], [0.8, 7.6, 0.0], [0.0, 0.5, 8.4]])
    s = dict(cell=cell, ecut=12.0, grid=(16, 18, 20), psi=gen.random_orbitals(cell, 12.0, 5, seed=21))
    piv, ref = _check_scdm(s, prec, True)
    if prec == "fp64":
        assert np.array_equal(piv, ref["pivots"])


def test_scdm_separated_gaussians_mixed():
    """Four rotated Gaussians come back as the Gaussians (mixed precision)."""
    L, ecut, grid = 16.0, 25.0, (32, 32, 32)
    cell = gen.cubic_cell(L)
    m = oracle.half_sphere(cell, ecut)
    centres = [np.array(c) for c in ((2.0, 2.0, 2.0), (10.0, 2.0, 2.0), (2.0, 10.0, 10.0), (10.0, 10.0, 2.0))]
    g = np.array([gen.gaussian_sum_coefficients(cell, m, [c], [0.9], [1.0]) for c in centres])
    U, _ = np.linalg.qr(np.random.default_rng(6).standard_normal((4, 4)))
    plan = ace.Plan(grid, cell, ecut, 4, "mixed")
    phi, piv, O, nc = ace.ace_scdm(plan, dev(U @ g, plan))
    C = oracle.gamma_gram(g, host(phi), m)
    assert np.abs(np.abs(C) - np.eye(4)[:, np.argmax(np.abs(C), 0)]).max() < 1e-5
    assert sorted(np.argmax(np.abs(C), 0).tolist()) == [0, 1, 2, 3]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_s_prime_mtace_chain(prec):
    """SCDM -> overlap screen -> screened build (the s'-MTACE outer step): the
    GPU's localised orbitals and pair list give the oracle's screened E_x and
    K psi; unscreened, the build of phi equals the build of psi."""
    s = gen.config_small()
    n = len(s["psi"])
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], n, prec)
    phi, piv, O, nc = ace.ace_scdm(plan, dev(s["psi"], plan))
    _, S = ace.ace_overlap_screen(plan, phi, 0.0)
    cut = float(np.median(S[np.triu_indices(n, 1)]))  # about half the pairs i < j go
    pairs, _ = ace.ace_overlap_screen(plan, phi, cut)
    assert n < pairs[0][-1] < n * (n + 1) // 2
    xi, E = ace.ace_build(plan, phi, s["alpha"], pairs=pairs)
    phi_h = host(phi)
    ref = oracle.ace_build(phi_h, s["cell"], s["grid"], s["ecut"], s["alpha"], pairs=pairs)
    tolE = 1e-10 * abs(ref["E_x"]) if prec == "fp64" else 1e-6 * s["n_atom"]
    assert abs(E - ref["E_x"]) <= tolE
    tr = gen.random_trials(s["cell"], s["ecut"], 4, seed=31)
    K = host(ace.ace_apply(plan, xi, dev(tr, plan)))
    Kref = oracle.ace_apply(ref["xi"], tr, ref["miller"])
    assert np.abs(K - Kref).max() <= (1e-10 if prec == "fp64" else 1e-6) * np.abs(Kref).max()
    _, E_phi = ace.ace_build(plan, phi, s["alpha"])
    _, E_psi = ace.ace_build(plan, dev(s["psi"], plan), s["alpha"])
    assert abs(E_phi - E_psi) <= (1e-10 * abs(E_psi) if prec == "fp64" else 1e-6 * s["n_atom"])


def test_scdm_rejections():
    s = gen.config_small()
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], 8, "mixed")
    psi = dev(s["psi"], plan)
    with pytest.raises(ace.AceError):
        ace.ace_scdm(plan, psi, phi_G=psi)  # in place
    dup = dev(np.concatenate([s["psi"][:4], s["psi"][:4]]), plan)
    with pytest.raises(ace.AceError):
        ace.ace_scdm(plan, dup, preselect=False)  # rank 4 < 8


def test_graph_replay_unaffected_by_scdm_overlap_and_exact_exchange():
    """A captured build replays the pair list of its capture even after SCDM,
    the overlap screen and the exact exchange ran eagerly on the plan with an
    odd orbital count (their quads differ from the build's)."""
    s = gen.config_small()
    n = len(s["psi"])
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], n, "mixed")
    psi = dev(s["psi"], plan)
    xi = torch.empty_like(psi)
    ace.ace_build_async(plan, psi, s["alpha"], xi=xi)
    ace.ace_build_result(plan)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ace.ace_build_async(plan, psi, s["alpha"], xi=xi)
    g.replay()
    E0 = ace.ace_build_result(plan)
    five = dev(s["psi"][:5], plan)
    ace.ace_scdm(plan, five)
    ace.ace_overlap_screen(plan, five, 0.1)
    ace.hfx_apply_exact(plan, five, s["alpha"], dev(gen.random_trials(s["cell"], s["ecut"], 3, seed=8), plan))
    g.replay()
    assert abs(ace.ace_build_result(plan) - E0) <= 1e-10 * abs(E0)
    ref = oracle.ace_build(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    assert abs(E0 - ref["E_x"]) / s["n_atom"] <= 1e-6
    del g
    plan.close()


def test_s_prime_mts_harness_matches_oracle():
    """The MTS loop with s'-MTACE outer steps (FP64): SCDM, the overlap screen
    and the screened build on Phi_0, then inner steps on drifting orbitals --
    pivots, the kept pairs and every step's energies against the oracle."""
    from paper_2110_07670_gb300 import mts
    s = gen.config_small()
    n = len(s["psi"])
    D = gen.random_orbitals(s["cell"], s["ecut"], n, seed=33)
    at = lambda k: mts.drifted_orbitals(s["psi"], D, 0.02, k)
    loc = oscdm.scdm(s["psi"], s["cell"], s["grid"], s["ecut"])
    S = oracle.overlap(loc["phi_G"], s["cell"], s["grid"], s["ecut"])
    cut = float(np.median(S[np.triu_indices(n, 1)]))
    assert np.abs(S - cut).min() > 1e-9 * cut  # no pair within rounding of the cut
    pairs = oracle.screened_pairs(S, cut)
    ref = oracle.ace_build(loc["phi_G"], s["cell"], s["grid"], s["ecut"], s["alpha"], pairs=pairs)
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], n, "fp64")
    rec = mts.run(plan, s["psi"], s["alpha"], at, n_inner=2, every=1, rho_cut=cut)
    plan.close()
    assert np.array_equal(rec[0]["pivots"], loc["pivots"])
    assert all(np.array_equal(a, b) for a, b in zip(rec[0]["pairs"], pairs))
    for r in rec:
        phik = at(r["k"]) if r["k"] else s["psi"]
        E_ace = _tr_gamma(phik, oracle.ace_apply(ref["xi"], phik, ref["miller"]))
        E_ex = oracle.exchange(phik, s["cell"], s["grid"], s["ecut"], s["alpha"])[1]
        assert abs(r["E_ACE"] - E_ace) <= 1e-10 * abs(E_ex)
        assert abs(r["E_exact"] - E_ex) <= 1e-10 * abs(E_ex)
        assert abs(r["dE"] - (E_ex - E_ace)) <= 2e-10 * abs(E_ex)
    assert abs(rec[0]["dE"]) > 1e-6  # the screening error


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("n", [1, 2, 3])
def test_scdm_few_orbitals(prec, n):
    """1 to 3 orbitals (empty row groups in the column pass, no second
    Gram-Schmidt pass at step 0, a 1 x 1 rotation)."""
    s = gen.config_small()
    piv, ref = _check_scdm(dict(s, psi=s["psi"][:n]), prec, True)
    if prec == "fp64":
        assert np.array_equal(piv, ref["pivots"])
