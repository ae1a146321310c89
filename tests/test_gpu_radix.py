"""GPU parity of the pair passes' alternative FFT radix plans (the plans the
autotuner times on 96^3, 120^3 and 160^3 boxes) against the FP64 oracle, and
the autotuner's choice among them.

The orbitals fill a sphere of radius 0.3 n in Miller units, so the pair
densities reach every frequency of the box (with the aliasing the oracle
computes too): a Coulomb factor or a frequency table laid out for the wrong
plan changes E_x, W_G and K psi.  Tolerances as in test_gpu_parity.py.
"""
import functools

import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2110_07670_gb300 as ace

pytestmark = pytest.mark.gpu

TOL = dict(E=1e-6, K=1e-6, W=2e-6)
N_ORB = 4


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a.astype(np.complex64))).cuda()


def host(t):
    return t.cpu().numpy().astype(np.complex128)


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2110_07670_gb300 import build
    build.build_library()
    ace.load()


@functools.lru_cache(maxsize=None)
def system(n):
    """4 orbitals on an n^3 box of edge n / 8 bohr, cutoff radius 0.3 n in
    Miller units (sqrt(ecut) = 0.3 n 2 pi / L), 3 trial vectors; the oracle's
    build and apply.  (Trials orthogonal to the orbitals, drawn at random over
    this 97k-wave sphere, make K psi a sum of cancelling terms two orders
    below the orbitals' scale: the split-TF32 products then reach 1.4e-6 of
    max |K psi| on the default plan too.)"""
    L = n / 8.0
    ecut = (0.3 * n * 2 * np.pi / L) ** 2
    cell = gen.cubic_cell(L)
    psi = gen.random_orbitals(cell, ecut, N_ORB, seed=50 + n)
    # trial vectors near the occupied space, as at an MTS inner step: random
    # combinations of the orbitals plus a random part
    mix = np.random.default_rng(70 + n).standard_normal((3, N_ORB))
    tr = mix @ psi + 0.3 * gen.random_trials(cell, ecut, 3, seed=60 + n)
    ref = oracle.ace_build(psi, cell, (n, n, n), ecut, 0.25)
    return dict(cell=cell, ecut=ecut, psi=psi, trials=tr, ref=ref,
                K=oracle.ace_apply(ref["xi"], tr, ref["miller"]))


# (box, first radix, variant): every radix plan with compile-time kernels,
# make_axis_plan's first, under every pair-pass variant the box has; 80^3
# (one plan) for its own rotation of the plane swizzle
CASES = [(80, 10, v) for v in (1, 2, 3, 4)] + \
        [(96, r, v) for r in (12, 8, 16) for v in (1, 2, 3, 4)] + \
        [(120, r, v) for r in (12, 10, 8) for v in (1, 2, 4, 5)] + \
        [(160, r, v) for r in (16, 10) for v in (1, 2, 3, 4)]


@pytest.mark.parametrize("n,radix,variant", CASES)
def test_radix_plans_match_oracle(monkeypatch, n, radix, variant):
    monkeypatch.setenv("ACE_PAIR_RADIX", str(radix))
    s = system(n)
    plan = ace.Plan((n, n, n), s["cell"], s["ecut"], N_ORB, "mixed", pair_variant=variant)
    cfg = plan.config()
    assert cfg["pair_variant"] == variant and cfg["radix_plan"] == f"{radix} x {n // radix}"
    xi, E = ace.ace_build(plan, dev(s["psi"]), 0.25)
    W, _ = ace.ace_last_intermediates(plan, N_ORB)
    ref = s["ref"]
    assert abs(E - ref["E_x"]) / (3 * N_ORB / 4) <= TOL["E"]
    assert rel(host(W), ref["W_G"]) <= TOL["W"]
    K = host(ace.ace_apply(plan, xi, dev(s["trials"])))
    assert rel(K, s["K"]) <= TOL["K"]
    plan.close()


def test_autotuner_times_every_radix_plan(monkeypatch, tmp_path):
    """A 96^3 plan with the automatic choice times the three radix plans,
    keeps one of them, and writes it to the tune cache; a second plan reads
    it back and builds the same E_x."""
    monkeypatch.delenv("ACE_PAIR_RADIX", raising=False)
    monkeypatch.delenv("ACE_ROW_BLOCK", raising=False)
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("ACE_TUNE_CACHE", str(path))
    s = system(96)
    p1 = ace.Plan((96, 96, 96), s["cell"], s["ecut"], N_ORB, "mixed")
    c1 = p1.config()
    assert set(c1["radix_ms"]) == {"12 x 8", "8 x 12", "16 x 6"}
    assert c1["radix_plan"] in c1["radix_ms"]
    assert c1["radix_ms"][c1["radix_plan"]] == min(c1["radix_ms"].values())
    r0 = int(c1["radix_plan"].split()[0])
    line = path.read_text().splitlines()[0]
    assert line.endswith(f"= {c1['pair_variant']} {c1['pair_streams']} {c1['row_block']} {0 if r0 == 12 else r0}")
    p2 = ace.Plan((96, 96, 96), s["cell"], s["ecut"], N_ORB, "mixed")
    c2 = p2.config()
    assert c2["from_tune_cache"] and c2["radix_plan"] == c1["radix_plan"]
    _, E1 = ace.ace_build(p1, dev(s["psi"]), 0.25)
    _, E2 = ace.ace_build(p2, dev(s["psi"]), 0.25)
    assert E1 == E2
    assert abs(E1 - s["ref"]["E_x"]) / (3 * N_ORB / 4) <= TOL["E"]
    p1.close()
    p2.close()


def test_radix_plan_rejections(monkeypatch):
    """ACE_PAIR_RADIX that names no candidate plan of the grid fails plan
    creation; grids without alternatives have one candidate."""
    s = system(96)
    monkeypatch.setenv("ACE_PAIR_RADIX", "7")
    with pytest.raises(ace.AceError):
        ace.Plan((96, 96, 96), s["cell"], s["ecut"], N_ORB, "mixed")
    monkeypatch.setenv("ACE_PAIR_RADIX", "4")
    cfg = gen.config_small()
    with pytest.raises(ace.AceError):  # 32^3 has make_axis_plan's 8 x 4 only
        ace.Plan(cfg["grid"], cfg["cell"], cfg["ecut"], 8, "mixed")
    monkeypatch.delenv("ACE_PAIR_RADIX")
    s120 = system(120)
    with pytest.raises(ace.AceError):  # the persistent pipeline needs n % 16 == 0
        ace.Plan((120, 120, 120), s120["cell"], s120["ecut"], N_ORB, "mixed", pair_variant=3)
    p = ace.Plan(cfg["grid"], cfg["cell"], cfg["ecut"], 8, "mixed")
    assert len(p.config()["radix_ms"]) <= 1
    p.close()
