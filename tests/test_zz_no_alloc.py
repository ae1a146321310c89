"""ace_apply_noalloc: the ACE apply for callers that cannot allocate device
memory (an inner loop that must not stall on cudaMalloc, or a host whose
device memory belongs to another allocator).  It must give the result of the
plan-based ace_apply, within the GPU parity tolerance, on consecutive calls
that reuse its one fixed scratch array.  Named to be collected last."""
import numpy as np
import pytest
import torch

import gen
import paper_2110_07670_gb300 as ace

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "mixed": 1e-6}  # max |diff| / max |reference|, as in the parity tests


def _dev(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a.astype(dtype))).cuda()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_apply_noalloc_matches_apply_on_two_calls(prec):
    from paper_2110_07670_gb300 import build
    build.build_library()
    cfg = gen.config_small()
    dt = np.complex64 if prec == "mixed" else np.complex128
    plan = ace.Plan(cfg["grid"], cfg["cell"], cfg["ecut"], 8, prec)
    xi, _ = ace.ace_build(plan, _dev(cfg["psi"], dt), cfg["alpha"])
    for seed, T in ((5, 9), (6, 4)):  # two calls in a row, different sizes and inputs
        tr = _dev(gen.random_trials(cfg["cell"], cfg["ecut"], T, seed), dt)
        ref = ace.ace_apply(plan, xi, tr).cpu().numpy()
        out = torch.full_like(tr, float("nan"))
        ace.ace_apply_noalloc(xi, tr, out)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= TOL[prec] * np.abs(ref).max()


def test_apply_noalloc_rejects_oversize():
    xi = torch.zeros((1024, 16), dtype=torch.complex64, device="cuda")
    psi = torch.zeros((600, 16), dtype=torch.complex64, device="cuda")
    out = torch.zeros_like(psi)
    with pytest.raises(ace.AceError) as e:
        ace.ace_apply_noalloc(xi, psi, out)
    assert e.value.code == -1 and "exceeds" in str(e.value)


def _gamma_random(rng, rows, npw, dtype):
    a = (rng.standard_normal((rows, npw)) + 1j * rng.standard_normal((rows, npw))) / np.sqrt(npw)
    a[:, 0] = a[:, 0].real
    return _dev(a, dtype)


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_apply_noalloc_at_the_size_limit(prec):
    """T * n_occ exactly at the limit (512 ACE vectors, 1024 trials): C and the
    Gram partials then just fit in the fixed array; the result must match the
    plan-based apply, and one more trial must be rejected before any work."""
    from paper_2110_07670_gb300 import build
    build.build_library()
    cfg = gen.config_small()
    dt = np.complex64 if prec == "mixed" else np.complex128
    plan = ace.Plan(cfg["grid"], cfg["cell"], cfg["ecut"], 8, prec)
    rng = np.random.default_rng(11)
    xi = _gamma_random(rng, 512, plan.n_pw_half, dt)
    tr = _gamma_random(rng, 1024, plan.n_pw_half, dt)
    assert xi.shape[0] * tr.shape[0] == 524288
    ref = ace.ace_apply(plan, xi, tr).cpu().numpy()
    out = torch.full_like(tr, float("nan"))
    ace.ace_apply_noalloc(xi, tr, out)
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    assert np.abs(got - ref).max() <= TOL[prec] * np.abs(ref).max()
    over = _gamma_random(rng, 1025, plan.n_pw_half, dt)
    with pytest.raises(ace.AceError) as e:
        ace.ace_apply_noalloc(xi, over, torch.empty_like(over))
    assert e.value.code == -1 and "exceeds" in str(e.value)
    plan.close()
