"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle,
element by element on the same seeded inputs.

Tolerances (written here, derived in the design notes):
  fp64 form : relative 1e-10 on every output (only rounding order differs);
  mixed form: |dE_x| <= 1e-6 Ha per atom (n_atom = 3 n_occ / 4) and
              max |K psi - K_oracle psi| / max |K_oracle psi| <= 1e-6;
              intermediates (W_G, M, V_X psi) to 2e-6 relative to their maximum.
"""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2110_07670_gb300 as ace

pytestmark = pytest.mark.gpu


def _tr_gamma(a, b):
    """sum_i <a_i|b_i> with the Gamma-point inner product (host arrays)."""
    return float(np.trace(gen.gamma_overlap(a, b)))

TOL = {"fp64": dict(E=1e-10, K=1e-10, W=1e-10), "mixed": dict(E=1e-6, K=1e-6, W=2e-6)}


def dev(a, plan):
    dt = np.complex64 if plan.prec == ace.ACE_MIXED else np.complex128
    return torch.from_numpy(np.ascontiguousarray(a.astype(dt))).cuda()


def host(t):
    return t.cpu().numpy().astype(np.complex128)


def rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2110_07670_gb300 import build
    build.build_library()
    ace.load()


def small_system(n=5, seed=11):
    cell = gen.cubic_cell(7.0)
    return dict(cell=cell, ecut=14.0, grid=(16, 16, 16), alpha=0.25, psi=gen.random_orbitals(cell, 14.0, n, seed),
                trials=gen.random_trials(cell, 14.0, 3, seed + 1), n_atom=3 * n / 4)


def check_build(s, prec, pairs=None, trials=None):
    tol = TOL[prec]
    n = len(s["psi"])
    ref = oracle.ace_build(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"], pairs=pairs)
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], n, prec)
    assert np.array_equal(ace.ace_gvec(plan), ref["miller"])
    xi, E = ace.ace_build(plan, dev(s["psi"], plan), s["alpha"], pairs=pairs)
    W, M = ace.ace_last_intermediates(plan, n)
    assert abs(E - ref["E_x"]) / s["n_atom"] <= tol["E"] * (1 if prec == "mixed" else abs(ref["E_x"]) + 1e-300)
    assert rel(host(W), ref["W_G"]) <= tol["W"]
    assert np.abs(M - ref["M"]).max() <= tol["W"] * np.abs(ref["M"]).max()
    tr = trials if trials is not None else gen.random_trials(s["cell"], s["ecut"], 6, seed=99)
    Kref = oracle.ace_apply(ref["xi"], tr, ref["miller"])
    K = host(ace.ace_apply(plan, xi, dev(tr, plan)))
    assert rel(K, Kref) <= tol["K"]
    if pairs is None:
        # exactness on the occupied span with the GPU's own vectors (a screened
        # list makes M unsymmetric, and exactness holds only without screening)
        Kphi = host(ace.ace_apply(plan, xi, dev(s["psi"], plan)))
        assert rel(Kphi, ref["W_G"]) <= tol["K"] * 2
    return E, ref


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_hfx_exact_matches_oracle(prec):
    s = small_system()
    ref = oracle.vx_apply(s["psi"], s["trials"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], len(s["psi"]), prec)
    out = host(ace.hfx_apply_exact(plan, dev(s["psi"], plan), s["alpha"], dev(s["trials"], plan)))
    assert rel(out, ref) <= TOL[prec]["W"]


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_build_small_random(prec):
    check_build(gen.config_small(), prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("grid", [(16, 18, 20), (20, 16, 18), (18, 20, 15)])
def test_build_odd_count_noncubic(prec, grid):
    """7 orbitals (last packed transform half empty), a skewed cell and
    non-cubic grids with radices 2, 3, 4, 5, 8 on different axes; x extents
    20 / 18 / 15 exercise the vector, scalar and non-bulk tile paths."""
    cell = np.array([[7.0, 0.0, 0.0], [0.6, 7.5, 0.0], [0.3, -0.4, 8.0]])
    ecut = 9.0
    psi = gen.random_orbitals(cell, ecut, 7, seed=31)
    s = dict(cell=cell, ecut=ecut, grid=grid, alpha=0.25, psi=psi, n_atom=3 * 7 / 4)
    check_build(s, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_build_single_orbital(prec):
    s = small_system(n=1, seed=41)
    check_build(s, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_build_screened_pairs(prec):
    s = small_system(n=6, seed=51)
    rng = np.random.default_rng(3)
    row_ptr, cols = [0], []
    for i in range(6):
        js = [j for j in range(i, 6) if j == i or rng.random() < 0.5]
        cols += js
        row_ptr.append(len(cols))
    pairs = (np.array(row_ptr, dtype=np.int32), np.array(cols, dtype=np.int32))
    check_build(s, prec, pairs=pairs)


def test_apply_empty_and_shapes():
    s = small_system()
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], 5, "mixed")
    xi, _ = ace.ace_build(plan, dev(s["psi"], plan), s["alpha"])
    out = ace.ace_apply(plan, xi, dev(s["trials"][:0], plan))
    assert out.shape[0] == 0


def test_error_paths():
    s = small_system()
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], 5, "mixed")
    zero = s["psi"].copy()
    zero[1] = 0.0  # a zero orbital makes M exactly singular
    with pytest.raises(ace.AceError) as e:
        ace.ace_build(plan, dev(zero, plan), s["alpha"])
    assert e.value.code == -3
    bad = s["psi"].copy()
    bad[2, 0] += 1e-3j
    with pytest.raises(ace.AceError) as e:
        ace.ace_build(plan, dev(bad, plan), s["alpha"])
    assert e.value.code == -1
    with pytest.raises(ace.AceError) as e:
        ace.Plan((8, 8, 8), s["cell"], s["ecut"], 5, "mixed")
    assert e.value.code == -2
    with pytest.raises(ace.AceError) as e:
        ace.Plan((21, 21, 21), s["cell"], s["ecut"], 5, "mixed")
    assert e.value.code == -2
    with pytest.raises(ace.AceError):
        ace.ace_build(plan, dev(gen.random_orbitals(s["cell"], s["ecut"], 6, 1), plan), s["alpha"])
    # the plan stays usable after errors
    xi, E = ace.ace_build(plan, dev(s["psi"], plan), s["alpha"])
    assert np.isfinite(E)


def test_tensor_core_gram_matches_cuda_cores():
    """The tcgen05 split-TF32 Gram (default for single precision) against the
    CUDA-core Gram, through ace_apply with ragged sizes (partial 128-row tiles,
    K = 2 n_pw_half not a multiple of the K tile), and through ace_build."""
    cfg = gen.config_small()
    rng = np.random.default_rng(17)
    npw = len(gen.half_sphere(cfg["cell"], cfg["ecut"]))
    xi = (rng.standard_normal((200, npw)) + 1j * rng.standard_normal((200, npw))) / np.sqrt(npw)
    xi[:, 0] = xi[:, 0].real
    psi = gen.random_trials(cfg["cell"], cfg["ecut"], 150, seed=18)
    out = []
    for kernels in (0, 1):
        plan = ace.Plan(cfg["grid"], cfg["cell"], cfg["ecut"], 200, "mixed", kernels=kernels)
        out.append(host(ace.ace_apply(plan, dev(xi, plan), dev(psi, plan))))
    ref = -xi.T @ oracle.gamma_gram(xi, psi, gen.half_sphere(cfg["cell"], cfg["ecut"]))
    assert rel(out[0], ref.T) <= 1e-6 and rel(out[1], ref.T) <= 1e-6
    assert rel(out[0], out[1]) <= 1e-6
    Es, Ms = [], []
    for kernels in (0, 1):
        plan = ace.Plan(cfg["grid"], cfg["cell"], cfg["ecut"], 8, "mixed", kernels=kernels)
        _, E = ace.ace_build(plan, dev(cfg["psi"], plan), cfg["alpha"])
        Es.append(E)
        Ms.append(ace.ace_last_intermediates(plan, 8)[1])
    assert np.abs(Ms[0] - Ms[1]).max() <= 1e-6 * np.abs(Ms[1]).max()


@pytest.mark.parametrize("prec", ["mixed"])
def test_generic_kernels_on_a_cube(prec):
    """The runtime-size FFT passes on a 32^3 box (normally served by the
    compile-time cube kernels) give the same build."""
    cfg = gen.config_small()
    ref = oracle.ace_build(cfg["psi"], cfg["cell"], cfg["grid"], cfg["ecut"], cfg["alpha"])
    plan = ace.Plan(cfg["grid"], cfg["cell"], cfg["ecut"], 8, prec, kernels=2)
    xi, E = ace.ace_build(plan, dev(cfg["psi"], plan), cfg["alpha"])
    assert abs(E - ref["E_x"]) / cfg["n_atom"] <= 1e-6
    tr = gen.random_trials(cfg["cell"], cfg["ecut"], 4, seed=5)
    assert rel(host(ace.ace_apply(plan, xi, dev(tr, plan))), oracle.ace_apply(ref["xi"], tr, ref["miller"])) <= 1e-6


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("world", [2, 3])
def test_split_build_over_shards_matches_oracle(prec, world):
    """ace_build_pairs on each shard of the pair list, W_G and E summed, then
    ace_build_finish: the multi-GPU path's arithmetic, run shard by shard on
    one GPU, against the oracle's single build (every pair, then screened)."""
    from paper_2110_07670_gb300 import shard
    tol = TOL[prec]
    s = gen.config_small()
    n = len(s["psi"])
    rp_all, col_all = gen.all_pairs_csr(n)
    keep = [(i, j) for i in range(n) for j in range(i, n) if i == j or (i + 2 * j) % 3 != 0]
    rp_s = np.zeros(n + 1, dtype=np.int32)
    for i, _ in keep:
        rp_s[i + 1] += 1
    screened = (np.cumsum(rp_s).astype(np.int32), np.array([j for _, j in keep], dtype=np.int32))
    for pairs in (None, screened):
        ref = oracle.ace_build(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"], pairs=pairs)
        plan = ace.Plan(s["grid"], s["cell"], s["ecut"], n, prec)
        psi = dev(s["psi"], plan)
        W_sum, E_sum = None, 0.0
        for r in range(world):
            W, E = ace.ace_build_pairs(plan, psi, s["alpha"], pairs=shard.shard_pairs(n, world, r, pairs))
            W_sum = W.clone() if W_sum is None else W_sum + W
            E_sum += E
        xi = ace.ace_build_finish(plan, psi, W_sum)
        assert abs(E_sum - ref["E_x"]) / s["n_atom"] <= tol["E"] * (1 if prec == "mixed" else abs(ref["E_x"]))
        assert rel(host(W_sum), ref["W_G"]) <= tol["W"]
        tr = gen.random_trials(s["cell"], s["ecut"], 6, seed=5)
        K = host(ace.ace_apply(plan, xi, dev(tr, plan)))
        K_ref = oracle.ace_apply(ref["xi"], tr, ref["miller"])
        assert rel(K, K_ref) <= tol["K"]
        plan.close()


@pytest.mark.parametrize("variant,streams", [(1, 1), (1, 2), (2, 1), (2, 2), (3, 0), (4, 1), (4, 2)])
def test_pair_variants_match_oracle(variant, streams):
    """Every pair-pass variant (tile passes, transposed-plane passes, the
    persistent pipeline), on one and two streams, all pairs and a screened
    list, on the 32^3 cube: E_x, W_G and K psi against the oracle."""
    tol = TOL["mixed"]
    s = gen.config_small()
    n = len(s["psi"])
    keep = [(i, j) for i in range(n) for j in range(i, n) if i == j or (3 * i + j) % 4 != 1]
    rp = np.zeros(n + 1, dtype=np.int32)
    for i, _ in keep:
        rp[i + 1] += 1
    screened = (np.cumsum(rp).astype(np.int32), np.array([j for _, j in keep], dtype=np.int32))
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], n, "mixed", pair_streams=streams, pair_variant=variant)
    cfg = plan.config()
    assert cfg["pair_variant"] == variant
    psi = dev(s["psi"], plan)
    tr = gen.random_trials(s["cell"], s["ecut"], 6, seed=7)
    for pairs in (None, screened):
        ref = oracle.ace_build(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"], pairs=pairs)
        xi, E = ace.ace_build(plan, psi, s["alpha"], pairs=pairs)
        W, _ = ace.ace_last_intermediates(plan, n)
        assert abs(E - ref["E_x"]) / s["n_atom"] <= tol["E"]
        assert rel(host(W), ref["W_G"]) <= tol["W"]
        K = host(ace.ace_apply(plan, xi, dev(tr, plan)))
        assert rel(K, oracle.ace_apply(ref["xi"], tr, ref["miller"])) <= tol["K"]
    plan.close()


@pytest.mark.parametrize("row_block", ["0", "2", "3", "4", "8"])
def test_row_blocks_match_oracle(monkeypatch, row_block):
    """Every pair-tile shape (row order; column-shared transforms in blocks of
    2, 3, 4, 8 rows, with blocks that do not divide the 13 orbitals and a
    screened list whose columns leave unpaired rows) gives the oracle's E_x,
    W_G and K psi."""
    monkeypatch.setenv("ACE_ROW_BLOCK", row_block)
    tol = TOL["mixed"]
    cell = gen.cubic_cell(9.0)
    ecut, grid, alpha = 20.0, (32, 32, 32), 0.25
    n = 13
    psi0 = gen.random_orbitals(cell, ecut, n, seed=41)
    keep = [(i, j) for i in range(n) for j in range(i, n) if i == j or (5 * i + 3 * j) % 7 < 4]
    rp = np.zeros(n + 1, dtype=np.int32)
    for i, _ in keep:
        rp[i + 1] += 1
    screened = (np.cumsum(rp).astype(np.int32), np.array([j for _, j in keep], dtype=np.int32))
    plan = ace.Plan(grid, cell, ecut, n, "mixed", pair_variant=4)
    assert plan.config()["row_block"] == int(row_block)
    psi = dev(psi0, plan)
    tr = gen.random_trials(cell, ecut, 5, seed=8)
    for pairs in (None, screened):
        ref = oracle.ace_build(psi0, cell, grid, ecut, alpha, pairs=pairs)
        xi, E = ace.ace_build(plan, psi, alpha, pairs=pairs)
        W, _ = ace.ace_last_intermediates(plan, n)
        assert abs(E - ref["E_x"]) / (3 * n / 4) <= tol["E"]
        assert rel(host(W), ref["W_G"]) <= tol["W"]
        K = host(ace.ace_apply(plan, xi, dev(tr, plan)))
        assert rel(K, oracle.ace_apply(ref["xi"], tr, ref["miller"])) <= tol["K"]
    plan.close()


@pytest.mark.parametrize("n,T", [(1, 1), (33, 300), (130, 257), (300, 5)])
def test_tensor_core_apply_ragged_shapes(n, T):
    """The streamed tcgen05 Gram and product on ragged shapes: one vector and
    one trial; a partial K stage of ACE vectors (33) and three trial blocks
    (300); 130 vectors (two 128-row Gram tiles) and 257 trials; 300 vectors
    (three Gram tiles, ten product stages) on 5 trials -- against an FP64
    evaluation of -xi (xi^T psi) on the same float inputs, and the fast
    energy against -sum C^2."""
    cfg = gen.config_small()
    plan = ace.Plan(cfg["grid"], cfg["cell"], cfg["ecut"], 8, "mixed")
    npw = plan.n_pw_half
    rng = np.random.default_rng(n * 1000 + T)
    xi = (rng.standard_normal((n, npw)) + 1j * rng.standard_normal((n, npw))) / np.sqrt(npw)
    xi[:, 0] = xi[:, 0].real
    tr = gen.random_trials(cfg["cell"], cfg["ecut"], T, seed=T)
    d_xi, d_tr = dev(xi, plan), dev(tr, plan)
    xh, th = host(d_xi), host(d_tr)  # the float inputs, exactly
    C = gen.gamma_overlap(th, xh)
    ref = -(C @ xh)
    K0 = ace.ace_apply(plan, d_xi, d_tr)
    K = host(K0)
    assert rel(K, ref) <= 1e-6
    E = ace.ace_apply_energy(plan, d_xi, d_tr)
    assert abs(E + np.sum(C * C)) <= 1e-6 * np.sum(C * C)
    # with xi's split image (ace_apply_prepare) the product takes xi by bulk
    # copies: the same hi / lo operands in the same order, so the same bits
    ace.ace_apply_prepare(plan, d_xi)
    assert torch.equal(ace.ace_apply(plan, d_xi, d_tr), K0)
    plan.close()


def test_apply_prepare_lifetime():
    """The split image of xi serves only the xi it was made from: a build
    clears it, another xi pointer or count does not use it, a new prepare
    after xi changes in place gives that xi's product; each against the FP64
    evaluation of -xi (xi^T psi) on the float inputs."""
    s = gen.config_small()
    n = len(s["psi"])
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], n, "mixed")
    tr = dev(gen.random_trials(s["cell"], s["ecut"], 9, seed=5), plan)
    th = host(tr)

    def ref(x):
        xh = host(x)
        return -(gen.gamma_overlap(th, xh) @ xh)

    xi, _ = ace.ace_build(plan, dev(s["psi"], plan), s["alpha"])
    ace.ace_apply_prepare(plan, xi)
    assert rel(host(ace.ace_apply(plan, xi, tr)), ref(xi)) <= 1e-6
    other = xi.clone().mul_(0.25)  # another pointer, same count, other contents
    assert rel(host(ace.ace_apply(plan, other, tr)), ref(other)) <= 1e-6
    assert rel(host(ace.ace_apply(plan, xi[:5], tr)), ref(xi[:5])) <= 1e-6  # same pointer, fewer vectors
    xi2 = xi.clone()
    xi.mul_(0.5)  # in place: the image is stale until prepared again
    ace.ace_apply_prepare(plan, xi)
    assert rel(host(ace.ace_apply(plan, xi, tr)), ref(xi)) <= 1e-6
    ace.ace_apply_prepare(plan, xi2)
    xi3, _ = ace.ace_build(plan, dev(s["psi"], plan), s["alpha"], xi=xi2)  # the build clears the image
    xi3.mul_(2.0)
    assert rel(host(ace.ace_apply(plan, xi3, tr)), ref(xi3)) <= 1e-6
    plan.close()


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_blocked_cholesky_70_orbitals(prec):
    """70 orbitals take the multi-block Cholesky and inverse (blocks of 32,
    padded to 96): E_x, M and K psi against the oracle; and a zero orbital in
    the third block (M exactly singular) is rejected as not positive
    definite."""
    tol = TOL[prec]
    s = gen.config_small()
    n = 70
    psi0 = gen.random_orbitals(s["cell"], s["ecut"], n, seed=61)
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], n, prec)
    ref = oracle.ace_build(psi0, s["cell"], s["grid"], s["ecut"], s["alpha"])
    xi, E = ace.ace_build(plan, dev(psi0, plan), s["alpha"])
    _, M = ace.ace_last_intermediates(plan, n)
    assert abs(E - ref["E_x"]) / (3 * n / 4) <= tol["E"]
    assert np.abs(M - ref["M"]).max() <= tol["W"] * np.abs(ref["M"]).max()
    tr = gen.random_trials(s["cell"], s["ecut"], 6, seed=62)
    K = host(ace.ace_apply(plan, xi, dev(tr, plan)))
    assert rel(K, oracle.ace_apply(ref["xi"], tr, ref["miller"])) <= tol["K"]
    dep = psi0.copy()
    dep[67] = 0.0
    with pytest.raises(ace.AceError) as e:
        ace.ace_build(plan, dev(dep, plan), s["alpha"])
    assert e.value.code == -3
    plan.close()


def test_tune_cache_round_trip(monkeypatch, tmp_path):
    """Plan creation with ACE_TUNE_CACHE: the first plan times the variants and
    row blocks and appends its choice; a second plan of the same grid, size
    and precision takes the same choice from the file without timing."""
    monkeypatch.delenv("ACE_ROW_BLOCK", raising=False)
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("ACE_TUNE_CACHE", str(path))
    s = gen.config_small()
    p1 = ace.Plan(s["grid"], s["cell"], s["ecut"], 8, "mixed")
    c1 = p1.config()
    assert not c1["from_tune_cache"] and c1["row_block_ms"] and c1["tune_ms"]
    lines = path.read_text().splitlines()
    assert len(lines) == 1 and lines[0].startswith("32x32x32 n8 f32 ")
    # variant, streams, row block, radix plan (0: make_axis_plan's, the only one at 32^3)
    assert lines[0].endswith(f"= {c1['pair_variant']} {c1['pair_streams']} {c1['row_block']} 0")
    p2 = ace.Plan(s["grid"], s["cell"], s["ecut"], 8, "mixed")
    c2 = p2.config()
    assert c2["from_tune_cache"] and not c2["tune_ms"] and not c2["row_block_ms"]
    assert (c2["pair_variant"], c2["pair_streams"], c2["row_block"]) == \
        (c1["pair_variant"], c1["pair_streams"], c1["row_block"])
    xi1, E1 = ace.ace_build(p1, dev(s["psi"], p1), s["alpha"])
    xi2, E2 = ace.ace_build(p2, dev(s["psi"], p2), s["alpha"])
    assert E1 == E2
    p1.close()
    p2.close()


def test_automatic_variant_choice_and_rejections():
    s = gen.config_small()
    n = len(s["psi"])
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], n, "mixed")  # 32^3: all variants apply, timed
    cfg = plan.config()
    # any timed candidate may win (the half-plane pairs are not one at 32^3)
    assert cfg["pair_variant"] in (1, 2, 3, 4) and cfg["pair_streams"] in (1, 2)
    assert set(cfg["tune_ms"]) == {"tile_1_stream", "tile_2_streams", "planes", "pipeline", "hybrid"}
    plan.close()
    p64 = ace.Plan(s["grid"], s["cell"], s["ecut"], n, "fp64")
    assert p64.config()["pair_variant"] == 1 and p64.config()["tune_ms"] == {}
    p64.close()
    small = small_system()
    for v in (2, 3, 4, 5):  # 16^3 has no compile-time kernels, double has none either
        with pytest.raises(ace.AceError):
            ace.Plan(small["grid"], small["cell"], small["ecut"], 5, "mixed", pair_variant=v)
        with pytest.raises(ace.AceError):
            ace.Plan(s["grid"], s["cell"], s["ecut"], n, "fp64", pair_variant=v)
    with pytest.raises(ace.AceError):  # the half-plane pairs exist for 120^3 only
        ace.Plan(s["grid"], s["cell"], s["ecut"], n, "mixed", pair_variant=5)
    with pytest.raises(ace.AceError):
        ace.Plan(s["grid"], s["cell"], s["ecut"], n, "mixed", pair_variant=6)


def _csr_set(pairs):
    rp, col = pairs
    return {(i, int(j)) for i in range(len(rp) - 1) for j in col[rp[i]:rp[i + 1]]}


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_overlap_screen_matches_oracle(prec):
    """s-MTACE screening (Section 2.4) on localised orbitals (32^3 cube): S
    element by element, the kept pairs at the paper's three rho_cut values
    (identical except pairs within the S tolerance of rho_cut, which may fall
    either way), and the screened build against the oracle's on the same list."""
    tol_S = 1e-12 if prec == "fp64" else 2e-5
    cell = gen.cubic_cell(14.0)
    ecut, grid, n = 30.0, (32, 32, 32), 16
    psi, _ = gen.localized_orbitals(14.0, ecut, n, seed=21)
    S_ref = oracle.overlap(psi, cell, grid, ecut)
    plan = ace.Plan(grid, cell, ecut, n, prec)
    d = dev(psi, plan)
    for rho_cut in (2.5e-2, 1.0e-2, 2.0e-3):
        pairs, S = ace.ace_overlap_screen(plan, d, rho_cut)
        assert np.abs(S - S_ref).max() <= tol_S
        got, ref = _csr_set(pairs), _csr_set(oracle.screened_pairs(S_ref, rho_cut))
        for i, j in got ^ ref:
            assert abs(S_ref[i, j] - rho_cut) <= tol_S
        assert all((i, i) in got for i in range(n))
    # the screened build on the GPU's list (rho_cut 1e-2) against the oracle's build on it
    pairs, _ = ace.ace_overlap_screen(plan, d, 1.0e-2)
    ref = oracle.ace_build(psi, cell, grid, ecut, 0.25, pairs=pairs)
    xi, E = ace.ace_build(plan, d, 0.25, pairs=pairs)
    tol = TOL[prec]
    assert abs(E - ref["E_x"]) / (3 * n / 4) <= tol["E"] * (1 if prec == "mixed" else abs(ref["E_x"]))
    tr = gen.random_trials(cell, ecut, 4, seed=3)
    K = host(ace.ace_apply(plan, xi, dev(tr, plan)))
    assert rel(K, oracle.ace_apply(ref["xi"], tr, ref["miller"])) <= tol["K"]
    plan.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_mts_harness_matches_oracle(prec):
    """The MTS loop (Section 2.3): ACE built once on Phi_0, inner steps on
    drifting orbitals; the fast energy sum <phi_k|K_0 phi_k>, the exact E_x on
    Phi_k and their difference against the oracle, and dE(0) = 0."""
    from paper_2110_07670_gb300 import mts
    s = gen.config_small()
    n = len(s["psi"])
    D = gen.random_orbitals(s["cell"], s["ecut"], n, seed=33)
    at = lambda k: mts.drifted_orbitals(s["psi"], D, 0.02, k)
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], n, prec)
    rec = mts.run(plan, s["psi"], s["alpha"], at, n_inner=3, every=1)
    plan.close()
    ref0 = oracle.ace_build(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    tol = 1e-10 if prec == "fp64" else 1e-6
    assert abs(rec[0]["dE"]) == 0.0
    for r in rec[1:]:
        phik = at(r["k"])
        E_ace = _tr_gamma(phik, oracle.ace_apply(ref0["xi"], phik, ref0["miller"]))
        E_ex = oracle.exchange(phik, s["cell"], s["grid"], s["ecut"], s["alpha"])[1]
        scale = 1.0 if prec == "mixed" else abs(E_ex)
        assert abs(r["E_ACE"] - E_ace) / s["n_atom"] <= tol * scale
        assert abs(r["E_exact"] - E_ex) / s["n_atom"] <= tol * scale
        assert abs(r["dE"] - (E_ex - E_ace)) / s["n_atom"] <= 2 * tol * scale
    # the ACE energy of Phi_0 itself is the exact one (exactness on span(Phi_0))
    assert abs(_tr_gamma(s["psi"], oracle.ace_apply(ref0["xi"], s["psi"], ref0["miller"])) - ref0["E_x"]) \
        <= 1e-10 * abs(ref0["E_x"])


@pytest.mark.parametrize("variant", [1, 3])
def test_cuda_graph_capture_of_build_and_apply(variant):
    """ace_build_async + ace_apply captured in one CUDA graph (after one run
    outside capture): replays match the oracle, and a replay after new
    orbitals are copied into the captured input buffer builds from them."""
    s = gen.config_small()
    n = len(s["psi"])
    psi2 = gen.random_orbitals(s["cell"], s["ecut"], n, seed=44)
    tr_h = gen.random_trials(s["cell"], s["ecut"], 5, seed=45)
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], n, "mixed", pair_variant=variant)
    psi = dev(s["psi"], plan)
    tr = dev(tr_h, plan)
    xi = torch.empty_like(psi)
    K = torch.empty_like(tr)
    ace.ace_build_async(plan, psi, s["alpha"], xi=xi)  # outside capture: allocations, attributes
    ace.ace_apply(plan, xi, tr, out=K)
    ace.ace_build_result(plan)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        ace.ace_build_async(plan, psi, s["alpha"], xi=xi)
        ace.ace_apply(plan, xi, tr, out=K)
    for orb in (s["psi"], psi2):
        psi.copy_(dev(orb, plan))
        g.replay()
        E = ace.ace_build_result(plan)
        ref = oracle.ace_build(orb, s["cell"], s["grid"], s["ecut"], s["alpha"])
        assert abs(E - ref["E_x"]) / s["n_atom"] <= TOL["mixed"]["E"]
        assert rel(host(K), oracle.ace_apply(ref["xi"], tr_h, ref["miller"])) <= TOL["mixed"]["K"]
    del g
    plan.close()


def test_bounded_wait_timeout_path_and_recovery():
    """A device wait that nothing completes gives up after its limit and the
    call returns ACE_ERR_TIMEOUT (no fault, nothing in flight); the plan and
    the context stay usable: a build right after matches the oracle."""
    s = small_system()
    n = len(s["psi"])
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], n, "mixed")
    assert ace.ace_check_timeout_path(plan, 50) == -6
    assert "timed out" in ace.last_error()
    ref = oracle.ace_build(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    _, E = ace.ace_build(plan, dev(s["psi"], plan), s["alpha"])
    assert abs(E - ref["E_x"]) / s["n_atom"] <= TOL["mixed"]["E"]
    assert ace.ace_check_timeout_path(plan, 0) == -1  # limit out of range
    plan.close()


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_hfx_exact_every_variant(variant):
    """The exact exchange on trial vectors (one-sided accumulation: trials x
    occupied pairs) through every pair-pass variant on the 32^3 cube, against
    the oracle's V_X psi; an odd number of trials leaves a half-empty
    transform."""
    s = gen.config_small()
    trials = gen.random_trials(s["cell"], s["ecut"], 7, seed=12)
    ref = oracle.vx_apply(s["psi"], trials, s["cell"], s["grid"], s["ecut"], s["alpha"])
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], len(s["psi"]), "mixed", pair_variant=variant)
    out = host(ace.hfx_apply_exact(plan, dev(s["psi"], plan), s["alpha"], dev(trials, plan)))
    assert rel(out, ref) <= TOL["mixed"]["W"]
    plan.close()


@pytest.mark.parametrize("grid", [60, 90, 108])
def test_hybrid_variant_on_cubes_without_transposed_planes(grid):
    """Pair variant 4 (plane-kernel forward pass into the tile layout, no
    slot swizzle when n % 16 != 0) on cubes the transposed passes do not
    cover: E_x, W_G and K psi against the oracle."""
    cell = gen.cubic_cell(12.0)
    ecut = 30.0
    psi = gen.random_orbitals(cell, ecut, 5, seed=grid)
    s = dict(cell=cell, grid=(grid,) * 3, ecut=ecut, alpha=0.25, psi=psi, n_atom=3 * 5 / 4)
    ref = oracle.ace_build(psi, cell, s["grid"], ecut, 0.25)
    plan = ace.Plan(s["grid"], cell, ecut, 5, "mixed", pair_variant=4)
    assert plan.config()["pair_variant"] == 4
    xi, E = ace.ace_build(plan, dev(psi, plan), 0.25)
    W, _ = ace.ace_last_intermediates(plan, 5)
    assert abs(E - ref["E_x"]) / s["n_atom"] <= TOL["mixed"]["E"]
    assert rel(host(W), ref["W_G"]) <= TOL["mixed"]["W"]
    tr = gen.random_trials(cell, ecut, 3, seed=1)
    assert rel(host(ace.ace_apply(plan, xi, dev(tr, plan))), oracle.ace_apply(ref["xi"], tr, ref["miller"])) \
        <= TOL["mixed"]["K"]
    plan.close()


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_pair_variants_odd_pair_count(variant):
    """Six orbitals on the 32^3 cube: 21 pairs, so the last packed transform
    carries one pair; every variant against the oracle."""
    s = gen.config_small()
    psi = s["psi"][:6]
    ref = oracle.ace_build(psi, s["cell"], s["grid"], s["ecut"], s["alpha"])
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], 6, "mixed", pair_variant=variant)
    xi, E = ace.ace_build(plan, dev(psi, plan), s["alpha"])
    W, _ = ace.ace_last_intermediates(plan, 6)
    assert abs(E - ref["E_x"]) / (3 * 6 / 4) <= TOL["mixed"]["E"]
    assert rel(host(W), ref["W_G"]) <= TOL["mixed"]["W"]
    plan.close()


# ---------------------------------------- the Coulomb interaction cut off at R_c

def _check_truncated(s, prec, rc, **plan_kw):
    return _check_coulomb(s, prec, oracle.coulomb_cutoff(rc), coulomb_rc=rc, **plan_kw)


def _check_coulomb(s, prec, ctx, **plan_kw):
    n = len(s["psi"])
    with ctx:
        ref = oracle.ace_build(s["psi"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], n, prec, **plan_kw)
    xi, E = ace.ace_build(plan, dev(s["psi"], plan), s["alpha"])
    W, M = ace.ace_last_intermediates(plan, n)
    tol = TOL[prec]
    n_atom = 3 * n / 4
    assert abs(E - ref["E_x"]) / n_atom <= tol["E"] * (1 if prec == "mixed" else abs(ref["E_x"]))
    assert rel(host(W), ref["W_G"]) <= tol["W"]
    tr = gen.random_trials(s["cell"], s["ecut"], 4, seed=98)
    K = host(ace.ace_apply(plan, xi, dev(tr, plan)))
    assert rel(K, oracle.ace_apply(ref["xi"], tr, ref["miller"])) <= tol["K"]
    plan.close()
    return E


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_truncated_coulomb_generic_passes(prec):
    """16^3 box (runtime-size passes): the Coulomb stage reads the cut-off
    kernel from the plan's table, in the plan's precision."""
    s = small_system()
    E = _check_truncated(s, prec, ace.sphere_radius(s["cell"]))
    # a different cutoff gives a different answer (the table is used)
    E2 = _check_truncated(s, prec, 2.0)
    assert abs(E - E2) > 1e-4


@pytest.mark.parametrize("variant", [1, 2, 3, 4])
def test_truncated_coulomb_every_variant(variant):
    """32^3 cube, mixed precision: the per-pencil pass's tables (natural and
    transposed planes) carry the cut-off kernel in every pair-pass variant."""
    s = gen.config_small()
    _check_truncated(s, "mixed", ace.sphere_radius(s["cell"]), pair_variant=variant)


@pytest.mark.parametrize("prec,kernels", [("fp64", 0), ("mixed", 2)])
def test_truncated_coulomb_cube_without_pencil_pass(prec, kernels):
    s = gen.config_small()
    _check_truncated(s, prec, ace.sphere_radius(s["cell"]), kernels=kernels)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_truncated_coulomb_hfx_exact(prec):
    s = small_system()
    rc = ace.sphere_radius(s["cell"])
    with oracle.coulomb_cutoff(rc):
        ref = oracle.vx_apply(s["psi"], s["trials"], s["cell"], s["grid"], s["ecut"], s["alpha"])
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], len(s["psi"]), prec, coulomb_rc=rc)
    out = host(ace.hfx_apply_exact(plan, dev(s["psi"], plan), s["alpha"], dev(s["trials"], plan)))
    assert rel(out, ref) <= TOL[prec]["W"]


def test_truncated_coulomb_checkpoint_and_rejections(tmp_path):
    s = gen.config_small()
    rc = ace.sphere_radius(s["cell"])
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], 8, "mixed", coulomb_rc=rc)
    xi, E = ace.ace_build(plan, dev(s["psi"], plan), s["alpha"])
    path = str(tmp_path / "xi_rc.ace")
    ace.ace_save(plan, path, xi, s["alpha"], E)
    same = ace.Plan(s["grid"], s["cell"], s["ecut"], 8, "mixed", coulomb_rc=rc)
    xi2, _, E2 = ace.ace_load(same, path)
    assert torch.equal(xi, xi2) and E2 == E
    bare = ace.Plan(s["grid"], s["cell"], s["ecut"], 8, "mixed")
    with pytest.raises(ace.AceError):
        ace.ace_load(bare, path)
    for bad in (-1.0, float("nan"), float("inf")):
        with pytest.raises(ace.AceError):
            ace.Plan(s["grid"], s["cell"], s["ecut"], 8, "mixed", coulomb_rc=bad)


# ------------------------- the auxiliary-function G = 0 term (Gygi-Baldereschi)

@pytest.mark.parametrize("prec,kw", [("mixed", dict(pair_variant=1)), ("mixed", dict(pair_variant=2)),
                                     ("mixed", dict(pair_variant=3)), ("mixed", dict(pair_variant=4)),
                                     ("mixed", dict(kernels=2)), ("fp64", {})])
def test_auxiliary_g0_every_path(prec, kw):
    """K(0) = 4 pi chi computed by the library against the oracle's own
    computation of it, through every Coulomb-table path (32^3 cube)."""
    s = gen.config_small()
    E = _check_coulomb(s, prec, oracle.coulomb_g0(oracle.auxiliary_function_k0(s["cell"])), coulomb_g0=True, **kw)
    # the G = 0 term shifts E_x by -alpha n K(0) / Omega from the dropped-term value
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], 8, prec)
    _, E0 = ace.ace_build(plan, dev(s["psi"], plan), s["alpha"])
    k0 = oracle.auxiliary_function_k0(s["cell"])
    assert abs((E - E0) - (-s["alpha"] * 8 * k0 / 1000.0)) <= (1e-6 * s["n_atom"] if prec == "mixed" else 1e-9)


def test_auxiliary_g0_generic_box_and_rejections(tmp_path):
    s = small_system()
    _check_coulomb(s, "mixed", oracle.coulomb_g0(oracle.auxiliary_function_k0(s["cell"])), coulomb_g0=True)
    with pytest.raises(ace.AceError):
        ace.Plan(s["grid"], s["cell"], s["ecut"], 5, "mixed", coulomb_g0=True, coulomb_rc=3.0)
    c = gen.config_small()
    plan = ace.Plan(c["grid"], c["cell"], c["ecut"], 8, "mixed", coulomb_g0=True)
    xi, E = ace.ace_build(plan, dev(c["psi"], plan), c["alpha"])
    path = str(tmp_path / "xi_g0.ace")
    ace.ace_save(plan, path, xi, c["alpha"], E)
    xi2, _, _ = ace.ace_load(ace.Plan(c["grid"], c["cell"], c["ecut"], 8, "mixed", coulomb_g0=True), path)
    assert torch.equal(xi, xi2)
    with pytest.raises(ace.AceError):
        ace.ace_load(ace.Plan(c["grid"], c["cell"], c["ecut"], 8, "mixed"), path)


def test_last_intermediates_survive_the_overlap_screen():
    """The overlap screen keeps its S apart from the last build's M and W."""
    s = gen.config_small()
    plan = ace.Plan(s["grid"], s["cell"], s["ecut"], 8, "mixed")
    psi = dev(s["psi"], plan)
    ace.ace_build(plan, psi, s["alpha"])
    W0, M0 = ace.ace_last_intermediates(plan, 8)
    W0 = W0.clone()
    ace.ace_overlap_screen(plan, psi, 0.1)
    W1, M1 = ace.ace_last_intermediates(plan, 8)
    assert np.array_equal(M0, M1) and torch.equal(W0, W1)
    plan.close()
