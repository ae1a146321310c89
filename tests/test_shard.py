"""Pair sharding of one ACE build over ranks (the multi-GPU path) on CPU.

The host logic is checked without a GPU: the shards partition the pair list,
and two gloo ranks that each compute their shard's W_G and E_x with the oracle
and sum them with the same allreduce helper the GPU path uses reproduce the
oracle's single-process build (Eq. 2-4 are sums over pairs).
"""
import multiprocessing as mp
import os
import socket
import tempfile

import numpy as np
import pytest

import gen
import oracle
from paper_2110_07670_gb300 import shard


def _screened_csr(n):
    """A screened-looking CSR: the diagonal plus about two thirds of i < j."""
    rp = [0]
    col = []
    for i in range(n):
        for j in range(i, n):
            if i == j or (i * 7 + j * 3) % 3 != 1:
                col.append(j)
        rp.append(len(col))
    return np.array(rp, dtype=np.int32), np.array(col, dtype=np.int32)


@pytest.mark.parametrize("n_occ", [1, 2, 7, 16])
@pytest.mark.parametrize("world", [1, 2, 3, 5])
@pytest.mark.parametrize("screened", [False, True])
def test_shards_partition_the_pair_list(n_occ, world, screened):
    pairs = _screened_csr(n_occ) if screened else None
    i_all, j_all = shard.pair_list(n_occ, pairs)
    full = list(zip(i_all.tolist(), j_all.tolist()))
    assert all(i <= j for i, j in full)
    got, sizes = [], []
    for r in range(world):
        rp, col = shard.shard_pairs(n_occ, world, r, pairs)
        assert rp.shape == (n_occ + 1,) and rp[0] == 0 and np.all(np.diff(rp) >= 0)
        assert rp[-1] == len(col)
        i, j = shard.pair_list(n_occ, (rp, col))
        got.extend(zip(i.tolist(), j.tolist()))
        sizes.append(len(col))
    assert got == full  # disjoint, complete and in row order
    assert max(sizes) - min(sizes) <= 1


def test_all_pairs_list_matches_generator_csr():
    n = 9
    rp, col = gen.all_pairs_csr(n)
    a = shard.pair_list(n, None)
    b = shard.pair_list(n, (rp, col))
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_shard_rank_out_of_range():
    with pytest.raises(ValueError):
        shard.shard_pairs(4, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, pairs, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg = gen.config_small()
        sp = shard.shard_pairs(cfg["psi"].shape[0], world, rank, pairs)
        W, E = oracle.exchange(cfg["psi"], cfg["cell"], cfg["grid"], cfg["ecut"], cfg["alpha"], pairs=sp,
                               nthreads=2)
        W_t = torch.from_numpy(np.ascontiguousarray(W))
        W_t, E_sum = shard.allreduce_partials(W_t, E)
        if rank == 0:
            np.savez(out_path, W=W_t.numpy(), E=E_sum)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("screened", [False, True])
def test_two_gloo_ranks_sum_to_the_full_build(screened):
    cfg = gen.config_small()
    n = cfg["psi"].shape[0]
    pairs = _screened_csr(n) if screened else None
    ctx = mp.get_context("spawn")
    with tempfile.TemporaryDirectory() as d:
        out = os.path.join(d, "sum.npz")
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, 2, port, pairs, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=300)
        codes = [p.exitcode for p in procs]
        for p in procs:
            if p.is_alive():
                p.kill()
        assert codes == [0, 0]
        got = np.load(out)
        W_sum, E_sum = got["W"], float(got["E"])
    ref = oracle.ace_build(cfg["psi"], cfg["cell"], cfg["grid"], cfg["ecut"], cfg["alpha"], pairs=pairs)
    assert abs(E_sum - ref["E_x"]) <= 1e-12 * abs(ref["E_x"])
    assert np.max(np.abs(W_sum - ref["W_G"])) <= 1e-12 * np.max(np.abs(ref["W_G"]))
    # the dense part from the summed W_G gives the same M as the full build
    M = oracle.gamma_gram(cfg["psi"], W_sum, ref["miller"])
    assert np.max(np.abs(M - ref["M"])) <= 1e-11 * np.max(np.abs(ref["M"]))
