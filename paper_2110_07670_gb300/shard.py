"""One ACE build split over several GPUs, one process per GPU.

The pair terms of the exchange (Eq. 2-4 of arXiv:2110.07670) are independent:
W_i = sum_j v_ij phi_j and E_x = -alpha sum (2 - d_ij) e_ij are sums over the
kept pairs.  Each rank takes a contiguous, nearly equal share of the pair list
(in row order, so a rank's pairs mostly share their row orbital), runs
ace_build_pairs on it, and the ranks sum W_G and E_x with one allreduce; every
rank then finishes the small dense part (M, Cholesky, xi) itself.  This is the
only exchange step of the path.
"""
import numpy as np


def pair_list(n_occ, pairs=None):
    """(i, j) int32 arrays of the kept pairs i <= j in row order; pairs is a
    (row_ptr, col) CSR or None for every pair."""
    if pairs is None:
        i, j = np.triu_indices(n_occ)
    else:
        rp = np.asarray(pairs[0], dtype=np.int64)
        i = np.repeat(np.arange(n_occ), np.diff(rp))
        j = np.asarray(pairs[1])
    return i.astype(np.int32), j.astype(np.int32)


def shard_pairs(n_occ, world, rank, pairs=None):
    """CSR (row_ptr [n_occ + 1], col) of rank's share: pairs lo..hi-1 of the
    row-ordered list with lo = n rank / world, hi = n (rank + 1) / world, so the
    shards partition the list and their sizes differ by at most one."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    i, j = pair_list(n_occ, pairs)
    n = len(i)
    lo, hi = n * rank // world, n * (rank + 1) // world
    i, j = i[lo:hi], j[lo:hi]
    counts = np.bincount(i, minlength=n_occ) if len(i) else np.zeros(n_occ, dtype=np.int64)
    rp = np.zeros(n_occ + 1, dtype=np.int32)
    rp[1:] = np.cumsum(counts)
    return rp, np.ascontiguousarray(j, dtype=np.int32)


def allreduce_partials(W_G, E_part, group=None):
    """Sum a shard's W_G (complex tensor on any device the process group
    serves) and its E_x share over the group; returns (W_G, E_x)."""
    import torch
    import torch.distributed as dist
    dist.all_reduce(torch.view_as_real(W_G), group=group)
    e = torch.tensor([float(E_part)], dtype=torch.float64, device=W_G.device)
    dist.all_reduce(e, group=group)
    return W_G, float(e.item())


def build_sharded(plan, psi_G, alpha, pairs=None, group=None, xi=None, W_G=None):
    """ace_build over the ranks of `group`: this rank's pair shard, one
    allreduce of W_G and E_x, then M / Cholesky / xi on every rank.
    Returns (xi, E_x), the same on every rank."""
    import torch.distributed as dist

    from . import ace_build_finish, ace_build_pairs
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    shard = shard_pairs(psi_G.shape[0], world, rank, pairs)
    W_G, E = ace_build_pairs(plan, psi_G, alpha, pairs=shard, W_G=W_G)
    W_G, E = allreduce_partials(W_G, E, group)
    xi = ace_build_finish(plan, psi_G, W_G, xi=xi)
    return xi, E
