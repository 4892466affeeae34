"""Several processes (one GPU each) sharing the k-points / spin channels of one
calculation (arXiv:1705.11191 sec. 2, SINGLE_PROC mode: each process solves its group of
k-points one after another).

The problems are independent except for the chemical potential, whose electron count is
summed over all k-points and spin channels (sec. 4.4). So the only exchange is one
all-gather of the eigenvalues (and their weights); every process then runs the same
occupation kernel on the same gathered list, and so obtains the same mu, and forms the
density matrices of its own problems. A single large problem is not split: several
processes given one problem each solve it as independent replicas.

``solver`` is anything with the three phase methods of ``Handle`` (batch_ev,
occupation_weighted, batch_dm); the collective is torch.distributed (NCCL for CUDA
tensors, gloo for CPU tensors).
"""
from __future__ import annotations

__all__ = ["partition", "max_states_per_rank", "allgather_varlen", "allgather_levels",
           "dm_batched_distributed"]


def partition(sizes, world_size: int):
    """Problem indices of each rank: longest-processing-time assignment by the n^3 cost
    of each problem (largest first, to the least loaded rank; ties to the lower rank),
    each rank's list in ascending index order. Deterministic, so every rank computes
    the same partition without communication."""
    if world_size < 1:
        raise ValueError("world_size must be >= 1")
    order = sorted(range(len(sizes)), key=lambda i: (-float(sizes[i]) ** 3, i))
    load = [0.0] * world_size
    parts = [[] for _ in range(world_size)]
    for i in order:
        r = min(range(world_size), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += float(sizes[i]) ** 3
    return [sorted(p) for p in parts]


def max_states_per_rank(sizes, n_states, world_size: int) -> int:
    """Largest number of states any rank holds under partition(sizes, world_size): the
    padded length of the packed exchange, computable by every rank without communication."""
    return max([sum(int(n_states[i]) for i in p) for p in partition(sizes, world_size)] + [0])


def allgather_levels(eps, wt, max_states: int, group=None):
    """One all-gather of this rank's eigenvalues and weights packed with their count,
    [count, eps (max_states), weights (max_states)] in binary64, max_states >= the count of
    every rank. Returns (all eigenvalues, all weights, per-rank counts), in rank order."""
    import torch
    import torch.distributed as dist
    m = int(eps.numel())
    if m > max_states:
        raise ValueError(f"{m} states exceed max_states = {max_states}")
    ws = dist.get_world_size(group)
    buf = torch.zeros(1 + 2 * max_states, dtype=torch.float64, device=eps.device)
    buf[0] = float(m)
    buf[1: 1 + m] = eps
    buf[1 + max_states: 1 + max_states + m] = wt
    bufs = [torch.zeros_like(buf) for _ in range(ws)]
    dist.all_gather(bufs, buf, group=group)
    lens = [int(b[0].item()) for b in bufs]
    eps_all = torch.cat([b[1: 1 + k] for b, k in zip(bufs, lens)])
    wt_all = torch.cat([b[1 + max_states: 1 + max_states + k] for b, k in zip(bufs, lens)])
    return eps_all, wt_all, lens


def allgather_varlen(t, group=None):
    """Concatenation, in rank order, of the 1-D tensors t of all ranks (lengths may
    differ). One all-gather of the lengths, one of the padded tensors."""
    import torch
    import torch.distributed as dist
    ws = dist.get_world_size(group)
    n = torch.tensor([t.numel()], dtype=torch.int64, device=t.device)
    ns = [torch.zeros_like(n) for _ in range(ws)]
    dist.all_gather(ns, n, group=group)
    lens = [int(x.item()) for x in ns]
    m = max(lens) if lens else 0
    pad = torch.zeros(m, dtype=t.dtype, device=t.device)
    pad[: t.numel()] = t
    bufs = [torch.zeros_like(pad) for _ in range(ws)]
    dist.all_gather(bufs, pad, group=group)
    return torch.cat([b[:k] for b, k in zip(bufs, lens)]), lens


def dm_batched_distributed(solver, hams, ovlps, n_states, weights, n_electron: float,
                           group=None, device=None, max_states: int | None = None):
    """This rank's problems (hams, ovlps, n_states, weights: lists over its problems) with
    one chemical potential over the problems of all ranks:
        sum over all ranks' problems i of weights[i] * sum_l f_il = n_electron.
    max_states (max_states_per_rank of the global problem list): the eigenvalues and
    weights travel in one all-gather; without it the counts are gathered first. A rank
    without problems takes part in the exchange only (its tensors live on ``device``).
    Returns (P list, W list, band energies, mu) for this rank's problems."""
    import torch
    import torch.distributed as dist
    if len(hams):
        eps = solver.batch_ev(hams, ovlps, n_states)
        wt = torch.cat([torch.full((int(k),), float(w), dtype=eps.dtype, device=eps.device)
                        for k, w in zip(n_states, weights)])
    else:
        eps = torch.empty(0, dtype=torch.float64, device=device or "cpu")
        wt = eps.clone()
    if max_states is None:
        import torch.distributed as dist
        cnt = torch.tensor([float(eps.numel())], dtype=torch.float64, device=eps.device)
        cnts = [torch.zeros_like(cnt) for _ in range(dist.get_world_size(group))]
        dist.all_gather(cnts, cnt, group=group)
        max_states = int(max(float(c.item()) for c in cnts))
    eps_all, wt_all, lens = allgather_levels(eps, wt, max_states, group)
    f_all, mu = solver.occupation_weighted(eps_all, wt_all, n_electron)
    r = dist.get_rank(group)
    off = sum(lens[:r])
    mine = f_all[off: off + lens[r]].contiguous()
    if not len(hams):
        return [], [], [], mu
    P, W, en = solver.batch_dm(mine)
    return P, W, en, mu
