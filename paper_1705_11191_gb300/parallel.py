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

__all__ = ["partition", "allgather_varlen", "dm_batched_distributed"]


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
                           group=None, device=None):
    """This rank's problems (hams, ovlps, n_states, weights: lists over its problems) with
    one chemical potential over the problems of all ranks:
        sum over all ranks' problems i of weights[i] * sum_l f_il = n_electron.
    A rank without problems takes part in the exchange only (its tensors live on
    ``device``). Returns (P list, W list, band energies, mu) for this rank's problems."""
    import torch
    import torch.distributed as dist
    if len(hams):
        eps = solver.batch_ev(hams, ovlps, n_states)
        wt = torch.cat([torch.full((int(k),), float(w), dtype=eps.dtype, device=eps.device)
                        for k, w in zip(n_states, weights)])
    else:
        eps = torch.empty(0, dtype=torch.float64, device=device or "cpu")
        wt = eps.clone()
    eps_all, lens = allgather_varlen(eps, group)
    wt_all, _ = allgather_varlen(wt, group)
    f_all, mu = solver.occupation_weighted(eps_all, wt_all, n_electron)
    r = dist.get_rank(group)
    off = sum(lens[:r])
    mine = f_all[off: off + lens[r]].contiguous()
    if not len(hams):
        return [], [], [], mu
    P, W, en = solver.batch_dm(mine)
    return P, W, en, mu
