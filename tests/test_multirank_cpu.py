"""Several-process k-point path on CPU ranks (gloo, world size 2): the partition of the
problems, the all-gather of eigenvalues and weights, one chemical potential on every
rank, and each rank's density matrices, checked against the single-process oracle
(arXiv:1705.11191 sec. 2 SINGLE_PROC mode; sec. 4.4 electron count summed over
k-points). The three phase calls are served by the oracle here, so that the exchange
logic of paper_1705_11191_gb300.parallel runs without a GPU."""
import os
import socket
import tempfile

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1705_11191_gb300 import parallel  # noqa: E402

SIZES = [40, 64, 28, 52, 36]
WEIGHTS = [0.1, 0.3, 0.2, 0.25, 0.15]


def _problem(i):
    import ksinputs
    return ksinputs.cluster_problem(SIZES[i], seed=300 + i)


class OracleSolver:
    """The phase interface of Handle, computed by the CPU oracle on CPU tensors."""

    def __init__(self, scheme, kt):
        self.scheme, self.kt = scheme, kt

    def batch_ev(self, hams, ovlps, n_states):
        import oracle
        self.kept = []
        evs = []
        for h, s, k in zip(hams, ovlps, n_states):
            r = oracle.solve(h.numpy(), s.numpy(), k, 0.0, want_pw=False)
            self.kept.append((r["eval"][:k], r["C"]))
            evs.append(r["eval"][:k])
        return torch.from_numpy(np.concatenate(evs))

    def occupation_weighted(self, eps, wt, n_el):
        import oracle
        f, mu = oracle.occupation_weighted(eps.numpy(), wt.numpy(), n_el, scheme=self.scheme,
                                           kt=self.kt)
        return torch.from_numpy(f), mu

    def batch_dm(self, occ):
        import oracle
        occ = occ.numpy()
        P, W, en = [], [], []
        off = 0
        for ev, c in self.kept:
            f = occ[off: off + ev.size]
            off += ev.size
            P.append(torch.from_numpy(oracle.weighted_outer(c, f)))
            W.append(torch.from_numpy(oracle.weighted_outer(c, f * ev)))
            en.append(float(np.sum(f * ev)))
        return P, W, en


def _rank_main(rank, world, port, outdir, scheme, kt, n_el, packed=True):
    import torch.distributed as dist
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    try:
        mine = parallel.partition(SIZES, world)[rank]
        probs = [_problem(i) for i in mine]
        ks = [p.n // 2 for p in probs]
        # one all-gather: the padded length comes from the global problem list
        mx = parallel.max_states_per_rank(SIZES, [n // 2 for n in SIZES], world) if packed else None
        P, W, en, mu = parallel.dm_batched_distributed(
            OracleSolver(scheme, kt), [torch.from_numpy(np.ascontiguousarray(p.h)) for p in probs],
            [torch.from_numpy(np.ascontiguousarray(p.s)) for p in probs], ks,
            [WEIGHTS[i] for i in mine], n_el, max_states=mx)
        for j, i in enumerate(mine):
            np.save(os.path.join(outdir, f"P{i}.npy"), P[j].numpy())
            np.save(os.path.join(outdir, f"W{i}.npy"), W[j].numpy())
            np.save(os.path.join(outdir, f"e{i}.npy"), np.array(en[j]))
        np.save(os.path.join(outdir, f"mu_rank{rank}.npy"), np.array(mu))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_partition_covers_and_balances():
    sizes = [256, 4096, 1024, 512, 2048, 300, 3000, 700]
    for ws in (1, 2, 3, 4):
        parts = parallel.partition(sizes, ws)
        assert sorted(i for p in parts for i in p) == list(range(len(sizes)))
        assert parts == parallel.partition(sizes, ws)
        loads = [sum(sizes[i] ** 3 for i in p) for p in parts]
        # longest-processing-time bound: max load <= average + largest single job
        assert max(loads) <= sum(loads) / ws + max(s ** 3 for s in sizes)
    assert parallel.partition([10], 3) == [[0], [], []]


@pytest.mark.parametrize("scheme,kt,n_el,packed", [(2, 0.01, 9.0, True), (0, 0.0, 10.0, True),
                                                   (2, 0.01, 9.0, False)])
def test_two_rank_shared_mu_matches_single_process(scheme, kt, n_el, packed):
    import torch.multiprocessing as tmp
    import oracle
    with tempfile.TemporaryDirectory() as outdir:
        port = _free_port()
        tmp.spawn(_rank_main, args=(2, port, outdir, scheme, kt, n_el, packed), nprocs=2, join=True)
        probs = [_problem(i) for i in range(len(SIZES))]
        ref, ref_mu = oracle.solve_batched([(p.h, p.s, p.n // 2) for p in probs], n_el,
                                           weights=WEIGHTS, scheme=scheme, kt=kt)
        mus = [float(np.load(os.path.join(outdir, f"mu_rank{r}.npy"))) for r in range(2)]
        assert mus[0] == mus[1]
        assert abs(mus[0] - ref_mu) <= 1e-12
        for i, r in enumerate(ref):
            P = np.load(os.path.join(outdir, f"P{i}.npy"))
            W = np.load(os.path.join(outdir, f"W{i}.npy"))
            e = float(np.load(os.path.join(outdir, f"e{i}.npy")))
            np.testing.assert_allclose(P, r["P"], rtol=0, atol=1e-12)
            np.testing.assert_allclose(W, r["W"], rtol=0, atol=1e-12)
            assert abs(e - r["energy"]) <= 1e-12 * max(1.0, abs(r["energy"]))
