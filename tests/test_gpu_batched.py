"""GPU parity of the several-problem entry points (elsi_dm_batched_real/_complex and the
phase calls elsi_batch_ev_*, elsi_occupation_weighted, elsi_batch_dm) against the FP64
CPU oracle's batched solve: k-points / spin channels of uneven size with one shared
chemical potential (arXiv:1705.11191 sec. 4.4, electron count summed over k-points and
spin channels) or one per problem. Tolerances as for one problem: eigenvalues 1e-10,
P and W 1e-9 relative Frobenius, band energies 1e-9 relative, mu 1e-10."""
import numpy as np
import pytest

import ksinputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1705_11191_gb300 as egb  # noqa: E402


def dev(a):
    if np.iscomplexobj(a):
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _handle(prec=0, b=16, scheme=None, kt=None):
    hd = egb.Handle(8, 1, 0.0)
    hd.use_current_stream()
    hd.set_band_width(b)
    hd.set_precision(prec)
    if scheme is not None:
        hd.set_broadening(scheme, kt)
    return hd


def _real_problems(sizes, seed0):
    return [ksinputs.cluster_problem(n, seed=seed0 + i) for i, n in enumerate(sizes)]


def _check(out, ref, mus, ref_mu, tol_mu=1e-10):
    P, W, en = out[0], out[1], out[2]
    for i, r in enumerate(ref):
        assert rel(P[i].cpu().numpy(), r["P"]) <= 1e-9, i
        assert rel(W[i].cpu().numpy(), r["W"]) <= 1e-9, i
        assert abs(en[i] - r["energy"]) <= 1e-9 * max(1.0, abs(r["energy"])), i
    if np.ndim(ref_mu) == 0:
        assert abs(mus - ref_mu) <= tol_mu
    else:
        np.testing.assert_allclose(mus, ref_mu, rtol=0, atol=tol_mu)


@pytest.mark.parametrize("scheme,kt", [(egb.OCC_FERMI, 0.01), (egb.OCC_GAUSSIAN, 0.02)])
def test_real_shared_mu_parity(scheme, kt):
    probs = _real_problems([70, 101, 150], 40)
    ks = [p.n // 2 for p in probs]
    wts = [0.5, 0.3, 0.2]
    n_el = sum(w * p.n / 4 for w, p in zip(wts, probs))
    ref, ref_mu = oracle.solve_batched([(p.h, p.s, k) for p, k in zip(probs, ks)], n_el,
                                       weights=wts, scheme=scheme, kt=kt)
    with _handle(scheme=scheme, kt=kt) as hd:
        out = hd.dm_batched([dev(p.h) for p in probs], [dev(p.s) for p in probs], ks, n_el,
                            weights=wts)
    _check(out, ref, out[3], ref_mu)


def test_real_shared_mu_integer_aufbau():
    probs = _real_problems([64, 90], 60)
    ks = [p.n // 2 for p in probs]
    wts = [0.25, 0.75]
    n_el = 31.0
    ref, ref_mu = oracle.solve_batched([(p.h, p.s, k) for p, k in zip(probs, ks)], n_el,
                                       weights=wts)
    with _handle() as hd:
        out = hd.dm_batched([dev(p.h) for p in probs], [dev(p.s) for p in probs], ks, n_el,
                            weights=wts)
    _check(out, ref, out[3], ref_mu)
    tot = sum(w * np.trace(P.cpu().numpy() @ p.s) for w, P, p in zip(wts, out[0], probs))
    assert abs(tot - n_el) < 1e-9


def test_real_per_problem_mu_equals_single_solves():
    probs = _real_problems([33, 80, 128, 47], 70)
    ks = [p.n_state for p in probs]
    nel = [p.n_electron for p in probs]
    ref = [oracle.solve(p.h, p.s, p.n_state, p.n_electron) for p in probs]
    with _handle() as hd:
        out = hd.dm_batched([dev(p.h) for p in probs], [dev(p.s) for p in probs], ks, nel,
                            shared_mu=False)
    _check(out, ref, out[3], [r["mu"] for r in ref])


def test_complex_kpoints_shared_mu_parity():
    n = 48
    ks_ = [(0.0, 0.0, 0.0), (0.25, 0.0, 0.0), (0.25, 0.25, 0.0), (0.5, 0.25, 0.25)]
    probs = [ksinputs.kpoint_problem(n, k, seed=9) for k in ks_]
    wts = [0.125, 0.375, 0.25, 0.25]
    k = 20
    n_el = 22.0
    ref, ref_mu = oracle.solve_batched([(p.h, p.s, k) for p in probs], n_el, weights=wts,
                                       is_complex=True, scheme=oracle.SCHEME_FERMI, kt=0.01)
    with _handle(scheme=egb.OCC_FERMI, kt=0.01) as hd:
        out = hd.dm_batched([dev(p.h) for p in probs], [dev(p.s) for p in probs], [k] * 4,
                            n_el, weights=wts)
    _check(out, ref, out[3], ref_mu)
    for P in out[0]:
        P = P.cpu().numpy()
        np.testing.assert_allclose(P, P.conj().T, rtol=0, atol=1e-12)


def test_complex_uneven_sizes_per_problem_mu():
    probs = [ksinputs.kpoint_problem(n, kf, seed=s) for n, kf, s in
             [(30, (0.5, 0.0, 0.0), 1), (57, (0.25, 0.5, 0.0), 2)]]
    ks = [p.n_state for p in probs]
    nel = [p.n_electron for p in probs]
    ref = [oracle.solve_complex(p.h, p.s, p.n_state, p.n_electron) for p in probs]
    with _handle() as hd:
        out = hd.dm_batched([dev(p.h) for p in probs], [dev(p.s) for p in probs], ks, nel,
                            shared_mu=False)
    _check(out, ref, out[3], [r["mu"] for r in ref])


def test_refined_precision_batch():
    probs = _real_problems([160, 220], 80)
    ks = [p.n // 4 for p in probs]
    wts = [0.5, 0.5]
    n_el = 0.5 * (probs[0].n // 4) + 0.5 * (probs[1].n // 4)
    ref, ref_mu = oracle.solve_batched([(p.h, p.s, k) for p, k in zip(probs, ks)], n_el,
                                       weights=wts, scheme=oracle.SCHEME_FERMI, kt=0.01)
    with _handle(prec=egb.PREC_FP32_REFINE, b=32, scheme=egb.OCC_FERMI, kt=0.01) as hd:
        out = hd.dm_batched([dev(p.h) for p in probs], [dev(p.s) for p in probs], ks, n_el,
                            weights=wts)
    _check(out, ref, out[3], ref_mu)


def test_phase_calls_match_all_in_one_and_split_groups():
    """Eigenvalues gathered from two groups of problems (two handles, as two processes
    would hold them), one occupation over the gathered list, densities per group: the
    result equals the single all-in-one call."""
    probs = _real_problems([50, 77, 96, 64], 90)
    ks = [p.n // 2 for p in probs]
    wts = [0.1, 0.2, 0.3, 0.4]
    n_el = sum(w * p.n / 4 for w, p in zip(wts, probs))
    hs, ss = [dev(p.h) for p in probs], [dev(p.s) for p in probs]
    with _handle(scheme=egb.OCC_FERMI, kt=0.01) as hd:
        P_all, W_all, e_all, mu_all = hd.dm_batched(hs, ss, ks, n_el, weights=wts)
    groups = [[0, 2], [1, 3]]
    hds = [_handle(scheme=egb.OCC_FERMI, kt=0.01) for _ in groups]
    try:
        evs = [h.batch_ev([hs[i] for i in g], [ss[i] for i in g], [ks[i] for i in g])
               for h, g in zip(hds, groups)]
        eps = torch.cat(evs)
        wt = torch.cat([torch.full((ks[i],), wts[i], dtype=torch.float64, device="cuda")
                        for g in groups for i in g])
        res = []
        off = 0
        for h, g, ev in zip(hds, groups, evs):
            f, mu = h.occupation_weighted(eps, wt, n_el)
            assert abs(mu - mu_all) <= 1e-12
            mine = f[off:off + ev.numel()].contiguous()
            off += ev.numel()
            res.append(h.batch_dm(mine))
    finally:
        for h in hds:
            h.close()
    for (P, W, en), g in zip(res, groups):
        for j, i in enumerate(g):
            assert rel(P[j].cpu().numpy(), P_all[i].cpu().numpy()) <= 1e-13
            assert rel(W[j].cpu().numpy(), W_all[i].cpu().numpy()) <= 1e-13
            assert abs(en[j] - e_all[i]) <= 1e-12 * abs(e_all[i])


def test_batch_errors():
    p = ksinputs.cluster_problem(40, seed=1)
    with _handle() as hd:
        with pytest.raises(egb.ElsiError) as ei:
            hd.batch_dm(torch.zeros(4, dtype=torch.float64, device="cuda"))
        assert ei.value.code == 8  # ELSI_ERR_STATE
        with pytest.raises(egb.ElsiError) as ei:
            hd.dm_batched([dev(p.h)], [dev(p.s)], [41], 10.0, weights=[1.0])
        assert ei.value.code == 1  # n_state > n_basis
        with pytest.raises(egb.ElsiError) as ei:
            hd.dm_batched([dev(p.h)], [dev(p.s)], [10], 20.5, weights=[1.0])
        assert ei.value.code == 1  # more electrons than 2 * weights * states
        # the handle stays usable
        P, W, en, mu = hd.dm_batched([dev(p.h)], [dev(p.s)], [20], 10.0, weights=[1.0])
        ref = oracle.solve(p.h, p.s, 20, 10.0)
        assert rel(P[0].cpu().numpy(), ref["P"]) <= 1e-9


def test_concurrent_workers_match_one_stream():
    """Problems solved by several concurrent solver instances (own streams and host
    threads) give the same result as one after another."""
    probs = _real_problems([64, 96, 80, 128, 72, 100, 90, 110], 120)
    ks = [p.n // 2 for p in probs]
    wts = [0.125] * 8
    n_el = sum(w * p.n / 4 for w, p in zip(wts, probs))
    hs, ss = [dev(p.h) for p in probs], [dev(p.s) for p in probs]
    out = {}
    for streams in (1, 4):
        with _handle(scheme=egb.OCC_FERMI, kt=0.01) as hd:
            hd.set_batch_streams(streams)
            out[streams] = hd.dm_batched(hs, ss, ks, n_el, weights=wts)
    assert abs(out[1][3] - out[4][3]) <= 1e-13
    for a, b in zip(out[1][0], out[4][0]):
        assert rel(a.cpu().numpy(), b.cpu().numpy()) <= 1e-13
    ref, ref_mu = oracle.solve_batched([(p.h, p.s, k) for p, k in zip(probs, ks)], n_el,
                                       weights=wts, scheme=oracle.SCHEME_FERMI, kt=0.01)
    _check(out[4], ref, out[4][3], ref_mu)
