"""GPU parity of the Methfessel-Paxton broadening schemes (sec. 4.5 broadening_scheme 3
and 4) against the oracle: density matrices, chemical potential, band energy and the
free energy with the order-1 entropy term and its gradient, for one problem and for
k-point batches with one shared chemical potential. Tolerances: P, W 1e-9 relative;
mu 1e-10; energies 1e-9 relative."""
import numpy as np
import pytest

import ksinputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1705_11191_gb300 as egb  # noqa: E402
from paper_1705_11191_gb300 import autograd as ega  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("scheme,kt,prec", [(egb.OCC_MP0, 0.02, 0), (egb.OCC_MP1, 0.02, 0),
                                            (egb.OCC_MP1, 0.03, 1)])
def test_mp_dm_parity(scheme, kt, prec):
    p = ksinputs.cluster_problem(120, seed=71)
    k, n_el = 60, 55.0
    ref = oracle.solve(p.h, p.s, k, n_el, scheme=scheme, kt=kt)
    with egb.Handle(p.n, k, n_el) as hd:
        hd.use_current_stream()
        hd.set_band_width(32)
        hd.set_precision(prec)
        hd.set_broadening(scheme, kt)
        P, e = hd.dm_real(dev(p.h), dev(p.s))
        W = hd.get_edm()
        mu = hd.get_mu()
    assert rel(P.cpu().numpy(), ref["P"]) <= 1e-9
    assert rel(W.cpu().numpy(), ref["W"]) <= 1e-9
    assert abs(mu - ref["mu"]) <= 1e-10
    assert abs(e - ref["energy"]) <= 1e-9 * abs(ref["energy"])


def test_mp1_free_energy_and_gradient():
    p = ksinputs.cluster_problem(80, seed=72)
    k, n_el, kt = 50, 37.0, 0.03
    ref = oracle.free_energy(p.h, p.s, k, n_el, scheme=oracle.SCHEME_MP1, kt=kt)
    with egb.Handle(p.n, k, n_el) as hd:
        hd.use_current_stream()
        hd.set_band_width(16)
        hd.set_broadening(egb.OCC_MP1, kt)
        H = dev(p.h).requires_grad_(True)
        S = dev(p.s).requires_grad_(True)
        F = ega.free_energy(H, S, hd)
        F.backward()
    assert abs(F.item() - ref["F"]) <= 1e-9 * abs(ref["F"])
    assert rel(H.grad.cpu().numpy(), ref["P"]) <= 1e-9
    assert rel(S.grad.cpu().numpy(), -ref["W"]) <= 1e-9


def test_mp1_kpoint_batch_shared_mu():
    probs = [ksinputs.kpoint_problem(40, kf, seed=73) for kf in
             [(0.0, 0.0, 0.0), (0.25, 0.0, 0.0), (0.5, 0.5, 0.0)]]
    wts = [0.25, 0.5, 0.25]
    k, n_el = 18, 19.0
    ref, ref_mu = oracle.solve_batched([(q.h, q.s, k) for q in probs], n_el, weights=wts,
                                       is_complex=True, scheme=oracle.SCHEME_MP1, kt=0.02)
    with egb.Handle(8, 1, 0.0) as hd:
        hd.use_current_stream()
        hd.set_band_width(16)
        hd.set_broadening(egb.OCC_MP1, 0.02)
        hs = [torch.from_numpy(np.ascontiguousarray(q.h)).cuda() for q in probs]
        ss = [torch.from_numpy(np.ascontiguousarray(q.s)).cuda() for q in probs]
        P, W, en, mu = hd.dm_batched(hs, ss, [k] * 3, n_el, weights=wts)
    assert abs(mu - ref_mu) <= 1e-10
    for Pi, r in zip(P, ref):
        assert rel(Pi.cpu().numpy(), r["P"]) <= 1e-9
