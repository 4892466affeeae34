"""GPU parity of the derivative entry points (elsi_get_entropy, elsi_dm_adjoint_real,
elsi_ev_adjoint_real) and of the autograd functions built on them, against the oracle's
free energy and eigenpair adjoint (themselves pinned by finite differences), plus central
finite differences through the GPU forward. Tolerances: 1e-9 relative for F, P, W;
1e-11 relative for the adjoint on identical inputs; 1e-8 for the adjoint through the
GPU's own eigenpairs; 1e-6 for finite differences (step 1e-6)."""
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


def _sym(rng, n):
    d = rng.standard_normal((n, n))
    return 0.5 * (d + d.T)


@pytest.mark.parametrize("scheme,kt", [(egb.OCC_FERMI, 0.02), (egb.OCC_GAUSSIAN, 0.03),
                                       (egb.OCC_INTEGER, 0.0)])
def test_entropy_and_free_energy_gradient(scheme, kt):
    p = ksinputs.cluster_problem(90, seed=31)
    k, n_el = 40, 45.0
    ref = oracle.free_energy(p.h, p.s, k, n_el, scheme=scheme, kt=kt)
    with egb.Handle(p.n, k, n_el) as hd:
        hd.use_current_stream()
        hd.set_band_width(16)
        if scheme != egb.OCC_INTEGER:
            hd.set_broadening(scheme, kt)
        H = dev(p.h).requires_grad_(True)
        S = dev(p.s).requires_grad_(True)
        F = ega.free_energy(H, S, hd)
        F.backward()
    assert abs(F.item() - ref["F"]) <= 1e-9 * abs(ref["F"])
    assert rel(H.grad.cpu().numpy(), ref["P"]) <= 1e-9
    assert rel(S.grad.cpu().numpy(), -ref["W"]) <= 1e-9


def test_free_energy_finite_differences_through_gpu_forward():
    p = ksinputs.cluster_problem(64, seed=32)
    k, n_el, kt = 40, 30.0, 0.02
    rng = np.random.default_rng(3)
    with egb.Handle(p.n, k, n_el) as hd:
        hd.use_current_stream()
        hd.set_band_width(16)
        hd.set_broadening(egb.OCC_FERMI, kt)
        H = dev(p.h).requires_grad_(True)
        S = dev(p.s).requires_grad_(True)
        ega.free_energy(H, S, hd).backward()
        gh, gs = H.grad.cpu().numpy(), S.grad.cpu().numpy()
        h = 1e-6
        for _ in range(3):
            d = _sym(rng, p.n)
            fp = ega.free_energy(dev(p.h + h * d), dev(p.s), hd).item()
            fm = ega.free_energy(dev(p.h - h * d), dev(p.s), hd).item()
            assert abs((fp - fm) / (2 * h) - np.sum(gh * d)) < 1e-6 * max(1.0, abs(np.sum(gh * d)))
            e = 0.05 * _sym(rng, p.n)
            fp = ega.free_energy(dev(p.h), dev(p.s + h * e), hd).item()
            fm = ega.free_energy(dev(p.h), dev(p.s - h * e), hd).item()
            assert abs((fp - fm) / (2 * h) - np.sum(gs * e)) < 1e-6 * max(1.0, abs(np.sum(gs * e)))


@pytest.mark.parametrize("n,k", [(40, 6), (130, 17), (77, 0)])
def test_ev_adjoint_parity_on_identical_inputs(n, k):
    p = ksinputs.cluster_problem(n, seed=33)
    r = oracle.solve(p.h, p.s, n, 0.0, want_pw=False)
    rng = np.random.default_rng(n)
    eb = rng.standard_normal(n)
    cb = rng.standard_normal((n, k)) if k else None
    hb, sb = oracle.ev_adjoint(r["eval"], r["C"], eb, cb)
    with egb.Handle(n, n, 0.0) as hd:
        hd.use_current_stream()
        ghb, gsb = hd.ev_adjoint(dev(r["eval"]), dev(r["C"]), dev(eb),
                                 dev(cb) if cb is not None else None)
    assert rel(ghb.cpu().numpy(), hb) <= 1e-11
    assert rel(gsb.cpu().numpy(), sb) <= 1e-11


def test_eigh_autograd_gauge_invariant_loss():
    p = ksinputs.cluster_problem(60, seed=34)
    n, k = p.n, 8
    rng = np.random.default_rng(4)
    eb = rng.standard_normal(n)
    ms = [_sym(rng, n) for _ in range(k)]
    r = oracle.solve(p.h, p.s, n, 0.0, want_pw=False)
    cb = np.stack([2 * ms[j] @ r["C"][:, j] for j in range(k)], axis=1)
    hb, sb = oracle.ev_adjoint(r["eval"], r["C"], eb, cb)
    M = torch.stack([dev(m) for m in ms])
    with egb.Handle(n, n, 0.0) as hd:
        hd.use_current_stream()
        hd.set_band_width(16)
        H = dev(p.h).requires_grad_(True)
        S = dev(p.s).requires_grad_(True)
        ev, C = ega.eigh(H, S, hd, k)
        loss = (ev * dev(eb)).sum() + torch.einsum("aj,jab,bj->", C, M, C)
        loss.backward()
    assert rel(H.grad.cpu().numpy(), hb) <= 1e-8
    assert rel(S.grad.cpu().numpy(), sb) <= 1e-8
