"""GPU parity of the singularity check and canonical orthogonalisation (sec. 4.4, Eq. 10;
elsi_set_sing_check / elsi_set_sing_tol / elsi_get_n_nonsing) against the oracle's
solve_sing: forced transformation without drops, an exactly duplicated basis function,
a nearly singular overlap, the binary32+refinement route on the reduced problem, reuse
of the transformation, and the argument errors. Tolerances as for the Cholesky route:
eigenvalues 1e-10, P and W 1e-9 relative Frobenius."""
import numpy as np
import pytest

import ksinputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1705_11191_gb300 as egb  # noqa: E402


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _dm(h, s, k, n_el, mode, tol, prec=0, b=16, reuse=False, calls=1):
    n = h.shape[0]
    with egb.Handle(n, k, n_el) as hd:
        hd.use_current_stream()
        hd.set_band_width(b)
        hd.set_precision(prec)
        hd.set_sing_check(mode, tol)
        if reuse:
            hd.set_reuse_ovlp_factor(True)
        for _ in range(calls):
            P, e = hd.dm_real(dev(h), dev(s))
        W = hd.get_edm()
        return P.cpu().numpy(), W.cpu().numpy(), e, hd.get_n_nonsing()


def _duplicate(p, idx):
    n = p.n
    e = np.vstack([np.eye(n), np.eye(n)[idx:idx + 1]])
    return e, e @ p.h @ e.T, e @ p.s @ e.T


def test_forced_transform_matches_cholesky_route():
    p = ksinputs.cluster_problem(80, seed=61)
    ref = oracle.solve(p.h, p.s, p.n_state, p.n_electron)
    P, W, e, nn = _dm(p.h, p.s, p.n_state, p.n_electron, 2, 1e-12)
    assert nn == p.n
    assert rel(P, ref["P"]) <= 1e-9 and rel(W, ref["W"]) <= 1e-9
    assert abs(e - ref["energy"]) <= 1e-9 * abs(ref["energy"])


def test_healthy_overlap_keeps_cholesky_route():
    p = ksinputs.cluster_problem(64, seed=62)
    ref = oracle.solve(p.h, p.s, p.n_state, p.n_electron)
    P, W, e, nn = _dm(p.h, p.s, p.n_state, p.n_electron, 1, 1e-6)
    assert nn == p.n
    assert rel(P, ref["P"]) <= 1e-9


@pytest.mark.parametrize("n,idx,prec", [(36, 5, 0), (150, 100, 1)])
def test_duplicated_basis_function(n, idx, prec):
    p = ksinputs.cluster_problem(n, seed=63)
    e_map, h2, s2 = _duplicate(p, idx)
    ref = oracle.solve_sing(h2, s2, p.n_state, p.n_electron, tau=1e-8)
    P, W, e, nn = _dm(h2, s2, p.n_state, p.n_electron, 1, 1e-8, prec=prec, b=32)
    assert nn == ref["n_nonsing"] == p.n
    assert rel(P, ref["P"]) <= 1e-9 and rel(W, ref["W"]) <= 1e-9
    assert abs(e - ref["energy"]) <= 1e-9 * abs(ref["energy"])
    r0 = oracle.solve(p.h, p.s, p.n_state, p.n_electron)
    assert rel(e_map.T @ P @ e_map, r0["P"]) <= 1e-9


def test_nearly_singular_overlap_ev_and_dm():
    p = ksinputs.cluster_problem(60, seed=54, tau=1e-9, force_tau=True)
    ref = oracle.solve_sing(p.h, p.s, p.n_state, p.n_electron, tau=1e-6)
    nn_ref = ref["n_nonsing"]
    assert nn_ref < p.n
    with egb.Handle(p.n, p.n_state, p.n_electron) as hd:
        hd.use_current_stream()
        hd.set_band_width(16)
        hd.set_sing_check(1, 1e-6)
        ev, C = hd.ev_real(dev(p.h), dev(p.s))
        assert hd.get_n_nonsing() == nn_ref
        P, e = hd.dm_real(dev(p.h), dev(p.s))
    ev, C, P = ev.cpu().numpy(), C.cpu().numpy(), P.cpu().numpy()
    np.testing.assert_allclose(ev[:nn_ref], ref["eval"][:nn_ref], rtol=0, atol=1e-10)
    assert np.all(ev[nn_ref:] == np.finfo(np.float64).max)
    np.testing.assert_allclose(C.T @ p.s @ C, np.eye(p.n_state), rtol=0, atol=1e-10)
    assert rel(P, ref["P"]) <= 1e-9


def test_reuse_of_the_transformation():
    p = ksinputs.cluster_problem(40, seed=64)
    e_map, h2, s2 = _duplicate(p, 3)
    ref = oracle.solve_sing(h2, s2, p.n_state, p.n_electron, tau=1e-8)
    P, W, e, nn = _dm(h2, s2, p.n_state, p.n_electron, 1, 1e-8, reuse=True, calls=2)
    assert nn == p.n
    assert rel(P, ref["P"]) <= 1e-9


def test_sing_check_errors():
    p = ksinputs.cluster_problem(30, seed=65)
    e_map, h2, s2 = _duplicate(p, 0)
    with egb.Handle(p.n + 1, p.n + 1, 2.0) as hd:
        hd.use_current_stream()
        with pytest.raises(egb.ElsiError) as ei:
            hd.set_sing_check(3)
        assert ei.value.code == 1
        with pytest.raises(egb.ElsiError) as ei:
            hd.set_sing_check(1, -1.0)
        assert ei.value.code == 1
        hd.set_sing_check(1, 1e-8)
        with pytest.raises(egb.ElsiError) as ei:  # n_state = n + 1 > N_nonsing = n
            hd.dm_real(dev(h2), dev(s2))
        assert ei.value.code == 1
