"""GPU parity of the one-stage tridiagonalisation route (Eq. 11 first form, elpa_solver 1,
sec. 4.5) against the oracle, in both precision routes: panel counts with ragged last
panels, the smallest sizes, eigenpairs, density matrices and a complex Hermitian problem.
Tolerances as for the two-stage route: eigenvalues 1e-10, P and W 1e-9 relative."""
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


@pytest.mark.parametrize("n,prec", [(33, 0), (100, 0), (257, 0), (300, 1)])
def test_onestage_dm_parity(n, prec):
    p = ksinputs.cluster_problem(n, seed=90 + n)
    ref = oracle.solve(p.h, p.s, p.n_state, p.n_electron)
    with egb.Handle(n, p.n_state, p.n_electron) as hd:
        hd.use_current_stream()
        hd.set_precision(prec)
        hd.set_elpa_solver(1)
        P, e = hd.dm_real(dev(p.h), dev(p.s))
        W = hd.get_edm()
    assert rel(P.cpu().numpy(), ref["P"]) <= 1e-9
    assert rel(W.cpu().numpy(), ref["W"]) <= 1e-9
    assert abs(e - ref["energy"]) <= 1e-9 * abs(ref["energy"])


@pytest.mark.parametrize("n", [2, 3, 5, 64, 129])
def test_onestage_ev_parity(n):
    p = ksinputs.cluster_problem(n, seed=7 + n, n_state=n, n_electron=float(n // 2))
    ref = oracle.solve(p.h, p.s, n, float(n // 2), want_pw=False)
    with egb.Handle(n, n, float(n // 2)) as hd:
        hd.use_current_stream()
        hd.set_elpa_solver(1)
        ev, C = hd.ev_real(dev(p.h), dev(p.s))
    ev, C = ev.cpu().numpy(), C.cpu().numpy()
    np.testing.assert_allclose(ev, ref["eval"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(C.T @ p.s @ C, np.eye(n), rtol=0, atol=1e-10)
    r = p.h @ C - (p.s @ C) * ev[None, :]
    assert np.abs(r).max() < 1e-9


def test_onestage_complex():
    p = ksinputs.kpoint_problem(60, (0.25, 0.5, 0.0), seed=3)
    ref = oracle.solve_complex(p.h, p.s, p.n_state, p.n_electron)
    with egb.Handle(p.n, p.n_state, p.n_electron) as hd:
        hd.use_current_stream()
        hd.set_elpa_solver(1)
        P, e = hd.dm_complex(dev(p.h), dev(p.s))
    assert rel(P.cpu().numpy(), ref["P"]) <= 1e-9


def test_elpa_solver_argument():
    with egb.Handle(8, 4, 2.0) as hd:
        with pytest.raises(egb.ElsiError) as ei:
            hd.set_elpa_solver(3)
        assert ei.value.code == 1
