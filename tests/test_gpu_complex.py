"""GPU parity of the complex Hermitian entry points (elsi_ev_complex, elsi_dm_complex,
elsi_get_edm_complex) against the FP64 CPU oracle on seeded k-point problems
H(k) = sum_R H_R e^{2 pi i k.R}. Tolerances as for the real path: eigenvalues 1e-10,
P and W 1e-9 relative Frobenius, band energy 1e-9 relative."""
import numpy as np
import pytest

import ksinputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1705_11191_gb300 as egb  # noqa: E402


def cdev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.complex128)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("n,kf,seed,b,prec", [
    (40, (0.0, 0.0, 0.0), 1, 16, 0),
    (101, (0.25, 0.5, 0.0), 2, 32, 0),
    (150, (0.5, 0.25, 0.75), 3, 64, 0),
    (120, (0.25, 0.0, 0.5), 4, 32, 1),
])
def test_complex_dm_parity(n, kf, seed, b, prec):
    p = ksinputs.kpoint_problem(n, kf, seed=seed)
    ref = oracle.solve_complex(p.h, p.s, p.n_state, p.n_electron)
    with egb.Handle(n, p.n_state, p.n_electron) as hd:
        hd.use_current_stream()
        hd.set_band_width(b)
        hd.set_precision(prec)
        P, e = hd.dm_complex(cdev(p.h), cdev(p.s))
        W = hd.get_edm_complex()
    P, W = P.cpu().numpy(), W.cpu().numpy()
    assert rel(P, ref["P"]) <= 1e-9
    assert rel(W, ref["W"]) <= 1e-9
    assert abs(e - ref["energy"]) <= 1e-9 * abs(ref["energy"])
    np.testing.assert_allclose(P, P.conj().T, atol=1e-12)


@pytest.mark.parametrize("n,kf,seed", [(64, (0.5, 0.5, 0.5), 5), (99, (0.25, 0.25, 0.0), 6)])
def test_complex_ev_parity(n, kf, seed):
    p = ksinputs.kpoint_problem(n, kf, seed=seed)
    k = p.n_state
    ref = oracle.solve_complex(p.h, p.s, k, p.n_electron, want_pw=False)
    with egb.Handle(n, k, p.n_electron) as hd:
        hd.use_current_stream()
        hd.set_band_width(16)
        ev, C = hd.ev_complex(cdev(p.h), cdev(p.s))
    ev, C = ev.cpu().numpy(), C.cpu().numpy()
    np.testing.assert_allclose(ev, ref["eval"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(C.conj().T @ p.s @ C, np.eye(k), atol=1e-10)
    r = p.h @ C - (p.s @ C) * ev[None, :k]
    assert np.abs(r).max() < 1e-9


def test_complex_gamma_point_real_hamiltonian_matches_real_path():
    """At k = 0 the k-point matrices are real: the complex route must reproduce the real one."""
    p = ksinputs.kpoint_problem(90, (0.0, 0.0, 0.0), seed=7)
    assert np.abs(p.h.imag).max() == 0.0
    with egb.Handle(p.n, p.n_state, p.n_electron) as hd:
        hd.use_current_stream()
        Pc, ec = hd.dm_complex(cdev(p.h), cdev(p.s))
        hr = torch.from_numpy(np.ascontiguousarray(p.h.real)).cuda()
        sr = torch.from_numpy(np.ascontiguousarray(p.s.real)).cuda()
        Pr, er = hd.dm_real(hr, sr)
    assert abs(ec - er) < 1e-10 * abs(er)
    assert rel(Pc.cpu().numpy().real, Pr.cpu().numpy()) < 1e-10
    assert np.abs(Pc.cpu().numpy().imag).max() < 1e-12
