"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle on the same
seeded inputs, at sizes the oracle finishes in seconds, spanning several panels / band
blocks and ragged tails. Tolerances (binary64 path): eigenvalues 1e-10 * max(1, |eps|max),
||P - P_oracle||_F / ||P_oracle||_F <= 1e-9, same for W, |E - E_oracle| <= 1e-9 max(1,|E|).
"""
import numpy as np
import pytest

import ksinputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1705_11191_gb300 as egb  # noqa: E402

EVAL_TOL = 1e-10
PW_TOL = 1e-9


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _problem(n, seed):
    if n <= 3:
        rng = np.random.default_rng(seed)
        a = rng.standard_normal((n, n))
        h = a + a.T
        b = rng.standard_normal((n, n))
        s = b @ b.T / n + np.eye(n)
        return ksinputs.Problem(np.asfortranarray(h), np.asfortranarray(s), float(n), n,
                                f"rand{n}", 0.0)
    return ksinputs.cluster_problem(n, seed=seed)


CASES = [(2, 1, 8), (3, 2, 8), (17, 3, 8), (64, 4, 16), (100, 5, 32), (150, 6, 64),
         (257, 7, 64), (300, 8, 16), (333, 9, 40)]


@pytest.mark.parametrize("n,seed,b", CASES)
def test_dm_parity(n, seed, b):
    p = _problem(n, seed)
    ref = oracle.solve(p.h, p.s, p.n_state, p.n_electron)
    out = egb.solve_dm(dev(p.h), dev(p.s), p.n_state, p.n_electron, band_width=b)
    P = out["P"].cpu().numpy()
    W = out["W"].cpu().numpy()
    assert rel(P, ref["P"]) <= PW_TOL
    assert rel(W, ref["W"]) <= PW_TOL
    assert abs(out["energy"] - ref["energy"]) <= PW_TOL * max(1.0, abs(ref["energy"]))
    np.testing.assert_allclose(P, P.T, atol=0)


@pytest.mark.parametrize("n,seed,b", CASES)
def test_ev_parity(n, seed, b):
    p = _problem(n, seed)
    k = max(1, min(n, p.n_state))
    ref = oracle.solve(p.h, p.s, k, p.n_electron, want_pw=False)
    out = egb.solve_ev(dev(p.h), dev(p.s), k, band_width=b)
    ev = out["eval"].cpu().numpy()
    C = out["C"].cpu().numpy()
    scale = max(1.0, np.abs(ref["eval"]).max())
    np.testing.assert_allclose(ev, ref["eval"], rtol=0, atol=EVAL_TOL * scale)
    # eigenvectors: S-orthonormal, and each matches the oracle's up to sign
    np.testing.assert_allclose(C.T @ p.s @ C, np.eye(k), atol=1e-10)
    overlap = np.abs(np.sum(C * (p.s @ ref["C"]), axis=0))
    gaps = np.diff(ref["eval"])
    isolated = np.ones(k, bool)
    tight = np.where(gaps < 1e-6)[0]
    isolated[tight] = False
    isolated[np.minimum(tight + 1, k - 1)] = False
    assert np.all(np.abs(overlap[isolated[:k]] - 1.0) < 1e-8)
    # residual H c = eps S c
    r = p.h @ C - (p.s @ C) * ev[None, :k]
    assert np.abs(r).max() < 1e-9 * scale


def test_chain512_parity():
    p = ksinputs.workload("chain-n512")
    ref = oracle.solve(p.h, p.s, p.n_state, p.n_electron)
    out = egb.solve_dm(dev(p.h), dev(p.s), p.n_state, p.n_electron)
    assert rel(out["P"].cpu().numpy(), ref["P"]) <= PW_TOL
    assert rel(out["W"].cpu().numpy(), ref["W"]) <= PW_TOL
    assert abs(out["energy"] - ref["energy"]) <= PW_TOL * abs(ref["energy"])
    ev = egb.solve_ev(dev(p.h), dev(p.s), p.n_state)
    np.testing.assert_allclose(ev["eval"].cpu().numpy(), ref["eval"], rtol=0,
                               atol=EVAL_TOL * np.abs(ref["eval"]).max())


def test_unit_overlap_chain_closed_form():
    """S = I path (overlap_is_unit): tight-binding chain eps_k = 2t cos(k pi/(n+1))."""
    n, t = 200, -0.8
    h = np.zeros((n, n))
    i = np.arange(n - 1)
    h[i, i + 1] = h[i + 1, i] = t
    out = egb.solve_ev(dev(h), None, n, overlap_is_unit=True, band_width=16)
    exact = np.sort(2 * t * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))
    np.testing.assert_allclose(out["eval"].cpu().numpy(), exact, rtol=0, atol=1e-12)


def test_fermi_smearing_parity():
    p = ksinputs.cluster_problem(240, seed=21)
    k = p.n  # all states can carry charge
    kt = 0.01
    ref = oracle.solve(p.h, p.s, k, p.n_electron, scheme=oracle.SCHEME_FERMI, kt=kt,
                       occ_accuracy=1e-12)
    with egb.Handle(p.n, k, p.n_electron) as hd:
        hd.use_current_stream()
        hd.set_broadening(egb.OCC_FERMI, kt)
        hd.set_occ_accuracy(1e-12)
        P, e = hd.dm_real(dev(p.h), dev(p.s))
        mu = hd.get_mu()
        f = hd.get_occ().cpu().numpy()
        W = hd.get_edm().cpu().numpy()
    assert abs(f.sum() - p.n_electron) <= 1e-11
    assert abs(mu - ref["mu"]) < 1e-9
    np.testing.assert_allclose(f, ref["f"], atol=1e-10)
    assert rel(P.cpu().numpy(), ref["P"]) <= PW_TOL
    assert rel(W, ref["W"]) <= PW_TOL
    assert abs(e - ref["energy"]) <= PW_TOL * abs(ref["energy"])


def test_gaussian_charge_correction():
    """mu_max_steps = 1: the surplus is removed from the top states so sum f = N_el."""
    p = ksinputs.cluster_problem(120, seed=22)
    k = p.n
    with egb.Handle(p.n, k, p.n_electron) as hd:
        hd.use_current_stream()
        hd.set_broadening(egb.OCC_GAUSSIAN, 0.05)
        hd.set_occ_accuracy(1e-14)
        hd.set_mu_max_steps(1)
        hd.dm_real(dev(p.h), dev(p.s))
        f = hd.get_occ().cpu().numpy()
    ref = oracle.solve(p.h, p.s, k, p.n_electron, scheme=oracle.SCHEME_GAUSSIAN, kt=0.05,
                       occ_accuracy=1e-14, mu_max_steps=1)
    assert abs(f.sum() - p.n_electron) < 1e-11
    assert np.all(f >= 0.0)
    np.testing.assert_allclose(f, ref["f"], atol=1e-10)


def test_reuse_cholesky_factor():
    p = ksinputs.cluster_problem(180, seed=23)
    rng = np.random.default_rng(5)
    a = rng.standard_normal((p.n, p.n)) * 0.01
    h2 = p.h + a + a.T
    ref = oracle.solve(h2, p.s, p.n_state, p.n_electron)
    with egb.Handle(p.n, p.n_state, p.n_electron) as hd:
        hd.use_current_stream()
        hd.set_reuse_ovlp_factor(True)
        hd.dm_real(dev(p.h), dev(p.s))
        P2, e2 = hd.dm_real(dev(h2), dev(p.s))
        times = hd.stage_times()
    assert rel(P2.cpu().numpy(), ref["P"]) <= PW_TOL
    assert times["cholesky"] < 0.5  # factorisation skipped


def test_not_positive_definite_reports_pivot():
    n = 64
    p = ksinputs.cluster_problem(n, seed=24)
    s = p.s.copy()
    s[40, 40] = -1.0
    with egb.Handle(n, p.n_state, p.n_electron) as hd:
        hd.use_current_stream()
        with pytest.raises(egb.ElsiError) as e:
            hd.dm_real(dev(p.h), dev(s))
    assert e.value.code == 3
    assert "pivot" in str(e.value)


def test_nonfinite_input_rejected():
    p = ksinputs.cluster_problem(64, seed=25)
    h = p.h.copy()
    h[3, 7] = np.nan
    with egb.Handle(p.n, p.n_state, p.n_electron) as hd:
        hd.use_current_stream()
        with pytest.raises(egb.ElsiError) as e:
            hd.dm_real(dev(h), dev(p.s))
    assert e.value.code == 4


def test_host_entry_point_matches_device():
    p = ksinputs.cluster_problem(150, seed=26)
    ref = oracle.solve(p.h, p.s, p.n_state, p.n_electron)
    P = np.zeros((p.n, p.n))
    W = np.zeros((p.n, p.n))
    with egb.Handle(p.n, p.n_state, p.n_electron) as hd:
        e = hd.dm_real_host(np.ascontiguousarray(p.h), np.ascontiguousarray(p.s), P, W)
    assert rel(P, ref["P"]) <= PW_TOL
    assert rel(W, ref["W"]) <= PW_TOL
    assert abs(e - ref["energy"]) <= PW_TOL * abs(ref["energy"])
