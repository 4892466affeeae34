"""Pins for the oracle's derivatives by central finite differences of the oracle's own
forward solve (step 1e-6, random symmetric directions): the Mermin free energy gives
dF/dH = P and dF/dS = -W (Hellmann-Feynman and Pulay terms), and the eigenvector adjoint
reproduces the directional derivative of gauge-invariant losses of eigenvalues and
eigenvectors. Also: kT -> 0 removes the entropy term, and an eigenvalue-only upstream
gives dL/dH = C diag(ev_bar) C^T."""
import numpy as np
import pytest

import ksinputs
import oracle


def _sym_dir(rng, n):
    d = rng.standard_normal((n, n))
    return 0.5 * (d + d.T)


@pytest.mark.parametrize("scheme", [oracle.SCHEME_FERMI, oracle.SCHEME_GAUSSIAN])
def test_free_energy_gradient_is_p_and_minus_w(scheme):
    p = ksinputs.cluster_problem(36, seed=12)
    k, n_el, kt = 24, 15.0, 0.02
    r = oracle.free_energy(p.h, p.s, k, n_el, scheme=scheme, kt=kt)
    rng = np.random.default_rng(6)
    h = 1e-6
    for _ in range(6):
        dh = _sym_dir(rng, p.n)
        fp = oracle.free_energy(p.h + h * dh, p.s, k, n_el, scheme=scheme, kt=kt, want_pw=False)["F"]
        fm = oracle.free_energy(p.h - h * dh, p.s, k, n_el, scheme=scheme, kt=kt, want_pw=False)["F"]
        # noise floor: the bisection's charge accuracy (1e-12) times mu, over 2h
        assert abs((fp - fm) / (2 * h) - np.sum(r["P"] * dh)) < 1e-6
        ds = 0.05 * _sym_dir(rng, p.n)
        fp = oracle.free_energy(p.h, p.s + h * ds, k, n_el, scheme=scheme, kt=kt, want_pw=False)["F"]
        fm = oracle.free_energy(p.h, p.s - h * ds, k, n_el, scheme=scheme, kt=kt, want_pw=False)["F"]
        assert abs((fp - fm) / (2 * h) + np.sum(r["W"] * ds)) < 1e-6


def test_band_energy_alone_is_not_stationary_under_smearing():
    """Without the entropy term the FD gradient differs from P (the term matters)."""
    p = ksinputs.cluster_problem(30, seed=13)
    k, n_el, kt = 20, 13.0, 0.05
    r = oracle.free_energy(p.h, p.s, k, n_el, scheme=oracle.SCHEME_FERMI, kt=kt)
    rng = np.random.default_rng(2)
    dh = _sym_dir(rng, p.n)
    h = 1e-6
    ep = oracle.solve(p.h + h * dh, p.s, k, n_el, scheme=oracle.SCHEME_FERMI, kt=kt, want_pw=False)["energy"]
    em = oracle.solve(p.h - h * dh, p.s, k, n_el, scheme=oracle.SCHEME_FERMI, kt=kt, want_pw=False)["energy"]
    assert abs((ep - em) / (2 * h) - np.sum(r["P"] * dh)) > 1e-4


def test_entropy_vanishes_at_zero_temperature():
    rng = np.random.default_rng(1)
    eps = np.sort(rng.uniform(-1, 1, 20))
    f, mu = oracle.occupation(eps, 10.0, scheme=oracle.SCHEME_FERMI, kt=1e-4)
    assert abs(oracle.entropy_term(eps, f, mu, oracle.SCHEME_FERMI, 1e-4)) < 1e-12
    # a half-filled level carries g ln 2 of entropy: -kT S = -kT g ln 2
    assert abs(oracle.entropy_term([0.0], [1.0], 0.0, oracle.SCHEME_FERMI, 0.1)
               + 0.1 * 2 * np.log(2)) < 1e-15
    # Gaussian at x = 0: -kT g / (2 sqrt(pi))
    assert abs(oracle.entropy_term([0.0], [1.0], 0.0, oracle.SCHEME_GAUSSIAN, 0.1)
               + 0.1 * 2 / (2 * np.sqrt(np.pi))) < 1e-15


def _ev_loss(h, s, eb, m, k):
    w, c, _ = oracle.jacobi(oracle.standard_form(h, oracle.cholesky(s)))
    cc = oracle.back_substitute(oracle.cholesky(s), c)
    return float(np.dot(eb, w) + sum(cc[:, j] @ m[j] @ cc[:, j] for j in range(k)))


def test_eigenvector_adjoint_matches_finite_differences():
    p = ksinputs.cluster_problem(24, seed=14)
    n, k = p.n, 5
    rng = np.random.default_rng(9)
    eb = rng.standard_normal(n)
    m = [_sym_dir(rng, n) for _ in range(k)]
    r = oracle.solve(p.h, p.s, n, 0.0, want_pw=False)
    ev, c = r["eval"], r["C"]
    cb = np.stack([2 * m[j] @ c[:, j] for j in range(k)], axis=1)
    hb, sb = oracle.ev_adjoint(ev, c, eb, cb)
    h = 1e-6
    for _ in range(4):
        dh = _sym_dir(rng, n)
        fd = (_ev_loss(p.h + h * dh, p.s, eb, m, k) - _ev_loss(p.h - h * dh, p.s, eb, m, k)) / (2 * h)
        assert abs(fd - np.sum(hb * dh)) < 1e-6 * max(1.0, abs(fd))
        ds = 0.05 * _sym_dir(rng, n)
        fd = (_ev_loss(p.h, p.s + h * ds, eb, m, k) - _ev_loss(p.h, p.s - h * ds, eb, m, k)) / (2 * h)
        assert abs(fd - np.sum(sb * ds)) < 1e-6 * max(1.0, abs(fd))


def test_eigenvalue_only_adjoint_closed_form():
    p = ksinputs.cluster_problem(20, seed=15)
    r = oracle.solve(p.h, p.s, p.n, 0.0, want_pw=False)
    eb = np.linspace(-1, 1, p.n)
    hb, sb = oracle.ev_adjoint(r["eval"], r["C"], eb, None)
    np.testing.assert_allclose(hb, (r["C"] * eb) @ r["C"].T, rtol=0, atol=1e-13)
    np.testing.assert_allclose(sb, -(r["C"] * (eb * r["eval"])) @ r["C"].T, rtol=0, atol=1e-13)
