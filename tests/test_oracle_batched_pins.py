"""Pins for the oracle's several-problem path (k-points / spin channels), independent of
the oracle itself: hand-computed aufbau fillings, the reduction to the single-problem
occupation, replication invariance, the symmetric-spectrum value mu = 0, the weighted
electron count, the zero-temperature limit and the density-matrix invariants per
problem (arXiv:1705.11191 sec. 4.4: the electron count of the chemical-potential search
is summed over k-points, spin channels and states)."""
import numpy as np
import pytest

import ksinputs
import oracle

G = 2.0


def test_weighted_integer_hand_filling():
    eps = np.array([0.3, -0.2, 0.1, -0.2, 0.5])
    wt = np.array([0.5, 0.25, 0.25, 0.25, 0.5])
    # lowest level -0.2 holds 2 * (0.25 + 0.25) = 1 electron
    f, mu = oracle.occupation_weighted(eps, wt, 1.0)
    np.testing.assert_array_equal(f, [0, 2, 0, 2, 0])
    assert mu == -0.2
    # 0.3 more electrons go to level 0.1 (weight 0.25): f = 0.3 / 0.25 = 1.2
    f, mu = oracle.occupation_weighted(eps, wt, 1.3)
    np.testing.assert_allclose(f, [0, 2, 1.2, 2, 0], rtol=0, atol=1e-15)
    assert mu == 0.1
    # full: every level at g
    f, mu = oracle.occupation_weighted(eps, wt, G * wt.sum())
    np.testing.assert_allclose(f, G, rtol=0, atol=1e-15)
    assert mu == 0.5


def test_weighted_integer_ties_share_by_weight():
    eps = np.array([0.0, 0.0, 1.0])
    wt = np.array([0.25, 0.75, 1.0])
    f, mu = oracle.occupation_weighted(eps, wt, 1.0)
    np.testing.assert_allclose(f, [1.0, 1.0, 0.0], rtol=0, atol=1e-15)
    assert mu == 0.0


@pytest.mark.parametrize("scheme,kt", [(oracle.SCHEME_INTEGER, 0.0),
                                       (oracle.SCHEME_FERMI, 0.02),
                                       (oracle.SCHEME_GAUSSIAN, 0.05)])
def test_unit_weights_reduce_to_single_problem(scheme, kt):
    rng = np.random.default_rng(11)
    eps = np.sort(rng.uniform(-1, 1, 40))
    f1, mu1 = oracle.occupation(eps, 23.0, scheme=scheme, kt=kt)
    f2, mu2 = oracle.occupation_weighted(eps, np.ones(40), 23.0, scheme=scheme, kt=kt)
    np.testing.assert_allclose(f2, f1, rtol=0, atol=1e-14)
    assert abs(mu2 - mu1) <= 1e-14


@pytest.mark.parametrize("scheme,kt", [(oracle.SCHEME_INTEGER, 0.0),
                                       (oracle.SCHEME_FERMI, 0.01)])
def test_replicated_problem_invariance(scheme, kt):
    """K copies of one spectrum with weights 1/K occupy like the spectrum alone."""
    rng = np.random.default_rng(5)
    eps = np.sort(rng.uniform(-1, 1, 30))
    f1, mu1 = oracle.occupation(eps, 17.0, scheme=scheme, kt=kt)
    K = 4
    fk, muk = oracle.occupation_weighted(np.tile(eps, K), np.full(30 * K, 1.0 / K), 17.0,
                                        scheme=scheme, kt=kt)
    for c in range(K):
        np.testing.assert_allclose(fk[30 * c:30 * (c + 1)], f1, rtol=0, atol=1e-9)
    assert abs(muk - mu1) < 1e-9


def test_symmetric_two_problem_spectrum_mu_zero():
    a = 0.37
    eps = np.array([-a, a, -a, a])
    wt = np.array([0.3, 0.3, 0.7, 0.7])
    f, mu = oracle.occupation_weighted(eps, wt, G * 1.0, scheme=oracle.SCHEME_FERMI, kt=0.05)
    assert mu == 0.0
    np.testing.assert_allclose(f[0] + f[1], G, rtol=0, atol=1e-15)


@pytest.mark.parametrize("scheme", [oracle.SCHEME_FERMI, oracle.SCHEME_GAUSSIAN])
def test_weighted_electron_count(scheme):
    rng = np.random.default_rng(3)
    eps = rng.uniform(-2, 1, 300)
    wt = np.repeat(rng.dirichlet(np.ones(6)), 50)
    f, mu = oracle.occupation_weighted(eps, wt, 0.8 * G * 0.5, scheme=scheme, kt=0.01)
    assert abs(np.dot(wt, f) - 0.8) <= 1e-12
    assert np.all((f >= 0) & (f <= G))
    # occupations are non-increasing in the eigenvalue
    o = np.argsort(eps)
    assert np.all(np.diff(f[o]) <= 1e-15)


def test_surplus_removed_from_the_top_when_bisection_capped():
    rng = np.random.default_rng(8)
    eps = rng.uniform(-1, 1, 60)
    wt = np.repeat([0.5, 0.5], 30)
    f_full, mu_cap = oracle.occupation_weighted(eps, wt, 21.0, scheme=oracle.SCHEME_FERMI,
                                                kt=0.2, mu_max_steps=2)
    assert abs(np.dot(wt, f_full) - 21.0) <= 1e-12
    phi = G / (1.0 + np.exp((eps - mu_cap) / 0.2))
    changed = np.abs(f_full - phi) > 1e-15
    assert changed.any()
    # every reduced entry lies above every unreduced one
    assert eps[changed].min() >= eps[~changed].max()
    assert np.all(f_full <= phi + 1e-15)


def test_zero_temperature_limit_matches_weighted_aufbau():
    rng = np.random.default_rng(4)
    eps = np.concatenate([rng.uniform(-1, -0.2, 20), rng.uniform(0.2, 1, 20)])
    wt = np.repeat([0.25, 0.75], 20)
    # the 20 levels below the gap hold exactly G * sum(wt[eps < 0]) electrons
    n_el = G * wt[eps < 0].sum()
    fi, _ = oracle.occupation_weighted(eps, wt, n_el)
    ff, mu = oracle.occupation_weighted(eps, wt, n_el, scheme=oracle.SCHEME_FERMI, kt=1e-4)
    np.testing.assert_allclose(ff, fi, rtol=0, atol=1e-12)
    assert -0.2 < mu < 0.2


def test_batched_single_problem_equals_solve():
    p = ksinputs.cluster_problem(60, seed=21)
    r = oracle.solve(p.h, p.s, p.n_state, p.n_electron)
    out, mu = oracle.solve_batched([(p.h, p.s, p.n_state)], p.n_electron, weights=[1.0])
    np.testing.assert_allclose(out[0]["P"], r["P"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(out[0]["W"], r["W"], rtol=0, atol=1e-13)
    assert mu == r["mu"]


def test_batched_kpoint_invariants():
    """Complex k-points with one mu: sum_i w_i Tr(P_i S_i) = N_el, Tr(P_i H_i) = E_i,
    and each P_i is Hermitian."""
    n = 30
    ks = [(0.0, 0.0, 0.0), (0.25, 0.0, 0.0), (0.25, 0.25, 0.0), (0.5, 0.25, 0.25)]
    probs = [ksinputs.kpoint_problem(n, k, seed=7) for k in ks]
    wts = np.array([0.1, 0.3, 0.3, 0.3])
    n_el = 14.0
    out, mu = oracle.solve_batched([(p.h, p.s, 12) for p in probs], n_el, weights=wts,
                                   is_complex=True, scheme=oracle.SCHEME_FERMI, kt=0.01)
    tot = sum(w * np.trace(o["P"] @ p.s).real for w, o, p in zip(wts, out, probs))
    assert abs(tot - n_el) < 1e-10
    for o, p in zip(out, probs):
        assert abs(np.trace(o["P"] @ p.h).real - o["energy"]) < 1e-10
        assert abs(np.trace(o["W"] @ p.s).real - o["energy"]) < 1e-10
        np.testing.assert_allclose(o["P"], o["P"].conj().T, rtol=0, atol=1e-13)
