"""Pins for the Methfessel-Paxton broadening of the oracle (sec. 4.5 broadening_scheme 3
and 4; Methfessel & Paxton, Phys. Rev. B 40, 3616 (1989)): order 0 is the Gaussian
scheme; the order-1 occupation is the integral from x to infinity of the order-1 delta
approximation delta_1(t) = (3/2 - t^2) exp(-t^2) / sqrt(pi), computed here by quadrature;
a symmetric spectrum at half filling gives mu = 0; the electron count is met; and the
free energy with the order-1 entropy term has dF/dH = P (central differences)."""
import numpy as np
import pytest
from scipy.integrate import quad

import ksinputs
import oracle


def test_mp0_is_gaussian():
    rng = np.random.default_rng(2)
    eps = np.sort(rng.uniform(-1, 1, 50))
    fg, mg = oracle.occupation(eps, 31.0, scheme=oracle.SCHEME_GAUSSIAN, kt=0.05)
    f0, m0 = oracle.occupation(eps, 31.0, scheme=oracle.SCHEME_MP0, kt=0.05)
    np.testing.assert_array_equal(f0, fg)
    assert m0 == mg


def test_mp1_occupation_is_integral_of_delta1():
    rng = np.random.default_rng(3)
    eps = np.sort(rng.uniform(-1, 1, 40))
    kt = 0.07
    f, mu = oracle.occupation(eps, 23.0, scheme=oracle.SCHEME_MP1, kt=kt)
    assert abs(f.sum() - 23.0) < 1e-11
    delta1 = lambda t: (1.5 - t * t) * np.exp(-t * t) / np.sqrt(np.pi)
    for e, fl in zip(eps, f):
        x = (e - mu) / kt
        phi = quad(delta1, x, np.inf, epsabs=1e-14, epsrel=1e-13)[0]
        assert abs(fl / 2.0 - phi) < 1e-11


def test_mp1_symmetric_spectrum_mu_zero():
    a = np.array([-0.4, -0.1, 0.1, 0.4])
    f, mu = oracle.occupation(a, 4.0, scheme=oracle.SCHEME_MP1, kt=0.2)
    assert mu == 0.0
    np.testing.assert_allclose(f + f[::-1], 2.0, rtol=0, atol=1e-15)


def test_mp1_free_energy_gradient_is_p():
    p = ksinputs.cluster_problem(32, seed=17)
    k, n_el, kt = 22, 13.0, 0.03
    r = oracle.free_energy(p.h, p.s, k, n_el, scheme=oracle.SCHEME_MP1, kt=kt)
    rng = np.random.default_rng(5)
    h = 1e-6
    for _ in range(4):
        d = rng.standard_normal((p.n, p.n))
        d = 0.5 * (d + d.T)
        fp = oracle.free_energy(p.h + h * d, p.s, k, n_el, scheme=oracle.SCHEME_MP1, kt=kt, want_pw=False)["F"]
        fm = oracle.free_energy(p.h - h * d, p.s, k, n_el, scheme=oracle.SCHEME_MP1, kt=kt, want_pw=False)["F"]
        g = np.sum(r["P"] * d)
        assert abs((fp - fm) / (2 * h) - g) < 1e-6 * max(1.0, abs(g))
