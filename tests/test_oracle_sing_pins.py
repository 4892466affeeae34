"""Pins for the oracle's singularity check and canonical orthogonalisation (sec. 4.4,
Eq. 10: S = X X^T with X = x sqrt(lambda), eigenvectors of S below the tolerance dropped):
  - with nothing dropped, the eigendecomposition route reproduces the Cholesky route;
  - an exactly duplicated basis function makes S singular; dropping its null direction
    must give back the eigenvalues of the original problem and, folded back onto the
    original basis, its density matrix;
  - on a nearly singular overlap the reduced solution is S-orthonormal and satisfies the
    Galerkin condition in the kept space, U^T (H C - S C eps) = 0 (the dropped direction
    is no longer part of the basis, so the full residual need not vanish)."""
import numpy as np
import pytest

import ksinputs
import oracle


def test_forced_transform_equals_cholesky_route():
    p = ksinputs.cluster_problem(48, seed=51)
    r0 = oracle.solve(p.h, p.s, p.n_state, p.n_electron)
    r1 = oracle.solve_sing(p.h, p.s, p.n_state, p.n_electron, tau=1e-12, force=True)
    assert r1["n_nonsing"] == p.n
    np.testing.assert_allclose(r1["eval"], r0["eval"], rtol=0, atol=1e-11)
    np.testing.assert_allclose(r1["P"], r0["P"], rtol=0, atol=1e-11)
    np.testing.assert_allclose(r1["W"], r0["W"], rtol=0, atol=1e-11)


def test_not_singular_uses_cholesky_route():
    p = ksinputs.cluster_problem(30, seed=52)
    r = oracle.solve_sing(p.h, p.s, p.n_state, p.n_electron, tau=1e-6)
    assert r["n_nonsing"] == p.n
    assert r["s_eval"][0] > 1e-6


def _duplicate(p, idx):
    """Basis extended by an exact copy of basis function idx: phi' = E phi."""
    n = p.n
    e = np.vstack([np.eye(n), np.eye(n)[idx:idx + 1]])
    return e, e @ p.h @ e.T, e @ p.s @ e.T


@pytest.mark.parametrize("idx", [0, 7, 29])
def test_duplicated_basis_function_is_dropped(idx):
    p = ksinputs.cluster_problem(36, seed=53)
    e, h2, s2 = _duplicate(p, idx)
    r0 = oracle.solve(p.h, p.s, p.n_state, p.n_electron)
    r2 = oracle.solve_sing(h2, s2, p.n_state, p.n_electron, tau=1e-8)
    assert r2["n_nonsing"] == p.n
    assert abs(r2["s_eval"][0]) < 1e-12
    np.testing.assert_allclose(r2["eval"][: p.n], r0["eval"], rtol=0, atol=1e-10)
    assert r2["eval"][p.n] == oracle.SING_FILL
    # the density operator is unique: folding the duplicate back gives the original P
    np.testing.assert_allclose(e.T @ r2["P"] @ e, r0["P"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(e.T @ r2["W"] @ e, r0["W"], rtol=0, atol=1e-10)
    assert abs(np.trace(r2["P"] @ s2) - p.n_electron) < 1e-10


def test_nearly_singular_overlap_invariants():
    p = ksinputs.cluster_problem(60, seed=54, tau=1e-9, force_tau=True)
    r = oracle.solve_sing(p.h, p.s, p.n_state, p.n_electron, tau=1e-6)
    nn = r["n_nonsing"]
    assert nn == int(np.sum(np.linalg.eigvalsh(p.s) >= 1e-6))
    assert nn < p.n
    c = r["C"]
    ev = r["eval"][: p.n_state]
    np.testing.assert_allclose(c.T @ p.s @ c, np.eye(p.n_state), rtol=0, atol=1e-10)
    u, _ = oracle.canonical_transform(p.s, 1e-6)
    res = u.T @ (p.h @ c - (p.s @ c) * ev[None, :])
    assert np.abs(res).max() < 1e-9
    assert abs(np.trace(r["P"] @ p.s) - p.n_electron) < 1e-10
