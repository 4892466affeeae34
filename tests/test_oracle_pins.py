"""Pins for the FP64 CPU oracle, independent of the oracle itself.

Each test checks the oracle against something the mathematics fixes: closed forms of
tridiagonal (chain) problems, a hand-solved 2x2 generalized problem, brute force with
LAPACK (scipy) on small inputs, and the invariants of the density matrices
(Tr(PS) = N_el, PSP = 2P for integer occupation, Tr(PH) = Tr(WS) = sum f eps).
Citations: arXiv:1705.11191 (ELSI), Eqs. 5, 7-9, 14-15, 17-18 and sec. 4.4.
"""
import os

import numpy as np
import pytest
import scipy.linalg as sla

import ksinputs
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_forms.txt")


def _golden():
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = np.array([float(v) for v in vals])
    return out


def _chain(n, alpha, t):
    a = np.zeros((n, n))
    i = np.arange(n - 1)
    a[i, i + 1] = t
    a[i + 1, i] = t
    a[np.arange(n), np.arange(n)] = alpha
    return a


def _chain_vectors(n):
    """Closed-form eigenvectors of the chain adjacency: s_k(i) = sqrt(2/(n+1)) sin(i k pi/(n+1))."""
    i = np.arange(1, n + 1)[:, None]
    k = np.arange(1, n + 1)[None, :]
    return np.sqrt(2.0 / (n + 1)) * np.sin(i * k * np.pi / (n + 1))


# ---------------------------------------------------------------- hand-derived goldens
def test_golden_2x2_generalized():
    g = _golden()
    h = np.array([[2.0, 1.0], [1.0, 3.0]])
    s = np.array([[2.0, 1.0], [1.0, 2.0]])
    r = oracle.solve(h, s, 2, 2.0)
    np.testing.assert_allclose(r["eval"], g["gen2x2"], rtol=0, atol=1e-14)


def test_golden_chain4():
    g = _golden()
    h = _chain(4, 0.0, -1.0)
    w, v, _ = oracle.jacobi(h)
    np.testing.assert_allclose(w, g["chain4"], rtol=0, atol=1e-14)


def test_golden_cholesky_2x2():
    g = _golden()
    l = oracle.cholesky(np.array([[4.0, 2.0], [2.0, 3.0]]))
    np.testing.assert_allclose([l[0, 0], l[1, 0], l[1, 1]], g["chol2x2"], atol=1e-15)
    assert l[0, 1] == 0.0


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("n", [5, 16, 33, 64])
def test_tight_binding_chain_closed_form(n):
    """S = I, H = t * chain: eps_k = 2 t cos(k pi/(n+1)) (textbook closed form)."""
    t = -0.7
    h = _chain(n, 0.0, t)
    r = oracle.solve(h, None, n, float(n), unit_ovlp=True)
    k = np.arange(1, n + 1)
    exact = np.sort(2 * t * np.cos(k * np.pi / (n + 1)))
    np.testing.assert_allclose(r["eval"], exact, rtol=0, atol=1e-13)
    # eigenvectors: each computed column is +-(closed-form vector) (t<0: ascending = k asc)
    s_exact = _chain_vectors(n)
    for j in range(n):
        dot = abs(s_exact[:, j] @ r["C"][:, j])
        assert abs(dot - 1.0) < 1e-12


@pytest.mark.parametrize("n,s_off", [(12, 0.2), (40, -0.3), (63, 0.45)])
def test_commuting_generalized_chain(n, s_off):
    """S = I + s A, H = alpha I + t A with A the chain adjacency: both share the sine
    vectors, eps_k = (alpha + 2t cos th_k)/(1 + 2 s cos th_k). Exercises Cholesky,
    the standard form and the back-substitution (Eqs. 8-9)."""
    alpha, t = 0.3, -0.5
    a = _chain(n, 0.0, 1.0)
    h = alpha * np.eye(n) + t * a
    s = np.eye(n) + s_off * a
    th = np.arange(1, n + 1) * np.pi / (n + 1)
    lam = (alpha + 2 * t * np.cos(th)) / (1 + 2 * s_off * np.cos(th))
    order = np.argsort(lam)
    r = oracle.solve(h, s, n, float(n))
    np.testing.assert_allclose(r["eval"], lam[order], rtol=0, atol=1e-13 * np.abs(lam).max())
    # S-normalised closed-form vectors: s_k / sqrt(1 + 2 s cos th_k)
    vec = _chain_vectors(n) / np.sqrt(1 + 2 * s_off * np.cos(th))[None, :]
    vec = vec[:, order]
    for j in range(n):
        assert abs(abs(vec[:, j] @ s @ r["C"][:, j]) - 1.0) < 1e-11
    # P and W with all n states occupied by f = 2 except none: use n_el = n (half)
    f = r["f"]
    p_exact = (vec * f[None, :]) @ vec.T
    w_exact = (vec * (f * lam[order])[None, :]) @ vec.T
    np.testing.assert_allclose(r["P"], p_exact, atol=1e-12 * np.abs(p_exact).max())
    np.testing.assert_allclose(r["W"], w_exact, atol=1e-12 * np.abs(w_exact).max())


def test_chain_density_matrix_closed_form():
    """S = I chain, half filling: P = 2 sum_{k occupied} s_k s_k^T with the sine vectors,
    W = 2 sum eps_k s_k s_k^T (Eq. 7 and its energy-weighted form)."""
    n, t = 30, -1.0
    h = _chain(n, 0.0, t)
    r = oracle.solve(h, None, n, float(n), unit_ovlp=True)
    s_exact = _chain_vectors(n)  # ascending order for t < 0 is k = 1..n
    eps = 2 * t * np.cos(np.arange(1, n + 1) * np.pi / (n + 1))
    occ = n // 2
    p = 2 * s_exact[:, :occ] @ s_exact[:, :occ].T
    w = 2 * (s_exact[:, :occ] * eps[:occ]) @ s_exact[:, :occ].T
    np.testing.assert_allclose(r["P"], p, atol=1e-13)
    np.testing.assert_allclose(r["W"], w, atol=1e-13)
    assert abs(r["energy"] - 2 * eps[:occ].sum()) < 1e-12


# ---------------------------------------------------------------- brute force vs LAPACK
@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (7, 2), (31, 3), (96, 4)])
def test_random_vs_lapack(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n))
    h = a + a.T
    b = rng.standard_normal((n, n))
    s = b @ b.T / max(n, 1) + 0.5 * np.eye(n)
    r = oracle.solve(h, s, n, float(n))
    ref = sla.eigh(h, s, eigvals_only=True)
    np.testing.assert_allclose(r["eval"], ref, rtol=0, atol=1e-11 * max(1, np.abs(ref).max()))
    c = r["C"]
    np.testing.assert_allclose(c.T @ s @ c, np.eye(n), atol=1e-12)
    np.testing.assert_allclose(h @ c, s @ c * r["eval"][None, :], atol=1e-10)


def test_cholesky_matches_lapack():
    rng = np.random.default_rng(11)
    b = rng.standard_normal((50, 50))
    s = b @ b.T + 50 * np.eye(50)
    np.testing.assert_allclose(oracle.cholesky(s), np.linalg.cholesky(s), atol=1e-13)


def test_cholesky_not_pd_reports_pivot():
    s = np.eye(6)
    s[3, 3] = -1.0
    with pytest.raises(oracle.OracleError, match="pivot 3"):
        oracle.cholesky(s)


def test_standard_form_definition():
    """L H~ L^T == H (Eq. 9 inverted)."""
    rng = np.random.default_rng(5)
    n = 40
    a = rng.standard_normal((n, n))
    h = a + a.T
    b = rng.standard_normal((n, n))
    s = b @ b.T / n + np.eye(n)
    l = oracle.cholesky(s)
    ht = oracle.standard_form(h, l)
    np.testing.assert_allclose(l @ ht @ l.T, h, atol=1e-12)
    np.testing.assert_allclose(ht, ht.T, atol=0)


def test_jacobi_diagonal_no_rotation():
    d = np.diag([3.0, -1.0, 2.0, 0.5])
    w, v, sweeps = oracle.jacobi(d)
    assert sweeps == 1
    np.testing.assert_array_equal(w, [-1.0, 0.5, 2.0, 3.0])


def test_back_substitution_definition():
    rng = np.random.default_rng(6)
    n = 25
    b = rng.standard_normal((n, n))
    l = np.tril(b) + 5 * np.eye(n)
    vt = rng.standard_normal((n, 7))
    c = oracle.back_substitute(l, vt)
    np.testing.assert_allclose(l.T @ c, vt, atol=1e-13)


# ---------------------------------------------------------------- occupation (sec. 4.4)
def test_integer_occupation_odd_electrons():
    eps = np.linspace(-1, 1, 10)
    f, mu = oracle.occupation(eps, 7.0)
    np.testing.assert_array_equal(f, [2, 2, 2, 1, 0, 0, 0, 0, 0, 0])
    assert mu == eps[3]


@pytest.mark.parametrize("scheme", [oracle.SCHEME_FERMI, oracle.SCHEME_GAUSSIAN])
def test_smeared_electron_count(scheme):
    rng = np.random.default_rng(3)
    eps = np.sort(rng.uniform(-2, 1, 200))
    f, mu = oracle.occupation(eps, 123.0, scheme=scheme, kt=0.01, occ_accuracy=1e-12)
    assert abs(f.sum() - 123.0) <= 1e-12
    assert np.all(f >= 0) and np.all(f <= 2)
    assert np.all(np.diff(f) <= 1e-15)  # monotone in eps


def test_fermi_symmetric_spectrum_mu_zero():
    """Chain at half filling has a spectrum symmetric about 0, so mu = 0 (Eq. 14-15)."""
    n = 40
    eps = np.sort(2 * -1.0 * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))
    f, mu = oracle.occupation(eps, float(n), scheme=oracle.SCHEME_FERMI, kt=0.05,
                              occ_accuracy=1e-13)
    assert abs(mu) < 1e-12


def test_fermi_matches_closed_form_at_returned_mu():
    rng = np.random.default_rng(8)
    eps = np.sort(rng.uniform(-1, 1, 50))
    kt = 0.02
    f, mu = oracle.occupation(eps, 40.0, scheme=oracle.SCHEME_FERMI, kt=kt)
    np.testing.assert_allclose(f, 2.0 / (1.0 + np.exp((eps - mu) / kt)), atol=1e-14)


def test_fermi_zero_temperature_limit_is_integer():
    rng = np.random.default_rng(9)
    eps = np.sort(rng.uniform(-1, 1, 60))
    fi, _ = oracle.occupation(eps, 30.0)
    ff, _ = oracle.occupation(eps, 30.0, scheme=oracle.SCHEME_FERMI, kt=1e-5)
    np.testing.assert_allclose(ff, fi, atol=1e-9)


def test_charge_correction_when_bisection_capped():
    """mu_max_steps = 1: bisection cannot reach occ_accuracy, so the surplus is removed
    from the highest occupied states down and sum f == N_el (sec. 4.4)."""
    rng = np.random.default_rng(10)
    eps = np.sort(rng.uniform(-1, 1, 80))
    f, mu = oracle.occupation(eps, 51.0, scheme=oracle.SCHEME_FERMI, kt=0.05,
                              occ_accuracy=1e-14, mu_max_steps=1)
    assert abs(f.sum() - 51.0) < 1e-12
    assert np.all(f >= 0)
    # only the tail was reduced: f(eps) at mu for the low states is untouched
    full = 2.0 / (1.0 + np.exp((eps - mu) / 0.05))
    assert np.all(f <= full + 1e-15)
    np.testing.assert_allclose(f[:20], full[:20], atol=1e-15)


# ---------------------------------------------------------------- invariants on the 512-function chain
@pytest.fixture(scope="module")
def chain512():
    p = ksinputs.workload("chain-n512")
    return p, oracle.solve(p.h, p.s, p.n_state, p.n_electron)


def test_chain512_vs_lapack(chain512):
    p, r = chain512
    ref_w, ref_v = sla.eigh(p.h, p.s)
    np.testing.assert_allclose(r["eval"], ref_w, rtol=0, atol=1e-11)
    occ = int(p.n_electron // 2)
    p_ref = 2 * ref_v[:, :occ] @ ref_v[:, :occ].T
    assert np.linalg.norm(r["P"] - p_ref) / np.linalg.norm(p_ref) < 1e-11


def test_chain512_invariants(chain512):
    p, r = chain512
    P, W, S, H = r["P"], r["W"], p.s, p.h
    assert abs(np.trace(P @ S) - p.n_electron) < 1e-9
    assert np.linalg.norm(P @ S @ P - 2 * P) / np.linalg.norm(P) < 1e-12
    e = r["energy"]
    assert abs(np.trace(P @ H) - e) < 1e-9 * abs(e)
    assert abs(np.trace(W @ S) - e) < 1e-9 * abs(e)
    C = r["C"]
    assert np.max(np.abs(C.T @ S @ C - np.eye(C.shape[1]))) < 1e-12


# ---------------------------------------------------------------- complex Hermitian path
def _complex_chain(n, t, phi):
    h = np.zeros((n, n), dtype=np.complex128)
    i = np.arange(n - 1)
    h[i, i + 1] = t * np.exp(1j * phi)
    h[i + 1, i] = t * np.exp(-1j * phi)
    return h


@pytest.mark.parametrize("n,phi", [(9, 0.3), (24, 1.1)])
def test_complex_chain_closed_form(n, phi):
    """H_{j,j+1} = t e^{i phi}: the gauge change c_j -> e^{i j phi} c_j maps it to the real
    chain, so eps_k = 2 t cos(k pi/(n+1)) for every phase."""
    t = -0.6
    r = oracle.solve_complex(_complex_chain(n, t, phi), None, n, float(n), unit_ovlp=True)
    exact = np.sort(2 * t * np.cos(np.arange(1, n + 1) * np.pi / (n + 1)))
    np.testing.assert_allclose(r["eval"], exact, rtol=0, atol=1e-13)
    C = r["C"]
    np.testing.assert_allclose(C.conj().T @ C, np.eye(n), atol=1e-12)


@pytest.mark.parametrize("n,seed", [(12, 1), (45, 2)])
def test_complex_random_vs_lapack(n, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    h = a + a.conj().T
    b = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    s = b @ b.conj().T / n + np.eye(n)
    k = n // 2
    r = oracle.solve_complex(h, s, k, float(k))
    w, v = sla.eigh(h, s)
    np.testing.assert_allclose(r["eval"], w, rtol=0, atol=1e-11 * max(1, np.abs(w).max()))
    f = r["f"]
    p_ref = (v[:, :k] * f) @ v[:, :k].conj().T
    np.testing.assert_allclose(r["P"], p_ref, atol=1e-11)
    C = r["C"]
    np.testing.assert_allclose(C.conj().T @ s @ C, np.eye(k), atol=1e-11)


def test_complex_kpoint_invariants():
    p = ksinputs.kpoint_problem(75, (0.25, 0.5, 0.0), seed=3)
    r = oracle.solve_complex(p.h, p.s, p.n_state, p.n_electron)
    P, S, H, W = r["P"], p.s, p.h, r["W"]
    assert abs(np.trace(P @ S).real - p.n_electron) < 1e-10
    np.testing.assert_allclose(P, P.conj().T, atol=1e-13)
    e = r["energy"]
    assert abs(np.trace(P @ H).real - e) < 1e-10 * abs(e)
    assert abs(np.trace(W @ S).real - e) < 1e-10 * abs(e)


def test_batch_generators_match_the_single_problem_recipe():
    """The batch generators (torch construction, used for the k-point and mixed-size
    batches) reproduce the numpy recipe of the single-problem generators."""
    torch = pytest.importorskip("torch")
    p = ksinputs.cluster_problem(150, seed=1007)
    h, s, ne, ns, lam = ksinputs.cluster_problem_torch(150, 1007, "cpu")
    assert np.abs(h.numpy() - p.h).max() < 1e-15 and np.abs(s.numpy() - p.s).max() < 1e-15
    assert (ne, ns) == (p.n_electron, p.n_state) and abs(lam - p.lambda_min_s) < 1e-12
    for kf, hk, sk, lk in ksinputs.kpoint_set(30, grid=2, seed=8)[::3]:
        q = ksinputs.kpoint_problem(30, kf, seed=8)
        assert np.abs(hk.numpy() - q.h).max() < 1e-15 and np.abs(sk.numpy() - q.s).max() < 1e-15
        assert abs(lk - q.lambda_min_s) < 1e-12
    sizes = ksinputs.mixed_sizes()
    assert len(sizes) == 200 and min(sizes) >= 256 and max(sizes) <= 4096
