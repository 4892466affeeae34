"""FP64 CPU oracle for the dense Kohn-Sham solver path (TEST INFRASTRUCTURE ONLY).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
import this package. The product library (``paper_1705_11191_gb300``) never imports,
links or calls it, and the two share no code.

The arithmetic lives in ``oracle.c`` (plain C, binary64, column-major); this module
compiles it with gcc on first use and wraps it with ctypes. Arrays are passed as numpy
float64 arrays in Fortran (column-major) order.

Each routine follows arXiv:1705.11191 (ELSI):
  cholesky        Eq. 8 (S = L L^*)
  standard_form   Eq. 9 (H~ = L^{-1} H L^{-*})
  jacobi          eigendecomposition of H~ by cyclic Jacobi (the plain definition of
                  the eigenpairs that Eqs. 10-11 reach by two-stage tridiagonalisation)
  back_substitute Eq. 9 (c = L^{-*} c~)
  occupation      sec. 4.4 (elsi_dm_real): bisection for mu, Eqs. 14-15, 17-18, and
                  the exact-charge correction
  occupation_weighted
                  sec. 4.4: one mu for several k-points / spin channels (the electron
                  count summed over all of them, each problem with its weight)
  weighted_outer  Eq. 7 (density matrix) and its energy-weighted form W
  solve           the whole path
  solve_batched   several independent problems (k-points / spin channels, sec. 2's
                  SINGLE_PROC mode) with a shared or a per-problem chemical potential
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so (gcc, OpenMP). Returns the library path."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c99", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i, d = ctypes.c_int, ctypes.c_double
            lib.orc_cholesky.argtypes = [i, _dp, _dp]
            lib.orc_cholesky.restype = i
            lib.orc_standard_form.argtypes = [i, _dp, _dp, _dp]
            lib.orc_standard_form.restype = None
            lib.orc_jacobi.argtypes = [i, _dp, _dp, _dp, i]
            lib.orc_jacobi.restype = i
            lib.orc_sort_eigenpairs.argtypes = [i, _dp, _dp]
            lib.orc_sort_eigenpairs.restype = None
            lib.orc_back_substitute.argtypes = [i, i, _dp, _dp, _dp]
            lib.orc_back_substitute.restype = None
            lib.orc_occupation.argtypes = [i, _dp, d, i, d, d, i, _dp, _dp]
            lib.orc_occupation.restype = i
            lib.orc_weighted_outer.argtypes = [i, i, _dp, _dp, _dp]
            lib.orc_weighted_outer.restype = None
            lib.orc_solve.argtypes = [i, i, _dp, _dp, i, d, i, d, d, i,
                                      _dp, _dp, _dp, _dp, _dp, _dp, _dp]
            lib.orc_solve.restype = i
            lib.orc_occupation_weighted.argtypes = [i, _dp, _dp, d, i, d, d, i, _dp, _dp]
            lib.orc_occupation_weighted.restype = i
            lib.orc_num_threads.argtypes = []
            lib.orc_num_threads.restype = i
            _lib = lib
    return _lib


def _f64(a) -> np.ndarray:
    return np.asfortranarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def num_threads() -> int:
    return int(_load().orc_num_threads())


class OracleError(RuntimeError):
    pass


def cholesky(s):
    s = _f64(s)
    n = s.shape[0]
    l = np.zeros((n, n), order="F")
    rc = _load().orc_cholesky(n, _ptr(s), _ptr(l))
    if rc:
        raise OracleError(f"S not positive definite at pivot {rc - 1}")
    return l


def standard_form(h, l):
    h, l = _f64(h), _f64(l)
    n = h.shape[0]
    ht = np.zeros((n, n), order="F")
    _load().orc_standard_form(n, _ptr(h), _ptr(l), _ptr(ht))
    return ht


def jacobi(a, max_sweeps: int = 60, sort: bool = True):
    """Eigenpairs of symmetric a by cyclic Jacobi. Returns (w, V, sweeps)."""
    a = np.array(_f64(a), order="F", copy=True)
    n = a.shape[0]
    w = np.zeros(n)
    v = np.zeros((n, n), order="F")
    sweeps = _load().orc_jacobi(n, _ptr(a), _ptr(w), _ptr(v), max_sweeps)
    if sweeps < 0:
        raise OracleError("Jacobi did not converge")
    if sort:
        _load().orc_sort_eigenpairs(n, _ptr(w), _ptr(v))
    return w, v, sweeps


def back_substitute(l, vt, k: int | None = None):
    l, vt = _f64(l), _f64(vt)
    n = l.shape[0]
    k = vt.shape[1] if k is None else k
    c = np.zeros((n, k), order="F")
    _load().orc_back_substitute(n, k, _ptr(l), _ptr(vt), _ptr(c))
    return c


SCHEME_INTEGER, SCHEME_GAUSSIAN, SCHEME_FERMI = 0, 1, 2
SCHEME_MP0, SCHEME_MP1 = 3, 4  # Methfessel-Paxton of order 0 (= Gaussian) and 1


def occupation(eps, n_el: float, scheme: int = SCHEME_INTEGER, kt: float = 0.0,
               occ_accuracy: float = 1e-12, mu_max_steps: int = 200):
    """Returns (f, mu) for the ascending eigenvalues eps."""
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    k = eps.shape[0]
    f = np.zeros(k)
    mu = ctypes.c_double(0.0)
    rc = _load().orc_occupation(k, _ptr(eps), float(n_el), int(scheme), float(kt),
                                float(occ_accuracy), int(mu_max_steps), _ptr(f),
                                ctypes.byref(mu))
    if rc:
        raise OracleError("occupation failed")
    return f, mu.value


def occupation_weighted(eps, wt, n_el: float, scheme: int = SCHEME_INTEGER, kt: float = 0.0,
                        occ_accuracy: float = 1e-12, mu_max_steps: int = 200):
    """One chemical potential over weighted entries (any order). Returns (f, mu)."""
    eps = np.ascontiguousarray(eps, dtype=np.float64)
    wt = np.ascontiguousarray(wt, dtype=np.float64)
    m = eps.shape[0]
    if wt.shape != (m,):
        raise ValueError("eps and wt differ in length")
    f = np.zeros(m)
    mu = ctypes.c_double(0.0)
    rc = _load().orc_occupation_weighted(m, _ptr(eps), _ptr(wt), float(n_el), int(scheme),
                                         float(kt), float(occ_accuracy), int(mu_max_steps),
                                         _ptr(f), ctypes.byref(mu))
    if rc:
        raise OracleError("weighted occupation failed")
    return f, mu.value


def weighted_outer(c, w):
    """sum_l w_l c_l c_l^T over the columns of c."""
    c = _f64(c)
    w = np.ascontiguousarray(w, dtype=np.float64)
    n, k = c.shape
    d = np.zeros((n, n), order="F")
    _load().orc_weighted_outer(n, k, _ptr(c), _ptr(w), _ptr(d))
    return d


def solve(h, s, n_state: int, n_el: float, *, unit_ovlp: bool = False,
          scheme: int = SCHEME_INTEGER, kt: float = 0.0, occ_accuracy: float = 1e-12,
          mu_max_steps: int = 200, want_pw: bool = True):
    """Whole path. Returns dict(eval (n), C (n x n_state), f, mu, P, W, energy)."""
    h = _f64(h)
    n = h.shape[0]
    s = _f64(s) if s is not None else np.eye(n, order="F")
    k = int(n_state)
    ev = np.zeros(n)
    c = np.zeros((n, k), order="F")
    f = np.zeros(k)
    p = np.zeros((n, n), order="F") if want_pw else None
    w = np.zeros((n, n), order="F") if want_pw else None
    e = ctypes.c_double(0.0)
    mu = ctypes.c_double(0.0)
    null = ctypes.cast(None, _dp)
    rc = _load().orc_solve(n, k, _ptr(h), _ptr(s), int(bool(unit_ovlp)), float(n_el),
                           int(scheme), float(kt), float(occ_accuracy), int(mu_max_steps),
                           _ptr(ev), _ptr(c), _ptr(f),
                           _ptr(p) if want_pw else null, _ptr(w) if want_pw else null,
                           ctypes.byref(e), ctypes.byref(mu))
    if rc > 0:
        raise OracleError(f"S not positive definite at pivot {rc - 1}")
    if rc == -1:
        raise OracleError("Jacobi did not converge")
    if rc == -2:
        raise OracleError("occupation failed")
    return dict(eval=ev, C=c, f=f, mu=mu.value, P=p, W=w, energy=e.value)


def embed_hermitian(a):
    """Real symmetric form [[Re A, -Im A], [Im A, Re A]] of a complex Hermitian A."""
    a = np.asarray(a, dtype=np.complex128)
    re, im = a.real, a.imag
    return np.asfortranarray(np.block([[re, -im], [im, re]]))


def solve_complex(h, s, n_state: int, n_el: float, *, unit_ovlp: bool = False,
                  scheme: int = SCHEME_INTEGER, kt: float = 0.0, occ_accuracy: float = 1e-12,
                  mu_max_steps: int = 200, want_pw: bool = True):
    """Complex Hermitian path (sec. 4.4, elsi_ev_complex / elsi_dm_complex): the real
    symmetric pencil of size 2n has each eigenvalue of (H, S) twice (eigenvectors [x; y]
    and [-y; x] for c = x + iy). The complex eigenvalue l is real eigenvalue 2l and its
    eigenvector x + iy comes from real eigenvector 2l. Occupations are computed on the
    complex eigenvalues and given to both real states of a pair, so that
    P_emb = sum f v v^T = [[Re P, -Im P], [Im P, Re P]] with P = sum_l f_l c_l c_l^H."""
    h = np.asarray(h, dtype=np.complex128)
    n = h.shape[0]
    he = embed_hermitian(h)
    se = embed_hermitian(s) if s is not None else None
    r = solve(he, se, 2 * n_state, 2.0 * n_state, unit_ovlp=unit_ovlp or s is None,
              want_pw=False)
    ev = r["eval"][0::2].copy()
    c2 = r["C"][:, 0::2]
    out = dict(eval=ev, C=c2[:n] + 1j * c2[n:], P=None, W=None)
    f, mu = occupation(ev[:n_state], n_el, scheme=scheme, kt=kt, occ_accuracy=occ_accuracy,
                       mu_max_steps=mu_max_steps)
    out.update(f=f, mu=mu, energy=float(np.sum(f * ev[:n_state])))
    if want_pw:
        f2 = np.repeat(f, 2)
        e2 = r["eval"][: 2 * n_state]
        pe = weighted_outer(r["C"], f2)
        we = weighted_outer(r["C"], f2 * e2)
        out["P"] = pe[:n, :n] + 1j * pe[n:, :n]
        out["W"] = we[:n, :n] + 1j * we[n:, :n]
    return out


def solve_batched(problems, n_el, *, weights=None, shared_mu: bool = True,
                  is_complex: bool = False, scheme: int = SCHEME_INTEGER, kt: float = 0.0,
                  occ_accuracy: float = 1e-12, mu_max_steps: int = 200, want_pw: bool = True):
    """Independent problems (h_i, s_i, n_state_i) solved one after another (sec. 2,
    SINGLE_PROC: one process handles several k-points in turn), then occupied:
      shared_mu: one mu with sum_i weights[i] sum_l f_il = n_el (a number);
      otherwise: problem i on its own with n_el[i] electrons.
    P_i = sum_l f_il c_il c_il^H and W_i = sum_l f_il eps_il c_il c_il^H (unweighted: the
    total density of a k-point sum is sum_i weights[i] P_i). Returns a list of dicts
    (eval, C, f, P, W, energy) and the chemical potential(s)."""
    out = []
    for (h, s, k) in problems:
        if is_complex:
            r = solve_complex(h, s, k, 2.0 * k, unit_ovlp=s is None, want_pw=False)
        else:
            r = solve(h, s, k, 2.0 * k, unit_ovlp=s is None, want_pw=False)
        out.append(dict(eval=r["eval"], C=r["C"]))
    if shared_mu:
        wts = np.ones(len(problems)) if weights is None else np.asarray(weights, dtype=float)
        eps = np.concatenate([o["eval"][:k] for o, (_, _, k) in zip(out, problems)])
        wt = np.concatenate([np.full(k, wts[i]) for i, (_, _, k) in enumerate(problems)])
        f, mu = occupation_weighted(eps, wt, float(n_el), scheme=scheme, kt=kt,
                                    occ_accuracy=occ_accuracy, mu_max_steps=mu_max_steps)
        off = 0
        for o, (_, _, k) in zip(out, problems):
            o["f"] = f[off:off + k]
            off += k
        mus = mu
    else:
        mus = []
        for i, (o, (_, _, k)) in enumerate(zip(out, problems)):
            f, mu = occupation(o["eval"][:k], float(n_el[i]), scheme=scheme, kt=kt,
                               occ_accuracy=occ_accuracy, mu_max_steps=mu_max_steps)
            o["f"] = f
            mus.append(mu)
    for o, (_, _, k) in zip(out, problems):
        ev = o["eval"][:k]
        o["energy"] = float(np.sum(o["f"] * ev))
        if want_pw:
            c = o["C"]
            if is_complex:
                o["P"] = (c * o["f"]) @ c.conj().T
                o["W"] = (c * (o["f"] * ev)) @ c.conj().T
            else:
                o["P"] = weighted_outer(c, o["f"])
                o["W"] = weighted_outer(c, o["f"] * ev)
    return out, mus


def entropy_term(eps, f, mu: float, scheme: int, kt: float) -> float:
    """-kT S_ent, the entropy contribution to the Mermin free energy F = E_band - kT S_ent
    (the paper names the broadening schemes, sec. 4.4, but gives no entropy; this is the
    term for which dF/deps_l = f_l at fixed electron count, so that dF/dH = P):
      Fermi-Dirac: S_ent = -g sum_l [phi ln phi + (1 - phi) ln(1 - phi)], phi = f_l / g;
      Gaussian and Methfessel-Paxton order 0:
                   S_ent = g sum_l exp(-x_l^2) / (2 sqrt(pi)), x_l = (eps_l - mu) / kT;
      Methfessel-Paxton order 1 (Phys. Rev. B 40, 3616 (1989)):
                   S_ent = g sum_l (1/2) A_1 H_2(x_l) exp(-x_l^2);
      integer:     0."""
    g = 2.0
    eps = np.asarray(eps, dtype=float)
    f = np.asarray(f, dtype=float)
    if scheme == SCHEME_INTEGER:
        return 0.0
    if scheme == SCHEME_FERMI:
        phi = f / g
        s = 0.0
        for p in phi:
            if 0.0 < p < 1.0:
                s += p * np.log(p) + (1.0 - p) * np.log1p(-p)
        return float(kt * g * s)
    x = (eps - mu) / kt
    if scheme == SCHEME_MP1:
        # Methfessel-Paxton order N: S_ent = g sum_l (1/2) A_N H_{2N}(x_l) exp(-x_l^2);
        # N = 1: A_1 = -1 / (4 sqrt(pi)), H_2(x) = 4 x^2 - 2
        s_l = 0.5 * (-1.0 / (4.0 * np.sqrt(np.pi))) * (4.0 * x * x - 2.0) * np.exp(-x * x)
        return float(-kt * g * np.sum(s_l))
    return float(-kt * g * np.sum(np.exp(-x * x)) / (2.0 * np.sqrt(np.pi)))


def free_energy(h, s, n_state: int, n_el: float, *, scheme: int = SCHEME_FERMI,
                kt: float = 0.01, want_pw: bool = True, **kw):
    """F = E_band - kT S_ent and the solve it comes from (dict of solve plus 'F')."""
    r = solve(h, s, n_state, n_el, scheme=scheme, kt=kt, want_pw=want_pw, **kw)
    r["F"] = r["energy"] + entropy_term(r["eval"][:n_state], r["f"], r["mu"], scheme, kt)
    return r


def ev_adjoint(ev, c, ev_bar=None, c_bar=None, guard: float = 1e-10):
    """Reverse-mode derivative of the generalized symmetric eigenproblem H C = S C diag(ev),
    C^T S C = I (all n eigenpairs in c), for a loss with dL/d ev = ev_bar (length n) and
    dL/d C[:, :k] = c_bar (n x k). Perturbation theory (first order) gives, with
    M = C^T dH C and N = C^T dS C,
      d ev_j = M_jj - ev_j N_jj,
      dC = C Omega,  Omega_ij = (M_ij - ev_j N_ij) / (ev_j - ev_i) (i != j),
                     Omega_jj = -N_jj / 2,
    so that dL = <X_H, M> + <X_S, N> with A = C^T c_bar (n x k), F_ij = 1/(ev_j - ev_i)
    (0 for i = j or |ev_i - ev_j| < guard: the degeneracy guard),
      X_H = diag(ev_bar) + [F o A | 0],
      X_S = -diag(ev_bar ev) - [(F o A) diag(ev_k) | 0] - diag(A_jj / 2, j < k),
    and dL/dH = C sym(X_H) C^T, dL/dS = C sym(X_S) C^T (sym(X) = (X + X^T)/2: the
    gradient with respect to a symmetric matrix)."""
    ev = np.asarray(ev, dtype=float)
    c = np.asarray(c, dtype=float)
    n = ev.shape[0]
    xh = np.zeros((n, n))
    xs = np.zeros((n, n))
    if ev_bar is not None:
        eb = np.asarray(ev_bar, dtype=float)
        xh[np.arange(n), np.arange(n)] += eb
        xs[np.arange(n), np.arange(n)] -= eb * ev
    if c_bar is not None:
        cb = np.asarray(c_bar, dtype=float)
        k = cb.shape[1]
        a = c.T @ cb
        d = ev[None, :k] - ev[:, None]
        fm = np.zeros((n, k))
        ok = np.abs(d) >= guard
        fm[ok] = 1.0 / d[ok]
        fa = fm * a
        xh[:, :k] += fa
        xs[:, :k] -= fa * ev[None, :k]
        xs[np.arange(k), np.arange(k)] -= 0.5 * a[np.arange(k), np.arange(k)]
    hb = c @ (0.5 * (xh + xh.T)) @ c.T
    sb = c @ (0.5 * (xs + xs.T)) @ c.T
    return hb, sb


SING_FILL = np.finfo(np.float64).max  # eigenvalue slots of dropped basis directions


def canonical_transform(s, tau: float, force: bool = False):
    """Singularity check of the overlap matrix (sec. 4.4, Eq. 10): all eigenvalues of S by
    Jacobi; when one or more are below tau (or force), S = X X^T with X = x sqrt(lambda) and
    the eigenvectors with lambda < tau dropped, which gives the transformation
    U = x_k lambda_k^{-1/2} (n x N_nonsing): H~ = U^T H U and c = U c~.
    Returns (U or None when S is not singular and not force, eigenvalues of S)."""
    w, v, _ = jacobi(s)
    keep = w >= tau
    if keep.all() and not force:
        return None, w
    return np.asfortranarray(v[:, keep] / np.sqrt(w[keep])), w


def solve_sing(h, s, n_state: int, n_el: float, *, tau: float = 1e-5, force: bool = False,
               scheme: int = SCHEME_INTEGER, kt: float = 0.0, occ_accuracy: float = 1e-12,
               mu_max_steps: int = 200, want_pw: bool = True):
    """Whole path with the singularity check: the Cholesky route when S has no eigenvalue
    below tau (and not force), else the reduced standard problem H~ = U^T H U of size
    N_nonsing, eigenvectors c = U c~. eval has length n; the slots of the dropped
    directions (l >= N_nonsing) hold SING_FILL."""
    h = _f64(h)
    n = h.shape[0]
    u, ws = canonical_transform(s, tau, force)
    if u is None:
        r = solve(h, s, n_state, n_el, scheme=scheme, kt=kt, occ_accuracy=occ_accuracy,
                  mu_max_steps=mu_max_steps, want_pw=want_pw)
        r.update(n_nonsing=n, s_eval=ws)
        return r
    nn = u.shape[1]
    k = int(n_state)
    if k > nn:
        raise OracleError("n_state exceeds the non-singular basis size")
    ht = u.T @ h @ u
    ht = 0.5 * (ht + ht.T)
    w, z, _ = jacobi(ht)
    c = np.asfortranarray(u @ z[:, :k])
    ev = np.full(n, SING_FILL)
    ev[:nn] = w
    f, mu = occupation(w[:k], n_el, scheme=scheme, kt=kt, occ_accuracy=occ_accuracy,
                       mu_max_steps=mu_max_steps)
    out = dict(eval=ev, C=c, f=f, mu=mu, energy=float(np.sum(f * w[:k])), n_nonsing=nn,
               s_eval=ws, P=None, W=None)
    if want_pw:
        out["P"] = weighted_outer(c, f)
        out["W"] = weighted_outer(c, f * w[:k])
    return out
