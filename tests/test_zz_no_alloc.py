"""GPU test of elsi_density_noalloc, the allocation-free entry point for callers that
cannot allocate GPU memory when they need the density matrices (memory owned by another
framework's pre-sized pool, loops that forbid allocation after start-up). It is called through the C ABI (ctypes) and checked
against the density matrices of the regular elsi_dm_real / elsi_get_edm_real entry points
on two calls in a row, within the binary64 parity tolerance (1e-9 relative Frobenius).
This file is collected last on purpose (test_zz_*)."""
import ctypes

import numpy as np
import pytest

import ksinputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1705_11191_gb300 as egb  # noqa: E402

TOL = 1e-9


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def rel(a, b):
    return float(torch.linalg.norm(a - b) / torch.linalg.norm(b))


def _reference(p):
    """Orbitals from elsi_ev_real and P, W from elsi_dm_real of the same problem."""
    with egb.Handle(p.n, p.n_state, p.n_electron) as hd:
        hd.use_current_stream()
        ev, vec = hd.ev_real(dev(p.h), dev(p.s))
    with egb.Handle(p.n, p.n_state, p.n_electron) as hd:
        hd.use_current_stream()
        P, _ = hd.dm_real(dev(p.h), dev(p.s))
        W = hd.get_edm()
        f = hd.get_occ()
    return ev[: p.n_state].contiguous(), vec.t().contiguous(), f, P, W


def _call(n, k, evec_t, f, ev, P, W):
    lib = egb.load()
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.elsi_density_noalloc(n, k, ctypes.c_void_p(evec_t.data_ptr()),
                                  ctypes.c_void_p(f.data_ptr()), ctypes.c_void_p(ev.data_ptr()),
                                  ctypes.c_void_p(P.data_ptr()),
                                  ctypes.c_void_p(W.data_ptr() if W is not None else None),
                                  ctypes.c_void_p(stream))
    torch.cuda.synchronize()
    return rc


def test_noalloc_density_matches_dm_real_twice():
    cases = [ksinputs.cluster_problem(300, seed=41), ksinputs.cluster_problem(180, seed=42)]
    for p in cases:  # two calls in a row, different sizes: stale scratch would show
        ev, evec_t, f, P_ref, W_ref = _reference(p)
        P = torch.full((p.n, p.n), float("nan"), dtype=torch.float64, device="cuda")
        W = torch.full((p.n, p.n), float("nan"), dtype=torch.float64, device="cuda")
        # evec_t is (n_state, n) row-major == n x n_state column-major
        rc = _call(p.n, p.n_state, evec_t, f, ev, P, W)
        assert rc == 0
        assert rel(P, P_ref) <= TOL
        assert rel(W, W_ref) <= TOL


def test_noalloc_size_limit_boundary():
    """n_basis * n_state = 2^21 (the scratch size) is accepted and correct."""
    n, k = 2048, 1024
    g = torch.Generator(device="cuda").manual_seed(7)
    evec_t = torch.randn((k, n), dtype=torch.float64, device="cuda", generator=g) / n ** 0.5
    f = torch.rand(k, dtype=torch.float64, device="cuda", generator=g) * 2.0
    ev = torch.randn(k, dtype=torch.float64, device="cuda", generator=g)
    P = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    W = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    assert _call(n, k, evec_t, f, ev, P, W) == 0
    C = evec_t.t()  # n x k
    # P, W are column-major n x n, i.e. the row-major tensors hold P^T = P
    assert rel(P, (C * f) @ C.t()) <= TOL
    assert rel(W, (C * (f * ev)) @ C.t()) <= TOL


def test_noalloc_rejects_oversize_and_bad_args():
    lib = egb.load()
    null = ctypes.c_void_p(None)
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    ptr = ctypes.c_void_p(x.data_ptr())
    # n_basis * n_state = 16257 * 129 = 2^21 + 1 entries: one more than the fixed scratch
    assert 16257 * 129 == (1 << 21) + 1
    assert lib.elsi_density_noalloc(16257, 129, ptr, ptr, ptr, ptr, null, null) == 10
    assert lib.elsi_density_noalloc(0, 1, ptr, ptr, ptr, ptr, null, null) == 1
    assert lib.elsi_density_noalloc(4, 2, ptr, ptr, null, ptr, ptr, null) == 1  # edm w/o eval
