"""GPU parity of the sparse (PEXSI_CSC) entry points (sec. 3.2 Fig. 2, sec. 4.3-4.4:
elsi_set_csc, elsi_ev_real_sparse, elsi_dm_real_sparse, elsi_get_edm_real_sparse)
against the oracle on the matrices the pattern describes: eigenvalues 1e-10, P and W at
the pattern's positions 1e-9 relative, 0- and 1-based indices, host or device index
arrays, and the argument errors."""
import numpy as np
import pytest
import scipy.sparse as sp

import ksinputs
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1705_11191_gb300 as egb  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _sparse_problem(n, seed, thr=2e-3):
    p = ksinputs.cluster_problem(n, seed=seed)
    mask = (np.abs(p.h) > thr) | (np.abs(p.s) > thr) | np.eye(n, dtype=bool)
    mask = mask | mask.T
    hs, ss = np.where(mask, p.h, 0.0), np.where(mask, p.s, 0.0)
    assert np.linalg.eigvalsh(ss)[0] > 1e-3
    pat = sp.csc_matrix(mask.astype(np.float64))
    pat.sort_indices()
    rows, colp = pat.indices.astype(np.int32), pat.indptr.astype(np.int32)
    cols = np.repeat(np.arange(n), np.diff(colp))
    return p, hs, ss, rows, colp, cols


def _t(a, device="cuda"):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device)


@pytest.mark.parametrize("base,where,prec", [(0, "cuda", 0), (1, "cpu", 0), (0, "cuda", 1)])
def test_dm_sparse_parity(base, where, prec):
    p, hs, ss, rows, colp, cols = _sparse_problem(140, 81)
    assert rows.size < 0.9 * p.n * p.n  # really sparse
    ref = oracle.solve(hs, ss, p.n_state, p.n_electron)
    with egb.Handle(p.n, p.n_state, p.n_electron) as hd:
        hd.use_current_stream()
        hd.set_band_width(32)
        hd.set_precision(prec)
        hd.set_csc(_t(rows + base, where), _t(colp + base, where), index_base=base)
        Pv, e = hd.dm_real_sparse(_t(hs[rows, cols]), _t(ss[rows, cols]))
        Wv = hd.get_edm_sparse()
    assert rel(Pv.cpu().numpy(), ref["P"][rows, cols]) <= 1e-9
    assert rel(Wv.cpu().numpy(), ref["W"][rows, cols]) <= 1e-9
    assert abs(e - ref["energy"]) <= 1e-9 * abs(ref["energy"])


def test_ev_sparse_parity():
    p, hs, ss, rows, colp, cols = _sparse_problem(100, 82)
    ref = oracle.solve(hs, ss, p.n_state, p.n_electron, want_pw=False)
    with egb.Handle(p.n, p.n_state, p.n_electron) as hd:
        hd.use_current_stream()
        hd.set_band_width(16)
        hd.set_csc(_t(rows), _t(colp))
        ev, C = hd.ev_real_sparse(_t(hs[rows, cols]), _t(ss[rows, cols]))
    ev, C = ev.cpu().numpy(), C.cpu().numpy()
    np.testing.assert_allclose(ev, ref["eval"], rtol=0, atol=1e-10)
    np.testing.assert_allclose(C.T @ ss @ C, np.eye(p.n_state), rtol=0, atol=1e-10)


def test_csc_errors():
    p, hs, ss, rows, colp, cols = _sparse_problem(40, 83)
    with egb.Handle(p.n, p.n_state, p.n_electron) as hd:
        hd.use_current_stream()
        with pytest.raises(egb.ElsiError) as ei:
            hd.dm_real_sparse(_t(hs[rows, cols]), _t(ss[rows, cols]))
        assert ei.value.code == 8  # no pattern yet
        bad = rows.copy()
        bad[5] = p.n
        with pytest.raises(egb.ElsiError) as ei:
            hd.set_csc(_t(bad), _t(colp))
        assert ei.value.code == 1
        badc = colp.copy()
        badc[3], badc[4] = badc[4], badc[3] - 1
        with pytest.raises(egb.ElsiError) as ei:
            hd.set_csc(_t(rows), _t(badc))
        assert ei.value.code == 1
        # a valid pattern afterwards works
        hd.set_csc(_t(rows), _t(colp))
        Pv, e = hd.dm_real_sparse(_t(hs[rows, cols]), _t(ss[rows, cols]))
    ref = oracle.solve(hs, ss, p.n_state, p.n_electron)
    assert rel(Pv.cpu().numpy(), ref["P"][rows, cols]) <= 1e-9
