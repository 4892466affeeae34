"""The binary32 panel factorisation of the full-to-band reduction (tall-skinny QR with
Householder reconstruction) against the defining properties of a Householder QR with
compact-WY factors, checked in binary64 with numpy:
  (I - V T V^T)[:, :b] R = P   (the panel is reproduced),
  T + T^T = T^T (V^T V) T      (I - V T V^T is orthogonal; the identity is that of
                                (I - V T^T V^T)(I - V T V^T) = I for full-rank V),
  V unit lower trapezoidal, T and R upper triangular.
Sizes: m from just above one block (257 rows) to a four-level tree, ragged last blocks,
b = 64 and 32. Tolerances follow binary32 arithmetic over a 64-column factorisation:
1e-5 relative for the reproduction, 1e-5 for the orthogonality identity (relative to
||T||^2 ||V||^2)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1705_11191_gb300 as egb  # noqa: E402


def _lib():
    lib = egb.load()
    v = ctypes.c_void_p
    lib.elsi_gb_tsqr_work.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.elsi_gb_tsqr_work.restype = ctypes.c_size_t
    lib.elsi_gb_tsqr_panel_f32.argtypes = [ctypes.c_int, ctypes.c_int, v, ctypes.c_int, v, ctypes.c_int,
                                           v, ctypes.c_int, v, ctypes.c_size_t, v]
    lib.elsi_gb_tsqr_panel_f32.restype = ctypes.c_int
    return lib


@pytest.mark.parametrize("m,b,seed", [(257, 64, 1), (1000, 64, 2), (4133, 32, 3), (16320, 64, 4)])
def test_tsqr_panel_is_a_householder_qr(m, b, seed):
    lib = _lib()
    rng = np.random.default_rng(seed)
    P0 = rng.standard_normal((m, b)).astype(np.float32)
    P0[:, 3] *= 1e-3  # uneven column scales
    P = torch.from_numpy(np.asfortranarray(P0).T.copy()).cuda()  # (b, m) = m x b column-major
    V = torch.full((b, m), float("nan"), dtype=torch.float32, device="cuda")
    T = torch.zeros((b, b), dtype=torch.float32, device="cuda")
    work = torch.zeros(lib.elsi_gb_tsqr_work(m, b), dtype=torch.float32, device="cuda")
    rc = lib.elsi_gb_tsqr_panel_f32(m, b, P.data_ptr(), m, V.data_ptr(), m, T.data_ptr(), b,
                                    work.data_ptr(), work.numel(), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == 0
    Rm = P.cpu().numpy().T.astype(np.float64)   # m x b
    Vm = V.cpu().numpy().T.astype(np.float64)   # m x b
    Tm = T.cpu().numpy().T.astype(np.float64)   # b x b
    R = Rm[:b]
    assert np.all(np.tril(R, -1) == 0) and np.all(Rm[b:] == 0)
    assert np.all(np.triu(Vm[:b], 1) == 0) and np.all(np.diag(Vm[:b]) == 1.0)
    assert np.all(np.tril(Tm, -1) == 0)
    # (I - V T V^T)[:, :b] R
    E = np.zeros((m, b))
    E[:b] = np.eye(b)
    Q = E - Vm @ (Tm @ Vm[:b].T)
    rec = Q @ R
    assert np.linalg.norm(rec - P0) / np.linalg.norm(P0) < 1e-5
    G = Vm.T @ Vm
    lhs = Tm + Tm.T
    rhs = Tm.T @ G @ Tm
    scale = np.linalg.norm(Tm) ** 2 * np.linalg.norm(G)
    assert np.linalg.norm(lhs - rhs) / scale < 1e-5
