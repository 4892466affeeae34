"""The binary32 back-transformation through Q2 (step (4) of the two-stage reduction) on the
tensor cores, against its definition applied in binary64 with numpy.

Random Householder reflectors stand in for the bulge chase's: reflector (sweep j, step t)
has v[0] = 1 and acts on rows j+1+tb .. j+tb+b (cut at row n-1), tau = 2 / v^T v, so every
H = I - tau v v^T is orthogonal. Q2 is their product in the order the sequential chase
generates them (sweep 0 steps 0, 1, ..., then sweep 1, ...), so Z <- Q2 Z applies them in
the reverse order. Sizes: n not a multiple of 64 or 8, k not a multiple of 128 (ragged
column tile), band widths 8, 40, 64.

The reference applies the reflectors as the kernel receives them (rounded to binary32),
in binary64, so the comparison measures the kernel's arithmetic alone: binary32 values
carried through about 2n/64 group applications per element (each a product of the group's
TF32 hi/lo splits, about binary32 accuracy) leave a relative error of a few 1e-6 at
n ~ 1000; the bound is 2e-5."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1705_11191_gb300 as egb  # noqa: E402


def _lib():
    lib = egb.load()
    v = ctypes.c_void_p
    lib.elsi_gb_q2_work.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.elsi_gb_q2_work.restype = ctypes.c_size_t
    lib.elsi_gb_q2_apply_f32.argtypes = [ctypes.c_int, ctypes.c_int, v, v, ctypes.c_int, v,
                                         ctypes.c_int, v, ctypes.c_size_t, v, v]
    lib.elsi_gb_q2_apply_f32.restype = ctypes.c_int
    return lib


def _reflectors(n, b, seed):
    rng = np.random.default_rng(seed)
    S = (n - 2) // b + 1
    v2 = np.zeros(((n - 2) * S, b))
    tau = np.zeros((n - 2) * S)
    for j in range(n - 2):
        for t in range((n - 2 - j) // b + 1):
            r = j + 1 + t * b
            L = min(b, n - r)
            if L <= 0:
                continue
            v = np.zeros(b)
            v[0] = 1.0
            v[1:L] = 0.4 * rng.standard_normal(L - 1)
            v2[j * S + t] = v
            tau[j * S + t] = 2.0 / float(v[:L] @ v[:L])
    return v2, tau, S


def _apply_ref(n, b, v2, tau, S, z):
    z = z.copy()
    for j in range(n - 3, -1, -1):
        for t in range((n - 2 - j) // b, -1, -1):
            r = j + 1 + t * b
            L = min(b, n - r)
            if L <= 0:
                continue
            v = v2[j * S + t, :L]
            z[r:r + L] -= tau[j * S + t] * np.outer(v, v @ z[r:r + L])
    return z


@pytest.mark.parametrize("n,b,k,seed", [(300, 64, 200, 1), (517, 40, 130, 2), (261, 8, 77, 3),
                                        (1100, 64, 300, 4)])
def test_q2_tensor_core_matches_binary64(n, b, k, seed):
    lib = _lib()
    v2, tau, S = _reflectors(n, b, seed)
    rng = np.random.default_rng(100 + seed)
    z0 = rng.standard_normal((n, k))
    v32, t32, z32 = v2.astype(np.float32), tau.astype(np.float32), z0.astype(np.float32)
    ref = _apply_ref(n, b, v32.astype(np.float64), t32.astype(np.float64), S, z32.astype(np.float64))
    dv2 = torch.from_numpy(v32).cuda().contiguous()
    dtau = torch.from_numpy(t32).cuda()
    zt = torch.from_numpy(np.asfortranarray(z32).T.copy()).cuda()  # (k, n) = n x k column-major
    work = torch.zeros(lib.elsi_gb_q2_work(n, b) + 16, dtype=torch.float32, device="cuda")
    st = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = lib.elsi_gb_q2_apply_f32(n, b, dv2.data_ptr(), dtau.data_ptr(), k, zt.data_ptr(), n,
                                  work.data_ptr(), work.numel(), st.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    assert rc == 0
    assert int(st[0]) == 0
    out = zt.cpu().numpy().T.astype(np.float64)
    err = float(np.linalg.norm(out - ref) / np.linalg.norm(ref))
    print(f"n={n} b={b} k={k}: relative error {err:.2e}")
    assert err < 2e-5
