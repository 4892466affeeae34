"""The symmetric panel product X = A V of the full-to-band reduction (A symmetric m x m,
V m x nv, nv <= 64; binary32 on the tensor cores, A split in shared memory, stream-K over
the SMs) against a float64 product of the same binary32 inputs.

Bound per element: 1e-5 (|A| |V|)_ic, which covers the TF32 split (about 2^-21 relative
per product term, the lo*lo term dropped) and binary32 accumulation over chunks of 64
along K (at most 2 (64 + m/64) 2^-24 relative to the sum of |terms|); a missing cross
term (2^-11) or a wrong partial tile exceeds it. Entries of X outside m x nv stay as
they were."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1705_11191_gb300 as egb  # noqa: E402


def _lib():
    lib = egb.load()
    v = ctypes.c_void_p
    lib.elsi_gb_symm_tall_f32_work.argtypes = [ctypes.c_int]
    lib.elsi_gb_symm_tall_f32_work.restype = ctypes.c_size_t
    lib.elsi_gb_symm_tall_f32.argtypes = [ctypes.c_int, ctypes.c_int, v, ctypes.c_int, v, ctypes.c_int,
                                          v, ctypes.c_int, v, ctypes.c_size_t, v, v]
    lib.elsi_gb_symm_tall_f32.restype = ctypes.c_int
    return lib


def _run(m, nv, seed, lda=None, ldv=None, ldx=None, scale_rows=False):
    lib = _lib()
    lda = lda or ((m + 3) // 4) * 4
    ldv = ldv or m + 3
    ldx = ldx or m + 5
    g = torch.Generator(device="cpu").manual_seed(seed)
    S = torch.randn(m, m, generator=g, dtype=torch.float64)
    S = S + S.t()
    if scale_rows:
        d = torch.pow(10.0, torch.empty(m, dtype=torch.float64).uniform_(-3, 3, generator=g))
        S = d[:, None] * S * d[None, :]
    Af = S.float()
    # column-major storage with leading dimension lda: a (m, lda) row-major tensor, row j =
    # column j
    Abuf = torch.full((m, lda), float("nan"), dtype=torch.float32)
    Abuf[:, :m] = Af.t()
    Vf = torch.randn(nv, ldv, generator=g, dtype=torch.float32)
    Vf[:, m:] = float("nan")
    X = torch.full((nv, ldx), 7.0, dtype=torch.float32)
    dA, dV, dX = Abuf.cuda(), Vf.cuda(), X.cuda()
    w = torch.zeros(lib.elsi_gb_symm_tall_f32_work(m) + 16, dtype=torch.float32, device="cuda")
    st = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = lib.elsi_gb_symm_tall_f32(m, nv, dA.data_ptr(), lda, dV.data_ptr(), ldv, dX.data_ptr(), ldx,
                                   w.data_ptr(), w.numel(), st.data_ptr(), None)
    torch.cuda.synchronize()
    assert rc == 0
    assert int(st[0]) == 0
    A64 = Af.double()
    V64 = Vf[:, :m].double().t()                   # m x nv
    ref = A64 @ V64
    bound = 1e-5 * (A64.abs() @ V64.abs())
    got = dX.cpu()
    err = (got[:, :m].double().t() - ref).abs()
    assert bool((err <= bound).all()), float((err / bound).max())
    assert bool((got[:, m:] == 7.0).all())
    return float((err / bound).max())


@pytest.mark.parametrize("m,nv", [(1, 1), (100, 8), (300, 33), (1000, 64), (4099, 64), (2051, 16)])
def test_symmetric_panel_product(m, nv):
    _run(m, nv, seed=m + nv)


def test_graded_magnitudes():
    _run(777, 64, seed=5, scale_rows=True)


def test_leading_dimensions():
    _run(513, 40, seed=6, lda=520, ldv=600, ldx=700)


def test_unaligned_leading_dimension_rejected():
    lib = _lib()
    m = 64
    A = torch.zeros(m * 67, dtype=torch.float32, device="cuda")
    V = torch.zeros(m * 64, dtype=torch.float32, device="cuda")
    X = torch.zeros(m * 64, dtype=torch.float32, device="cuda")
    w = torch.zeros(lib.elsi_gb_symm_tall_f32_work(m) + 16, dtype=torch.float32, device="cuda")
    st = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = lib.elsi_gb_symm_tall_f32(m, 8, A.data_ptr(), 67, V.data_ptr(), m, X.data_ptr(), m,
                                   w.data_ptr(), w.numel(), st.data_ptr(), None)
    assert rc == 1  # ELSI_ERR_ARG: lda not a multiple of 4
