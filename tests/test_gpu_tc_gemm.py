"""The binary32 tensor-core GEMM (tcgen05, three TF32 products of hi/lo splits) against a
plain PyTorch float64 product of the same binary32 inputs: every transpose combination,
ragged tails in m, n and k, beta != 0, and the lower-triangle mode. The tolerance
3e-6 * ||op(A)|| ||op(B)|| per element bounds the split error (2^-21 relative per
product term) plus binary32 accumulation over k <= 1024."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1705_11191_gb300 as egb  # noqa: E402


def _lib():
    lib = egb.load()
    lib.elsi_gb_gemm_f32_work.argtypes = [ctypes.c_int] * 3
    lib.elsi_gb_gemm_f32_work.restype = ctypes.c_size_t
    v = ctypes.c_void_p
    lib.elsi_gb_gemm_f32.argtypes = [ctypes.c_int] * 5 + [ctypes.c_float, v, ctypes.c_int, v,
                                                          ctypes.c_int, ctypes.c_float, v,
                                                          ctypes.c_int, ctypes.c_int, v,
                                                          ctypes.c_size_t, v, v]
    lib.elsi_gb_gemm_f32.restype = ctypes.c_int
    return lib


def _run(ta, tb, m, n, k, alpha=1.0, beta=0.0, uplo=0, seed=0):
    lib = _lib()
    g = torch.Generator(device="cpu").manual_seed(seed)
    # column-major storage: a tensor of shape (cols, rows) row-major is the same memory
    ar, ac = (m, k) if ta == 0 else (k, m)
    br, bc = (k, n) if tb == 0 else (n, k)
    A = torch.randn(ac, ar, generator=g, dtype=torch.float32).cuda()
    B = torch.randn(bc, br, generator=g, dtype=torch.float32).cuda()
    C = torch.randn(n, m, generator=g, dtype=torch.float32).cuda()
    C0 = C.clone()
    w = torch.zeros(lib.elsi_gb_gemm_f32_work(m, n, k) + 16, dtype=torch.float32, device="cuda")
    st = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = lib.elsi_gb_gemm_f32(ta, tb, m, n, k, alpha, A.data_ptr(), ar, B.data_ptr(), br, beta,
                              C.data_ptr(), m, uplo, w.data_ptr(), w.numel(), st.data_ptr(), None)
    torch.cuda.synchronize()
    assert rc == 0
    assert int(st[0]) == 0
    opA = A.double().t() if ta == 0 else A.double()        # (m, k)
    opB = B.double().t() if tb == 0 else B.double()        # (k, n)
    ref = alpha * opA @ opB + beta * C0.double().t()       # (m, n)
    got = C.double().t()
    tol = 3e-6 * np.sqrt(k) * 1.0 + 1e-6
    if uplo:
        mask = torch.tril(torch.ones(m, n, dtype=torch.bool, device="cuda"))
        assert torch.equal(got[~mask], C0.double().t()[~mask])
        got, ref = got[mask], ref[mask]
    err = (got - ref).abs().max().item()
    assert err <= tol * max(1.0, abs(alpha)) * 4, err
    return err


@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_transposes_ragged(ta, tb):
    _run(ta, tb, 200, 130, 70, seed=ta * 2 + tb)


def test_exact_tiles_and_beta():
    _run(0, 0, 256, 384, 128, alpha=-1.0, beta=1.0, seed=5)


def test_lower_triangle_mode():
    _run(0, 1, 300, 300, 96, alpha=0.5, beta=0.25, uplo=1, seed=6)


def test_large_k():
    _run(1, 0, 512, 256, 1024, seed=7)


def test_small_shapes():
    _run(0, 0, 1, 1, 1, seed=8)
    _run(0, 0, 17, 5, 3, beta=1.0, seed=9)
