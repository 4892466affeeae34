"""The binary64-accurate digit product (Ozaki splitting into signed 7-bit digits, exact
bf16 digit products on the tcgen05 tensor cores) through its testing entry.

Pins that do not depend on another floating-point product:
- dyadic inputs (integers of at most 11 bits times a power of two) have at most two
  nonzero digits per entry and an exact binary64 product, so the digit product must equal
  numpy's float64 product bit for bit, for every transpose pair, ragged m, n, k, beta,
  alpha and the lower-triangle mode;
- constant matrices whose level-2 digit sums pass 2^31 over the whole K (K = 140 000 >
  131 072 = 2^31 / 128^2) must still give k x^2 (the K segments keep each int32 level
  sum exact);
- random normal data against a binary128 (or x87 extended) product: the error is within
  the truncation bound k 2^(e_i + f_j) 2^(-7 D + 3) for D digits (e_i, f_j the power-of-two
  scales of row i of op(A) and column j of op(B)), and with 7 digits it is at the binary64
  level.
"""
import ctypes
from fractions import Fraction

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1705_11191_gb300 as egb  # noqa: E402


def _lib():
    lib = egb.load()
    v = ctypes.c_void_p
    lib.elsi_gb_gemm_f64_digits_planes.argtypes = [ctypes.c_int] * 3
    lib.elsi_gb_gemm_f64_digits_planes.restype = ctypes.c_size_t
    lib.elsi_gb_gemm_f64_digits_exps.argtypes = [ctypes.c_int] * 2
    lib.elsi_gb_gemm_f64_digits_exps.restype = ctypes.c_size_t
    lib.elsi_gb_gemm_f64_digits.argtypes = (
        [ctypes.c_int] * 5 + [ctypes.c_double, v, ctypes.c_int, v, ctypes.c_int, ctypes.c_double, v,
                              ctypes.c_int, ctypes.c_int, ctypes.c_int, v, ctypes.c_size_t, v,
                              ctypes.c_size_t, v, v])
    lib.elsi_gb_gemm_f64_digits.restype = ctypes.c_int
    return lib


def _digits_gemm(ta, tb, A, B, C, alpha, beta, uplo, digits):
    """A, B, C: numpy float64 arrays in the shapes op() expects before transposition
    (A is m x k if ta == 0 else k x m). Returns the new C (m x n)."""
    lib = _lib()
    m = A.shape[1] if ta else A.shape[0]
    k = A.shape[0] if ta else A.shape[1]
    n = B.shape[0] if tb else B.shape[1]
    # column-major device copies: the transpose of a C-contiguous array
    dA = torch.from_numpy(np.ascontiguousarray(A.T)).cuda()
    dB = torch.from_numpy(np.ascontiguousarray(B.T)).cuda()
    dC = torch.from_numpy(np.ascontiguousarray(C.T)).cuda()
    npl = lib.elsi_gb_gemm_f64_digits_planes(m, n, k)
    nex = lib.elsi_gb_gemm_f64_digits_exps(m, n)
    planes = torch.zeros(npl + 8, dtype=torch.bfloat16, device="cuda")
    exps = torch.zeros(nex, dtype=torch.int32, device="cuda")
    st = torch.zeros(8, dtype=torch.int32, device="cuda")
    rc = lib.elsi_gb_gemm_f64_digits(ta, tb, m, n, k, alpha, dA.data_ptr(), A.shape[0],
                                     dB.data_ptr(), B.shape[0], beta, dC.data_ptr(), m, uplo,
                                     digits, planes.data_ptr(), planes.numel(), exps.data_ptr(),
                                     exps.numel(), st.data_ptr(), None)
    torch.cuda.synchronize()
    assert rc == 0
    assert int(st[0]) == 0
    return dC.cpu().numpy().T


def _op(X, t):
    return X.T if t else X


def _dyadic(rng, shape, bits=10):
    return rng.integers(-(1 << bits), (1 << bits) + 1, size=shape).astype(np.float64) * 2.0 ** -bits


@pytest.mark.parametrize("ta,tb", [(0, 0), (0, 1), (1, 0), (1, 1)])
@pytest.mark.parametrize("digits", [3, 7])
def test_dyadic_exact(ta, tb, digits):
    rng = np.random.default_rng(10 * ta + 3 * tb + digits)
    m, n, k = 200, 130, 70
    A = _dyadic(rng, (k, m) if ta else (m, k))
    B = _dyadic(rng, (n, k) if tb else (k, n))
    # rows of different magnitude: the per-row scale must follow them
    if ta:
        A *= 2.0 ** rng.integers(-6, 7, size=(1, m))
    else:
        A *= 2.0 ** rng.integers(-6, 7, size=(m, 1))
    C = _dyadic(rng, (m, n))
    got = _digits_gemm(ta, tb, A, B, C, 0.5, 0.25, 0, digits)
    ref = 0.5 * (_op(A, ta) @ _op(B, tb)) + 0.25 * C
    assert np.array_equal(got, ref)


def test_dyadic_lower_triangle_and_tiles():
    rng = np.random.default_rng(3)
    m = n = 300
    k = 257
    A = _dyadic(rng, (m, k))
    B = _dyadic(rng, (n, k))
    C = _dyadic(rng, (m, n))
    got = _digits_gemm(0, 1, A, B, C, -1.0, 1.0, 1, 7)
    ref = -(A @ B.T) + C
    low = np.tril(np.ones((m, n), dtype=bool))
    assert np.array_equal(got[low], ref[low])
    assert np.array_equal(got[~low], C[~low])


def test_level_sums_beyond_int32_are_segmented():
    k = 140000
    x = 1.0 - 2.0 ** -20          # leading digit 128 in every entry: level 2 sums 128^2 per term
    A = np.full((16, k), x)
    B = np.full((k, 16), x)
    C = np.zeros((16, 16))
    got = _digits_gemm(0, 0, A, B, C, 1.0, 0.0, 0, 7)
    exact = float(Fraction(x) * Fraction(x) * k)
    assert np.abs(got - exact).max() <= 1e-15 * exact


def _scale(v):
    """2^e with max|v| = m 2^e, m in [0.5, 1) (the digit split's power-of-two scale)."""
    mx = np.abs(v).max()
    return 2.0 ** np.frexp(mx)[1] if mx > 0 else 0.0


@pytest.mark.parametrize("digits", [4, 7])
def test_random_normal_within_truncation_bound(digits):
    rng = np.random.default_rng(20 + digits)
    m, n, k = 150, 140, 1000
    A = rng.standard_normal((m, k)) * 10.0 ** rng.uniform(-3, 3, size=(m, 1))
    B = rng.standard_normal((k, n))
    got = _digits_gemm(0, 0, A, B, np.zeros((m, n)), 1.0, 0.0, 0, digits)
    ref = A.astype(np.longdouble) @ B.astype(np.longdouble)
    err = np.abs(got.astype(np.longdouble) - ref).astype(np.float64)
    ea = np.array([_scale(A[i]) for i in range(m)])[:, None]
    eb = np.array([_scale(B[:, j]) for j in range(n)])[None, :]
    bound = k * ea * eb * 2.0 ** (-7 * digits + 3)
    assert (err <= bound).all(), float((err / bound).max())
    if digits == 7:
        # binary64 accuracy: within a few units of the exact product's magnitude scale
        assert (err <= 1e-14 * k ** 0.5 * ea * eb).all()
