"""Host-side checks of the C ABI that need no GPU: the library loads, exports every
function declared in include/elsi_gb.h, and rejects bad arguments before any CUDA call."""
import ctypes
import os
import re

import pytest

import paper_1705_11191_gb300 as egb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", "elsi_gb.h"),
           os.path.join(ROOT, "include", "elsi_gb_testing.h")]


def _declared():
    names = set()
    for hdr in HEADERS:
        txt = open(hdr).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names |= set(re.findall(r"\b(elsi_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1705_11191_gb300 import build
    build.build()
    return egb.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name


def test_init_rejects_bad_arguments(lib):
    h = ctypes.c_void_p()
    assert lib.elsi_init(ctypes.byref(h), 2, 1, 2, 10, 5, 4.0) == 2   # libOMM: unsupported
    assert lib.elsi_init(ctypes.byref(h), 1, 3, 2, 10, 5, 4.0) == 2   # unknown format
    assert lib.elsi_init(ctypes.byref(h), 1, 1, 3, 10, 5, 4.0) == 1   # bad mode
    assert lib.elsi_init(ctypes.byref(h), 1, 1, 2, 10, 11, 4.0) == 1  # n_state > n
    assert lib.elsi_init(ctypes.byref(h), 1, 1, 2, 10, 2, 5.0) == 1   # too many electrons
    assert lib.elsi_init(ctypes.byref(h), 1, 1, 2, 0, 1, 0.0) == 1


def test_handle_lifecycle_and_setters(lib):
    h = egb.Handle(16, 8, 8.0)
    h.set_band_width(16)
    h.set_broadening(egb.OCC_FERMI, 0.01)
    h.set_occ_accuracy(1e-10)
    h.set_mu_max_steps(50)
    h.set_precision(egb.PREC_FP32_REFINE)
    h.set_broadening(egb.OCC_MP1, 0.01)  # Methfessel-Paxton order 1
    with pytest.raises(egb.ElsiError) as e:
        h.set_broadening(5)
    assert e.value.code == 1
    with pytest.raises(egb.ElsiError):
        h.set_band_width(7)
    with pytest.raises(egb.ElsiError) as e:
        h.get_mu()  # no dm solve yet
    assert e.value.code == 8
    h.close()
    # use after finalize is rejected by the library
    assert lib.elsi_set_band_width(ctypes.c_void_p(None), 16) == 8


def test_stage_names(lib):
    names = egb.stage_names()
    assert names[0] == "cholesky" and "full_to_band" in names and "density" in names


def test_customisation_setters_reject_bad_values(lib):
    h = egb.Handle(16, 8, 8.0)
    for call, bad in [(h.set_elpa_solver, 3), (h.set_elpa_solver, 0), (h.set_batch_streams, 17),
                      (h.set_batch_streams, -1), (h.set_sing_check, 3), (h.set_broadening, 5)]:
        with pytest.raises(egb.ElsiError) as e:
            call(bad)
        assert e.value.code == 1
    with pytest.raises(egb.ElsiError) as e:
        h.set_sing_check(1, 0.0)  # tolerance must be > 0
    assert e.value.code == 1
    h.set_elpa_solver(1)
    h.set_batch_streams(0)
    h.set_sing_check(2, 1e-7)
    h.set_broadening(egb.OCC_MP0, 0.02)
    assert h.get_n_nonsing() == 16  # no solve yet: the full basis
    h.close()


def test_csc_format_accepted_by_init(lib):
    h = ctypes.c_void_p()
    assert lib.elsi_init(ctypes.byref(h), 1, 2, 2, 10, 5, 4.0) == 0
    assert lib.elsi_finalize(ctypes.byref(h)) == 0


def test_spin_limit_setter(lib):
    """The runtime limit of the SIMT spin waits is host state: set, read back, reject < 0."""
    old = lib.elsi_gb_get_spin_limit()
    assert old == 1 << 26
    try:
        assert lib.elsi_gb_set_spin_limit(5) == 0
        assert lib.elsi_gb_get_spin_limit() == 5
        assert lib.elsi_gb_set_spin_limit(-1) == 1
        assert lib.elsi_gb_get_spin_limit() == 5
    finally:
        assert lib.elsi_gb_set_spin_limit(old) == 0


def _testing_protos(lib):
    v = ctypes.c_void_p
    lib.elsi_gb_symm_tall_f32_work.argtypes = [ctypes.c_int]
    lib.elsi_gb_symm_tall_f32_work.restype = ctypes.c_size_t
    lib.elsi_gb_symm_tall_f32.argtypes = [ctypes.c_int, ctypes.c_int, v, ctypes.c_int, v, ctypes.c_int,
                                          v, ctypes.c_int, v, ctypes.c_size_t, v, v]
    lib.elsi_gb_gemm_f64_digits_planes.argtypes = [ctypes.c_int] * 3
    lib.elsi_gb_gemm_f64_digits_planes.restype = ctypes.c_size_t
    lib.elsi_gb_gemm_f64_digits_exps.argtypes = [ctypes.c_int] * 2
    lib.elsi_gb_gemm_f64_digits_exps.restype = ctypes.c_size_t
    lib.elsi_gb_gemm_f64_digits.argtypes = (
        [ctypes.c_int] * 5 + [ctypes.c_double, v, ctypes.c_int, v, ctypes.c_int, ctypes.c_double, v,
                              ctypes.c_int, ctypes.c_int, ctypes.c_int, v, ctypes.c_size_t, v,
                              ctypes.c_size_t, v, v])


def test_testing_entry_scratch_sizes(lib):
    """Scratch sizes of the testing entries are host arithmetic: the digit planes hold 7
    planes of (rows padded to 128) x (K padded to 16) bf16 values per operand; the
    symmetric panel product holds the V hi/lo planes (64 x K padded to 32 each) and at most
    tiles_m + 3 G partial 128 x 64 tiles, G = min(256, tiles_m * k-tiles)."""
    _testing_protos(lib)

    def up(x, q):
        return (x + q - 1) // q * q

    for m, n, k in [(1, 1, 1), (200, 130, 70), (4099, 64, 40000)]:
        assert lib.elsi_gb_gemm_f64_digits_planes(m, n, k) == 7 * (up(m, 128) + up(n, 128)) * up(k, 16)
        assert lib.elsi_gb_gemm_f64_digits_exps(m, n) == up(m, 128) + up(n, 128)
    for m in [1, 100, 4099, 16384]:
        kp = up(m, 32)
        tiles = (m + 127) // 128
        G = min(256, tiles * (kp // 32))
        assert lib.elsi_gb_symm_tall_f32_work(m) == 2 * 64 * kp + (tiles + 3 * G) * 128 * 64 + 64
    assert lib.elsi_gb_symm_tall_f32_work(0) == 0


def test_testing_entries_reject_bad_arguments(lib):
    """Bad sizes, digit counts and missing buffers come back as ELSI_ERR_ARG (1) before any
    CUDA call (the pointers below are never dereferenced)."""
    _testing_protos(lib)
    p = ctypes.c_void_p(16)
    # symmetric panel product: nv > 64, nv < 1, m < 1, null scratch
    assert lib.elsi_gb_symm_tall_f32(64, 65, p, 64, p, 64, p, 64, p, 1 << 20, p, None) == 1
    assert lib.elsi_gb_symm_tall_f32(64, 0, p, 64, p, 64, p, 64, p, 1 << 20, p, None) == 1
    assert lib.elsi_gb_symm_tall_f32(0, 8, p, 64, p, 64, p, 64, p, 1 << 20, p, None) == 1
    assert lib.elsi_gb_symm_tall_f32(64, 8, p, 64, p, 64, p, 64, None, 1 << 20, p, None) == 1
    # digit product: digits outside 1..7, short leading dimensions, short scratch
    args = lambda digits, lda, pe: (0, 0, 64, 32, 48, 1.0, p, lda, p, 48, 0.0, p, 64, 0, digits,
                                    p, pe, p, 1 << 10, p, None)
    big = lib.elsi_gb_gemm_f64_digits_planes(64, 32, 48)
    assert lib.elsi_gb_gemm_f64_digits(*args(0, 64, big)) == 1
    assert lib.elsi_gb_gemm_f64_digits(*args(8, 64, big)) == 1
    assert lib.elsi_gb_gemm_f64_digits(*args(7, 63, big)) == 1
    assert lib.elsi_gb_gemm_f64_digits(*args(7, 64, big - 1)) == 1
