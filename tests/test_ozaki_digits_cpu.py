"""The digit split of the binary64-accurate products (Ozaki scheme) is computed on the GPU
from the bit pattern of each element with integer operations. This checks, on the CPU,
the identity that form relies on: for r = x 2^-e (|r| < 1) the binary64 steps
t = 128 r, d_s = rint(t), r = t - d_s give digits with A_s = sum_{i<=s} d_i 128^(s-i) =
rint(x 2^(7s-e)) (rounding half to even), so d_s = A_s - 128 A_(s-1), where
rint(x 2^(7s-e)) = +-rne(M / 2^(e-E-7s)) for x = +-M 2^E. Random values over a wide
exponent range, zeros, subnormals and exact ties at every digit level."""
import struct

import numpy as np

DIGITS, BITS = 7, 7


def digits_by_steps(x: float, e: int) -> list[int]:
    r = np.ldexp(np.float64(x), -e)
    out = []
    for _ in range(DIGITS):
        t = r * 128.0
        d = np.rint(t)
        r = t - d
        out.append(int(d))
    return out


def digits_by_bits(x: float, e: int) -> list[int]:
    u = struct.unpack("<Q", struct.pack("<d", x))[0]
    sign = -1 if u >> 63 else 1
    xf, frac = (u >> 52) & 0x7FF, u & ((1 << 52) - 1)
    m, ex = (frac | (1 << 52), xf - 1075) if xf else (frac, -1074)
    out, prev = [], 0
    for s in range(1, DIGITS + 1):
        k = e - ex - BITS * s
        if m == 0:
            a = 0
        elif k <= 0:
            a = m << (-k)
        else:
            q, rem, half = m >> k, m & ((1 << k) - 1), 1 << (k - 1)
            a = q + (1 if rem > half or (rem == half and q & 1) else 0)
        a *= sign
        out.append(a - 128 * prev)
        prev = a
    return out


def row_exponent(v: np.ndarray) -> int:
    mx = float(np.max(np.abs(v)))
    return int(np.frexp(mx)[1]) if mx > 0 else 0


def test_random_rows_match():
    rng = np.random.default_rng(7)
    for trial in range(300):
        v = rng.standard_normal(32) * 10.0 ** rng.integers(-300, 300)
        if trial % 4 == 1:
            v[rng.integers(32)] = 0.0
        if trial % 4 == 2:
            v[:8] *= 1e-200
        e = row_exponent(v)
        for x in v:
            assert digits_by_steps(float(x), e) == digits_by_bits(float(x), e)


def test_subnormal_row():
    v = np.array([5e-324, -3e-320, 2.2e-310, 0.0])
    e = row_exponent(v)
    for x in v:
        assert digits_by_steps(float(x), e) == digits_by_bits(float(x), e)


def test_exact_ties_at_every_level():
    rng = np.random.default_rng(8)
    for s in range(1, DIGITS + 1):
        for trial in range(200):
            e = int(rng.integers(-30, 30))
            j = int(rng.integers(0, 2 ** min(7 * s, 50)))
            x = (2 * j + 1) * 2.0 ** (-7 * s - 1) * 2.0 ** e
            if not abs(x) < 2.0 ** e:
                continue
            x = -x if trial % 2 else x
            assert digits_by_steps(x, e) == digits_by_bits(x, e)
