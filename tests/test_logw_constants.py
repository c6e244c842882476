"""CPU: the constants of the log-weight exponential (k_logw.cu) against their
definitions, computed here independently: the table 2^(j/256) in units 2^-62
by exact integer roots, and the reduction constants by 300-bit ln 2.  The
table and constants are read from the kernel source as text."""
import os
import re

import pytest

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_2604_01356_gb300", "csrc", "k_logw.cu")


def _source():
    with open(SRC) as f:
        return f.read()


def _nearest_root(j):
    """The integer nearest to 2^((62 * 256 + j) / 256), exactly."""
    P = 62 * 256 + j
    lo, hi = 1 << 62, 1 << 63
    while hi - lo > 1:  # largest t with t^256 <= 2^P
        mid = (lo + hi) // 2
        if mid ** 256 <= 1 << P:
            lo = mid
        else:
            hi = mid
    # t + 1/2 rounds up iff (2t + 1)^256 <= 2^(P + 256)
    return lo + 1 if (2 * lo + 1) ** 256 <= 1 << (P + 256) else lo


def test_exp2_table_is_nearest_integer_root():
    body = re.search(r"kExp2Tab\[256\]\s*=\s*\{(.*?)\};", _source(), re.S).group(1)
    vals = [int(v, 16) for v in re.findall(r"0x([0-9a-fA-F]+)ULL", body)]
    assert len(vals) == 256
    for j in (0, 1, 2, 63, 64, 127, 128, 200, 254, 255):
        assert vals[j] == _nearest_root(j), j
    assert vals[0] == 1 << 62
    assert all(a < b for a, b in zip(vals, vals[1:])) and vals[-1] < 1 << 63


def test_reduction_constants():
    mp = pytest.importorskip("mpmath")
    mp.mp.prec = 300
    ln2 = mp.log(2)
    body = _source()
    K1 = int(mp.nint(ln2 / 256 * 2 ** 51))
    K2 = int(mp.nint((ln2 / 256 * 2 ** 51 - K1) * 2 ** 32))
    C = int(mp.nint(256 / ln2 * 2 ** 22))
    lim = int(mp.ceil(mp.mpf("745.14") * 2 ** 51))
    for name, v in (("K1", K1), ("K2", K2), ("n multiplier", C), ("underflow limit", lim)):
        assert f"{v}LL" in body, name
    # the underflow limit lies beyond -1075 ln2, below which exp rounds to 0
    assert lim > 1075 * ln2 * 2 ** 51
    # the n estimate stays within 1e-3 of x 256/ln2 over |x| <= 745.14:
    # the multiplier's rounding plus the 2^-19 truncation of the high word
    assert abs(C / 2 ** 22 - 256 / ln2) * 745.14 + 2 ** -19 * 256 / ln2 < 1e-3
    # K1 shifted left by 8 stays below 2^63 (r is formed at units 2^-59)
    assert K1 << 8 < 1 << 63 and "6096987078286LL << 8" in body
    # binary32 literals of the series and of the scales
    for lit in ("0.16666667f", "0.041666668f", "0.008333334f", "9.094947017729282e-13f",
                "4.611686018427388e18f"):
        assert lit in body, lit
    import numpy as np
    assert np.float32(9.094947017729282e-13) == np.float32(2.0 ** -40)
    assert np.float32(4.611686018427388e18) == np.float32(2.0 ** 62)
