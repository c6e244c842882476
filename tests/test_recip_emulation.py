"""CPU: the precision argument of the reciprocal of Z_{N+1} used by every
path (seg_common.cuh, recip_total), checked on an exact-integer emulation of
its steps with the same truncations: a binary32 estimate of 1/u for the
mantissa u in [1, 2), two Newton steps y <- y + y (2^126 - y U) 2^-126 on
the top 64 bits U of the mantissa, then one step y (2 - m y) on the 128-bit
mantissa with the truncating product and difference of the xf format.  The
claim is a relative error below 2^-122.5 for every total; the device code
itself is checked by the GPU parity tests (identical indices on every path,
U against the oracle)."""
import math
import random
import struct
from fractions import Fraction

TOP = 125  # top mantissa bit of the xf format
M64 = (1 << 64) - 1


def xf_make(m, e):
    if m == 0:
        return (0, None)
    sh = TOP - (m.bit_length() - 1)
    return (m << sh, e - sh) if sh >= 0 else (m >> -sh, e - sh)


def xf_mul(a, b):  # top 128 bits of the 256-bit product (bits 126..253), renormalised
    if a[0] == 0 or b[0] == 0:
        return (0, None)
    return xf_make((a[0] * b[0] >> 126) & ((1 << 128) - 1), a[1] + b[1] + 126)


def xf_sub(a, b):  # a - b for a >= b, b aligned to a by truncation
    if b[0] == 0:
        return a
    d = a[1] - b[1]
    bm = b[0] >> min(d, 128)
    return xf_make(a[0] - bm, a[1])


def f32(x):
    return struct.unpack("<f", struct.pack("<f", x))[0]


def recip(t, rcp_ulps=0):
    m = xf_make(t, 0)
    U = ((m[0] >> 64) << 2 | ((m[0] & M64) >> 62)) & M64  # u = U 2^-63
    uf = f32(f32(float(U >> 40)) * 2.0 ** -23)
    yf = f32(1.0 / uf)
    if rcp_ulps:  # rcp.approx is not correctly rounded: perturb the estimate
        yf = f32(yf * (1.0 + rcp_ulps * 2.0 ** -23))
    Y = round(f32(yf * 2.0 ** 63))
    for _ in range(2):
        D = (1 << 126) - Y * U
        Y = Y + ((Y * (D >> 62)) >> 64)
        assert 0 < Y <= (1 << 63) + 8
    r = xf_make(Y, -63 - TOP - m[1])
    return xf_mul(r, xf_sub(xf_make(2, 0), xf_mul(m, r)))


def test_reciprocal_error_below_bound():
    rng = random.Random(5)
    cases = [1, 2, 3, 5, (1 << 126) - 1, 1 << 125, (1 << 88) + 1]
    cases += [(1 << k) - 1 for k in range(2, 127)] + [(1 << k) + 1 for k in range(2, 126)]
    cases += [rng.getrandbits(rng.randint(1, 126)) | 1 for _ in range(3000)]
    worst = 0
    for t in cases:
        for ulps in (0, 2, -2):
            r = recip(t, ulps)
            err = abs(Fraction(r[0]) * Fraction(2) ** r[1] * t - 1)
            worst = max(worst, err)
    assert float(worst) < 2.0 ** -122.5, math.log2(worst)
