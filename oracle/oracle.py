"""ctypes front end of the C oracle (``oracle/oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the library.

Every function takes and returns numpy arrays; indices are 0-based int32.
The paper references are to arXiv 2604.01356: Eq. 2-3 (inverse CDF and the
cumulative weights), Algorithm 1 (SortedUniform), Algorithm 2 (modified binary
search), Algorithms 3-5 (binary, CCF and divide-and-conquer samplers).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_int = ctypes.c_int
_p = ctypes.c_void_p


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.orc_philox4x64_10.argtypes = [_p, _p, _p]
        L.orc_philox4x64_10.restype = None
        L.orc_stream_word.argtypes = [_u64, _u64, _u64]
        L.orc_stream_word.restype = _u64
        L.orc_uniform_draws.argtypes = [_u64, _u64, _i64, _int, _p]
        L.orc_uniform_draws.restype = None
        L.orc_sorted_uniform.argtypes = [_u64, _u64, _i64, _int, _p]
        L.orc_sorted_uniform.restype = None
        L.orc_cumulative.argtypes = [_p, _i64, _p, _p]
        L.orc_cumulative.restype = _int
        L.orc_cumulative_f32.argtypes = [_p, _i64, _p, _p]
        L.orc_cumulative_f32.restype = _int
        L.orc_inverse_cdf.argtypes = [_p, _i64, _p, _i64, _p]
        L.orc_inverse_cdf.restype = None
        L.orc_inverse_cdf_walk.argtypes = [_p, _i64, _p, _i64, _p]
        L.orc_inverse_cdf_walk.restype = _int
        L.orc_alg2_binary_search.argtypes = [_p, _i64, _i64, ctypes.c_double]
        L.orc_alg2_binary_search.restype = _i64
        L.orc_alg2_probes.argtypes = [_int]
        L.orc_alg2_probes.restype = _i64
        L.orc_alg3_binary_map.argtypes = [_p, _i64, _p, _i64, _p]
        L.orc_alg3_binary_map.restype = None
        L.orc_alg4_ccf_map.argtypes = [_p, _i64, _p, _i64, _p]
        L.orc_alg4_ccf_map.restype = None
        L.orc_alg5_dac_map.argtypes = [_p, _i64, _p, _i64, _p, _p, _i64]
        L.orc_alg5_dac_map.restype = _i64
        L.orc_resample.argtypes = [_p, _int, _i64, _i64, _u64, _u64, _int, _p, _p, _p]
        L.orc_resample.restype = _int
        L.orc_softmax_weights.argtypes = [_p, _i64, _p]
        L.orc_softmax_weights.restype = _int
        L.orc_scheme_uniform.argtypes = [_u64, _u64, _i64, _int, _int, _p]
        L.orc_scheme_uniform.restype = None
        L.orc_resample_scheme.argtypes = [_p, _int, _i64, _i64, _u64, _u64, _int, _int, _p, _p, _p]
        L.orc_resample_scheme.restype = _int
        L.orc_resample_batched.argtypes = [_p, _int, _p, _p, _i64, _u64, _int, _p]
        L.orc_resample_batched.restype = _int
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class OracleError(ValueError):
    """Raised for invalid weights: 1 = negative or non-finite, 2 = zero total."""


def philox4x64_10(counter, key):
    """Philox-4x64-10 block function (Salmon et al., SC'11)."""
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    lib().orc_philox4x64_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def stream_words(seed, instance, n):
    """Raw 64-bit words 0..n-1 of the stream (seed, instance)."""
    L = lib()
    return np.array([L.orc_stream_word(seed, instance, k) for k in range(n)], dtype=np.uint64)


def uniform_draws(seed, instance, n, single=False):
    """Open-interval draws v_k in (0,1), k = 0..n-1 (binary32 draws widened)."""
    v = np.zeros(max(n, 1), dtype=np.float64)
    lib().orc_uniform_draws(seed, instance, n, int(bool(single)), _ptr(v))
    return v[:n]


def sorted_uniform(N, seed, instance=0, single=False):
    """Algorithm 1 with normaliser Z_{N+1}: N sorted uniforms in (0,1]."""
    U = np.zeros(max(N, 1), dtype=np.float64)
    lib().orc_sorted_uniform(seed, instance, N, int(bool(single)), _ptr(U))
    return U[:N]


def softmax_weights(l):
    """w_j = exp(l_j - max l) in binary64 (the largest weight is 1)."""
    ll = _f64(l)
    w = np.zeros(max(ll.shape[0], 1), dtype=np.float64)
    rc = lib().orc_softmax_weights(_ptr(ll), ll.shape[0], _ptr(w))
    if rc:
        raise OracleError(rc)
    return w[: ll.shape[0]]


SCHEMES = {"multinomial": 0, "stratified": 1, "systematic": 2}


def scheme_uniform(N, seed, instance=0, scheme="stratified", single=False):
    """N uniforms of a scheme: Algorithm 1 ('multinomial'), or one point per
    stratum ((i-1)/N, i/N]: U_i = (i-1+v_{i-1})/N ('stratified') or
    (i-1+v_0)/N ('systematic'), with Algorithm 1's draws v_k."""
    U = np.zeros(max(N, 1), dtype=np.float64)
    lib().orc_scheme_uniform(seed, instance, N, int(bool(single)), SCHEMES[scheme], _ptr(U))
    return U[:N]


def cumulative(w):
    """Eq. 3 with normalisation.  Returns (W, total) with W_M == 1."""
    if w.dtype == np.float32:
        ww = np.ascontiguousarray(w)
        fn = lib().orc_cumulative_f32
    else:
        ww = _f64(w)
        fn = lib().orc_cumulative
    M = ww.shape[0]
    W = np.zeros(max(M, 1), dtype=np.float64)
    tot = ctypes.c_double(0.0)
    rc = fn(_ptr(ww), M, _ptr(W), ctypes.byref(tot))
    if rc:
        raise OracleError(rc)
    return W[:M], tot.value


def inverse_cdf(W, U):
    """Eq. 2-3 by brute force (per-u linear scan, clamped to the last index)."""
    W = _f64(W)
    U = _f64(U)
    r = np.zeros(max(U.shape[0], 1), dtype=np.int32)
    lib().orc_inverse_cdf(_ptr(W), W.shape[0], _ptr(U), U.shape[0], _ptr(r))
    return r[: U.shape[0]]


def inverse_cdf_walk(W, U):
    """Same result as inverse_cdf for non-decreasing U, in one monotone walk."""
    W = _f64(W)
    U = _f64(U)
    r = np.zeros(max(U.shape[0], 1), dtype=np.int32)
    rc = lib().orc_inverse_cdf_walk(_ptr(W), W.shape[0], _ptr(U), U.shape[0], _ptr(r))
    if rc:
        raise ValueError("U is not sorted")
    return r[: U.shape[0]]


def alg2_binary_search(Z, X, a=1, b=None):
    """Algorithm 2 over Z[a..b] (1-based inclusive); returns a 1-based index."""
    Z = _f64(Z)
    b = Z.shape[0] if b is None else b
    base = np.concatenate([[np.nan], Z])  # 1-based view
    return int(lib().orc_alg2_binary_search(_ptr(base), a, b, float(X)))


def alg2_probe_count(reset=True):
    """Number of W comparisons Algorithm 2 made since the last reset."""
    return int(lib().orc_alg2_probes(int(bool(reset))))


def alg3_binary_map(W, U):
    W, U = _f64(W), _f64(U)
    r = np.zeros(max(U.shape[0], 1), dtype=np.int32)
    lib().orc_alg3_binary_map(_ptr(W), W.shape[0], _ptr(U), U.shape[0], _ptr(r))
    return r[: U.shape[0]]


def alg4_ccf_map(W, U):
    W, U = _f64(W), _f64(U)
    r = np.zeros(max(U.shape[0], 1), dtype=np.int32)
    lib().orc_alg4_ccf_map(_ptr(W), W.shape[0], _ptr(U), U.shape[0], _ptr(r))
    return r[: U.shape[0]]


def alg5_dac_map(W, U, trace=False):
    """Algorithm 5.  With trace=True also returns the (depth, m_U, m_W) triples
    (1-based) of every binary search, in visit order."""
    W, U = _f64(W), _f64(U)
    N = U.shape[0]
    r = np.zeros(max(N, 1), dtype=np.int32)
    cap = 2 * N + 4
    tr = np.zeros(3 * cap, dtype=np.int64)
    n = lib().orc_alg5_dac_map(_ptr(W), W.shape[0], _ptr(U), N, _ptr(r), _ptr(tr), cap)
    if trace:
        return r[:N], tr[: 3 * min(n, cap)].reshape(-1, 3)
    return r[:N]


def resample(w, N, seed, instance=0, single=False):
    """Whole path for one instance: (r, W, U).  binary32 w selects the binary32
    weights; single=True selects the binary32 draws."""
    is32 = w.dtype == np.float32
    ww = np.ascontiguousarray(w) if is32 else _f64(w)
    M = ww.shape[0]
    r = np.zeros(max(N, 1), dtype=np.int32)
    W = np.zeros(max(M, 1), dtype=np.float64)
    U = np.zeros(max(N, 1), dtype=np.float64)
    rc = lib().orc_resample(_ptr(ww), int(is32), M, N, seed, instance, int(bool(single)), _ptr(r), _ptr(W), _ptr(U))
    if rc:
        raise OracleError(rc)
    return r[:N], W[:M], U[:N]


def resample_scheme(w, N, seed, scheme, instance=0, single=False):
    """Whole path with the uniforms of `scheme`: (r, W, U)."""
    is32 = w.dtype == np.float32
    ww = np.ascontiguousarray(w) if is32 else _f64(w)
    M = ww.shape[0]
    r = np.zeros(max(N, 1), dtype=np.int32)
    W = np.zeros(max(M, 1), dtype=np.float64)
    U = np.zeros(max(N, 1), dtype=np.float64)
    rc = lib().orc_resample_scheme(_ptr(ww), int(is32), M, N, seed, instance, int(bool(single)), SCHEMES[scheme],
                                   _ptr(r), _ptr(W), _ptr(U))
    if rc:
        raise OracleError(rc)
    return r[:N], W[:M], U[:N]


def resample_batched(w, woff, roff, seed, single=False):
    """K independent instances (instance id k = its position)."""
    is32 = w.dtype == np.float32
    ww = np.ascontiguousarray(w) if is32 else _f64(w)
    wo = np.ascontiguousarray(woff, dtype=np.int64)
    ro = np.ascontiguousarray(roff, dtype=np.int64)
    K = wo.shape[0] - 1
    r = np.zeros(max(int(ro[-1]), 1), dtype=np.int32)
    rc = lib().orc_resample_batched(_ptr(ww), int(is32), _ptr(wo), _ptr(ro), K, seed, int(bool(single)), _ptr(r))
    if rc:
        raise OracleError(rc)
    return r[: int(ro[-1])]
