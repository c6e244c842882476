"""ctypes marshalling for libgbresample.so.  No computation happens here."""
import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(HERE, "libgbresample.so")

RS_OK, RS_EINVAL, RS_ENOMEM, RS_ECUDA, RS_ENONFINITE, RS_EZEROSUM, RS_ETIMEOUT, RS_ECAPACITY = range(8)
RS_STATIC_MAX_N = 65536
RS_MAP_DAC, RS_MAP_BINARY, RS_MAP_LINEAR = 0, 1, 2
RS_F64, RS_F32_COMP = 0, 1
RS_SCHEME_MULTINOMIAL, RS_SCHEME_STRATIFIED, RS_SCHEME_SYSTEMATIC = 0, 1, 2
_NAMES = {0: "RS_OK", 1: "RS_EINVAL", 2: "RS_ENOMEM", 3: "RS_ECUDA", 4: "RS_ENONFINITE", 5: "RS_EZEROSUM",
          6: "RS_ETIMEOUT", 7: "RS_ECAPACITY"}


class ResampleError(RuntimeError):
    def __init__(self, code, msg=""):
        self.code = code
        super().__init__("%s%s" % (_NAMES.get(code, str(code)), (": " + msg) if msg else ""))


class rs_opts(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("prec", ctypes.c_int32), ("leaf_L", ctypes.c_int32),
                ("stage_max", ctypes.c_int32), ("spin_limit", ctypes.c_int32), ("debug_flags", ctypes.c_int32),
                ("tile_threads", ctypes.c_int32), ("scheme", ctypes.c_int32)]


def opts(algo=RS_MAP_DAC, prec=RS_F64, leaf_L=0, stage_max=0, spin_limit=0, debug_flags=0, tile_threads=0,
         scheme=RS_SCHEME_MULTINOMIAL):
    return rs_opts(algo, prec, leaf_L, stage_max, spin_limit, debug_flags, tile_threads, scheme)


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_U64 = ctypes.c_uint64
_I32 = ctypes.c_int32
_ST = ctypes.c_int
_OPTS = ctypes.POINTER(rs_opts)


def lib():
    """Load the library; raises if it was not built (no fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise ImportError("libgbresample.so is not built (run __graft_entry__.build()); "
                              "this package has no CPU fallback")
        L = ctypes.CDLL(library_path)
        sig = {
            "rs_create": (_ST, [ctypes.POINTER(_P)]),
            "rs_destroy": (_ST, [_P]),
            "rs_get_status": (_ST, [_P, _P]),
            "rs_last_error": (ctypes.c_char_p, [_P]),
            "rs_version": (ctypes.c_char_p, []),
            "rs_resample_w": (_ST, [_P, _P, _I64, _I64, _U64, _U64, _P, _P, _OPTS, _P]),
            "rs_resample_W": (_ST, [_P, _P, _I64, _I64, _U64, _U64, _P, _OPTS, _P]),
            "rs_sorted_uniform": (_ST, [_P, _I64, _U64, _U64, _P, _OPTS, _P]),
            "rs_sorted_uniform_static": (_ST, [_I64, _U64, _U64, _I32, _P, _P, _P]),
            "rs_cumulative": (_ST, [_P, _P, _I64, _P, _OPTS, _P]),
            "rs_map": (_ST, [_P, _P, _I64, _P, _I64, _P, _OPTS, _P]),
            "rs_philox": (_ST, [_P, _U64, _U64, _U64, _I64, _P, _P]),
            "rs_gather": (_ST, [_P, _P, _I64, _I64, _P, _I64, _P, _P]),
            "rs_softmax_weights": (_ST, [_P, _P, _I64, _P, _P]),
            "rs_resample_logw": (_ST, [_P, _P, _I64, _I64, _U64, _U64, _P, _OPTS, _P]),
            "rs_resample_batched": (_ST, [_P, _P, _P, _P, _I32, _P, _P, _U64, _P, _OPTS, _P]),
            "rs_autotune_batched": (_ST, [_P, _P, _P, _P, _I32, _P, _P, _U64, _P, _OPTS, _OPTS, _P]),
            "rs_autotune_map": (_ST, [_P, _P, _I64, _I64, _U64, _P, _OPTS, _P]),
            "rs_tuning_save": (_ST, [_P, ctypes.c_char_p]),
            "rs_tuning_load": (_ST, [_P, ctypes.c_char_p]),
            "rs_tuning_get": (_ST, [_P, _I32, _I32, _I64, _I64, _OPTS]),
            "rs_trace_enable": (_ST, [_P, ctypes.c_int]),
            "rs_trace_collect": (_ST, [_P, ctypes.c_int]),
            "rs_trace_report": (_ST, [_P, ctypes.c_char_p, _I64]),
            "rs_trace_reset": (_ST, [_P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(t):
    """Device (or host) address of a tensor / int / None."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _opt(o):
    return ctypes.byref(o) if o is not None else None


def _check(h, rc):
    if rc != RS_OK:
        msg = lib().rs_last_error(h).decode() if h else ""
        raise ResampleError(rc, msg)


def rs_version():
    return lib().rs_version().decode()


def rs_create():
    h = _P()
    _check(None, lib().rs_create(ctypes.byref(h)))
    return h


def rs_destroy(h):
    _check(None, lib().rs_destroy(h))


def rs_last_error(h):
    return lib().rs_last_error(h).decode()


def rs_get_status(h, stream=None):
    """Synchronise the stream; return (and clear) the latched device status code."""
    return lib().rs_get_status(h, _stream(stream))


def rs_resample_w(h, w, M, N, seed, instance, out_idx, W_out=None, o=None, stream=None):
    _check(h, lib().rs_resample_w(h, _ptr(w), M, N, seed, instance, _ptr(out_idx), _ptr(W_out), _opt(o),
                                  _stream(stream)))


def rs_resample_W(h, W, M, N, seed, instance, out_idx, o=None, stream=None):
    _check(h, lib().rs_resample_W(h, _ptr(W), M, N, seed, instance, _ptr(out_idx), _opt(o), _stream(stream)))


def rs_softmax_weights(h, logw, M, w_out, stream=None):
    _check(h, lib().rs_softmax_weights(h, _ptr(logw), M, _ptr(w_out), _stream(stream)))


def rs_resample_logw(h, logw, M, N, seed, instance, out_idx, o=None, stream=None):
    _check(h, lib().rs_resample_logw(h, _ptr(logw), M, N, seed, instance, _ptr(out_idx), _opt(o), _stream(stream)))


def rs_gather(h, x, M, row_bytes, idx, N, x_out, stream=None):
    _check(h, lib().rs_gather(h, _ptr(x), M, row_bytes, _ptr(idx), N, _ptr(x_out), _stream(stream)))


def rs_sorted_uniform(h, N, seed, instance, U_out, o=None, stream=None):
    _check(h, lib().rs_sorted_uniform(h, N, seed, instance, _ptr(U_out), _opt(o), _stream(stream)))


def rs_sorted_uniform_static(N, seed, instance, U_out, precision=RS_F64, status=None, stream=None):
    """Allocation-free sorted uniforms; returns the rs_status code (no handle,
    so no error text)."""
    return lib().rs_sorted_uniform_static(N, seed, instance, precision, _ptr(U_out), _ptr(status), _stream(stream))


def rs_cumulative(h, w, M, W_out, o=None, stream=None):
    _check(h, lib().rs_cumulative(h, _ptr(w), M, _ptr(W_out), _opt(o), _stream(stream)))


def rs_map(h, W, M, U, N, out_idx, o=None, stream=None):
    _check(h, lib().rs_map(h, _ptr(W), M, _ptr(U), N, _ptr(out_idx), _opt(o), _stream(stream)))


def rs_philox(h, seed, instance, first, n, out, stream=None):
    _check(h, lib().rs_philox(h, seed, instance, first, n, _ptr(out), _stream(stream)))


def _host_offsets(a):
    import numpy as np
    return None if a is None else np.ascontiguousarray(a, dtype=np.int64)


def rs_resample_batched(h, w, w_off, r_off, K, seed, out_idx, h_w_off=None, h_r_off=None, o=None, stream=None):
    """w_off, r_off: device int64 tensors [K+1]; h_w_off, h_r_off: optional host
    int64 arrays with the same offsets."""
    hw, hr = _host_offsets(h_w_off), _host_offsets(h_r_off)
    _check(h, lib().rs_resample_batched(h, _ptr(w), _ptr(w_off), _ptr(r_off), K,
                                        None if hw is None else hw.ctypes.data,
                                        None if hr is None else hr.ctypes.data, seed, _ptr(out_idx), _opt(o),
                                        _stream(stream)))


def rs_autotune_batched(h, w, w_off, r_off, K, seed, out_idx, h_w_off=None, h_r_off=None, o=None, stream=None):
    """Runs the tuner; returns the chosen rs_opts (tile_threads, leaf_L, prec)."""
    hw, hr = _host_offsets(h_w_off), _host_offsets(h_r_off)
    best = rs_opts()
    _check(h, lib().rs_autotune_batched(h, _ptr(w), _ptr(w_off), _ptr(r_off), K,
                                        None if hw is None else hw.ctypes.data,
                                        None if hr is None else hr.ctypes.data, seed, _ptr(out_idx), _opt(o),
                                        ctypes.byref(best), _stream(stream)))
    return best


def rs_autotune_map(h, W, M, N, seed, out_idx, stream=None):
    """Tunes the DaC map's leaf size on W; returns the chosen rs_opts."""
    best = rs_opts()
    _check(h, lib().rs_autotune_map(h, _ptr(W), M, N, seed, _ptr(out_idx), ctypes.byref(best), _stream(stream)))
    return best


def rs_tuning_save(h, path):
    _check(h, lib().rs_tuning_save(h, str(path).encode()))


def rs_tuning_load(h, path):
    _check(h, lib().rs_tuning_load(h, str(path).encode()))


def rs_tuning_get(h, kind, precision, M, N):
    """kind 0: the DaC map given W, 1: the batched kernel; returns rs_opts."""
    out = rs_opts()
    _check(h, lib().rs_tuning_get(h, kind, precision, M, N, ctypes.byref(out)))
    return out


def rs_trace_enable(h, on=True):
    _check(h, lib().rs_trace_enable(h, int(bool(on))))


def rs_trace_collect(h, keep=False):
    _check(h, lib().rs_trace_collect(h, int(bool(keep))))


def rs_trace_report(h):
    """{kernel name: (launches, total_ms)} accumulated by rs_trace_collect."""
    buf = ctypes.create_string_buffer(8192)
    _check(h, lib().rs_trace_report(h, buf, len(buf)))
    out = {}
    for line in buf.value.decode().splitlines():
        name, n, ms = line.split()
        out[name] = (int(n), float(ms))
    return out


def rs_trace_reset(h):
    _check(h, lib().rs_trace_reset(h))


class Handle:
    """Owns one rs_handle (grow-only workspace on the current CUDA device)."""

    def __init__(self):
        self.h = rs_create()

    def close(self):
        if self.h:
            rs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def status(self, stream=None):
        return rs_get_status(self.h, stream)
