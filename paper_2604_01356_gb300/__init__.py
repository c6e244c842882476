"""GB300-native multinomial resampling (arXiv 2604.01356).

Thin Python binding over the C ABI of ``libgbresample.so`` (declared in
``include/gbresample.h``).  Functions keep the C names; tensors are passed as
device pointers and the current torch CUDA stream is used unless one is
given.  Every computation runs in the library's CUDA kernels: there is no
CPU path, and importing fails loudly when the library is missing.
"""
from ._binding import (  # noqa: F401
    RS_EINVAL, RS_ENOMEM, RS_ECUDA, RS_ENONFINITE, RS_EZEROSUM, RS_ETIMEOUT, RS_ECAPACITY, RS_OK, RS_STATIC_MAX_N,
    RS_F32_COMP, RS_F64, RS_MAP_BINARY, RS_MAP_DAC, RS_MAP_LINEAR,
    RS_SCHEME_MULTINOMIAL, RS_SCHEME_STRATIFIED, RS_SCHEME_SYSTEMATIC,
    ResampleError, Handle, lib, library_path, opts,
    rs_create, rs_destroy, rs_get_status, rs_last_error, rs_version,
    rs_resample_w, rs_resample_W, rs_sorted_uniform, rs_sorted_uniform_static, rs_cumulative, rs_map, rs_philox, rs_gather,
    rs_softmax_weights, rs_resample_logw,
    rs_resample_batched, rs_autotune_batched, rs_autotune_map, rs_tuning_save, rs_tuning_load, rs_tuning_get,
    rs_trace_enable, rs_trace_collect, rs_trace_report, rs_trace_reset,
)
