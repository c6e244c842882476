"""Helpers shared by the GPU parity tests (comparison logic only)."""
import numpy as np

# End-to-end tolerances on a cumulative-weight boundary (relative for the
# binary64 path; absolute 4 ulp of binary32 at 1 for the compensated path).
REL_F64 = 1e-12
ABS_F32 = 4 * 2.0**-23
# What the compensated binary32 path achieves beside that stated bound: its
# spacings -log v of binary32 draws are evaluated in binary32-pair arithmetic
# (about 2^-45 relative) and summed exactly, so U agrees with the oracle's
# binary64 evaluation of the same draws far inside 1e-12 relative, and an
# index can differ only where U lies within about 1e-13 of a boundary.
REL_U_F32 = 1e-12


def boundary_only(r_gpu, r_ref, W, U, rel=None, abs_tol=None):
    """Indices may differ only where U_i lies within the tolerance of every
    cumulative weight W_k between the two answers (k in [min, max))."""
    r_gpu = np.asarray(r_gpu, dtype=np.int64)
    r_ref = np.asarray(r_ref, dtype=np.int64)
    mism = np.nonzero(r_gpu != r_ref)[0]
    bad = []
    for i in mism:
        a, b = sorted((int(r_gpu[i]), int(r_ref[i])))
        Wk = W[a:b]
        tol = rel * Wk if rel is not None else abs_tol
        if not np.all(np.abs(U[i] - Wk) <= tol):
            bad.append(int(i))
    return mism, bad


def assert_boundary_only(r_gpu, r_ref, W, U, rel=None, abs_tol=None, max_frac=1e-3):
    M = W.shape[0]
    assert r_gpu.min() >= 0 and r_gpu.max() < M
    mism, bad = boundary_only(r_gpu, r_ref, W, U, rel, abs_tol)
    assert not bad, "non-boundary mismatches at %s (gpu %s, ref %s)" % (bad[:5], r_gpu[bad[:5]], r_ref[bad[:5]])
    assert mism.size <= max(2, max_frac * r_gpu.size), mism.size
    return mism.size
