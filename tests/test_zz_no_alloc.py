"""rs_sorted_uniform_static: the allocation-free entry point.

Compared bit for bit with rs_sorted_uniform (same kernels, so the results
must be identical) on two calls in a row, for both precisions, plus its
size limit and a check that repeated calls leave the device's free memory
unchanged.  This file is collected last on purpose: it must pass both alone
in a fresh process and after every other GPU test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01356_gb300 as g
    return g


def _handle_uniforms(g, N, seed, inst, prec):
    h = g.Handle()
    try:
        U = torch.empty(N, dtype=torch.float64, device="cuda")
        g.rs_sorted_uniform(h.h, N, seed, inst, U, g.opts(prec=prec))
        torch.cuda.synchronize()
        assert h.status() == g.RS_OK
        return U.cpu().numpy()
    finally:
        h.close()


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_static_matches_handle_path_two_calls(g, prec):
    p = g.RS_F64 if prec == "f64" else g.RS_F32_COMP
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    # two calls in a row on the same stream: a larger N, then a smaller one,
    # so stale scratch from the first call would show in the second
    cases = [(g.RS_STATIC_MAX_N, 2024, 7), (1000, 5, 0)]
    outs = []
    for N, seed, inst in cases:
        U = torch.full((N,), -1.0, dtype=torch.float64, device="cuda")
        assert g.rs_sorted_uniform_static(N, seed, inst, U, precision=p, status=status) == g.RS_OK
        outs.append(U)
    torch.cuda.synchronize()
    assert int(status.item()) == g.RS_OK
    for (N, seed, inst), U in zip(cases, outs):
        got = U.cpu().numpy()
        ref = _handle_uniforms(g, N, seed, inst, p)
        assert np.array_equal(got, ref), (N, seed, inst)
        assert np.all(np.diff(got) >= 0) and got[0] > 0 and got[-1] <= 1.0


def test_static_size_limit_and_arguments(g):
    U = torch.empty(8, dtype=torch.float64, device="cuda")
    assert g.rs_sorted_uniform_static(g.RS_STATIC_MAX_N + 1, 1, 0, U) == g.RS_ECAPACITY
    assert g.rs_sorted_uniform_static(-1, 1, 0, U) == g.RS_EINVAL
    assert g.rs_sorted_uniform_static(8, 1, 0, U, precision=5) == g.RS_EINVAL
    assert g.rs_sorted_uniform_static(8, 1, 0, None) == g.RS_EINVAL
    assert g.rs_sorted_uniform_static(0, 1, 0, None) == g.RS_OK


def test_static_repeated_calls_keep_free_memory(g):
    """Twenty calls after the set-up call leave the device's free memory
    unchanged.  The reading is device-wide, so another process allocating
    meanwhile could move it: the measurement is repeated (up to three
    times) and one unchanged reading suffices, while an entry point that
    allocated per call would lower every one of them."""
    N = 4096
    U = torch.empty(N, dtype=torch.float64, device="cuda")
    assert g.rs_sorted_uniform_static(N, 3, 1, U) == g.RS_OK  # set-up on this device
    torch.cuda.synchronize()
    deltas = []
    for attempt in range(3):
        free0, _ = torch.cuda.mem_get_info()
        for k in range(20):
            assert g.rs_sorted_uniform_static(N, 3 + k, 1, U) == g.RS_OK
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        deltas.append(free0 - free1)
        if free1 == free0:
            break
    assert deltas[-1] == 0, deltas
