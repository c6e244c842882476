"""GPU parity: the CUDA path through the C ABI against the oracle.

Bit-exact where the work is integer or exact comparison (Philox words, the
three maps on given W and U); within the derived tolerance where floating
point is involved (cumulative weights, uniforms); boundary-only index
differences end to end.
"""
import numpy as np
import pytest

import oracle
import workloads
from parity_util import ABS_F32, REL_F64, REL_U_F32, assert_boundary_only

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01356_gb300 as g
    return g


@pytest.fixture(scope="module")
def h(g):
    hd = g.Handle()
    yield hd
    hd.close()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


# ------------------------------------------------------------- Philox ----
@pytest.mark.parametrize("seed,inst,first,n", [(0, 0, 0, 4096), (12, 3, 1, 1001), (2**64 - 1, 2**63, 2**40 - 3, 777),
                                               (99, 0, 5, 100_003)])
def test_philox_words_bit_exact(g, h, seed, inst, first, n):
    out = torch.empty(n, dtype=torch.int64, device="cuda")
    g.rs_philox(h.h, seed, inst, first, n, out)
    got = host(out).view(np.uint64)
    if first == 0 and n <= 4096:
        ref = oracle.stream_words(seed, inst, n)
    else:
        ks = np.unique(np.concatenate([np.arange(min(n, 64)), np.linspace(0, n - 1, 200).astype(np.int64)]))
        L = oracle.lib()
        ref_s = np.array([L.orc_stream_word(seed, inst, first + int(k)) for k in ks], dtype=np.uint64)
        assert np.array_equal(got[ks], ref_s)
        return
    assert np.array_equal(got, ref)


# ----------------------------------------------------------- uniforms ----
@pytest.mark.parametrize("N", [1, 2, 31, 4095, 4096, 4097, 3 * 4096 + 77, 100_000])
def test_sorted_uniform_f64(g, h, N):
    U = torch.empty(N, dtype=torch.float64, device="cuda")
    g.rs_sorted_uniform(h.h, N, 5, 7, U)
    assert h.status() == g.RS_OK
    got = host(U)
    ref = oracle.sorted_uniform(N, 5, 7)
    assert np.all(np.diff(got) >= 0)
    assert got[0] > 0 and got[-1] <= 1.0
    rel = np.max(np.abs(got - ref) / ref)
    assert rel <= 1e-13, rel


@pytest.mark.parametrize("N", [1, 4097, 65_536])
def test_sorted_uniform_f32_comp(g, h, N):
    U = torch.empty(N, dtype=torch.float64, device="cuda")
    g.rs_sorted_uniform(h.h, N, 9, 1, U, g.opts(prec=g.RS_F32_COMP))
    assert h.status() == g.RS_OK
    got = host(U)
    ref = oracle.sorted_uniform(N, 9, 1, single=True)
    assert np.all(np.diff(got) >= 0)
    assert np.max(np.abs(got - ref)) <= ABS_F32  # the stated bound
    assert np.max(np.abs(got - ref) / ref) <= REL_U_F32  # what the path achieves


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("scheme", ["multinomial", "stratified", "systematic"])
@pytest.mark.parametrize("N", [1, 2, 1023, 1024, 2046, 2047, 2048])
def test_sorted_uniform_one_cta_equals_lookback(g, h, prec, scheme, N):
    """Up to 2,047 samples the sorted uniforms come from one CTA in one
    launch; they must equal, bit for bit, those of the multi-tile look-back
    scan (debug bit 2 forces it)."""
    p = g.RS_F32_COMP if prec == "f32" else g.RS_F64
    sc = {"multinomial": g.RS_SCHEME_MULTINOMIAL, "stratified": g.RS_SCHEME_STRATIFIED,
          "systematic": g.RS_SCHEME_SYSTEMATIC}[scheme]
    a = torch.empty(N, dtype=torch.float64, device="cuda")
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    g.rs_sorted_uniform(h.h, N, 31, 2, a, g.opts(prec=p, scheme=sc))
    g.rs_sorted_uniform(h.h, N, 31, 2, b, g.opts(prec=p, scheme=sc, debug_flags=4))
    assert h.status() == g.RS_OK
    assert np.array_equal(host(a).view(np.int64), host(b).view(np.int64))


# ----------------------------------------------------- cumulative (Eq.3) --
SIZES = [1, 2, 511, 512, 513, 4095, 4096, 4097, 37 * 4096 + 123]


@pytest.mark.parametrize("M", SIZES)
def test_cumulative_f64_sizes(g, h, M):
    w = workloads.weights_lognormal(M, 2.0, seed=M)
    W = torch.empty(M, dtype=torch.float64, device="cuda")
    g.rs_cumulative(h.h, dev(w), M, W)
    assert h.status() == g.RS_OK
    got = host(W)
    ref, _ = oracle.cumulative(w)
    assert got[-1] == 1.0
    assert np.all(np.diff(got) >= 0)
    assert np.all(np.abs(got - ref) <= REL_F64 * ref + 1e-300)


@pytest.mark.parametrize("kind", workloads.ADVERSARIAL)
def test_cumulative_f64_adversarial(g, h, kind):
    M = 9 * 4096 + 5
    w = workloads.adversarial_weights(kind, M, seed=2)
    W = torch.empty(M, dtype=torch.float64, device="cuda")
    g.rs_cumulative(h.h, dev(w), M, W)
    assert h.status() == g.RS_OK
    got = host(W)
    ref, _ = oracle.cumulative(w)
    assert got[-1] == 1.0 and np.all(np.diff(got) >= 0)
    assert np.all(np.abs(got - ref) <= REL_F64 * ref + 1e-300), kind


@pytest.mark.parametrize("M", [513, 4097, 50_003])
def test_cumulative_f32_comp(g, h, M):
    w = workloads.weights_lognormal(M, 1.5, seed=M).astype(np.float32)
    W = torch.empty(M, dtype=torch.float64, device="cuda")
    g.rs_cumulative(h.h, dev(w), M, W, g.opts(prec=g.RS_F32_COMP))
    assert h.status() == g.RS_OK
    got = host(W)
    ref, _ = oracle.cumulative(w)
    assert got[-1] == 1.0 and np.all(np.diff(got) >= 0)
    assert np.max(np.abs(got - ref)) <= ABS_F32


# ---------------------------------------------------- maps, bit-exact ----
def _map_case(kind, M, N, seed):
    rng = np.random.default_rng(seed)
    w = workloads.adversarial_weights(kind, M, seed) if kind in workloads.ADVERSARIAL else \
        workloads.weights_lognormal(M, 2.0, seed)
    W, _ = oracle.cumulative(w)
    # sorted u's including exact ties with W, values above W_M and tiny values
    picks = W[rng.integers(0, M, size=min(N, 64))]
    U = np.sort(np.concatenate([rng.random(max(N - picks.size - 2, 0)), picks, [1e-300, 1.0]])[:N])
    return W, U


MAP_CASES = [("lognormal", 4096, 1024), ("lognormal", 16 * 4096 + 7, 300), ("lognormal", 1000, 5000),
             ("zeros_runs", 20_000, 2000), ("dyadic", 3000, 3000), ("spike", 5000, 100), ("first", 700, 64),
             ("last", 700, 64), ("lognormal", 1, 10), ("lognormal", 2, 1), ("equal", 4096, 4096),
             ("lognormal", 300_000, 4099)]


@pytest.mark.parametrize("algo", ["dac", "binary", "linear"])
@pytest.mark.parametrize("kind,M,N", MAP_CASES)
def test_map_bit_exact(g, h, algo, kind, M, N):
    W, U = _map_case(kind, M, N, seed=M + N)
    ref = oracle.inverse_cdf_walk(W, U)
    if M * N <= 5_000_000:
        assert np.array_equal(ref, oracle.inverse_cdf(W, U))
    a = {"dac": g.RS_MAP_DAC, "binary": g.RS_MAP_BINARY, "linear": g.RS_MAP_LINEAR}[algo]
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    g.rs_map(h.h, dev(W), M, dev(U), N, out, g.opts(algo=a))
    got = host(out)
    assert np.array_equal(got, ref)


@pytest.mark.parametrize("L", [1, 2, 8, 32, 64, 256])
def test_map_dac_leaf_sizes(g, h, L):
    W, U = _map_case("lognormal", 50_000, 6000, seed=L)
    ref = oracle.inverse_cdf_walk(W, U)
    out = torch.empty(U.size, dtype=torch.int32, device="cuda")
    g.rs_map(h.h, dev(W), W.size, dev(U), U.size, out, g.opts(algo=g.RS_MAP_DAC, leaf_L=L))
    assert np.array_equal(host(out), ref)


# --------------------------------------------------------- end to end ----
E2E = [(4096, 1024), (37 * 4096 + 123, 3 * 4096 + 77), (1, 5), (513, 1), (2000, 9000), (200_000, 200_000)]


@pytest.mark.parametrize("M,N", E2E)
def test_resample_w_f64(g, h, M, N):
    w = workloads.weights_lognormal(M, 2.0, seed=M + 1)
    seed = 1234 + M
    r_ref, W_ref, U_ref = oracle.resample(w, N, seed)
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    Wd = torch.empty(M, dtype=torch.float64, device="cuda")
    g.rs_resample_w(h.h, dev(w), M, N, seed, 0, out, Wd)
    assert h.status() == g.RS_OK
    r = host(out)
    assert_boundary_only(r, r_ref, W_ref, U_ref, rel=REL_F64)
    Wg = host(Wd)
    assert Wg[-1] == 1.0 and np.all(np.abs(Wg - W_ref) <= REL_F64 * W_ref + 1e-300)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_resample_w_unaligned_weights(g, h, prec):
    """Weights starting one element past a 16-byte boundary (no bulk copies:
    the cooperative launch reads them with plain loads), ragged M, against
    the multi-kernel path and the oracle; N = 0 is a no-op."""
    M, N = 300_001, 5000
    w = workloads.weights_lognormal(M, 2.0, seed=71)
    dt = torch.float32 if prec == "f32" else torch.float64
    if prec == "f32":
        w = w.astype(np.float32)
    p = g.RS_F32_COMP if prec == "f32" else g.RS_F64
    buf = torch.zeros(M + 1, dtype=dt, device="cuda")
    buf[1:] = torch.from_numpy(w).cuda()
    wd = buf[1:]
    assert wd.data_ptr() % 16 != 0
    a = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    b = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    g.rs_resample_w(h.h, wd, M, N, 5, 1, a, None, g.opts(prec=p))
    g.rs_resample_w(h.h, wd, M, N, 5, 1, b, None, g.opts(prec=p, debug_flags=2))
    assert h.status() == g.RS_OK
    ra = host(a)
    assert np.array_equal(ra, host(b))
    r_ref, W_ref, U_ref = oracle.resample(w, N, 5, instance=1, single=prec == "f32")
    if prec == "f32":
        assert_boundary_only(ra, r_ref, W_ref, U_ref, abs_tol=ABS_F32, max_frac=0.0)
    else:
        assert_boundary_only(ra, r_ref, W_ref, U_ref, rel=REL_F64)
    z = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    g.rs_resample_w(h.h, wd, M, 0, 5, 1, z, None, g.opts(prec=p))
    assert h.status() == g.RS_OK and int(host(z)[0]) == -7


@pytest.mark.parametrize("kind", workloads.ADVERSARIAL)
def test_resample_w_adversarial(g, h, kind):
    M, N = 5 * 4096 + 17, 4096
    w = workloads.adversarial_weights(kind, M, seed=3)
    r_ref, W_ref, U_ref = oracle.resample(w, N, 77)
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    g.rs_resample_w(h.h, dev(w), M, N, 77, 0, out)
    assert h.status() == g.RS_OK
    r = host(out)
    assert_boundary_only(r, r_ref, W_ref, U_ref, rel=REL_F64)
    # zero-weight indices are never drawn
    assert np.all(w[r] > 0)


@pytest.mark.parametrize("M,N", [(4096, 1024), (9 * 4096 + 3, 5000)])
def test_resample_w_f32_comp(g, h, M, N):
    w = workloads.weights_lognormal(M, 1.5, seed=M).astype(np.float32)
    r_ref, W_ref, U_ref = oracle.resample(w, N, 31, single=True)
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    g.rs_resample_w(h.h, dev(w), M, N, 31, 0, out, None, g.opts(prec=g.RS_F32_COMP))
    assert h.status() == g.RS_OK
    assert_boundary_only(host(out), r_ref, W_ref, U_ref, abs_tol=ABS_F32, max_frac=0.0)


@pytest.mark.parametrize("algo", ["dac", "binary", "linear"])
def test_resample_W_map_only(g, h, algo):
    M, N = 100_000, 3000
    w = workloads.weights_lognormal(M, 2.0, seed=4)
    W, _ = oracle.cumulative(w)
    U_ref = oracle.sorted_uniform(N, 8, 0)
    r_ref = oracle.inverse_cdf_walk(W, U_ref)
    a = {"dac": g.RS_MAP_DAC, "binary": g.RS_MAP_BINARY, "linear": g.RS_MAP_LINEAR}[algo]
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    g.rs_resample_W(h.h, dev(W), M, N, 8, 0, out, g.opts(algo=a))
    assert h.status() == g.RS_OK
    assert_boundary_only(host(out), r_ref, W, U_ref, rel=REL_F64)


SMALL_W_CASES = [(1, 1), (7, 2047), (600, 3), (4096, 1024), (5000, 300), (12_288, 2047)]


@pytest.mark.parametrize("scheme", ["multinomial", "stratified", "systematic"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("algo", ["dac", "binary", "linear"])
@pytest.mark.parametrize("M,N", SMALL_W_CASES)
def test_resample_W_one_cta_equals_multilaunch(g, h, M, N, algo, prec, scheme):
    """rs_resample_W on one CTA (W in shared memory, at most 12,288 weights
    and 2047 samples) against the multi-launch form (debug bit 2), index for
    index, for the three maps, both draw precisions, every scheme, and an
    8-byte (not 16-byte) aligned W; ties with W and an all-zero head."""
    w = workloads.adversarial_weights("zeros_runs", M + 1, seed=M + N)
    W, _ = oracle.cumulative(w)
    a = {"dac": g.RS_MAP_DAC, "binary": g.RS_MAP_BINARY, "linear": g.RS_MAP_LINEAR}[algo]
    sc = {"multinomial": g.RS_SCHEME_MULTINOMIAL, "stratified": g.RS_SCHEME_STRATIFIED,
          "systematic": g.RS_SCHEME_SYSTEMATIC}[scheme]
    p = g.RS_F64 if prec == "f64" else g.RS_F32_COMP
    Wd = dev(W)
    outs = []
    for Wv in (Wd[:M], Wd[1:]):  # 16-byte aligned, then 8-byte aligned
        for flags in (0, 4):
            r = torch.full((N,), -1, dtype=torch.int32, device="cuda")
            g.rs_resample_W(h.h, Wv, M, N, 13, 2, r, g.opts(algo=a, prec=p, scheme=sc, debug_flags=flags))
            outs.append(host(r))
    assert h.status() == g.RS_OK
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[2], outs[3])
    assert outs[0].min() >= 0 and outs[0].max() < M


@pytest.mark.parametrize("L", [1, 4, 64, 1024])
def test_resample_W_one_cta_leaf_sizes(g, h, L):
    """The one-CTA divide and conquer with explicit leaf sizes (one sample a
    leaf up to one leaf for all) against the oracle's walk on the same U."""
    M, N = 4096, 1024
    w = workloads.weights_lognormal(M, 2.0, seed=L)
    W, _ = oracle.cumulative(w)
    U_ref = oracle.sorted_uniform(N, 8, 0)
    r_ref = oracle.inverse_cdf_walk(W, U_ref)
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    g.rs_resample_W(h.h, dev(W), M, N, 8, 0, out, g.opts(algo=g.RS_MAP_DAC, leaf_L=L))
    assert h.status() == g.RS_OK
    assert_boundary_only(host(out), r_ref, W, U_ref, rel=REL_F64)


def test_resample_batched_matches_instances(g, h):
    w, woff, roff = workloads.weights_batched(K=24, seed=5, nmin=8, nmax=300, pmax=9)
    K = 24
    r_ref = oracle.resample_batched(w, woff, roff, seed=3, single=True)
    out = torch.empty(int(roff[-1]), dtype=torch.int32, device="cuda")
    g.rs_resample_batched(h.h, dev(w), dev(woff), dev(roff), K, 3, out, woff, roff)
    assert h.status() == g.RS_OK
    got = host(out)
    assert np.count_nonzero(got != r_ref) <= 2
    for k in range(K):
        a, b = int(roff[k]), int(roff[k + 1])
        wk = w[woff[k]:woff[k + 1]]
        Wk, _ = oracle.cumulative(wk)
        Uk = oracle.sorted_uniform(b - a, 3, k, single=True)
        assert_boundary_only(got[a:b], r_ref[a:b], Wk, Uk, abs_tol=ABS_F32, max_frac=0.0)


# ----------------------------------------------------- device errors ----
@pytest.mark.parametrize("bad,code", [(-1.0, "RS_ENONFINITE"), (np.nan, "RS_ENONFINITE"), (np.inf, "RS_ENONFINITE")])
def test_invalid_weight_latches_status(g, h, bad, code):
    w = workloads.weights_small(20_000, seed=1)
    w[12_345] = bad
    out = torch.empty(100, dtype=torch.int32, device="cuda")
    g.rs_resample_w(h.h, dev(w), w.size, 100, 1, 0, out)
    assert h.status() == getattr(g, code)
    assert h.status() == g.RS_OK  # cleared
    r = host(out)
    assert r.min() >= 0 and r.max() < w.size  # outputs stay in bounds


def test_zero_sum_latches_status(g, h):
    w = np.zeros(5000)
    out = torch.empty(10, dtype=torch.int32, device="cuda")
    g.rs_resample_w(h.h, dev(w), w.size, 10, 1, 0, out)
    assert h.status() == g.RS_EZEROSUM


def test_bounded_wait_times_out_and_context_survives(g, h):
    """Fault injection on the host side: the first look-back tile of the
    spacing scan withholds its publication; every later tile's wait runs out
    after spin_limit polls (tiles of 1024 draws, so 10 tiles here)."""
    N = 10_000
    U = torch.empty(N, dtype=torch.float64, device="cuda")
    g.rs_sorted_uniform(h.h, N, 5, 7, U, g.opts(spin_limit=200, debug_flags=1))
    assert h.status() == g.RS_ETIMEOUT
    # the context is still usable and a normal call is correct again
    g.rs_sorted_uniform(h.h, N, 5, 7, U)
    assert h.status() == g.RS_OK
    ref = oracle.sorted_uniform(N, 5, 7)
    assert np.max(np.abs(host(U) - ref) / ref) <= 1e-13


def test_host_argument_errors(g, h):
    out = torch.empty(4, dtype=torch.int32, device="cuda")
    w = torch.ones(8, dtype=torch.float64, device="cuda")
    with pytest.raises(g.ResampleError) as e:
        g.rs_resample_w(h.h, w, 0, 4, 1, 0, out)
    assert e.value.code == g.RS_EINVAL
    with pytest.raises(g.ResampleError):
        g.rs_resample_w(h.h, w, 8, -1, 1, 0, out)
    with pytest.raises(g.ResampleError):
        g.rs_map(h.h, w, 8, w, 4, out, g.opts(algo=7))
    with pytest.raises(g.ResampleError):
        g.rs_resample_w(h.h, None, 8, 4, 1, 0, out)
    g.rs_resample_w(h.h, w, 8, 0, 1, 0, None)  # N = 0 is a no-op
    assert h.status() == g.RS_OK


# -------------------------------------------------------------- tracing ----
def test_tracing_outside_capture_reports_kernels(g, h):
    w = workloads.weights_lognormal(300_000, 2.0, seed=4)
    out = torch.empty(500, dtype=torch.int32, device="cuda")
    wd = dev(w)
    g.rs_trace_enable(h.h, True)
    try:
        for _ in range(3):
            g.rs_resample_w(h.h, wd, w.size, 500, 1, 0, out)  # one cooperative launch
            g.rs_resample_w(h.h, wd, w.size, 500, 1, 0, out, None, g.opts(debug_flags=2))  # multi-kernel
            g.rs_resample_w(h.h, wd, 20_000, 500, 1, 0, out)  # a small instance: one CTA
        g.rs_trace_collect(h.h)
        rep = g.rs_trace_report(h.h)
    finally:
        g.rs_trace_enable(h.h, False)
        g.rs_trace_reset(h.h)
    assert h.status() == g.RS_OK
    for name in ("fused", "w_reduce", "seg_prefix", "uniform_scan", "map_seg", "single_cta"):
        n, ms = rep[name]
        assert n == 3 and ms > 0.0, (name, rep[name])


# ------------------------------------ fused launch vs multi-kernel path ----
FUSED_CASES = [(1, 1), (2, 5), (513, 1000), (4096, 1024), (131_072, 2048), (9 * 4096 + 5, 4097), (300_000, 64),
               (1_000_003, 300_001), (4_000_000, 4000)]


@pytest.mark.parametrize("path", ["auto", "cooperative"])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("M,N", FUSED_CASES)
def test_fused_equals_multikernel(g, h, prec, M, N, path):
    """The one-launch forms of rs_resample_w (the one-CTA path of small
    instances, and the cooperative launch, forced with debug bit 2) against
    the multi-kernel path, index for index."""
    w = workloads.weights_lognormal(M, 2.0, seed=M)
    p = g.RS_F64 if prec == "f64" else g.RS_F32_COMP
    if prec == "f32":
        w = w.astype(np.float32)
    wd = dev(w)
    a = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    b = torch.full((N,), -2, dtype=torch.int32, device="cuda")
    g.rs_resample_w(h.h, wd, M, N, 9, 2, a, None, g.opts(prec=p, debug_flags=0 if path == "auto" else 4))
    g.rs_resample_w(h.h, wd, M, N, 9, 2, b, None, g.opts(prec=p, debug_flags=2))
    assert h.status() == g.RS_OK
    assert np.array_equal(host(a), host(b))


SMALL_CASES = [(1, 1), (3, 2047), (511, 7), (512, 512), (4096, 1024), (5000, 2047), (12_287, 300), ("max", 2047)]


@pytest.mark.parametrize("scheme", ["multinomial", "stratified", "systematic"])
@pytest.mark.parametrize("aligned", [True, False])
@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("M,N", SMALL_CASES)
def test_small_smem_equals_other_forms(g, h, prec, M, N, aligned, scheme):
    """The one-CTA form with the weights staged in shared memory (at most
    12,288 weights, 2047 samples) against the cooperative launch and the
    multi-kernel path, index for index, for 16-byte aligned weights (copied
    asynchronously) and unaligned ones (plain loads), under every scheme."""
    if M == "max":
        M = 12_288
    w = workloads.weights_lognormal(M + 1, 2.0, seed=M + N)
    p = g.RS_F64 if prec == "f64" else g.RS_F32_COMP
    if prec == "f32":
        w = w.astype(np.float32)
    base = dev(w)
    wd = base[:M] if aligned else base[1:]  # one element in: 4- or 8-byte aligned only
    sc = {"multinomial": g.RS_SCHEME_MULTINOMIAL, "stratified": g.RS_SCHEME_STRATIFIED,
          "systematic": g.RS_SCHEME_SYSTEMATIC}[scheme]
    outs = []
    for flags in (0, 4, 2):
        r = torch.full((N,), -1, dtype=torch.int32, device="cuda")
        g.rs_resample_w(h.h, wd, M, N, 21, 5, r, None, g.opts(prec=p, debug_flags=flags, scheme=sc))
        outs.append(host(r))
    assert h.status() == g.RS_OK
    assert np.array_equal(outs[0], outs[2]) and np.array_equal(outs[1], outs[2])
    assert outs[0].min() >= 0 and outs[0].max() < M


@pytest.mark.parametrize("kind", workloads.ADVERSARIAL)
@pytest.mark.parametrize("M,N", [(12_288, 2047), (1500, 700)])
def test_small_smem_adversarial(g, h, kind, M, N):
    """Adversarial binary64 weights (ties, zero runs, head segments, a spike)
    on the shared-memory one-CTA form against the multi-kernel path."""
    w = workloads.adversarial_weights(kind, M, seed=6)
    wd = dev(w)
    a = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    b = torch.full((N,), -2, dtype=torch.int32, device="cuda")
    g.rs_resample_w(h.h, wd, M, N, 8, 1, a)
    g.rs_resample_w(h.h, wd, M, N, 8, 1, b, None, g.opts(debug_flags=2))
    assert h.status() == g.RS_OK
    assert np.array_equal(host(a), host(b))


@pytest.mark.parametrize("N", [300, 1024])
def test_small_smem_error_paths(g, N):
    """The shared-memory small-instance forms (one CTA below 384 samples, a
    cluster of four from there) latch RS_EZEROSUM with zero indices for an
    all-zero instance, and RS_ENONFINITE for a NaN weight; the handle keeps
    working afterwards."""
    M = 4096
    out = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    hz = g.Handle()
    try:
        g.rs_resample_w(hz.h, dev(np.zeros(M)), M, N, 3, 0, out)
        assert hz.status() == g.RS_EZEROSUM
        assert np.all(host(out) == 0)
    finally:
        hz.close()
    w = workloads.weights_lognormal(M, 2.0, seed=5)
    w[1234] = np.nan
    hn = g.Handle()
    try:
        g.rs_resample_w(hn.h, dev(w), M, N, 3, 0, out)
        assert hn.status() == g.RS_ENONFINITE
    finally:
        hn.close()
    hk = g.Handle()
    try:
        w[1234] = 1.0
        g.rs_resample_w(hk.h, dev(w), M, N, 3, 0, out)
        assert hk.status() == g.RS_OK
        r = host(out)
        assert r.min() >= 0 and r.max() < M and np.all(np.diff(r) >= 0)
    finally:
        hk.close()


def test_small_smem_is_taken(g, h):
    """The small workload's shape (M = 4096, N = 1024) runs on the
    shared-memory one-CTA form; 20,000 binary64 weights on the other one."""
    out = torch.empty(1024, dtype=torch.int32, device="cuda")
    wd = dev(workloads.weights_lognormal(20_000, 2.0, seed=2))
    g.rs_trace_enable(h.h, True)
    try:
        g.rs_resample_w(h.h, wd, 4096, 1024, 1, 0, out)
        g.rs_resample_w(h.h, wd, 20_000, 1024, 1, 0, out)
        g.rs_trace_collect(h.h)
        rep = g.rs_trace_report(h.h)
    finally:
        g.rs_trace_enable(h.h, False)
        g.rs_trace_reset(h.h)
    assert h.status() == g.RS_OK
    assert rep["small_smem"][0] == 1 and rep["single_cta"][0] == 1, rep


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("which", ["all_few", "mixed", "all_many"])
def test_fused_draw_split_modes(g, h, prec, which):
    """The cooperative launch splits a CTA's draws over 15 warps when it holds
    at most 2048 of them, else over all 16 with per-warp prefixes.  N = 2048 B - 1
    (every CTA exactly 2048 draws), N = 2048 B (one CTA 2049: both modes in one
    launch) and N = 600,000 (every CTA above 2048) against the multi-kernel path."""
    B = torch.cuda.get_device_properties(0).multi_processor_count
    N = {"all_few": 2048 * B - 1, "mixed": 2048 * B, "all_many": 600_000}[which]
    M = N + 12_345
    w = workloads.weights_lognormal(M, 2.0, seed=N)
    if prec == "f32":
        w = w.astype(np.float32)
    p = g.RS_F32_COMP if prec == "f32" else g.RS_F64
    wd = dev(w)
    a = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    b = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    g.rs_resample_w(h.h, wd, M, N, 17, 3, a, None, g.opts(prec=p))
    g.rs_resample_w(h.h, wd, M, N, 17, 3, b, None, g.opts(prec=p, debug_flags=2))
    assert h.status() == g.RS_OK
    ra = host(a)
    assert np.array_equal(ra, host(b))
    assert ra.min() >= 0 and ra.max() < M and np.all(np.diff(ra) >= 0)


@pytest.mark.parametrize("kind", workloads.ADVERSARIAL)
@pytest.mark.parametrize("M,N", [(7 * 4096 + 3, 5000), (7 * 4096 + 3, 2000)])
def test_fused_equals_multikernel_adversarial(g, h, kind, M, N):
    """Adversarial weights on the cooperative launch (N = 5000) and on the
    one-CTA path of small instances (N = 2000) against the multi-kernel path."""
    w = workloads.adversarial_weights(kind, M, seed=4)
    wd = dev(w)
    a = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    b = torch.full((N,), -2, dtype=torch.int32, device="cuda")
    g.rs_resample_w(h.h, wd, M, N, 5, 0, a)
    g.rs_resample_w(h.h, wd, M, N, 5, 0, b, None, g.opts(debug_flags=2))
    assert h.status() == g.RS_OK
    assert np.array_equal(host(a), host(b))


def test_fused_bounded_wait_times_out_and_context_survives(g, h):
    w = workloads.weights_lognormal(50_000, 2.0, seed=3)
    wd = dev(w)
    out = torch.empty(5000, dtype=torch.int32, device="cuda")
    g.rs_resample_w(h.h, wd, w.size, 5000, 1, 0, out, None, g.opts(spin_limit=200, debug_flags=1))
    assert h.status() == g.RS_ETIMEOUT
    g.rs_resample_w(h.h, wd, w.size, 5000, 1, 0, out)
    assert h.status() == g.RS_OK
    r = host(out)
    assert r.min() >= 0 and r.max() < w.size
