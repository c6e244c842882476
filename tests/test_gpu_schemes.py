"""GPU parity of the stratified and systematic points (rs_opts.scheme).

U_i = (i-1+v_{i-1})/N or (i-1+v_0)/N with Algorithm 1's draws, through every
entry point that generates points: rs_sorted_uniform, rs_resample_W (the three
maps), rs_resample_w (single cooperative launch and multi-kernel path) and
rs_resample_batched; checked against the oracle's definition.
"""
import numpy as np
import pytest

import oracle
import workloads
from parity_util import ABS_F32, REL_F64, assert_boundary_only

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCHEMES = ["stratified", "systematic"]


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


def code(g, scheme):
    return {"stratified": g.RS_SCHEME_STRATIFIED, "systematic": g.RS_SCHEME_SYSTEMATIC}[scheme]


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("N", [1, 2, 1023, 1024, 1025, 4097, 100_003])
def test_scheme_points_f64(g, h, scheme, N):
    U = torch.empty(N, dtype=torch.float64, device="cuda")
    g.rs_sorted_uniform(h.h, N, 21, 4, U, g.opts(scheme=code(g, scheme)))
    assert h.status() == g.RS_OK
    got = host(U)
    ref = oracle.scheme_uniform(N, 21, 4, scheme)
    assert np.all(np.diff(got) >= 0) and got[-1] <= 1.0
    assert np.max(np.abs(got - ref) / ref) <= 1e-13


@pytest.mark.parametrize("scheme", SCHEMES)
def test_scheme_points_f32(g, h, scheme):
    N = 5000
    U = torch.empty(N, dtype=torch.float64, device="cuda")
    g.rs_sorted_uniform(h.h, N, 3, 1, U, g.opts(prec=g.RS_F32_COMP, scheme=code(g, scheme)))
    assert h.status() == g.RS_OK
    ref = oracle.scheme_uniform(N, 3, 1, scheme, single=True)
    assert np.max(np.abs(host(U) - ref)) <= ABS_F32


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("M,N", [(1, 3), (513, 1000), (9 * 4096 + 5, 4097), (1_000_003, 300_001), (200_000, 200_000),
                                 (600_001, 600_000)])
def test_scheme_resample_w_fused_and_multikernel(g, h, scheme, M, N):
    w = workloads.weights_lognormal(M, 2.0, seed=M + 7)
    r_ref, W_ref, U_ref = oracle.resample_scheme(w, N, 99, scheme)
    a = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    b = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    wd = dev(w)
    g.rs_resample_w(h.h, wd, M, N, 99, 0, a, None, g.opts(scheme=code(g, scheme)))
    g.rs_resample_w(h.h, wd, M, N, 99, 0, b, None, g.opts(scheme=code(g, scheme), debug_flags=2))
    assert h.status() == g.RS_OK
    ra, rb = host(a), host(b)
    assert np.array_equal(ra, rb)
    assert_boundary_only(ra, r_ref, W_ref, U_ref, rel=REL_F64)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("algo", ["dac", "binary", "linear"])
def test_scheme_resample_W_maps(g, h, scheme, algo):
    M, N = 100_000, 3000
    w = workloads.weights_lognormal(M, 2.0, seed=12)
    r_ref, W_ref, U_ref = oracle.resample_scheme(w, N, 5, scheme)
    a = {"dac": g.RS_MAP_DAC, "binary": g.RS_MAP_BINARY, "linear": g.RS_MAP_LINEAR}[algo]
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    g.rs_resample_W(h.h, dev(W_ref), M, N, 5, 0, out, g.opts(algo=a, scheme=code(g, scheme)))
    assert h.status() == g.RS_OK
    assert_boundary_only(host(out), r_ref, W_ref, U_ref, rel=REL_F64)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_scheme_batched_equals_instances(g, h, scheme):
    K = 60
    w, woff, roff = workloads.weights_batched(K=K, seed=9, nmin=1, nmax=700, pmax=40)
    out = torch.full((int(roff[-1]),), -1, dtype=torch.int32, device="cuda")
    o = g.opts(prec=g.RS_F32_COMP, scheme=code(g, scheme))
    g.rs_resample_batched(h.h, dev(w), dev(woff), dev(roff), K, 8, out, woff, roff, o)
    assert h.status() == g.RS_OK
    got = host(out)
    for k in range(K):
        a, b = int(roff[k]), int(roff[k + 1])
        Mk = int(woff[k + 1] - woff[k])
        ok = torch.empty(b - a, dtype=torch.int32, device="cuda")
        g.rs_resample_w(h.h, dev(w[woff[k]:woff[k + 1]]), Mk, b - a, 8, k, ok, None, o)
        assert np.array_equal(host(ok), got[a:b]), k


def test_systematic_counts_floor_or_ceil_gpu(g, h):
    # equally spaced points: index j is drawn floor(N w_j) or ceil(N w_j)
    # times (up to the rounding of W at a point exactly on a boundary)
    M, N = 300_000, 100_000
    w = workloads.weights_lognormal(M, 1.0, seed=31)
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    g.rs_resample_w(h.h, dev(w), M, N, 4, 0, out, None, g.opts(scheme=g.RS_SCHEME_SYSTEMATIC))
    assert h.status() == g.RS_OK
    c = np.bincount(host(out), minlength=M)
    e = N * w / w.sum()
    off = (c < np.floor(e - 1e-9)) | (c > np.ceil(e + 1e-9))
    assert np.all(np.abs(c - e) <= 2) and off.sum() <= 2


def test_scheme_engmf_full_graph(g, h):
    """The engmf instance (M = 16,777,216, N = 4,096), stratified, replayed
    from a CUDA graph as the benchmark launches it."""
    wl = workloads.make("engmf")
    r_ref, W_ref, U_ref = oracle.resample_scheme(wl.w, wl.N, wl.seed, "stratified")
    wd = dev(wl.w)
    out = torch.full((wl.N,), -1, dtype=torch.int32, device="cuda")
    o = g.opts(scheme=g.RS_SCHEME_STRATIFIED)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        g.rs_resample_w(h.h, wd, wl.M, wl.N, wl.seed, 0, out, None, o, stream=stream)
    stream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        g.rs_resample_w(h.h, wd, wl.M, wl.N, wl.seed, 0, out, None, o, stream=torch.cuda.current_stream())
    out.fill_(-1)
    graph.replay()
    torch.cuda.synchronize()
    assert h.status() == g.RS_OK
    assert_boundary_only(host(out), r_ref, W_ref, U_ref, rel=REL_F64)


def test_scheme_invalid_rejected(g, h):
    U = torch.empty(4, dtype=torch.float64, device="cuda")
    with pytest.raises(g.ResampleError):
        g.rs_sorted_uniform(h.h, 4, 1, 0, U, g.opts(scheme=3))
