"""GPU: the batched persistent path (many instances in one launch).

Its indices must equal, bit for bit, those of rs_resample_w's multi-kernel
path run on each instance alone (same precision, binary32 or binary64): both
use the same exact integer arithmetic.  The per-instance path is itself checked against the oracle in
test_gpu_parity; here the batched result is also checked against the oracle
directly on a small batch.
"""
import numpy as np
import pytest

import oracle
import workloads
from parity_util import ABS_F32, assert_boundary_only

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


def _mixed_batch(seed):
    """Ragged sizes, instances with N_k = 0, odd offsets (unaligned starts),
    one instance above the persistent kernel's 262,144-weight limit."""
    rng = np.random.default_rng(seed)
    Mk = [1, 2, 511, 512, 513, 4097, 300_001, 70_000, 1, 9_999, 262_144, 262_145, 33, 0, 5000]
    Nk = [1, 7, 100, 512, 3, 4097, 2000, 1, 0, 10_000, 300, 17, 64, 0, 2048]
    woff = np.zeros(len(Mk) + 1, dtype=np.int64)
    roff = np.zeros(len(Mk) + 1, dtype=np.int64)
    np.cumsum(Mk, out=woff[1:])
    np.cumsum(Nk, out=roff[1:])
    w = np.exp(rng.normal(0.0, 1.5, size=int(woff[-1]))).astype(np.float32)
    w[rng.random(w.size) < 0.1] = 0.0  # zero runs
    for k in range(len(Mk)):  # keep every instance's total positive
        if Mk[k]:
            w[woff[k]] = 1.0
    return w, woff, roff


def _per_instance(g, h, w, woff, roff, seed, prec=None):
    """Every instance through rs_resample_w's multi-kernel path (debug bit
    1), which shares no kernel with the persistent one."""
    prec = g.RS_F32_COMP if prec is None else prec
    K = len(woff) - 1
    out = torch.empty(max(int(roff[-1]), 1), dtype=torch.int32, device="cuda")
    wd = dev(w)
    for k in range(K):
        Mk, Nk = int(woff[k + 1] - woff[k]), int(roff[k + 1] - roff[k])
        if Nk == 0:
            continue
        wk = wd[int(woff[k]):int(woff[k + 1])]
        ok = out[int(roff[k]):int(roff[k + 1])]
        g.rs_resample_w(h.h, wk, Mk, Nk, seed, k, ok, None, g.opts(prec=prec, debug_flags=2))
    assert h.status() == g.RS_OK
    return host(out)[: int(roff[-1])]


@pytest.mark.parametrize("prec", ["f32", "f64"])
@pytest.mark.parametrize("threads", [128, 256, 512])
@pytest.mark.parametrize("leaf", [1, 4, 32, 1024])
def test_batched_equals_per_instance_bit_exact(g, h, threads, leaf, prec):
    w, woff, roff = _mixed_batch(11)
    p = g.RS_F32_COMP if prec == "f32" else g.RS_F64
    if prec == "f64":
        w = w.astype(np.float64)
    ref = _per_instance(g, h, w, woff, roff, seed=5, prec=p)
    out = torch.full((int(roff[-1]),), -1, dtype=torch.int32, device="cuda")
    g.rs_resample_batched(h.h, dev(w), dev(woff), dev(roff), len(woff) - 1, 5, out, woff, roff,
                          g.opts(prec=p, tile_threads=threads, leaf_L=leaf))
    assert h.status() == g.RS_OK
    assert np.array_equal(host(out), ref)


@pytest.mark.parametrize("kind", workloads.ADVERSARIAL)
def test_batched_f64_adversarial_heads(g, h, kind):
    """Binary64 weights through the persistent kernel: adversarial weight
    vectors (zero runs, ties, a spike, tiny/huge/wide dynamic ranges) whose
    head segments need the exact per-element decision, against the
    multi-kernel path on each instance."""
    Mk = [4096, 513, 20_000, 1, 777]
    Nk = [1000, 513, 2048, 5, 300]
    woff = np.zeros(len(Mk) + 1, dtype=np.int64)
    roff = np.zeros(len(Mk) + 1, dtype=np.int64)
    np.cumsum(Mk, out=woff[1:])
    np.cumsum(Nk, out=roff[1:])
    w = np.concatenate([workloads.adversarial_weights(kind, m, seed=i) for i, m in enumerate(Mk)])
    ref = _per_instance(g, h, w, woff, roff, seed=21, prec=g.RS_F64)
    out = torch.full((int(roff[-1]),), -1, dtype=torch.int32, device="cuda")
    g.rs_resample_batched(h.h, dev(w), dev(woff), dev(roff), len(Mk), 21, out, woff, roff, g.opts(prec=g.RS_F64))
    assert h.status() == g.RS_OK
    assert np.array_equal(host(out), ref)


def test_batched_without_host_offsets(g, h):
    w, woff, roff = workloads.weights_batched(K=300, seed=7, nmin=16, nmax=600, pmax=40)
    ref = _per_instance(g, h, w, woff, roff, seed=9)
    out = torch.full((int(roff[-1]),), -1, dtype=torch.int32, device="cuda")
    g.rs_resample_batched(h.h, dev(w), dev(woff), dev(roff), 300, 9, out)
    assert h.status() == g.RS_OK
    assert np.array_equal(host(out), ref)


def test_batched_against_oracle(g, h):
    K = 40
    w, woff, roff = workloads.weights_batched(K=K, seed=8, nmin=8, nmax=700, pmax=70)
    r_ref = oracle.resample_batched(w, woff, roff, seed=4, single=True)
    out = torch.empty(int(roff[-1]), dtype=torch.int32, device="cuda")
    g.rs_resample_batched(h.h, dev(w), dev(woff), dev(roff), K, 4, out, woff, roff)
    assert h.status() == g.RS_OK
    got = host(out)
    assert np.count_nonzero(got != r_ref) <= 2
    for k in range(K):
        a, b = int(roff[k]), int(roff[k + 1])
        Wk, _ = oracle.cumulative(w[woff[k]:woff[k + 1]])
        Uk = oracle.sorted_uniform(b - a, 4, k, single=True)
        assert_boundary_only(got[a:b], r_ref[a:b], Wk, Uk, abs_tol=ABS_F32, max_frac=0.0)


def test_batched_large_k_identity_order(g, h):
    # more instances than the device sort handles: identity work order
    K = 20_000
    woff, roff, _ = workloads.batched_layout(K=K, seed=12, nmin=1, nmax=8, pmax=3)
    rng = np.random.default_rng(1)
    w = rng.exponential(size=int(woff[-1])).astype(np.float32)
    out = torch.full((int(roff[-1]),), -1, dtype=torch.int32, device="cuda")
    g.rs_resample_batched(h.h, dev(w), dev(woff), dev(roff), K, 2, out, woff, roff)
    assert h.status() == g.RS_OK
    got = host(out)
    # spot-check 50 instances against the single-instance path
    for k in rng.choice(K, size=50, replace=False):
        a, b = int(roff[k]), int(roff[k + 1])
        Mk = int(woff[k + 1] - woff[k])
        ok = torch.empty(b - a, dtype=torch.int32, device="cuda")
        g.rs_resample_w(h.h, dev(w[woff[k]:woff[k + 1]]), Mk, b - a, 2, int(k), ok, None,
                        g.opts(prec=g.RS_F32_COMP))
        assert np.array_equal(host(ok), got[a:b]), k


def test_batched_zero_sum_instance_latches(g, h):
    w, woff, roff = workloads.weights_batched(K=5, seed=2, nmin=8, nmax=64, pmax=4)
    w[woff[3]:woff[4]] = 0.0
    out = torch.empty(int(roff[-1]), dtype=torch.int32, device="cuda")
    g.rs_resample_batched(h.h, dev(w), dev(woff), dev(roff), 5, 1, out, woff, roff)
    assert h.status() == g.RS_EZEROSUM
    got = host(out)
    assert got.min() >= 0


def test_autotune_batched(g, h):
    w, woff, roff = workloads.weights_batched(K=64, seed=6, nmin=32, nmax=512, pmax=32)
    out = torch.empty(int(roff[-1]), dtype=torch.int32, device="cuda")
    best = g.rs_autotune_batched(h.h, dev(w), dev(woff), dev(roff), 64, 3, out, woff, roff)
    assert best.tile_threads in (128, 256, 512) and best.leaf_L in (4, 16, 64)
    ref = _per_instance(g, h, w, woff, roff, seed=3)
    out2 = torch.full((int(roff[-1]),), -1, dtype=torch.int32, device="cuda")
    g.rs_resample_batched(h.h, dev(w), dev(woff), dev(roff), 64, 3, out2, woff, roff)  # uses the tuned values
    assert h.status() == g.RS_OK
    assert np.array_equal(host(out2), ref)
