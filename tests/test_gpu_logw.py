"""GPU parity of the log-weight input: rs_softmax_weights against the oracle's
binary64 exp(l - max l), and rs_resample_logw end to end (boundary-only
index differences on the oracle's cumulative weights)."""
import numpy as np
import pytest

import oracle
from parity_util import REL_F64, assert_boundary_only

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


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def softmax_gpu(g, h, l):
    w = torch.full((l.size,), np.nan, dtype=torch.float64, device="cuda")
    g.rs_softmax_weights(h.h, torch.from_numpy(l).cuda(), l.size, w)
    return w


@pytest.mark.parametrize("sigma,M,shift", [(1.0, 1, 3.0), (2.0, 513, 3.0), (2.0, 100_003, 3.0),
                                           (10.0, 1_000_000, 3.0), (100.0, 50_000, 3.0),
                                           (1e-3, 20_000, 0.0), (50.0, 30_000, -1e6), (2.0, 30_000, 4e4)])
def test_softmax_weights_accuracy(g, h, sigma, M, shift):
    l = np.random.default_rng(M).normal(0.0, sigma, size=M) + shift
    w = host(softmax_gpu(g, h, l))
    assert h.status() == g.RS_OK
    ref = oracle.softmax_weights(l)
    x = l - l.max()
    # the GPU takes exp of the exact l - m in integer arithmetic (below 2^-49
    # relative); the oracle rounds l - m to binary64 first, which moves exp by
    # up to 2^-53 |l - m| relative, and its exp by about 2^-52; subnormal
    # results to an absolute 2^-1060
    tol = np.maximum((2.0 ** -48 + 2.0 ** -52 * (np.abs(x) + 1.0)) * ref, 2.0 ** -1060)
    bad = np.abs(w - ref) > tol
    assert not bad.any(), (x[bad][:3], w[bad][:3], ref[bad][:3])
    assert w[np.argmax(l)] == 1.0


def test_softmax_subnormal_band(g, h):
    """Results from 2^-1022 down to the underflow to 0 (x in [-746, -700])."""
    l = np.concatenate([[0.0], -700.0 - 46.0 * np.random.default_rng(3).random(20_000)])
    w = host(softmax_gpu(g, h, l))
    assert h.status() == g.RS_OK
    ref = oracle.softmax_weights(l)
    assert np.all(np.abs(w - ref) <= np.maximum(2.0 ** -1072, 2.0 ** -46 * ref))
    assert np.all(w[l < -745.2] == 0.0)


def test_softmax_special_values(g, h):
    l = np.array([-np.inf, 0.5, -3.0, -np.inf, 0.5, -800.0, -1e-200, 2e-130])
    w = host(softmax_gpu(g, h, l))
    assert h.status() == g.RS_OK
    ref = oracle.softmax_weights(l)
    assert w[0] == 0 and w[3] == 0 and w[1] == 1.0 and w[4] == 1.0
    assert w[5] == 0.0  # exp(-800.5) is below the binary64 range
    assert np.allclose(w[[2, 6, 7]], ref[[2, 6, 7]], rtol=2e-13, atol=0)


@pytest.mark.parametrize("bad,code", [(np.nan, "RS_ENONFINITE"), (np.inf, "RS_ENONFINITE"), (3e38, "RS_ENONFINITE")])
def test_softmax_invalid_latches(g, h, bad, code):
    l = np.zeros(1000)
    l[77] = bad
    softmax_gpu(g, h, l)
    assert h.status() == getattr(g, code)


def test_softmax_all_minus_inf_latches(g, h):
    w = host(softmax_gpu(g, h, np.full(300, -np.inf)))
    assert h.status() == g.RS_EZEROSUM
    assert np.all(w == 0)


@pytest.mark.parametrize("sigma,M,N", [(2.0, 4096, 1024), (2.0, 1_000_003, 4097), (10.0, 2_000_000, 100_000),
                                       (1.5, 5000, 9000)])
def test_resample_logw_end_to_end(g, h, sigma, M, N):
    l = np.random.default_rng(N).normal(-5.0, sigma, size=M)
    w_ref = oracle.softmax_weights(l)
    r_ref, W_ref, U_ref = oracle.resample(w_ref, N, 41)
    out = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    g.rs_resample_logw(h.h, torch.from_numpy(l).cuda(), M, N, 41, 0, out)
    assert h.status() == g.RS_OK
    assert_boundary_only(host(out), r_ref, W_ref, U_ref, rel=REL_F64)


def test_resample_logw_engmf_full(g, h):
    """The engmf instance from its log-weights (M = 16,777,216, N = 4,096)."""
    import workloads
    rng = np.random.default_rng(workloads.CONFIGS["engmf"]["seed"])
    l = rng.normal(0.0, 2.0, size=workloads.CONFIGS["engmf"]["M"])
    N = workloads.CONFIGS["engmf"]["N"]
    w_ref = oracle.softmax_weights(l)
    r_ref, W_ref, U_ref = oracle.resample(w_ref, N, 12)
    out = torch.full((N,), -1, dtype=torch.int32, device="cuda")
    g.rs_resample_logw(h.h, torch.from_numpy(l).cuda(), l.size, N, 12, 0, out)
    assert h.status() == g.RS_OK
    assert_boundary_only(host(out), r_ref, W_ref, U_ref, rel=REL_F64)
