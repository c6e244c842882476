"""GPU parity of rs_gather (x'_i = x_{r_i}): byte-exact against numpy
indexing, for row sizes and alignments that take each copy width."""
import numpy as np
import pytest

import oracle
import workloads
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


@pytest.mark.parametrize("dtype,D", [(np.float64, 1), (np.float64, 2), (np.float64, 4), (np.float64, 7),
                                     (np.float32, 1), (np.float32, 3), (np.float32, 4), (np.float32, 33),
                                     (np.float64, 64)])
@pytest.mark.parametrize("M,N", [(1, 1), (1000, 3001), (100_003, 50_000)])
def test_gather_matches_numpy(g, h, dtype, D, M, N):
    rng = np.random.default_rng(M + D)
    x = rng.standard_normal((M, D)).astype(dtype)
    idx = rng.integers(0, M, size=N).astype(np.int32)
    xd = torch.from_numpy(x).cuda()
    out = torch.full((N, D), np.nan, dtype=xd.dtype, device="cuda")
    g.rs_gather(h.h, xd, M, D * x.itemsize, torch.from_numpy(idx).cuda(), N, out)
    assert h.status() == g.RS_OK
    assert np.array_equal(out.cpu().numpy().view(np.uint8), x[idx].view(np.uint8))


def test_gather_unaligned_offset(g, h):
    # an x pointer 4 bytes past a 16-byte boundary takes the 4-byte copies
    M, D, N = 5000, 4, 7000
    rng = np.random.default_rng(1)
    base = torch.from_numpy(rng.standard_normal(M * D + 1).astype(np.float32)).cuda()
    x = base[1:]
    idx = rng.integers(0, M, size=N).astype(np.int32)
    out = torch.empty(N * D, dtype=torch.float32, device="cuda")
    g.rs_gather(h.h, x, M, D * 4, torch.from_numpy(idx).cuda(), N, out)
    assert h.status() == g.RS_OK
    ref = base.cpu().numpy()[1:].reshape(M, D)[idx].reshape(-1)
    assert np.array_equal(out.cpu().numpy(), ref)


def test_gather_after_resampling(g, h):
    """The filter step: resample the bootstrap-shaped weights, then move the
    particles: the moved rows are those the (oracle-checked) indices select."""
    M, N, D = 200_000, 200_000, 4
    w = workloads.weights_bootstrap(M, seed=3)
    x = np.random.default_rng(2).standard_normal((M, D))
    out_idx = torch.empty(N, dtype=torch.int32, device="cuda")
    g.rs_resample_w(h.h, torch.from_numpy(w).cuda(), M, N, 7, 0, out_idx)
    xo = torch.empty((N, D), dtype=torch.float64, device="cuda")
    g.rs_gather(h.h, torch.from_numpy(x).cuda(), M, D * 8, out_idx, N, xo)
    assert h.status() == g.RS_OK
    r = out_idx.cpu().numpy()
    r_ref, W_ref, U_ref = oracle.resample(w, N, 7)
    assert_boundary_only(r, r_ref, W_ref, U_ref, rel=REL_F64)
    assert np.array_equal(xo.cpu().numpy(), x[r])


def test_gather_bad_index_latches(g, h):
    x = torch.arange(40, dtype=torch.float32, device="cuda").reshape(10, 4)
    idx = torch.tensor([0, 9, 10, -1], dtype=torch.int32, device="cuda")
    out = torch.full((4, 4), 7.0, dtype=torch.float32, device="cuda")
    g.rs_gather(h.h, x, 10, 16, idx, 4, out)
    assert h.status() == g.RS_EINVAL
    o = out.cpu().numpy()
    assert np.array_equal(o[:2], x.cpu().numpy()[[0, 9]]) and np.all(o[2:] == 0)
    with pytest.raises(g.ResampleError):
        g.rs_gather(h.h, x, 10, 6, idx, 4, out)  # row_bytes not a multiple of 4
