"""GPU: the autotuners and the persistence of their settings.

The tuned settings only choose among equivalent kernels (leaf sizes, CTA
sizes), so every choice must give the same indices; the tests tune, save,
reload (explicitly and through rs_create's GBRESAMPLE_TUNING), and check that
a reloaded handle uses the saved values and reproduces the indices.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def g():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2604_01356_gb300 as g
    return g


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def test_map_tune_save_reload_identical(g, tmp_path):
    M, N = 200_000, 2000
    W, _ = oracle.cumulative(workloads.weights_lognormal(M, 2.0, seed=3))
    Wd = dev(W)
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    h = g.Handle()
    best = g.rs_autotune_map(h.h, Wd, M, N, 5, out)
    assert best.algo == g.RS_MAP_DAC and best.leaf_L in [1 << k for k in range(9)]
    assert g.rs_tuning_get(h.h, 0, g.RS_F64, M, N).leaf_L == best.leaf_L
    # the tuned leaf is used when leaf_L is 0, and gives the explicit leaf's indices
    a = torch.empty(N, dtype=torch.int32, device="cuda")
    b = torch.empty(N, dtype=torch.int32, device="cuda")
    g.rs_resample_W(h.h, Wd, M, N, 9, 0, a, g.opts(algo=g.RS_MAP_DAC))
    g.rs_resample_W(h.h, Wd, M, N, 9, 0, b, g.opts(algo=g.RS_MAP_DAC, leaf_L=best.leaf_L))
    assert h.status() == g.RS_OK
    assert np.array_equal(host(a), host(b))
    U = oracle.sorted_uniform(N, 9, 0)
    assert np.array_equal(host(a), oracle.inverse_cdf_walk(W, U))
    path = tmp_path / "tuning.json"
    g.rs_tuning_save(h.h, path)
    doc = json.loads(path.read_text())
    ent = [e for e in doc["entries"] if e["kind"] == "map_dac"]
    assert ent and ent[0]["leaf_L"] == best.leaf_L and ent[0]["dtype"] == "f64"
    assert ent[0]["gpu"] == torch.cuda.get_device_name(0)
    h.close()
    # a fresh handle: nothing tuned, then the file's value
    h2 = g.Handle()
    assert g.rs_tuning_get(h2.h, 0, g.RS_F64, M, N).leaf_L == 0
    g.rs_tuning_load(h2.h, path)
    assert g.rs_tuning_get(h2.h, 0, g.RS_F64, M, N).leaf_L == best.leaf_L
    c = torch.empty(N, dtype=torch.int32, device="cuda")
    g.rs_resample_W(h2.h, Wd, M, N, 9, 0, c, g.opts(algo=g.RS_MAP_DAC))
    assert h2.status() == g.RS_OK
    assert np.array_equal(host(c), host(a))
    h2.close()


def test_batched_tune_persist_and_entries_of_other_gpus_kept(g, tmp_path):
    w, woff, roff = workloads.weights_batched(K=64, seed=4, nmin=16, nmax=400, pmax=20)
    K = 64
    out = torch.empty(int(roff[-1]), dtype=torch.int32, device="cuda")
    h = g.Handle()
    best = g.rs_autotune_batched(h.h, dev(w), dev(woff), dev(roff), K, 3, out, woff, roff)
    r1 = host(out).copy()
    path = tmp_path / "tuning.json"
    path.write_text(json.dumps({"entries": [{"gpu": "some other GPU", "kind": "map_dac", "dtype": "f64",
                                             "mn_bucket": 3, "tile_threads": 0, "leaf_L": 64}]}))
    g.rs_tuning_save(h.h, path)
    doc = json.loads(path.read_text())
    kinds = {(e["gpu"] == "some other GPU", e["kind"]) for e in doc["entries"]}
    assert (True, "map_dac") in kinds and (False, "batched") in kinds
    h.close()
    h2 = g.Handle()
    g.rs_tuning_load(h2.h, path)
    t = g.rs_tuning_get(h2.h, 1, g.RS_F32_COMP, int(woff[-1]), int(roff[-1]))
    assert (t.tile_threads, t.leaf_L) == (best.tile_threads, best.leaf_L)
    assert g.rs_tuning_get(h2.h, 0, g.RS_F64, 8, 1).leaf_L == 0  # the other GPU's entry is not taken
    out2 = torch.full_like(out, -1)
    g.rs_resample_batched(h2.h, dev(w), dev(woff), dev(roff), K, 3, out2, woff, roff)
    assert h2.status() == g.RS_OK
    assert np.array_equal(host(out2), r1)
    h2.close()


def test_rs_create_loads_the_tuning_file(g, tmp_path):
    """GBRESAMPLE_TUNING is read by rs_create (in a fresh process, so that the
    variable is seen from the start); a malformed file leaves the defaults."""
    path = tmp_path / "tuning.json"
    name = torch.cuda.get_device_name(0)
    path.write_text(json.dumps({"entries": [{"gpu": name, "kind": "map_dac", "dtype": "f64", "mn_bucket": 7,
                                             "tile_threads": 0, "leaf_L": 16}]}))
    bad = tmp_path / "bad.json"
    bad.write_text("not json")
    code = ("import paper_2604_01356_gb300 as g, sys\n"
            "h = g.Handle()\n"
            "print(g.rs_tuning_get(h.h, 0, g.RS_F64, 128 * 1000, 1000).leaf_L)\n")
    for p, want in [(path, "16"), (bad, "0")]:
        env = dict(os.environ, GBRESAMPLE_TUNING=str(p))
        r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                           timeout=300)
        assert r.returncode == 0, r.stderr
        assert r.stdout.strip().splitlines()[-1] == want
