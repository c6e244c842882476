"""The benchmark's reference arm on CPU: one JSON line with the required keys
(the oracle timed on a bounded sample of the engmf workload), and silence
from every rank but 0."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(env_extra):
    env = dict(os.environ)
    env.update(env_extra)
    return subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                           "--warmup", "0"], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_reference_arm_json_line():
    p = run_bench({"RANK": "0", "WORLD_SIZE": "1"})
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference"
    assert d["value"] > 0 and d["ms_per_step"] > 0 and d["steps"] == 1 and d["warmup"] == 0
    assert d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"].startswith("engmf")
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    e = d["e2e"]
    assert e["value"] == d["value"] and e["unit"] == d["unit"]
    assert e["h2d_bytes_per_step"] == 0 and e["d2h_bytes_per_step"] == 0


def test_reference_arm_other_ranks_silent():
    p = run_bench({"RANK": "1", "WORLD_SIZE": "2"})
    assert p.returncode == 0, p.stderr[-2000:]
    assert p.stdout.strip() == ""


def test_gpu_arm_runs_no_oracle():
    """The GPU arm's measurements take their inputs from the workload
    generators or the library itself: no function of that arm names the
    oracle, and run_ours calls the oracle legs (CPU baselines, the paper
    sweep's serial maps, the accuracy report) only under the CPU-baseline
    switch."""
    import ast
    import inspect
    sys.path.insert(0, ROOT)
    import bench
    for fn in (bench.e2e_measure, bench.map_only, bench.gather_measure, bench.logw_measure, bench.batched_measure,
               bench.single_measure, bench.small_measure, bench.batched_probe, bench.small_probe, bench.logw_probe,
               bench._time_calls, bench._time_graph_calls, bench.make_flush):
        assert "oracle" not in inspect.getsource(fn), fn.__name__
    tree = ast.parse(inspect.getsource(bench.run_ours))
    legs = {"paper_sweep", "accuracy_report", "cpu_baseline", "cpu_allcore"}
    gated = set()

    def walk(node, under_switch):
        if isinstance(node, ast.If) and "no_cpu_baseline" in ast.unparse(node.test):
            for child in node.body:
                walk(child, True)
            for child in node.orelse:
                walk(child, under_switch)
            return
        if isinstance(node, ast.Call) and isinstance(node.func, ast.Name) and node.func.id in legs:
            assert under_switch, node.func.id
            gated.add(node.func.id)
        for child in ast.iter_child_nodes(node):
            walk(child, under_switch)

    walk(tree, False)
    assert gated == legs
