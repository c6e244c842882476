#!/usr/bin/env python
"""Benchmark of the multinomial resampling path on GB300.

Workload (one step = one pass of the whole path over one instance):
  engmf  M = 16,777,216 binary64 weights w = exp(l - max l), l ~ Normal(0, 2^2),
         N = 4,096 samples: cumulative weights (Eq. 3), N sorted uniforms
         (Algorithm 1), divide-and-conquer inverse-CDF map (Algorithm 5),
         through one rs_resample_w call replayed as a CUDA graph.

Prints ONE JSON line (rank 0).  `value` is resampled particles/s over all
ranks (each rank resamples its own instance: weak scaling, no collective on
the data path).  L2 is flushed (256 MiB write, read back) before every timed step and
each step is timed with CUDA events on its stream.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--path fused|multikernel] [--no-extras] [--no-cpu-baseline]
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

METRIC = "resampled particles/s and HBM GB/s vs roofline; batched FP32 vs per-instance FP64"
UNIT = "particles/s"
FALLBACK_HBM_GBS = 6800.0
L2_FLUSH_BYTES = 256 << 20


def make_flush(dev):
    """An L2 flush: write a 256 MiB buffer (larger than L2), then read it back
    so that no dirty flush lines remain to be written back inside the timed
    region.  Returns the function that flushes (outside the timed events)."""
    import torch
    buf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    sink = torch.zeros(1, dtype=torch.int64, device=dev)
    state = {"k": 0}

    def flush():
        state["k"] += 1
        buf.fill_(state["k"] & 255)
        sink.add_(buf.view(torch.int64).sum())
    return flush


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true",
                    help="skip everything that runs the oracle: the CPU baselines (one core, all cores), "
                         "the paper sweep's serial CPU maps and the accuracy report against the oracle")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the sub-measurements (e2e, map only, batched, bootstrap, stress)")
    ap.add_argument("--batched-probe", type=int, default=0, metavar="K",
                    help="only run the batched launch on the first K instances of the batched workload "
                         "(binary32, default settings; 3 + 2 launches) and print their times: a small "
                         "case for profiling the persistent kernel")
    ap.add_argument("--small-probe", action="store_true",
                    help="only run rs_resample_w and rs_resample_W (binary search) on the small workload "
                         "(M = 4096, N = 1024), 3 + 2 calls each, and print their times: a small case for "
                         "profiling the shared-memory kernels")
    ap.add_argument("--logw-probe", action="store_true",
                    help="only run rs_resample_logw on the engmf log-weights (M = 16,777,216 binary64, "
                         "N = 4,096), 3 + 2 calls, and print their times: a case for profiling the "
                         "maximum and exponent passes")
    ap.add_argument("--path", choices=["fused", "multikernel"], default="fused",
                    help="rs_resample_w as one cooperative launch (default) or through the "
                         "multi-kernel path (identical indices; for profiling and comparison)")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return FALLBACK_HBM_GBS, "fallback"


def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


_CSRC = "paper_2604_01356_gb300/csrc/"
# sources each profiled kernel is compiled from (a recorded ncu traffic figure
# is used only while they are unchanged)
KERNEL_SOURCES = {
    "w_reduce": [_CSRC + "k_weights.cu", _CSRC + "common.cuh", _CSRC + "seg_common.cuh"],
    "fused": [_CSRC + f for f in ("k_fused.cu", "map_common.cuh", "seg_common.cuh", "common.cuh")],
}


def recorded_traffic(kernel, M):
    """dram bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source (else None).  Scaled by M when captured smaller."""
    p = os.path.join(ROOT, "profiles", "ncu_counters.json")
    if not os.path.exists(p) or kernel not in KERNEL_SOURCES:
        return None
    d = json.load(open(p)).get(kernel)
    if not d or d.get("source_hash") != source_hash(KERNEL_SOURCES[kernel]):
        return None
    return d["dram_bytes_per_launch"] * (M / d["M"])


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(w, N, seed, budget_s=12.0):
    """The oracle as it stands, single-threaded, on full engmf instances."""
    import oracle
    oracle.lib()
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.resample(w, N, seed, instance=reps)
        reps += 1
        el = time.perf_counter() - t0
        if el >= budget_s or reps >= 64:
            break
    return {"value": N * reps / el, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": "%d full engmf instances (M=%d, N=%d) end to end, %.1f s" % (reps, w.size, N, el)}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.lib()
    wl = workloads.make("engmf")
    # size each step so that warmup + steps stay within about two minutes
    t0 = time.perf_counter()
    oracle.resample(wl.w, wl.N, wl.seed)
    full = time.perf_counter() - t0
    per_step = 120.0 / max(1, args.steps + args.warmup)
    frac = min(1.0, per_step / full)
    M = max(4096, int(wl.M * frac))
    N = max(1, int(wl.N * M / wl.M))
    w = wl.w[:M]
    for k in range(args.warmup):
        oracle.resample(w, N, wl.seed, instance=k)
    times = []
    for k in range(args.steps):
        t = time.perf_counter()
        oracle.resample(w, N, wl.seed, instance=k)
        times.append(time.perf_counter() - t)
    ms = 1e3 * statistics.mean(times)
    value = N / (ms * 1e-3)
    sample = "first %d weights of the engmf instance with N=%d (M/N as in the full workload)" % (M, N)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "engmf (oracle sample)", "M": M, "N": N},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def rank_instance(rank):
    """Instance id (the Philox stream) a rank resamples: every rank draws its
    own independent instance, so ranks never exchange data."""
    return rank


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (the whole job ends with its slowest
    rank); x itself when there is one rank."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world_size, units_per_rank_step, steps, total_ms):
    """Units all ranks processed per second over the (max-over-ranks) time."""
    return world_size * units_per_rank_step * steps / (total_ms * 1e-3)


def run_ours(args):
    import torch
    import paper_2604_01356_gb300 as g

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    wl = workloads.make("engmf")
    M, N, seed = wl.M, wl.N, wl.seed
    wd = torch.from_numpy(wl.w).to(dev)
    out = torch.empty(N, dtype=torch.int32, device=dev)
    flush = make_flush(dev)
    h = g.Handle()
    stream = torch.cuda.Stream(device=dev)
    inst = rank_instance(rank)

    o_path = g.opts(debug_flags=2) if args.path == "multikernel" else None

    def step(s):
        g.rs_resample_w(h.h, wd, M, N, seed, inst, out, None, o_path, stream=s)

    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):
            flush()
            step(stream)
    stream.synchronize()
    if h.status() != g.RS_OK:
        raise RuntimeError("device status after warm-up")

    # one step captured as a CUDA graph, with per-kernel trace events inside
    g.rs_trace_enable(h.h, True)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        step(torch.cuda.current_stream())
    torch.cuda.synchronize()
    g.rs_trace_reset(h.h)

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    sampler = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    time.sleep(0.3)
    with torch.cuda.stream(stream):
        for k in range(K):
            flush()
            ev[k][0].record(stream)
            graph.replay()
            ev[k][1].record(stream)
            g.rs_trace_collect(h.h, keep=True)  # per-kernel event pairs of this replay
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    trace = g.rs_trace_report(h.h)
    g.rs_trace_enable(h.h, False)
    total_ms = max_over_ranks(float(sum(step_ms)), dist, dev)
    if h.status() != g.RS_OK:
        raise RuntimeError("device status after the timed region")
    ms_per_step = total_ms / K
    value = whole_job_rate(ws, N, K, total_ms)

    hbm, peak_kind = peaks()
    # dominant kernel: the single cooperative launch when the device holds it
    # (reads w, writes the indices), else the weights pass of the multi-kernel
    # path (reads w)
    kname = "fused" if "fused" in trace else "w_reduce"
    n_tr, ms_tr = trace.get(kname, (0, 0.0))
    dom_ms = ms_tr / n_tr if n_tr else None
    alg_dom = 8 * M + 4 * N if kname == "fused" else 8 * M
    achieved = alg_dom / (dom_ms * 1e-3) / 1e9 if dom_ms else None
    traffic = recorded_traffic(kname, M)
    roofline = {"bound": "hbm", "kernel": "k_" + kname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": (achieved / hbm) if achieved else None, "traffic": traffic,
                "peak_source": peak_kind, "algorithmic_bytes_per_launch": alg_dom,
                "avg_launch_us": dom_ms * 1e3 if dom_ms else None}
    path_bytes = 8 * M + 4 * N
    kernels_per_step = sum(n for name, (n, _) in trace.items() if name != "clear") / max(1, n_tr)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "engmf: M=16,777,216 binary64 weights exp(l - max l), l~Normal(0,2^2); N=4,096; "
                               "rs_resample_w (Eq.3 + Alg.1 + segmented DaC map) as a CUDA graph",
                   "M": M, "N": N, "precision": "f64", "l2": "flushed before every timed step (256 MiB write, then read back so no dirty lines remain)",
                   "parallelism": "independent instance per GPU" if ws > 1 else "single GPU",
                   "path": args.path},
        "roofline": roofline,
        "path": {"algorithmic_bytes": path_bytes, "GBps": path_bytes / (ms_per_step * 1e-3) / 1e9,
                 "frac": path_bytes / (ms_per_step * 1e-3) / 1e9 / hbm,
                 "kernel_avg_us": {k: 1e3 * v[1] / v[0] for k, v in trace.items() if v[0]}},
        "clocks": clocks,
        "gpu_launches": int(round(kernels_per_step * K)),
    }

    if not args.no_extras:
        line["e2e"] = e2e_measure(g, h, wl, dev, stream, min(K, 100), inst)
        if ws == 1:
            line["map_only"] = map_only(g, h, wl, dev, stream)
            line["gather"] = gather_measure(g, h, dev, stream, hbm)
            line["logw"] = logw_measure(g, h, dev, stream, hbm)
            if not args.no_cpu_baseline:  # its CPU half is the oracle's serial maps
                line["paper_sweep"] = paper_sweep(g, h, dev, stream)
            del wd, flush, graph
            torch.cuda.empty_cache()
            line["batched"] = batched_measure(g, h, dev, stream, hbm)
            torch.cuda.empty_cache()
            line["bootstrap"] = single_measure(g, h, dev, stream, "bootstrap", hbm)
            line["stress"] = single_measure(g, h, dev, stream, "stress", hbm)
            line["small"] = small_measure(g, h, dev, stream)
            if not args.no_cpu_baseline:  # the oracle as the checker
                line["accuracy_vs_oracle"] = accuracy_report(g, h, dev, stream)
    else:
        line["e2e"] = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(wl.w, N, seed)
        line["cpu_allcore"] = cpu_allcore()
    h.close()
    if dist:
        dist.destroy_process_group()
    if rank == 0:
        print(json.dumps(line), flush=True)


def e2e_measure(g, h, wl, dev, stream, K, inst):
    """Same metric through the public call with host buffers: pinned host
    weights copied in and indices copied out inside every timed step."""
    import torch
    M, N, seed = wl.M, wl.N, wl.seed
    w_host = torch.from_numpy(wl.w).pin_memory()
    out_host = torch.empty(N, dtype=torch.int32).pin_memory()
    wd = torch.empty(M, dtype=torch.float64, device=dev)
    out = torch.empty(N, dtype=torch.int32, device=dev)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with torch.cuda.stream(stream):
        for k in range(3 + K):
            e = ev[k - 3] if k >= 3 else None
            if e:
                e[0].record(stream)
            wd.copy_(w_host, non_blocking=True)
            g.rs_resample_w(h.h, wd, M, N, seed, inst, out, None, None, stream=stream)
            out_host.copy_(out, non_blocking=True)
            if e:
                e[1].record(stream)
    torch.cuda.synchronize()
    ms = statistics.mean(a.elapsed_time(b) for a, b in ev)
    # the same two copies with no resampling between them: the host link's
    # share of the step (the step cannot be faster than its copies)
    cev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    with torch.cuda.stream(stream):
        for a, b in cev:
            a.record(stream)
            wd.copy_(w_host, non_blocking=True)
            out_host.copy_(out, non_blocking=True)
            b.record(stream)
    torch.cuda.synchronize()
    cms = statistics.mean(a.elapsed_time(b) for a, b in cev)
    return {"value": N / (ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": 8 * M, "d2h_bytes_per_step": 4 * N,
            "ms_per_step": ms, "copies_only_ms_per_step": cms, "h2d_link_GBps": 8 * M / (cms * 1e-3) / 1e9,
            "frac_of_copy_bound": cms / ms}


def map_only(g, h, wl, dev, stream, K=50):
    """The paper's timing protocol: sampling steps only (W given): sorted
    uniforms + map, for the three maps, on the engmf instance; the DaC map
    with the leaf size its autotuner picks (kept in the handle)."""
    import torch
    M, N, seed = wl.M, wl.N, wl.seed
    wd = torch.from_numpy(wl.w).to(dev)
    W = torch.empty(M, dtype=torch.float64, device=dev)
    out = torch.empty(N, dtype=torch.int32, device=dev)
    res = {}
    with torch.cuda.stream(stream):
        g.rs_cumulative(h.h, wd, M, W, stream=stream)
        # the DaC leaf size picked by the library's autotuner for this M/N
        best = g.rs_autotune_map(h.h, W, M, N, seed, out, stream=stream)
        res["dac_tuned_leaf_L"] = best.leaf_L
        for name, algo in [("dac", g.RS_MAP_DAC), ("binary", g.RS_MAP_BINARY), ("linear", g.RS_MAP_LINEAR)]:
            o = g.opts(algo=algo)
            for _ in range(3):
                g.rs_resample_W(h.h, W, M, N, seed, 0, out, o, stream=stream)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
            for a, b in ev:
                a.record(stream)
                g.rs_resample_W(h.h, W, M, N, seed, 0, out, o, stream=stream)
                b.record(stream)
            torch.cuda.synchronize()
            ms = statistics.median(a.elapsed_time(b) for a, b in ev)
            res[name] = {"us_per_call": ms * 1e3, "particles_per_s": N / (ms * 1e-3)}
    return res


def gather_measure(g, h, dev, stream, hbm, reps=20):
    """The step after resampling, x'_i = x_{r_i}: N = M = 4,194,304 particles
    of 4 binary64 components (the bootstrap-filter size), gathered by the
    resampled indices of the bootstrap instance."""
    import torch
    wl = workloads.make("bootstrap")
    M, N, D = wl.M, wl.N, 4
    x = torch.randn((M, D), dtype=torch.float64, device=dev, generator=torch.Generator(device=dev).manual_seed(0))
    idx = torch.empty(N, dtype=torch.int32, device=dev)
    xo = torch.empty((N, D), dtype=torch.float64, device=dev)
    with torch.cuda.stream(stream):
        g.rs_resample_w(h.h, torch.from_numpy(wl.w).to(dev), M, N, wl.seed, 0, idx, stream=stream)
    ms = _time_calls(lambda: g.rs_gather(h.h, x, M, D * 8, idx, N, xo, stream=stream), stream, reps)
    if h.status() != g.RS_OK:
        raise RuntimeError("device status after the gather")
    bytes_ = 2 * N * D * 8 + 4 * N
    return {"workload": "N=M=4,194,304 rows of 4 binary64, bootstrap indices", "us_per_call": ms * 1e3,
            "GBps": bytes_ / (ms * 1e-3) / 1e9, "frac_of_hbm": bytes_ / (ms * 1e-3) / 1e9 / hbm,
            "bytes_per_call": bytes_}


def logw_measure(g, h, dev, stream, hbm, reps=20):
    """The engmf instance from its log-weights (l ~ Normal(0, 2^2), binary64):
    rs_resample_logw = the weights exp(l - max l) (maximum pass, exponent
    pass writing w) and the cooperative path on w."""
    import torch
    c = workloads.CONFIGS["engmf"]
    M, N = c["M"], c["N"]
    l = torch.from_numpy(np.random.default_rng(c["seed"]).normal(0.0, 2.0, size=M)).to(dev)
    out = torch.empty(N, dtype=torch.int32, device=dev)
    ms = _time_calls(lambda: g.rs_resample_logw(h.h, l, M, N, 12, 0, out, stream=stream), stream, reps)
    if h.status() != g.RS_OK:
        raise RuntimeError("device status after the log-weight run")
    alg = 8 * M + 4 * N
    moved = 8 * M * 4 + 4 * N  # max pass, exponent pass (read + write), the path's read
    return {"workload": "engmf from log-weights: M=16,777,216 binary64 l~Normal(0,2^2), N=4,096",
            "us_per_call": ms * 1e3, "particles_per_s": N / (ms * 1e-3),
            "GBps_algorithmic": alg / (ms * 1e-3) / 1e9, "frac_of_hbm_algorithmic": alg / (ms * 1e-3) / 1e9 / hbm,
            "GBps_moved": moved / (ms * 1e-3) / 1e9}


def paper_sweep(g, h, dev, stream, reps=20):
    """Figure 2's experiment shape: the sampling steps (sorted uniforms plus
    the map, W given) for N from 1e2 to 1e4 and M/N in {1, 100, 1000}, on the
    GPU (rs_resample_W per map) and with the oracle's serial Algorithms 3, 4
    and 5 on the host (sorted uniforms included), weights exp(l), l~N(0,2^2)."""
    import torch
    import oracle
    oracle.lib()
    rows = []
    for ratio in (1, 100, 1000):
        for N in (100, 316, 1000, 3162, 10000):
            M = N * ratio
            w = workloads.weights_lognormal(M, 2.0, seed=1000 + N + ratio)
            wdev = torch.from_numpy(w).to(dev)  # kept alive while the side stream reads it
            Wd = torch.empty(M, dtype=torch.float64, device=dev)
            g.rs_cumulative(h.h, wdev, M, Wd, stream=stream)  # the GPU leg's W
            W, _ = oracle.cumulative(w)  # the serial CPU algorithms' W
            out = torch.empty(N, dtype=torch.int32, device=dev)
            row = {"N": N, "M": M}
            for name, algo in [("dac", g.RS_MAP_DAC), ("binary", g.RS_MAP_BINARY), ("linear", g.RS_MAP_LINEAR)]:
                o = g.opts(algo=algo)
                row["gpu_us_" + name] = 1e3 * _time_calls(
                    lambda: g.rs_resample_W(h.h, Wd, M, N, 7, 0, out, o, stream=stream), stream, reps)
            for name, fn in [("dac", oracle.alg5_dac_map), ("binary", oracle.alg3_binary_map),
                             ("ccf", oracle.alg4_ccf_map)]:
                ts = []
                for _ in range(3):
                    t = time.perf_counter()
                    U = oracle.sorted_uniform(N, 7, 0)
                    fn(W, U)
                    ts.append(time.perf_counter() - t)
                row["cpu_us_" + name] = 1e6 * statistics.median(ts)
            rows.append(row)
    if h.status() != g.RS_OK:
        raise RuntimeError("device status after the sweep")
    return {"what": "sampling steps (sorted uniforms + map, W given); GPU maps vs the oracle's serial "
                    "Algorithms 3/4/5 on 1 host core", "rows": rows}


def _time_calls(fn, stream, reps, warm=2):
    import torch
    with torch.cuda.stream(stream):
        for _ in range(warm):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _time_graph_calls(fn, stream, calls=64, reps=10):
    """Device time per call: `calls` back-to-back calls captured as one CUDA
    graph, replayed `reps` times (host issue cost amortised)."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(2):
            fn(stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        for _ in range(calls):
            fn(torch.cuda.current_stream())
    torch.cuda.synchronize()
    ms = _time_calls(graph.replay, stream, reps)
    del graph
    return ms / calls


def batched_measure(g, h, dev, stream, hbm, reps=20):
    """8192 EnGMF-shaped instances (N_k ~ U{64..2048}, P_k ~ U{1..64},
    M_k = N_k P_k, binary32 weights): the persistent batched launch (autotuned,
    replayed as a CUDA graph) against the same persistent launch in binary64
    (the weights widened) and, for context, one binary64 rs_resample_w per
    instance (plain launches, and the same loop captured in a graph), plus
    the binary32 cumulative-weight error against binary64 on a sample of
    instances."""
    import torch
    wl = workloads.make("batched")
    w32, woff, roff, K = wl.w, wl.woff, wl.roff, wl.info["K"]
    sumM, sumN = int(woff[-1]), int(roff[-1])
    wd = torch.from_numpy(w32).to(dev)
    wo, ro = torch.from_numpy(woff).to(dev), torch.from_numpy(roff).to(dev)
    out = torch.empty(sumN, dtype=torch.int32, device=dev)
    best = g.rs_autotune_batched(h.h, wd, wo, ro, K, wl.seed, out, woff, roff, stream=stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        g.rs_resample_batched(h.h, wd, wo, ro, K, wl.seed, out, woff, roff, stream=stream)
    torch.cuda.synchronize()
    with torch.cuda.graph(graph, stream=stream):
        g.rs_resample_batched(h.h, wd, wo, ro, K, wl.seed, out, woff, roff, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    ms32 = _time_calls(graph.replay, stream, reps)
    if h.status() != g.RS_OK:
        raise RuntimeError("device status after the batched run")
    del graph
    # binary64 comparisons on the same weights widened: the same persistent
    # launch in binary64 (the like-for-like comparator), and, for context, one
    # rs_resample_w per instance (plain launches, and the same loop in a graph)
    w64 = wd.double()
    del wd
    o64 = g.opts(prec=g.RS_F64)
    with torch.cuda.stream(stream):
        g.rs_resample_batched(h.h, w64, wo, ro, K, wl.seed, out, woff, roff, o64, stream=stream)
    torch.cuda.synchronize()
    gp = torch.cuda.CUDAGraph()
    with torch.cuda.graph(gp, stream=stream):
        g.rs_resample_batched(h.h, w64, wo, ro, K, wl.seed, out, woff, roff, o64, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    ms64p = _time_calls(gp.replay, stream, reps)
    del gp

    # one rs_resample_w per instance inside the library (debug bit 2: every
    # instance through the cooperative single-instance launch)
    o64i = g.opts(prec=g.RS_F64, debug_flags=4)
    per_instance = lambda s=None: g.rs_resample_batched(  # noqa: E731
        h.h, w64, wo, ro, K, wl.seed, out, woff, roff, o64i, stream=s or stream)
    ms64 = _time_calls(per_instance, stream, 2, warm=1)
    g64 = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g64, stream=stream):
        per_instance(torch.cuda.current_stream())
    torch.cuda.synchronize()
    ms64g = _time_calls(g64.replay, stream, 3, warm=1)
    del g64
    if h.status() != g.RS_OK:
        raise RuntimeError("device status after the binary64 batched runs")
    # binary32-compensated W against binary64 W on 64 instances
    rng = np.random.default_rng(0)
    err = 0.0
    for k in rng.choice(K, size=64, replace=False):
        a, b = int(woff[k]), int(woff[k + 1])
        W32 = torch.empty(b - a, dtype=torch.float64, device=dev)
        W64 = torch.empty(b - a, dtype=torch.float64, device=dev)
        w32k = torch.from_numpy(w32[a:b]).to(dev)
        g.rs_cumulative(h.h, w32k, b - a, W32, g.opts(prec=g.RS_F32_COMP), stream=stream)
        g.rs_cumulative(h.h, w64[a:b].contiguous(), b - a, W64, g.opts(prec=g.RS_F64), stream=stream)
        torch.cuda.synchronize()
        err = max(err, float((W32 - W64).abs().max().item()))
    bytes32 = 4 * sumM + 4 * sumN
    return {"workload": "K=8192 instances, N_k~U{64..2048}, P_k~U{1..64}, M_k=N_k*P_k, binary32 exp(l-max), "
                        "l~Normal(0,1.5^2)", "K": K, "sum_M": sumM, "sum_N": sumN,
            "tuned": {"tile_threads": best.tile_threads, "leaf_L": best.leaf_L},
            "f32_batched_graph_us": ms32 * 1e3, "f32_particles_per_s": sumN / (ms32 * 1e-3),
            "f32_GBps": bytes32 / (ms32 * 1e-3) / 1e9, "f32_frac_of_hbm": bytes32 / (ms32 * 1e-3) / 1e9 / hbm,
            "batched_f64_persistent_us": ms64p * 1e3, "f64_GBps": (8 * sumM + 4 * sumN) / (ms64p * 1e-3) / 1e9,
            "f64_frac_of_hbm": (8 * sumM + 4 * sumN) / (ms64p * 1e-3) / 1e9 / hbm,
            "speedup_f32_vs_f64_persistent": ms64p / ms32,
            "f64_per_instance_launches_us": ms64 * 1e3, "f64_per_instance_graph_us": ms64g * 1e3,
            "speedup_vs_f64_launches": ms64 / ms32, "speedup_vs_f64_graph": ms64g / ms32,
            "max_abs_W_err_f32comp_vs_f64": err, "W_err_bound": 4 * 2.0 ** -23, "err_sample": "64 instances"}


def single_measure(g, h, dev, stream, name, hbm, reps=20):
    """rs_resample_w on the bootstrap (M = N) or precision-stress instance, in
    binary64 and, for the stress case, compensated binary32 with the error
    report (max |W32c - W64|, max |U32c - U64|, index mismatches)."""
    import torch
    wl = workloads.make(name)
    M, N, seed = wl.M, wl.N, wl.seed
    out = torch.empty(N, dtype=torch.int32, device=dev)
    res = {"M": M, "N": N}
    variants = [("f64", torch.from_numpy(wl.w).to(dev), g.RS_F64)]
    if wl.w32 is not None:
        variants.append(("f32comp", torch.from_numpy(wl.w32).to(dev), g.RS_F32_COMP))
    outs = {}
    for tag, wd, prec in variants:
        o = g.opts(prec=prec)
        ms = _time_calls(lambda: g.rs_resample_w(h.h, wd, M, N, seed, 0, out, None, o, stream=stream), stream, reps)
        bytes_ = wd.element_size() * M + 4 * N
        res[tag] = {"us_per_call": ms * 1e3, "particles_per_s": N / (ms * 1e-3),
                    "GBps": bytes_ / (ms * 1e-3) / 1e9, "frac_of_hbm": bytes_ / (ms * 1e-3) / 1e9 / hbm}
        outs[tag] = out.clone()
    if len(variants) == 2:
        W64 = torch.empty(M, dtype=torch.float64, device=dev)
        W32 = torch.empty(M, dtype=torch.float64, device=dev)
        g.rs_cumulative(h.h, variants[0][1], M, W64, g.opts(prec=g.RS_F64), stream=stream)
        g.rs_cumulative(h.h, variants[1][1], M, W32, g.opts(prec=g.RS_F32_COMP), stream=stream)
        U64 = torch.empty(N, dtype=torch.float64, device=dev)
        U32 = torch.empty(N, dtype=torch.float64, device=dev)
        g.rs_sorted_uniform(h.h, N, seed, 0, U64, g.opts(prec=g.RS_F64), stream=stream)
        g.rs_sorted_uniform(h.h, N, seed, 0, U32, g.opts(prec=g.RS_F32_COMP), stream=stream)
        torch.cuda.synchronize()
        res["max_abs_W_err_f32comp_vs_f64"] = float((W32 - W64).abs().max().item())
        res["max_abs_U_err_f32comp_vs_f64"] = float((U32 - U64).abs().max().item())
        res["index_mismatches_f32comp_vs_f64"] = int((outs["f32comp"] != outs["f64"]).sum().item())
    if h.status() != g.RS_OK:
        raise RuntimeError("device status after the %s run" % name)
    return res


def small_measure(g, h, dev, stream, reps=200):
    """The small workload (M = 4,096 Exp(1) weights, N = 1,024): the whole
    path per call (rs_resample_w, back-to-back calls on one stream) and the
    sampling steps on a given W (sorted uniforms + each of the three maps,
    rs_resample_W), as per-call microseconds; a launch-latency regime."""
    import torch
    wl = workloads.make("small")
    M, N, seed = wl.M, wl.N, wl.seed
    wd = torch.from_numpy(wl.w).to(dev)
    W = torch.empty(M, dtype=torch.float64, device=dev)
    g.rs_cumulative(h.h, wd, M, W, stream=stream)  # W for the sampling steps, by the library
    out = torch.empty(N, dtype=torch.int32, device=dev)
    res = {"M": M, "N": N, "bytes": 8 * M + 4 * N,
           "timing": "*_us_per_call: back-to-back calls from Python (includes the host's issue cost per call); "
                     "*_graph_us_per_call: 64 calls captured as one CUDA graph (device time per call)"}
    whole = lambda s: g.rs_resample_w(h.h, wd, M, N, seed, 0, out, stream=s)  # noqa: E731
    ms = _time_calls(lambda: whole(stream), stream, reps)
    res["whole_path_us_per_call"] = ms * 1e3
    res["whole_path_particles_per_s"] = N / (ms * 1e-3)
    ms = _time_graph_calls(whole, stream)
    res["whole_path_graph_us_per_call"] = ms * 1e3
    res["whole_path_graph_particles_per_s"] = N / (ms * 1e-3)
    for name, algo in [("dac", g.RS_MAP_DAC), ("binary", g.RS_MAP_BINARY), ("linear", g.RS_MAP_LINEAR)]:
        o = g.opts(algo=algo)
        mapf = lambda s, o=o: g.rs_resample_W(h.h, W, M, N, seed, 0, out, o, stream=s)  # noqa: E731
        ms = _time_calls(lambda: mapf(stream), stream, reps)
        res["map_only_us_per_call_" + name] = ms * 1e3
        res["map_only_graph_us_per_call_" + name] = _time_graph_calls(mapf, stream) * 1e3
    if h.status() != g.RS_OK:
        raise RuntimeError("device status after the small workload")
    return res


def accuracy_report(g, h, dev, stream):
    """Every workload against the binary64 oracle: max |W - W_oracle| of the
    cumulative weights, max |U - U_oracle| (absolute and relative) of the
    sorted uniforms, and the index mismatches of the whole path with how many
    of them lie on a boundary within the stated tolerance (1e-12 relative for
    binary64; 4 * 2^-23 absolute for compensated binary32).  Binary32 rows use
    the oracle evaluated on the same binary32 weights and draws; the stress
    row also gives W32 against the oracle's binary64 W of the unrounded
    weights.  The batched row covers a sample of 64 instances."""
    import torch
    import oracle
    oracle.lib()

    def one(w_np, N, seed, inst, prec):
        f32 = prec == "f32comp"
        M = w_np.shape[0]
        o = g.opts(prec=g.RS_F32_COMP if f32 else g.RS_F64)
        wd = torch.from_numpy(w_np).to(dev)
        Wg = torch.empty(M, dtype=torch.float64, device=dev)
        Ug = torch.empty(N, dtype=torch.float64, device=dev)
        r = torch.empty(N, dtype=torch.int32, device=dev)
        with torch.cuda.stream(stream):
            g.rs_cumulative(h.h, wd, M, Wg, o, stream=stream)
            g.rs_sorted_uniform(h.h, N, seed, inst, Ug, o, stream=stream)
            g.rs_resample_w(h.h, wd, M, N, seed, inst, r, None, o, stream=stream)
        torch.cuda.synchronize()
        if h.status() != g.RS_OK:
            raise RuntimeError("device status in the accuracy report")
        r_ref, W_ref, U_ref = oracle.resample(w_np, N, seed, instance=inst, single=f32)
        Wh, Uh, rh = Wg.cpu().numpy(), Ug.cpu().numpy(), r.cpu().numpy()
        mism = np.nonzero(rh != r_ref)[0]
        on_b = 0
        for i in mism:
            a, b = sorted((int(rh[i]), int(r_ref[i])))
            Wk = W_ref[a:b]
            tol = 4 * 2.0 ** -23 if f32 else 1e-12 * Wk
            on_b += int(np.all(np.abs(U_ref[i] - Wk) <= tol))
        res = {"max_abs_W_err": float(np.max(np.abs(Wh - W_ref))),
               "max_rel_W_err": float(np.max(np.abs(Wh - W_ref) / np.maximum(W_ref, 1e-300))),
               "max_abs_U_err": float(np.max(np.abs(Uh - U_ref))),
               "max_rel_U_err": float(np.max(np.abs(Uh - U_ref) / U_ref)),
               "index_mismatches": int(mism.size), "mismatches_on_boundary": on_b, "N": int(N), "M": int(M)}
        if f32:
            # the compensated binary32 bound is absolute: cumulative weights
            # below the unit of the global grid read 0, so their relative
            # error can reach 1 while the absolute error stays tiny
            big = W_ref >= 2.0 ** -40
            res["max_rel_W_err_above_2^-40"] = float(np.max(np.abs(Wh[big] - W_ref[big]) / W_ref[big])) if big.any() else 0.0
            res["W_err_bound_abs"] = 4 * 2.0 ** -23
        return res

    rep = {}
    for name in ("small", "engmf", "bootstrap", "stress"):
        wl = workloads.make(name)
        rep[name + ".f64"] = one(wl.w, wl.N, wl.seed, 0, "f64")
        if wl.w32 is not None:
            row = one(wl.w32, wl.N, wl.seed, 0, "f32comp")
            Wg = torch.empty(wl.M, dtype=torch.float64, device=dev)
            g.rs_cumulative(h.h, torch.from_numpy(wl.w32).to(dev), wl.M, Wg, g.opts(prec=g.RS_F32_COMP),
                            stream=stream)
            torch.cuda.synchronize()
            W64, _ = oracle.cumulative(wl.w)
            row["max_abs_W_err_vs_f64_weights"] = float(np.max(np.abs(Wg.cpu().numpy() - W64)))
            rep[name + ".f32comp"] = row
        del wl
        torch.cuda.empty_cache()
    wl = workloads.make("batched")
    rng = np.random.default_rng(0)
    agg = {}
    for k in sorted(rng.choice(wl.info["K"], size=64, replace=False)):
        a, b = int(wl.woff[k]), int(wl.woff[k + 1])
        Nk = int(wl.roff[k + 1] - wl.roff[k])
        for prec, wk in (("f32comp", wl.w[a:b]), ("f64", wl.w[a:b].astype(np.float64))):
            row = one(wk, Nk, wl.seed, int(k), prec)
            t = agg.setdefault("batched." + prec, {"sample": "64 instances", "index_mismatches": 0,
                                                    "mismatches_on_boundary": 0, "N": 0, "max_abs_W_err": 0.0,
                                                    "max_abs_U_err": 0.0, "max_rel_U_err": 0.0})
            for key in ("index_mismatches", "mismatches_on_boundary", "N"):
                t[key] += row[key]
            for key in ("max_abs_W_err", "max_abs_U_err", "max_rel_U_err"):
                t[key] = max(t[key], row[key])
    rep.update(agg)
    return rep


def _allcore_worker(job):
    """One process of the all-core CPU leg: the oracle as it stands on whole
    instances (engmf instances, or a slice of the batched instances)."""
    kind, lo, hi = job
    import oracle
    oracle.lib()
    t0 = time.perf_counter()
    n = 0
    if kind == "engmf":
        wl = workloads.make("engmf")
        t0 = time.perf_counter()
        for inst in range(lo, hi):
            oracle.resample(wl.w, wl.N, wl.seed, instance=inst)
            n += wl.N
    else:
        w, woff, roff = workloads.weights_batched(K=workloads.CONFIGS["batched"]["K"],
                                                  seed=workloads.CONFIGS["batched"]["seed"])
        t0 = time.perf_counter()
        for k in range(lo, hi):
            a, b = int(woff[k]), int(woff[k + 1])
            Nk = int(roff[k + 1] - roff[k])
            oracle.resample(w[a:b], Nk, workloads.PHILOX_SEED["batched"], instance=k, single=True)
            n += Nk
    return n, time.perf_counter() - t0


def cpu_allcore():
    """The oracle as it stands, one process per host core (spawned), on
    independent instances: engmf instances (instance ids 0..P-1, two each) and
    a slice of the batched workload's instances; particles/s over the slowest
    process, with the core count and CPU model."""
    import multiprocessing as mp
    import platform
    P = os.cpu_count() or 1
    model = platform.processor() or platform.machine()
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part", "hardware")):
                model = ln.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    res = {"cores": P, "cpu_model": model, "kind": "oracle", "unit": UNIT}
    ctx = mp.get_context("spawn")
    with ctx.Pool(P) as pool:
        out = pool.map(_allcore_worker, [("engmf", 2 * p, 2 * p + 2) for p in range(P)])
        n = sum(o[0] for o in out)
        res["engmf"] = {"value": n / max(o[1] for o in out),
                        "sample": "%d full engmf instances (2 per process) end to end" % (2 * P)}
        per = 16
        out = pool.map(_allcore_worker, [("batched", per * p, per * p + per) for p in range(P)])
        n = sum(o[0] for o in out)
        res["batched"] = {"value": n / max(o[1] for o in out),
                          "sample": "the first %d batched instances (%d per process, binary32 weights and draws)"
                                    % (per * P, per)}
    return res


def batched_probe(K):
    """The persistent batched launch on the first K instances of the batched
    workload (binary32 weights, default settings): three warm-up launches,
    then two, each timed with CUDA events; prints one line."""
    import torch
    import paper_2604_01356_gb300 as g
    wl = workloads.make("batched")
    K = min(K, wl.info["K"])
    woff, roff = wl.woff[:K + 1].copy(), wl.roff[:K + 1].copy()
    wd = torch.from_numpy(wl.w[: int(woff[-1])]).cuda()
    wo, ro = torch.from_numpy(woff).cuda(), torch.from_numpy(roff).cuda()
    out = torch.empty(int(roff[-1]), dtype=torch.int32, device="cuda")
    h = g.Handle()
    ev = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.rs_resample_batched(h.h, wd, wo, ro, K, wl.seed, out, woff, roff, g.opts(prec=g.RS_F32_COMP))
        e1.record()
        ev.append((e0, e1))
    torch.cuda.synchronize()
    if h.status() != g.RS_OK:
        raise RuntimeError("device status after the batched probe")
    h.close()
    print(json.dumps({"batched_probe": {"K": K, "sum_M": int(woff[-1]), "sum_N": int(roff[-1]),
                                        "algorithmic_bytes": 4 * int(woff[-1]) + 4 * int(roff[-1]),
                                        "us": [round(a.elapsed_time(b) * 1e3, 1) for a, b in ev]}}))


def small_probe():
    """rs_resample_w, then rs_resample_W with the binary-search map, on the
    small workload: three warm-up calls each, then two timed with CUDA
    events; prints one line."""
    import torch
    import paper_2604_01356_gb300 as g
    wl = workloads.make("small")
    wd = torch.from_numpy(wl.w).cuda()
    out = torch.empty(wl.N, dtype=torch.int32, device="cuda")
    h = g.Handle()
    W = torch.empty(wl.M, dtype=torch.float64, device="cuda")
    g.rs_cumulative(h.h, wd, wl.M, W)  # W for the sampling steps, by the library
    res = {}
    for name, fn in [("resample_w", lambda: g.rs_resample_w(h.h, wd, wl.M, wl.N, wl.seed, 0, out)),
                     ("resample_W_binary", lambda: g.rs_resample_W(h.h, W, wl.M, wl.N, wl.seed, 0, out,
                                                                   g.opts(algo=g.RS_MAP_BINARY)))]:
        ev = []
        for _ in range(5):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            ev.append((e0, e1))
        torch.cuda.synchronize()
        res[name] = [round(a.elapsed_time(b) * 1e3, 1) for a, b in ev]
    if h.status() != g.RS_OK:
        raise RuntimeError("device status after the small probe")
    h.close()
    print(json.dumps({"small_probe": {"M": wl.M, "N": wl.N, "us": res}}))


def logw_probe():
    """rs_resample_logw on the engmf log-weights: three warm-up calls, then
    two timed with CUDA events; prints one line."""
    import torch
    import paper_2604_01356_gb300 as g
    c = workloads.CONFIGS["engmf"]
    M, N = c["M"], c["N"]
    l = torch.from_numpy(np.random.default_rng(c["seed"]).normal(0.0, 2.0, size=M)).cuda()
    out = torch.empty(N, dtype=torch.int32, device="cuda")
    h = g.Handle()
    ev = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        g.rs_resample_logw(h.h, l, M, N, 12, 0, out)
        e1.record()
        ev.append((e0, e1))
    torch.cuda.synchronize()
    if h.status() != g.RS_OK:
        raise RuntimeError("device status after the log-weight probe")
    h.close()
    print(json.dumps({"logw_probe": {"M": M, "N": N, "us": [round(a.elapsed_time(b) * 1e3, 1) for a, b in ev]}}))


def main():
    args = parse()
    if args.logw_probe:
        logw_probe()
        return
    if args.small_probe:
        small_probe()
        return
    if args.batched_probe:
        batched_probe(args.batched_probe)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
