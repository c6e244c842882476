"""Seeded synthetic inputs for the resampling workloads.

This module only draws inputs (numpy PCG64); it contains none of the
resampling arithmetic, and both the CUDA path's tests/benchmark and the oracle
consume what it returns.  Weights are returned UNNORMALISED: normalising them
is the first step of the path itself (Eq. 3 of arXiv 2604.01356).

The five workloads mirror the paper's setting (Sec. I: M = N*P weights of an
ensemble Gaussian mixture filter, Sec. IV: N up to 1e4, M/N up to 1e3) at the
sizes the library is measured on:

  small     M=4,096,       N=1,024      e ~ Exp(1)
  engmf     M=16,777,216,  N=4,096      w = exp(l - max l), l ~ Normal(0, 2^2)
  bootstrap M=N=4,194,304               w = exp(-0.5((0.5 - x)/0.1)^2), x ~ Normal(0,1)
  batched   K=8,192 instances, N_k ~ U{64..2048}, P_k ~ U{1..64}, M_k = N_k P_k,
            w = exp(l - max l) per instance, l ~ Normal(0, 1.5^2), binary32
  stress    M=67,108,864,  N=65,536     w = exp(l - max l), l ~ Normal(0, 10^2),
            rescaled to total 1e-9, plus one spike of mass 1 - 1e-9
"""
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

CONFIGS = {
    "small": dict(seed=0, M=4096, N=1024),
    "engmf": dict(seed=1, M=16_777_216, N=4096),
    "bootstrap": dict(seed=2, M=4_194_304, N=4_194_304),
    "batched": dict(seed=3, K=8192),
    "stress": dict(seed=4, M=67_108_864, N=65_536),
}

# Seeds of the method's own Philox stream used by the benchmark and tests.
PHILOX_SEED = {"small": 11, "engmf": 12, "bootstrap": 13, "batched": 14, "stress": 15}


@dataclass
class Workload:
    name: str
    w: np.ndarray                  # weights, float64 (or float32 for 'batched')
    N: int                         # samples per instance (single instance)
    seed: int                      # Philox seed of the path
    woff: Optional[np.ndarray] = None   # batched: int64 [K+1]
    roff: Optional[np.ndarray] = None   # batched: int64 [K+1]
    w32: Optional[np.ndarray] = None    # binary32 copy (stress)
    info: dict = field(default_factory=dict)

    @property
    def M(self):
        return int(self.w.shape[0])


def weights_small(M=4096, seed=0):
    rng = np.random.default_rng(seed)
    return rng.exponential(1.0, size=M)


def weights_lognormal(M, sigma, seed):
    rng = np.random.default_rng(seed)
    l = rng.normal(0.0, sigma, size=M)
    return np.exp(l - l.max())


def weights_bootstrap(M, seed, y=0.5, h=0.1):
    rng = np.random.default_rng(seed)
    x = rng.normal(0.0, 1.0, size=M)
    return np.exp(-0.5 * ((y - x) / h) ** 2)


def weights_stress(M, seed, sigma=10.0, spike=1.0 - 1e-9):
    rng = np.random.default_rng(seed)
    l = rng.normal(0.0, sigma, size=M)
    w = np.exp(l - l.max())
    s = int(rng.integers(0, M))
    w[s] = 0.0
    w *= (1.0 - spike) / w.sum()
    w[s] = spike
    return w, s


def batched_layout(K=8192, seed=3, nmin=64, nmax=2048, pmax=64):
    rng = np.random.default_rng(seed)
    Nk = rng.integers(nmin, nmax + 1, size=K)
    Pk = rng.integers(1, pmax + 1, size=K)
    Mk = Nk * Pk
    woff = np.zeros(K + 1, dtype=np.int64)
    roff = np.zeros(K + 1, dtype=np.int64)
    np.cumsum(Mk, out=woff[1:])
    np.cumsum(Nk, out=roff[1:])
    return woff, roff, rng


def weights_batched(K=8192, seed=3, sigma=1.5, nmin=64, nmax=2048, pmax=64):
    woff, roff, rng = batched_layout(K, seed, nmin, nmax, pmax)
    total = int(woff[-1])
    w = np.empty(total, dtype=np.float32)
    l = rng.normal(0.0, sigma, size=total)
    for k in range(K):
        a, b = int(woff[k]), int(woff[k + 1])
        seg = l[a:b]
        w[a:b] = np.exp(seg - seg.max()).astype(np.float32)
    return w, woff, roff


def make(name, scale=1.0):
    """Build a workload.  scale < 1 shrinks M and N (and K) proportionally while
    keeping the value distribution, for oracle-sized parity cases."""
    c = CONFIGS[name]
    ps = PHILOX_SEED[name]
    if name == "small":
        M = max(1, int(c["M"] * scale)); N = max(1, int(c["N"] * scale))
        return Workload(name, weights_small(M, c["seed"]), N, ps)
    if name == "engmf":
        M = max(1, int(c["M"] * scale)); N = max(1, int(c["N"] * scale))
        return Workload(name, weights_lognormal(M, 2.0, c["seed"]), N, ps)
    if name == "bootstrap":
        M = max(1, int(c["M"] * scale))
        return Workload(name, weights_bootstrap(M, c["seed"]), M, ps)
    if name == "stress":
        M = max(2, int(c["M"] * scale)); N = max(1, int(c["N"] * scale))
        w, s = weights_stress(M, c["seed"])
        return Workload(name, w, N, ps, w32=w.astype(np.float32), info={"spike": s})
    if name == "batched":
        K = max(1, int(c["K"] * scale))
        w, woff, roff = weights_batched(K, c["seed"])
        return Workload(name, w, int(roff[-1]), ps, woff=woff, roff=roff, info={"K": K})
    raise KeyError(name)


def adversarial_weights(kind, M, seed=0):
    """Edge-case weight vectors: runs of zeros, dyadic ties, a single spike,
    all-equal weights, one non-zero weight at either end."""
    rng = np.random.default_rng(seed)
    if kind == "zeros_runs":
        w = rng.exponential(size=M)
        mask = rng.random(M) < 0.5
        w[mask] = 0.0
        if w.sum() == 0:
            w[0] = 1.0
        return w
    if kind == "dyadic":
        return rng.integers(0, 4, size=M).astype(np.float64) + (np.arange(M) == M - 1)
    if kind == "spike":
        w = np.zeros(M)
        w[int(rng.integers(0, M))] = 1.0
        return w
    if kind == "equal":
        return np.full(M, 1.0 / M)
    if kind == "first":
        w = np.zeros(M); w[0] = 2.0
        return w
    if kind == "last":
        w = np.zeros(M); w[-1] = 0.5
        return w
    if kind == "tiny":
        return rng.exponential(size=M) * 1e-300
    if kind == "huge":
        return rng.exponential(size=M) * 1e300
    if kind == "wide":
        return np.exp(rng.normal(0.0, 150.0, size=M))
    raise KeyError(kind)


ADVERSARIAL = ["zeros_runs", "dyadic", "spike", "equal", "first", "last", "tiny", "huge", "wide"]
