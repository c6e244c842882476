"""Pins of the CPU oracle against facts the paper and mathematics fix.

No test here re-types an oracle formula: each compares the oracle with an
independent library routine, an exact (rational) computation, a closed form, a
distributional law, or the paper's worked example (Figure 1).
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- Philox ----
@pytest.mark.parametrize("key", [(0, 0), (1, 0), (0, 1), (0x0123456789ABCDEF, 0xFEDCBA9876543210), (2**64 - 1, 2**64 - 1)])
@pytest.mark.parametrize("block", [0, 1, 2, 3, 1000, 2**32 - 1, 2**32, 2**63])
def test_philox_matches_numpy_bit_generator(key, block):
    """numpy.random.Philox is an independent Philox-4x64-10 implementation.
    It increments its 256-bit counter before each block, so start at block-1."""
    v = (block - 1) % 2**256
    ctr_prev = np.array([(v >> (64 * i)) & (2**64 - 1) for i in range(4)], dtype=np.uint64)
    g = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=ctr_prev)
    ref = g.random_raw(4)
    ours = oracle.philox4x64_10(np.array([block, 0, 0, 0], dtype=np.uint64), np.array(key, dtype=np.uint64))
    assert np.array_equal(ours, ref)


def test_stream_words_are_consecutive_numpy_blocks():
    seed, inst = 987654321, 42
    g = np.random.Philox(key=np.array([seed, inst], dtype=np.uint64),
                         counter=np.array([2**64 - 1] * 4, dtype=np.uint64))
    ref = g.random_raw(4 * 16)
    assert np.array_equal(oracle.stream_words(seed, inst, 64), ref)


# --------------------------------------------------------- uniform draws ----
def test_uniform_draws_open_interval_and_exact_grid():
    v = oracle.uniform_draws(5, 0, 20000)
    assert v.min() > 0.0 and v.max() < 1.0
    k = v * 2.0**53
    assert np.all(k == np.round(k)) and np.all(np.mod(k, 2) == 1)  # odd multiples of 2^-53
    v32 = oracle.uniform_draws(5, 0, 20000, single=True)
    k32 = v32 * 2.0**24
    assert np.all(k32 == np.round(k32)) and np.all(np.mod(k32, 2) == 1)
    assert np.all(v32.astype(np.float32).astype(np.float64) == v32)  # representable in binary32
    # both precisions come from the same words: they agree to the binary32 grid
    assert np.max(np.abs(v32 - v)) <= 2.0**-24


def test_uniform_draws_are_uniform():
    from scipy import stats
    v = oracle.uniform_draws(77, 3, 200000)
    assert stats.kstest(v, "uniform").pvalue > 1e-3
    assert abs(v.mean() - 0.5) < 5 * math.sqrt(1 / 12 / v.size)


# ------------------------------------------------------- Algorithm 1 -------
@pytest.mark.parametrize("N", [1, 2, 5, 100, 4097])
def test_sorted_uniform_sorted_in_unit_interval(N):
    U = oracle.sorted_uniform(N, seed=3, instance=N)
    assert U.shape == (N,)
    assert np.all(np.diff(U) >= 0)
    assert U[0] > 0 and U[-1] < 1.0


def test_sorted_uniform_order_statistic_means():
    """U_i is the i-th order statistic of N iid U(0,1): E[U_i] = i/(N+1).
    (Normalising by Z_{i+1}, the printed typo, would give E = i/(i+1).)"""
    N, R = 8, 4000
    acc = np.zeros(N)
    for s in range(R):
        acc += oracle.sorted_uniform(N, seed=1000 + s)
    mean = acc / R
    expect = np.arange(1, N + 1) / (N + 1)
    # Var of the i-th order statistic <= 1/(4(N+2)); 5-sigma band
    assert np.all(np.abs(mean - expect) < 5 * math.sqrt(0.25 / (N + 2) / R))


def test_sorted_uniform_pooled_ks():
    from scipy import stats
    pooled = np.concatenate([oracle.sorted_uniform(64, seed=50 + s) for s in range(300)])
    assert stats.kstest(pooled, "uniform").pvalue > 1e-3


def test_sorted_uniform_n1_is_beta11():
    """For N=1, U_1 = z_1/(z_1+z_2) with z iid Exp(1) is exactly U(0,1)."""
    from scipy import stats
    u = np.array([oracle.sorted_uniform(1, seed=s)[0] for s in range(4000)])
    assert stats.kstest(u, "uniform").pvalue > 1e-3


def test_sorted_uniform_deterministic_and_stream_separated():
    a = oracle.sorted_uniform(100, seed=9, instance=0)
    b = oracle.sorted_uniform(100, seed=9, instance=0)
    c = oracle.sorted_uniform(100, seed=9, instance=1)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


def test_sorted_uniform_spacings_are_exponential():
    """Differences of the unnormalised partial sums are the draws' -log(v):
    the spacings n*(U_{i+1} - U_i) of uniform order statistics are ~Exp(1)
    for large n (Pyke 1965)."""
    from scipy import stats
    N = 20000
    U = oracle.sorted_uniform(N, seed=12)
    d = np.diff(U) * (N + 1)
    assert stats.kstest(d, "expon").pvalue > 1e-3


# ----------------------------------------------------------- Eq. 3 ---------
def _exact_cumulative(w):
    fr = [Fraction(float(x)) for x in w]
    S = sum(fr)
    out, acc = [], Fraction(0)
    for x in fr:
        acc += x
        out.append(acc / S)
    return out


def _ulp(x):
    return math.ulp(x) if x != 0 else 5e-324


@pytest.mark.parametrize("kind", workloads.ADVERSARIAL)
def test_cumulative_matches_exact_rational(kind):
    w = workloads.adversarial_weights(kind, 300, seed=4)
    W, S = oracle.cumulative(w)
    ex = _exact_cumulative(w)
    for j in range(len(w)):
        assert abs(Fraction(W[j]) - ex[j]) <= Fraction(_ulp(float(ex[j]))), (kind, j)
    assert W[-1] == 1.0
    assert np.all(np.diff(W) >= 0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_cumulative_random_vs_exact_and_fsum(seed):
    rng = np.random.default_rng(seed)
    w = np.exp(rng.normal(0, 3, size=2000))
    W, S = oracle.cumulative(w)
    assert S == math.fsum(w)  # correctly rounded total
    ex = _exact_cumulative(w)
    err = max(abs(float(Fraction(W[j]) - ex[j])) / float(ex[j]) for j in range(len(w)))
    assert err <= 2.2e-16


def test_cumulative_equal_weights_closed_form():
    M = 1 << 12
    W, S = oracle.cumulative(np.full(M, 1.0 / M))
    assert np.array_equal(W, np.arange(1, M + 1) / M)


def test_cumulative_large_prefix_against_fsum():
    w = workloads.weights_lognormal(100_000, 2.0, seed=7)
    W, S = oracle.cumulative(w)
    S_ref = math.fsum(w)
    for j in [0, 1, 17, 999, 50_000, 99_998, 99_999]:
        pj = math.fsum(w[: j + 1])
        assert abs(W[j] - pj / S_ref) <= 2 * _ulp(pj / S_ref)


def test_cumulative_binary32_input_is_widened():
    w32 = workloads.weights_lognormal(5000, 1.5, seed=8).astype(np.float32)
    W32, _ = oracle.cumulative(w32)
    W64, _ = oracle.cumulative(w32.astype(np.float64))
    assert np.array_equal(W32, W64)


@pytest.mark.parametrize("bad,code", [([1.0, -1e-300, 2.0], 1), ([1.0, float("nan")], 1), ([float("inf"), 1.0], 1), ([0.0, 0.0], 2), ([-0.0, 0.0], 2)])
def test_cumulative_rejects_invalid(bad, code):
    with pytest.raises(oracle.OracleError) as e:
        oracle.cumulative(np.array(bad))
    assert e.value.args[0] == code


# -------------------------------------------------------- Eq. 2-3 map -------
def _searchsorted_ref(W, U):
    """Lower bound (numpy library routine) clamped to the last index."""
    return np.minimum(np.searchsorted(W, U, side="left"), len(W) - 1).astype(np.int32)


def test_inverse_cdf_exhaustive_tiny_dyadic():
    """All W of length <= 5 over dyadic weights in {0,1,2}/4 and u on a grid that
    contains every W_j exactly, their midpoints and values above W_M."""
    import itertools
    for M in range(1, 6):
        for wts in itertools.product([0, 1, 2], repeat=M):
            if sum(wts) == 0:
                continue
            W = np.cumsum(np.array(wts, dtype=np.float64)) / sum(wts)
            grid = np.unique(np.concatenate([W, (np.concatenate([[0.0], W[:-1]]) + W) / 2, [1e-9, 0.5, 1.0, 1.0 + 2**-52]]))
            grid = grid[grid > 0]
            r = oracle.inverse_cdf(W, grid)
            assert np.array_equal(r, _searchsorted_ref(W, grid)), (wts,)
            # ties go to the tied index (Eq. 3: u <= W_i)
            for j in range(M):
                if j == 0 or W[j] > W[j - 1]:
                    assert oracle.inverse_cdf(W, np.array([W[j]]))[0] == j


@pytest.mark.parametrize("kind", workloads.ADVERSARIAL)
def test_paper_algorithms_agree_with_brute_force(kind):
    w = workloads.adversarial_weights(kind, 257, seed=11)
    W, _ = oracle.cumulative(w)
    for N in [1, 2, 7, 64, 300]:
        U = np.sort(np.concatenate([np.random.default_rng(N).random(N - min(N, 3)), W[: min(N, 3)]]))
        ref = oracle.inverse_cdf(W, U)
        assert np.array_equal(ref, _searchsorted_ref(W, U))
        assert np.array_equal(oracle.inverse_cdf_walk(W, U), ref)
        assert np.array_equal(oracle.alg3_binary_map(W, U), ref)
        assert np.array_equal(oracle.alg4_ccf_map(W, U), ref)
        assert np.array_equal(oracle.alg5_dac_map(W, U), ref)


def test_alg2_special_cases():
    Z = np.array([0.1, 0.2, 0.2, 0.7, 1.0])
    assert oracle.alg2_binary_search(Z, 0.2) == 2       # first tie (1-based)
    assert oracle.alg2_binary_search(Z, 0.05) == 1
    assert oracle.alg2_binary_search(Z, 0.9) == 5
    assert oracle.alg2_binary_search(Z, 2.0) == 5       # above W_M: clamped to M
    assert oracle.alg2_binary_search(Z, 0.7, a=2, b=3) == 3  # restricted range


def test_figure1_trace():
    g = json.load(open(os.path.join(GOLDEN, "fig1_trace.json")))
    W, U = np.array(g["W"]), np.array(g["U"])
    r, tr = oracle.alg5_dac_map(W, U, trace=True)
    assert list(r + 1) == g["r_1based"]
    assert list(oracle.inverse_cdf(W, U) + 1) == g["r_1based"]
    # group the algorithm's binary searches by recursion depth = figure step
    steps = {}
    for depth, mu, mw in tr:
        steps.setdefault(int(depth), []).append([int(mu), int(mw)])
    assert [steps[k] for k in sorted(steps)] == g["steps"]


def test_dac_comparison_count_matches_table1():
    """Table I: the divide and conquer sampler costs about log2(M/N + 1)
    comparisons per sample, the binary sampler log2(M).  Count Algorithm 2's
    W comparisons inside each sampler."""
    for M, N in [(1 << 16, 1 << 6), (1 << 18, 1 << 8), (1 << 12, 1 << 12)]:
        W, _ = oracle.cumulative(workloads.weights_small(M, seed=5))
        U = oracle.sorted_uniform(N, seed=5)
        oracle.alg2_probe_count(reset=True)
        _, tr = oracle.alg5_dac_map(W, U, trace=True)
        dac = oracle.alg2_probe_count(reset=True) / N
        oracle.alg3_binary_map(W, U)
        binary = oracle.alg2_probe_count(reset=True) / N
        assert abs(binary - math.log2(M)) <= 1.0
        assert dac <= math.log2(M / N + 1) + 3.0
        assert len(tr) <= N  # at most one binary search per sample


# ------------------------------------------------------- whole path --------
def test_resample_consistent_with_parts():
    w = workloads.weights_lognormal(3000, 2.0, seed=1)
    r, W, U = oracle.resample(w, 500, seed=3, instance=2)
    W2, _ = oracle.cumulative(w)
    U2 = oracle.sorted_uniform(500, seed=3, instance=2)
    assert np.array_equal(W, W2) and np.array_equal(U, U2)
    assert np.array_equal(r, oracle.inverse_cdf(W, U))


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_resample_chi_square_against_weights(seed):
    """The multiset of indices is Multinomial(N, w): chi-square goodness of fit."""
    from scipy import stats
    M, N = 40, 200_000
    w = workloads.weights_small(M, seed=seed)
    r, _, _ = oracle.resample(w, N, seed=seed)
    counts = np.bincount(r, minlength=M)
    expect = N * w / w.sum()
    assert stats.chisquare(counts, expect).pvalue > 1e-3


def test_resample_spike_degenerate():
    w = workloads.adversarial_weights("spike", 1000, seed=3)
    r, _, _ = oracle.resample(w, 777, seed=1)
    assert np.all(r == int(np.argmax(w)))


def test_resample_binary32_stream():
    w = workloads.weights_lognormal(2000, 1.5, seed=2).astype(np.float32)
    r, W, U = oracle.resample(w, 300, seed=4, single=True)
    U64 = oracle.sorted_uniform(300, seed=4, single=False)
    # same words on the binary32 grid; -log amplifies the grid error of small v
    assert np.max(np.abs(U - U64)) < 1e-4 and not np.array_equal(U, U64)
    assert np.array_equal(r, oracle.inverse_cdf(W, U))


def test_resample_batched_equals_instance_loop():
    w, woff, roff = workloads.weights_batched(K=6, seed=9, nmin=3, nmax=40, pmax=5)
    r = oracle.resample_batched(w, woff, roff, seed=21, single=True)
    for k in range(6):
        rk, _, _ = oracle.resample(w[woff[k]:woff[k + 1]], int(roff[k + 1] - roff[k]), seed=21, instance=k, single=True)
        assert np.array_equal(r[roff[k]:roff[k + 1]], rk)


# ---------------------------------------------- stratified / systematic ----
# The variants the paper's concluding section names: one point per stratum
# ((i-1)/N, i/N], with the draws of Algorithm 1.

@pytest.mark.parametrize("scheme", ["stratified", "systematic"])
@pytest.mark.parametrize("N", [1, 2, 7, 1000, 4097])
def test_scheme_one_point_per_stratum(scheme, N):
    U = oracle.scheme_uniform(N, 11, 3, scheme)
    i = np.arange(N, dtype=np.float64)
    assert np.all(U >= i / N) and np.all(U <= (i + 1) / N)
    assert np.all(np.diff(U) >= 0) and U[-1] <= 1.0 and U[0] > 0


def test_systematic_points_equally_spaced():
    N = 1000
    U = oracle.scheme_uniform(N, 4, 0, "systematic")
    assert np.allclose(np.diff(U), 1.0 / N, rtol=0, atol=1e-15)


def test_stratified_strata_are_independent_draws():
    # the position inside each stratum, N U_i - (i-1), is Uniform(0,1): KS
    from scipy import stats
    N = 20000
    U = oracle.scheme_uniform(N, 8, 1, "stratified")
    frac = N * U - np.arange(N)
    assert stats.kstest(frac, "uniform").pvalue > 1e-3


def _counts(r, M):
    return np.bincount(r, minlength=M)


def test_systematic_counts_are_floor_or_ceil():
    # N equally spaced points: an interval of W of length w_j holds
    # floor(N w_j) or ceil(N w_j) of them
    rng = np.random.default_rng(5)
    for M, N in [(50, 40), (1000, 5000), (3000, 700)]:
        w = rng.exponential(size=M)
        r, W, _ = oracle.resample_scheme(w, N, 17, "systematic")
        e = N * w / w.sum()
        c = _counts(r, M)
        assert np.all(c >= np.floor(e - 1e-9)) and np.all(c <= np.ceil(e + 1e-9))


def test_stratified_counts_within_one_and_unbiased():
    rng = np.random.default_rng(6)
    M, N = 40, 100
    w = rng.exponential(size=M)
    e = N * w / w.sum()
    mean = np.zeros(M)
    seeds = 400
    for seed in range(seeds):
        r, _, _ = oracle.resample_scheme(w, N, seed, "stratified")
        c = _counts(r, M)
        # an interval of length w_j meets at most ceil(N w_j) + 1 strata
        assert np.all(c >= np.floor(e) - 1) and np.all(c <= np.ceil(e) + 1)
        mean += c
    mean /= seeds
    # each stratum's point falls in j with its probability: E[count_j] = N w_j
    assert np.all(np.abs(mean - e) <= 4 * np.sqrt(np.maximum(e, 0.25) / seeds) + 1e-9)


def test_scheme_zero_is_algorithm_1():
    U0 = oracle.scheme_uniform(333, 9, 2, "multinomial")
    assert np.array_equal(U0, oracle.sorted_uniform(333, 9, 2))


# ------------------------------------------------------ log-weight input ----
def test_softmax_shift_invariance_and_max():
    rng = np.random.default_rng(3)
    l = rng.normal(0.0, 10.0, size=5000)
    w = oracle.softmax_weights(l)
    assert w.max() == 1.0 and np.all(w >= 0)
    # adding a constant to every log-weight leaves the cumulative weights unchanged
    W1, _ = oracle.cumulative(w)
    W2, _ = oracle.cumulative(oracle.softmax_weights(l + 1234.5))
    assert np.max(np.abs(W1 - W2)) <= 1e-13


def test_softmax_closed_forms():
    # equal log-weights: W_j = j / M exactly (M a power of two)
    W, _ = oracle.cumulative(oracle.softmax_weights(np.full(1024, -7.25)))
    assert np.array_equal(W, np.arange(1, 1025) / 1024.0)
    # l = (0, log 3): w proportional to (1, 3) -> W = (1/4, 1)
    W, _ = oracle.cumulative(oracle.softmax_weights(np.array([0.0, np.log(3.0)])))
    assert abs(W[0] - 0.25) <= 1e-16 and W[1] == 1.0
    # -inf gives a zero weight, never drawn
    w = oracle.softmax_weights(np.array([-np.inf, 0.0, -np.inf]))
    assert np.array_equal(w, [0.0, 1.0, 0.0])


def test_softmax_invalid():
    with pytest.raises(oracle.OracleError):
        oracle.softmax_weights(np.array([0.0, np.nan]))
    with pytest.raises(oracle.OracleError):
        oracle.softmax_weights(np.array([0.0, np.inf]))
    with pytest.raises(oracle.OracleError):
        oracle.softmax_weights(np.array([-np.inf, -np.inf]))
