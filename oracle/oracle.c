/*
 * Oracle for multinomial resampling (arXiv 2604.01356, "A divide and conquer
 * strategy for multinomial particle filter resampling").
 *
 * TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct CPU
 * statement of what the resampling path computes.  It shares no code, header,
 * table or constant with the CUDA library; only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  All arithmetic is
 * IEEE binary64 unless a function says otherwise.
 *
 * Contents
 *   orc_philox4x64_10     Philox-4x64 with 10 rounds, from its published
 *                         definition (Salmon, Moraes, Dror, Shaw, SC'11,
 *                         "Parallel random numbers: as easy as 1, 2, 3").
 *                         It plays the role of rand[0,1] in Algorithms 1 and 3.
 *   orc_uniform_draws     The open-interval uniform draws v_k of one stream.
 *   orc_sorted_uniform    Algorithm 1 (exponential spacings), with the
 *                         normaliser read as Z_{N+1}.
 *   orc_cumulative        Eq. 3: W_j = sum_{k<=j} w_k / sum_k w_k.
 *   orc_inverse_cdf       Eq. 2-3 by brute force: r_i = smallest j with
 *                         W_j >= U_i, clamped to the last index.
 *   orc_inverse_cdf_walk  The same result by one monotone walk (valid only
 *                         for sorted U); used where the per-u scan is too slow.
 *   orc_alg2_binary_search, orc_alg3_binary_map, orc_alg4_ccf_map,
 *   orc_alg5_dac_map      The samplers of Algorithms 2-5 (Sec. II-III),
 *                         restated from the result each computes (the
 *                         Eq. 3 lower bound) and the split argument of
 *                         Sec. III; cross-checks, the Figure 1 trace and
 *                         Table I's comparison counts.
 *   orc_resample          Whole path for one instance: Eq. 3 + Algorithm 1 +
 *                         Eq. 2.
 *   orc_resample_batched  The same for K independent instances.
 *
 * Indices returned to callers are 0-based (paper index j <-> j-1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Philox-4x64-10.  Round function (SC'11, Sec. 3.4 / Table 2 constants):    */
/*   (hi0,lo0) = M0 * X0, (hi1,lo1) = M1 * X2   (full 128-bit products)     */
/*   X' = (hi1 ^ X1 ^ K0, lo1, hi0 ^ X3 ^ K1, lo0)                           */
/* and the key is bumped by the Weyl constants between rounds.               */
/* ------------------------------------------------------------------------ */
static const uint64_t PHILOX_M0 = 0xD2E7470EE14C6C93ULL;
static const uint64_t PHILOX_M1 = 0xCA5A826395121157ULL;
static const uint64_t PHILOX_W0 = 0x9E3779B97F4A7C15ULL; /* golden ratio */
static const uint64_t PHILOX_W1 = 0xBB67AE8584CAA73BULL; /* sqrt(3) - 1 */

void orc_philox4x64_10(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]) {
  uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
  uint64_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += PHILOX_W0;
      k1 += PHILOX_W1;
    }
    unsigned __int128 p0 = (unsigned __int128)PHILOX_M0 * x0;
    unsigned __int128 p1 = (unsigned __int128)PHILOX_M1 * x2;
    uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
    uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
    uint64_t y0 = hi1 ^ x1 ^ k0;
    uint64_t y1 = lo1;
    uint64_t y2 = hi0 ^ x3 ^ k1;
    uint64_t y3 = lo0;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Raw 64-bit word k of the stream (seed, instance): key = (seed, instance),
 * counter = (floor(k/4), 0, 0, 0), word k mod 4 of the block. */
uint64_t orc_stream_word(uint64_t seed, uint64_t instance, uint64_t k) {
  uint64_t ctr[4] = {k / 4, 0, 0, 0};
  uint64_t key[2] = {seed, instance};
  uint64_t out[4];
  orc_philox4x64_10(ctr, key, out);
  return out[k % 4];
}

/* rand[0,1] read as the open interval (0,1) so that -log is finite.
 *   binary64 draw:  v = (2*(x >> 12) + 1) * 2^-53   in [2^-53, 1 - 2^-53]
 *   binary32 draw:  v = (2*(x >> 41) + 1) * 2^-24   in [2^-24, 1 - 2^-24]
 * Both are exact in their format; the binary32 draw is returned widened. */
double orc_uniform_from_word(uint64_t x, int single) {
  if (single) return (double)(2 * (x >> 41) + 1) * 0x1p-24;
  return (double)(2 * (x >> 12) + 1) * 0x1p-53;
}

void orc_uniform_draws(uint64_t seed, uint64_t instance, int64_t n, int single, double* v) {
  for (int64_t k = 0; k < n; ++k) v[k] = orc_uniform_from_word(orc_stream_word(seed, instance, (uint64_t)k), single);
}

/* ------------------------------------------------------------------------ */
/* Exact-to-one-rounding prefix sums.  The running sum is kept as an         */
/* unevaluated pair (s, c) with s + c equal to the true partial sum up to    */
/* 2^-104 relative (Knuth's TwoSum), so every reported prefix is the exact    */
/* real prefix rounded once.  This is the plain definition of a sum, written  */
/* so that the oracle's own rounding error is negligible.                     */
/* ------------------------------------------------------------------------ */
typedef struct { double s, c; } orc_dd;

static orc_dd dd_add_double(orc_dd a, double x) {
  double t = a.s + x;
  double bp = t - a.s;
  double err = (a.s - (t - bp)) + (x - bp); /* exact: a.s + x = t + err */
  double c = a.c + err;
  orc_dd r;
  r.s = t + c;
  r.c = c - (r.s - t);
  return r;
}

/* (a.s + a.c) / (b.s + b.c) rounded to binary64 (one Newton correction). */
static double dd_div(orc_dd a, orc_dd b) {
  double q = a.s / b.s;
  /* remainder a - q*b, with q*b.s formed exactly by fma */
  double p = q * b.s;
  double pe = fma(q, b.s, -p);
  double rem = ((a.s - p) - pe) + a.c - q * b.c;
  return q + rem / b.s;
}

/* Eq. 3 with normalisation: W_j = (sum_{k<=j} w_k) / (sum_k w_k).
 * Returns 0 on success, 1 if some weight is negative or not finite, 2 if the
 * total is zero.  W_{M-1} is exactly 1 (x/x). */
int orc_cumulative(const double* w, int64_t M, double* W, double* total) {
  orc_dd acc = {0.0, 0.0};
  for (int64_t j = 0; j < M; ++j) {
    if (!(w[j] >= 0.0) || isinf(w[j])) return 1;
    acc = dd_add_double(acc, w[j]);
  }
  if (total) *total = acc.s;
  if (acc.s == 0.0) return 2;
  orc_dd S = acc;
  acc.s = 0.0;
  acc.c = 0.0;
  for (int64_t j = 0; j < M; ++j) {
    acc = dd_add_double(acc, w[j]);
    W[j] = dd_div(acc, S);
  }
  return 0;
}

/* Same, for binary32 weights (widened exactly to binary64 first). */
int orc_cumulative_f32(const float* w, int64_t M, double* W, double* total) {
  double* wd = (double*)malloc((size_t)(M > 0 ? M : 1) * sizeof(double));
  if (!wd) return 3;
  for (int64_t j = 0; j < M; ++j) wd[j] = (double)w[j];
  int rc = orc_cumulative(wd, M, W, total);
  free(wd);
  return rc;
}

/* Algorithm 1, SortedUniform(N): z_k = -log(v_k) for k = 1..N+1,
 * Z_i = sum_{k<=i} z_k, U_i = Z_i / Z_{N+1} for i = 1..N.
 * (The printed normaliser Z_{i+1} is read as Z_{N+1}: only the latter yields
 * the sorted uniform order statistics the algorithm promises.) */
void orc_sorted_uniform(uint64_t seed, uint64_t instance, int64_t N, int single, double* U) {
  if (N <= 0) return;
  orc_dd Z = {0.0, 0.0};
  double* zs = (double*)malloc((size_t)(N + 1) * sizeof(double));
  orc_dd* pref = (orc_dd*)malloc((size_t)N * sizeof(orc_dd));
  for (int64_t k = 0; k <= N; ++k) {
    double v = orc_uniform_from_word(orc_stream_word(seed, instance, (uint64_t)k), single);
    zs[k] = -log(v);
  }
  for (int64_t k = 0; k <= N; ++k) {
    Z = dd_add_double(Z, zs[k]);
    if (k < N) pref[k] = Z;
  }
  for (int64_t i = 0; i < N; ++i) U[i] = dd_div(pref[i], Z);
  free(zs);
  free(pref);
}

/* Eq. 2-3 by brute force: for each u, scan j = 1..M for the first W_j >= u;
 * if none (u above W_M through rounding) the answer is clamped to M. */
void orc_inverse_cdf(const double* W, int64_t M, const double* U, int64_t N, int32_t* r) {
  for (int64_t i = 0; i < N; ++i) {
    int64_t ans = M - 1;
    for (int64_t j = 0; j < M; ++j) {
      if (W[j] >= U[i]) { ans = j; break; }
    }
    r[i] = (int32_t)ans;
  }
}

/* The same result for sorted U by one monotone walk over W (each W_j and
 * each u visited once).  Requires U non-decreasing; returns 1 otherwise. */
int orc_inverse_cdf_walk(const double* W, int64_t M, const double* U, int64_t N, int32_t* r) {
  int64_t j = 0;
  for (int64_t i = 0; i < N; ++i) {
    if (i > 0 && U[i] < U[i - 1]) return 1;
    while (j < M && !(W[j] >= U[i])) ++j;
    r[i] = (int32_t)(j < M ? j : M - 1);
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* The paper's samplers (Sec. II-III), restated from what they compute.      */
/* Each returns the Eq. 3 answer; they differ only in how they reach it, and  */
/* the probe counter lets the tests compare their costs with Table I.         */
/* ------------------------------------------------------------------------ */

static int64_t g_probes = 0; /* comparisons of a search key with an entry of W */

int64_t orc_alg2_probes(int reset) {
  int64_t p = g_probes;
  if (reset) g_probes = 0;
  return p;
}

/* Algorithm 2's result: over the non-decreasing entries Z1[a..b] (1-based,
 * inclusive) the first index whose entry reaches X, and b when no entry
 * before b does (so b also stands for "X lies above every entry").
 * Bisection on the count of leading entries below X: the candidates are
 * lo .. lo+len, where lo+len = b is the fallback, so Z1[b] is never read. */
int64_t orc_alg2_binary_search(const double* Z1, int64_t a, int64_t b, double X) {
  int64_t lo = a, len = b - a;
  while (len > 0) {
    const int64_t half = len / 2;
    ++g_probes;
    if (Z1[lo + half] < X) {
      lo += half + 1;
      len -= half + 1;
    } else {
      len = half;
    }
  }
  return lo;
}

/* Algorithm 3 on given U: one search over the whole of W per sample. */
void orc_alg3_binary_map(const double* W, int64_t M, const double* U, int64_t N, int32_t* r) {
  for (int64_t i = 0; i < N; ++i) r[i] = (int32_t)(orc_alg2_binary_search(W - 1, 1, M, U[i]) - 1);
}

/* Algorithm 4 (CCF) on given sorted U: one forward pass over W shared by all
 * samples, never moving past the last index. */
void orc_alg4_ccf_map(const double* W, int64_t M, const double* U, int64_t N, int32_t* r) {
  int64_t j = 0;
  for (int64_t i = 0; i < N; ++i) {
    while (j + 1 < M && W[j] < U[i]) ++j;
    r[i] = (int32_t)j;
  }
}

/* Algorithm 5 (divide and conquer) on given sorted U.  The answer of the
 * middle sample of a sample range splits the W range: samples before it
 * have answers at or below it, samples after it at or above it (U sorted,
 * W non-decreasing), so each side recurses on its own part of W, both parts
 * keeping the split index.  A W range of one index answers every sample in
 * it without a search.  trace (optional) receives, in visit order, triples
 * (depth, sample, answer) (1-based) for every search made; the count of
 * searches is returned. */
typedef struct {
  const double* W;
  const double* U;
  int32_t* r;
  int64_t* trace;
  int64_t ntrace, cap;
} dac_ctx;

static void dac_split(dac_ctx* c, int64_t i0, int64_t i1, int64_t lo, int64_t hi, int64_t depth) {
  /* samples [i0, i1) have their answers in W[lo..hi] (0-based, inclusive) */
  if (i0 >= i1) return;
  if (lo == hi) {
    for (int64_t i = i0; i < i1; ++i) c->r[i] = (int32_t)lo;
    return;
  }
  const int64_t mid = i0 + (i1 - 1 - i0) / 2; /* the lower middle */
  const int64_t ans = orc_alg2_binary_search(c->W - 1, lo + 1, hi + 1, c->U[mid]) - 1;
  c->r[mid] = (int32_t)ans;
  if (c->trace && c->ntrace < c->cap) {
    c->trace[3 * c->ntrace] = depth;
    c->trace[3 * c->ntrace + 1] = mid + 1;
    c->trace[3 * c->ntrace + 2] = ans + 1;
  }
  c->ntrace++;
  dac_split(c, i0, mid, lo, ans, depth + 1);
  dac_split(c, mid + 1, i1, ans, hi, depth + 1);
}

int64_t orc_alg5_dac_map(const double* W, int64_t M, const double* U, int64_t N, int32_t* r,
                         int64_t* trace, int64_t trace_cap) {
  if (N <= 0) return 0;
  dac_ctx c = {W, U, r, trace, 0, trace_cap};
  dac_split(&c, 0, N, 0, M - 1, 1);
  return c.ntrace;
}

/* ------------------------------------------------------------------------ */
/* Whole path.                                                                */
/* ------------------------------------------------------------------------ */

/* One instance: W from w (Eq. 3), U from Algorithm 1, r from Eq. 2.
 * w_is_f32 selects binary32 weights; single selects binary32 draws (the
 * compensated-binary32 path's stream), both evaluated here in binary64.
 * W_out, U_out may be NULL.  Returns the orc_cumulative status. */
/* Weights from log-weights, the step the paper places before resampling
 * (Sec. I: the filter carries log-likelihood weights): w_j = exp(l_j - m),
 * m = max_k l_k, so the largest weight is 1 and nothing overflows; -inf
 * gives a zero weight.  Returns 1 for a NaN or +inf log-weight, 2 when every
 * l_j is -inf (zero total), else 0. */
int orc_softmax_weights(const double* l, int64_t M, double* w) {
  double m = -INFINITY;
  for (int64_t j = 0; j < M; ++j) {
    if (isnan(l[j]) || l[j] == INFINITY) return 1;
    if (l[j] > m) m = l[j];
  }
  if (m == -INFINITY) return 2;
  for (int64_t j = 0; j < M; ++j) w[j] = exp(l[j] - m);
  return 0;
}

/* Stratified and systematic uniforms, the variants the paper's concluding
 * section says the method extends to: N points, one per stratum
 * ((i-1)/N, i/N], i = 1..N, with the same draws v_k as Algorithm 1:
 *   stratified  U_i = (i - 1 + v_{i-1}) / N   (a fresh draw per stratum)
 *   systematic  U_i = (i - 1 + v_0) / N       (one draw for all strata)
 * scheme 0 is Algorithm 1 itself. */
void orc_scheme_uniform(uint64_t seed, uint64_t instance, int64_t N, int single, int scheme, double* U) {
  if (N <= 0) return;
  if (scheme == 0) {
    orc_sorted_uniform(seed, instance, N, single, U);
    return;
  }
  const double v0 = orc_uniform_from_word(orc_stream_word(seed, instance, 0), single);
  for (int64_t i = 0; i < N; ++i) {
    const double v = scheme == 1 ? orc_uniform_from_word(orc_stream_word(seed, instance, (uint64_t)i), single) : v0;
    U[i] = ((double)i + v) / (double)N;
  }
}

/* Whole path with the uniforms of `scheme` (0: Algorithm 1, 1: stratified,
 * 2: systematic). */
int orc_resample_scheme(const void* w, int w_is_f32, int64_t M, int64_t N, uint64_t seed, uint64_t instance,
                        int single, int scheme, int32_t* r, double* W_out, double* U_out) {
  double* W = W_out ? W_out : (double*)malloc((size_t)M * sizeof(double));
  double* U = U_out ? U_out : (double*)malloc((size_t)(N > 0 ? N : 1) * sizeof(double));
  int rc = w_is_f32 ? orc_cumulative_f32((const float*)w, M, W, NULL) : orc_cumulative((const double*)w, M, W, NULL);
  if (rc == 0 && N > 0) {
    orc_scheme_uniform(seed, instance, N, single, scheme, U);
    orc_inverse_cdf_walk(W, M, U, N, r);
  }
  if (!W_out) free(W);
  if (!U_out) free(U);
  return rc;
}

int orc_resample(const void* w, int w_is_f32, int64_t M, int64_t N, uint64_t seed, uint64_t instance,
                 int single, int32_t* r, double* W_out, double* U_out) {
  return orc_resample_scheme(w, w_is_f32, M, N, seed, instance, single, 0, r, W_out, U_out);
}

/* K instances laid out back to back: instance k owns w[woff[k] .. woff[k+1])
 * and r[roff[k] .. roff[k+1]); its stream is (seed, instance = k).
 * Returns the first non-zero instance status, or 0. */
int orc_resample_batched(const void* w, int w_is_f32, const int64_t* woff, const int64_t* roff, int64_t K,
                         uint64_t seed, int single, int32_t* r) {
  int first = 0;
  for (int64_t k = 0; k < K; ++k) {
    int64_t M = woff[k + 1] - woff[k], N = roff[k + 1] - roff[k];
    const void* wk = w_is_f32 ? (const void*)((const float*)w + woff[k]) : (const void*)((const double*)w + woff[k]);
    int rc = orc_resample(wk, w_is_f32, M, N, seed, (uint64_t)k, single, r + roff[k], NULL, NULL);
    if (rc && !first) first = rc;
  }
  return first;
}
