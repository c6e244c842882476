/*
 * gbresample -- multinomial particle-filter resampling on NVIDIA GB300 (sm_103a).
 *
 * C ABI of libgbresample.so.  It computes the multinomial resampling map of
 * arXiv 2604.01356 ("A divide and conquer strategy for multinomial particle
 * filter resampling"):
 *
 *   Eq. 3   cumulative weights  W_j = sum_{k<=j} w_k / sum_k w_k,  j = 1..M
 *   Alg. 1  N sorted uniforms    U_i = Z_i / Z_{N+1},  Z_i = sum_{k<=i} -log(v_k)
 *           (the printed normaliser Z_{i+1} is read as Z_{N+1})
 *   Eq. 2   r_i = P^{-1}(U_i) = the smallest j with W_j >= U_i (ties go to j,
 *           a U above W_M is clamped to M), i = 1..N
 *
 * and the three maps the paper compares: divide and conquer (Alg. 5), binary
 * search (Alg. 3 with Alg. 2) and the Carpenter-Clifford-Fearnhead linear walk
 * (Alg. 4).  The draws v_k in (0,1) come from Philox-4x64-10 (Salmon et al.,
 * SC'11): key = (seed, instance), counter = (k/4, 0, 0, 0), 64-bit word k mod 4;
 * binary64 draws are (2*(x>>12)+1)*2^-53, binary32 draws (2*(x>>41)+1)*2^-24.
 *
 * Conventions shared by every entry point
 *  - Pointers named w, W, U, out_* and the batched offset arrays are DEVICE
 *    pointers owned by the caller.  The library never frees them and never
 *    keeps them after the call returns.  Weight and output arrays must be
 *    8-byte aligned; 16-byte alignment enables vectorised loads.
 *  - Indices are 0-based int32: paper index j is returned as j-1.
 *  - Sizes: M >= 1, M < 2^31; N >= 0 (N = 0 is a no-op); N > M is allowed.
 *  - stream is a cudaStream_t (NULL = the legacy default stream).  Every call
 *    only enqueues work on that stream and returns; it does not synchronise.
 *  - Errors found on the host (bad sizes, NULL pointers, bad options, CUDA
 *    launch failures, workspace allocation failure) are returned at once and
 *    enqueue nothing.  Errors found on the device (a negative, NaN or infinite
 *    weight; a zero total; a bounded wait that ran out) are latched in the
 *    handle's device status word and reported by the next rs_get_status();
 *    the outputs of that call are then unspecified but every write stays in
 *    bounds and every kernel terminates.
 *  - A handle owns a grow-only device workspace; calls on one handle must not
 *    overlap (use one handle per concurrent stream).  Handles are not
 *    thread-safe; distinct handles may be used from distinct threads.
 */
#ifndef GBRESAMPLE_H
#define GBRESAMPLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct rs_handle rs_handle;

typedef enum {
  RS_OK = 0,
  RS_EINVAL = 1,      /* bad argument (size, pointer, option) */
  RS_ENOMEM = 2,      /* workspace allocation failed */
  RS_ECUDA = 3,       /* a CUDA runtime call failed */
  RS_ENONFINITE = 4,  /* a weight is negative, NaN or infinite (device-detected) */
  RS_EZEROSUM = 5,    /* the weights sum to zero (device-detected) */
  RS_ETIMEOUT = 6,    /* a bounded inter-block wait gave up (device-detected) */
  RS_ECAPACITY = 7    /* a size exceeds a fixed capacity (rs_sorted_uniform_static) */
} rs_status;

/* Inverse-CDF map used after the cumulative weights and uniforms exist. */
typedef enum {
  RS_MAP_DAC = 0,     /* Alg. 5: split U, search the split points, walk the leaves */
  RS_MAP_BINARY = 1,  /* Alg. 3: one full-range binary search per sample */
  RS_MAP_LINEAR = 2   /* Alg. 4: every W element visited once (merge walk) */
} rs_map_algo;

/* Arithmetic of the path.
 *  RS_F64      binary64 weights and binary64 draws; results carry binary64
 *              accuracy (cumulative weights within 1e-12 relative of exact).
 *  RS_F32_COMP binary32 weights and binary32 draws; spacings and scans run in
 *              binary32 with compensation (error-free transforms / exact
 *              integer segment sums), binary64 only at segment boundaries and
 *              for the final normalisation; W within 4*2^-23 of exact. */
typedef enum { RS_F64 = 0, RS_F32_COMP = 1 } rs_precision;

/* The N points U_1 <= ... <= U_N fed to the inverse CDF (Eq. 2).
 *  RS_SCHEME_MULTINOMIAL  Alg. 1: the order statistics of N uniforms
 *                         (N+1 draws, exponential spacings); the paper's method.
 *  RS_SCHEME_STRATIFIED   one point per stratum ((i-1)/N, i/N]:
 *                         U_i = (i - 1 + v_{i-1}) / N, draws v_0 .. v_{N-1}.
 *  RS_SCHEME_SYSTEMATIC   U_i = (i - 1 + v_0) / N, one draw.
 * The last two are the variants the paper's concluding section says the
 * method extends to; only the points change, the map is the same.  The draws
 * v_k are those of Alg. 1 (same Philox words). */
typedef enum { RS_SCHEME_MULTINOMIAL = 0, RS_SCHEME_STRATIFIED = 1, RS_SCHEME_SYSTEMATIC = 2 } rs_scheme;

/* Options.  A NULL rs_opts pointer, or a zeroed struct, selects defaults. */
typedef struct {
  int32_t algo;        /* rs_map_algo (default RS_MAP_DAC) */
  int32_t prec;        /* rs_precision (default RS_F64) */
  int32_t leaf_L;      /* DaC: samples per leaf (power of two 1..1024; 0 = choose from M/N).
                          rs_resample_batched: the leaf threshold - a segment holding at
                          most leaf_L samples is resolved per sample from its 32 lane
                          prefixes and the one 16-weight block holding the target, a
                          fuller one from all 512 prefixes by per-sample binary search
                          (0 = the autotuned or default value) */
  int32_t stage_max;   /* DaC: largest W range a leaf stages in shared memory (0 = default 512) */
  int32_t spin_limit;  /* bounded-wait iterations before RS_ETIMEOUT (0 = default) */
  int32_t debug_flags; /* test hook, 0 in normal use.  Bit 0: the first tile of every
                          look-back scan of the call (spacings, segment prefixes)
                          withholds its publication, so every later tile's bounded
                          wait runs out and RS_ETIMEOUT is latched (results are then
                          unspecified).  Nothing faults.  Bit 1: rs_resample_w uses
                          the multi-kernel path instead of the single cooperative
                          launch (identical results; for comparison).  Bit 2: the
                          one-CTA paths of small instances (rs_resample_w up to
                          32,768 weights and 2,048 samples, both forms;
                          rs_resample_W up to 12,288 weights and 2,047
                          samples; the sorted uniforms of
                          rs_sorted_uniform and rs_resample_W up to 2,047
                          samples) are not taken (identical results; for
                          comparison).  Bit 0 also keeps the uniforms on the
                          look-back scan whose wait it exercises. */
  int32_t tile_threads; /* rs_resample_batched: threads per CTA, 128, 256 or 512
                           (0 = the autotuned or default value); ignored elsewhere */
  int32_t scheme;      /* rs_scheme of the N uniforms (default RS_SCHEME_MULTINOMIAL) */
} rs_opts;

/* Create a handle bound to the CUDA device current on the calling thread.
 * Allocates the device status word and an initial workspace. */
rs_status rs_create(rs_handle** out);

/* Destroy a handle and free its workspace.  Synchronises the device. */
rs_status rs_destroy(rs_handle* h);

/* Whole path from weights (Eq. 3 + Alg. 1 + Eq. 2).
 *  w       [M] binary64 weights (opts->prec == RS_F64) or binary32 weights
 *          (RS_F32_COMP); non-negative, finite, not all zero; unnormalised.
 *  out_idx [N] int32 sample indices, written.
 *  W_out   [M] binary64 cumulative weights W (Eq. 3), written if not NULL.
 *  seed, instance select the Philox stream of the N+1 draws.
 * Launch forms, all giving identical indices: an instance of at most 12,288
 * weights and 2,047 samples runs with its weights staged in shared memory on
 * one CTA, or from 384 samples on a cluster of four CTAs (each making a
 * quarter of the draws and mapping those samples); one of at most 32,768
 * weights and 2,048 samples on one CTA reading them from global memory
 * (one launch each); otherwise one cooperative launch of one CTA per SM (a
 * multi-kernel sequence when the device cannot hold that grid, or when W_out
 * is requested).  The map is the
 * segmented divide and conquer (exact segment sums and their prefixes, the
 * segment of each key, the element from that segment's exact prefixes);
 * opts->algo is ignored here. */
rs_status rs_resample_w(rs_handle* h, const void* w, int64_t M, int64_t N, uint64_t seed, uint64_t instance,
                        int32_t* out_idx, double* W_out, const rs_opts* opts, void* stream);

/* Sampling from given cumulative weights (Alg. 1 + Eq. 2; the paper's timed
 * "sampling steps", W excluded).
 *  W       [M] binary64 cumulative weights, non-decreasing, W_M = 1 expected
 *          (not checked: a U above W_M is clamped to M-1).
 *  out_idx [N] int32, written.  opts->algo selects the map.
 * Launch forms, all giving identical indices: M <= 12,288 and N <= 2,047 run
 * with W staged in shared memory on one CTA, or from 384 samples on a cluster
 * of four CTAs (the DaC leaves one per thread unless opts->leaf_L is set); otherwise the sorted uniforms (one CTA up to 2,047
 * samples, else a look-back scan) and then the map kernel. */
rs_status rs_resample_W(rs_handle* h, const double* W, int64_t M, int64_t N, uint64_t seed, uint64_t instance,
                        int32_t* out_idx, const rs_opts* opts, void* stream);

/* Alg. 1: N sorted uniforms.  U_out [N] binary64, written.  With
 * opts->prec == RS_F32_COMP the binary32 draws and compensated binary32
 * arithmetic are used and the (hi+lo) result is returned widened. */
rs_status rs_sorted_uniform(rs_handle* h, int64_t N, uint64_t seed, uint64_t instance, double* U_out,
                            const rs_opts* opts, void* stream);

/* rs_sorted_uniform without any memory allocation.  The paper has no
 * counterpart: this entry point exists for callers that must not allocate
 * device memory once they are running -- for example a filter loop that
 * reserved all of its memory at start-up and must keep a fixed footprint, or
 * code that runs while the device is out of memory.  rs_sorted_uniform needs a
 * handle, whose workspace grows by cudaMalloc when a call needs more; this
 * call needs no handle and keeps its scratch (spacing sums, scan descriptors,
 * per-call constants, about 1 MiB) in one fixed device array that is part of
 * the loaded library.  It calls no cudaMalloc, cudaFree or other allocating
 * routine.
 *
 * Results are bit-identical to rs_sorted_uniform with the same N, seed,
 * instance and precision (same kernels, same arithmetic).
 *
 *  N          number of uniforms, 0 <= N <= RS_STATIC_MAX_N (65,536).  A
 *             larger N returns RS_ECAPACITY and enqueues nothing; use
 *             rs_sorted_uniform for it.  N = 0 is a no-op.
 *  precision  RS_F64 or RS_F32_COMP (as opts->prec of rs_sorted_uniform).
 *  U_out      [N] binary64, device, 8-byte aligned, caller-owned; written.
 *  status     optional device pointer to one int32, caller-owned.  A bounded
 *             wait that runs out on the device stores RS_ETIMEOUT there if it
 *             holds 0; the call never clears it.  NULL: such an error is not
 *             reported.
 *  stream     cudaStream_t; the call only enqueues work on it.
 *
 * Host-detected errors (N out of range, bad precision, NULL or misaligned
 * U_out, a failed CUDA call) are returned at once: RS_EINVAL, RS_ECAPACITY or
 * RS_ECUDA.
 *
 * Set-up: the first call on each device (the current device) looks up the
 * scratch array's device address and uploads a 2 KB table used by the
 * logarithm, synchronously; later calls on that device only enqueue work.
 * Make that first call before any stream capture begins.
 *
 * Every call on one device uses the same scratch array, and each call first
 * clears its scan counters there.  Calls whose GPU work can overlap (issued to
 * different streams without ordering, or from different host threads) race on
 * the scratch and give wrong results: issue them on one stream, or order them
 * with events.  Host threads may call it concurrently only if their GPU work
 * is ordered in that way. */
#define RS_STATIC_MAX_N 65536
rs_status rs_sorted_uniform_static(int64_t N, uint64_t seed, uint64_t instance, int32_t precision, double* U_out,
                                   int32_t* status, void* stream);

/* Eq. 3: cumulative weights.  w as in rs_resample_w; W_out [M] binary64,
 * written, non-decreasing, W_out[M-1] == 1 exactly. */
rs_status rs_cumulative(rs_handle* h, const void* w, int64_t M, double* W_out, const rs_opts* opts, void* stream);

/* Eq. 2 only: r_i = smallest j with W_j >= U_i, clamped to M-1.
 *  W [M], U [N] binary64 (U non-decreasing for RS_MAP_DAC and RS_MAP_LINEAR);
 *  out_idx [N] int32, written.  Bit-exact: every comparison is an exact
 *  binary64 comparison, so all three maps return identical indices. */
rs_status rs_map(rs_handle* h, const double* W, int64_t M, const double* U, int64_t N, int32_t* out_idx,
                 const rs_opts* opts, void* stream);

/* Raw Philox-4x64-10 stream words first .. first+n-1 of (seed, instance).
 * out [n] uint64, written.  Exposed so the generator can be checked bit for bit. */
rs_status rs_philox(rs_handle* h, uint64_t seed, uint64_t instance, uint64_t first, int64_t n, uint64_t* out,
                    void* stream);

/* Weights from log-weights (the filter of Sec. I carries log-likelihoods):
 * w_out[j] = exp(logw[j] - max_k logw[k]), binary64, the largest weight 1.
 *  logw  [M] binary64 log-weights, device; -inf gives a zero weight.
 *  w_out [M] binary64, written (may not overlap logw).
 * Computed without binary64 arithmetic per element: the exponential is
 * evaluated in 64-bit integer arithmetic from the difference l - m in fixed
 * point (relative error below 2^-49.5 of the binary64 value, about 2^-52 when
 * |l|, |m| >= 1; subnormal results within 2 units of 2^-1074, and 0 below
 * exp(-745.14)).  NaN, +inf or |l| >= 2^126
 * latch RS_ENONFINITE; all -inf latches RS_EZEROSUM (rs_get_status).
 * Two passes over logw (maximum, then exponent) and one write of w_out. */
rs_status rs_softmax_weights(rs_handle* h, const double* logw, int64_t M, double* w_out, void* stream);

/* rs_resample_w from log-weights: rs_softmax_weights into the handle's
 * workspace (M * 8 bytes more), then the whole path (Eq. 3 + Alg. 1 + Eq. 2).
 * opts as for rs_resample_w; opts->prec must be RS_F64. */
rs_status rs_resample_logw(rs_handle* h, const double* logw, int64_t M, int64_t N, uint64_t seed, uint64_t instance,
                           int32_t* out_idx, const rs_opts* opts, void* stream);

/* The resampled particle set (Sec. I: the filter continues with the particles
 * the indices select): x_out[i] = x[idx[i]], i = 0..N-1, rows of row_bytes
 * bytes.
 *  x       [M rows] particles, row-major, device; 4-byte aligned (16-byte
 *          aligned rows and pointers move 16 bytes per access).
 *  idx     [N] int32 row indices (e.g. the out_idx of a resampling call).
 *  x_out   [N rows], written; must not overlap x.
 *  row_bytes  a positive multiple of 4 (D elements of 4 or 8 bytes).
 * An index outside [0, M) writes a zero row and latches RS_EINVAL in the
 * device status word (rs_get_status).  Bit-exact copy; HBM-bound. */
rs_status rs_gather(rs_handle* h, const void* x, int64_t M, int64_t row_bytes, const int32_t* idx, int64_t N,
                    void* x_out, void* stream);

/* K independent instances (the many-filter setting of Sec. I: M_k = N_k * P_k
 * weights per filter).  Instance k owns w[w_off[k] .. w_off[k+1]) and
 * out_idx[r_off[k] .. r_off[k+1]) and draws from the Philox stream
 * (seed, instance = k); its indices equal those of rs_resample_w on that
 * instance alone (same precision), bit for bit.
 *  w      [w_off[K]] binary32 (RS_F32_COMP, the default for this call when
 *         opts is NULL) or binary64 (RS_F64) weights; 4- resp. 8-byte aligned.
 *  w_off, r_off  [K+1] int64 DEVICE arrays, non-decreasing, starting at 0;
 *         every instance needs M_k >= 1 unless N_k = 0.
 *  h_w_off, h_r_off  optional HOST copies of the same offsets (may be NULL).
 *         When NULL the call copies the offsets to the host and synchronises
 *         the stream (not allowed during stream capture); when given it reads
 *         nothing back from the device.
 *  out_idx [r_off[K]] int32 indices, local to each instance, written.
 * One persistent launch (either precision) processes every instance of at
 * most 262,144 weights and 2,048 samples (one CTA per instance, taken from an
 * atomic queue in order of decreasing M_k); larger instances go through the
 * single-instance path first, on the same stream.  opts->debug_flags bit 2
 * sends every instance through rs_resample_w's cooperative launch instead
 * (identical indices; the per-instance comparison).  opts->tile_threads and
 * opts->leaf_L select the CTA size and the leaf threshold; 0 takes the values
 * rs_autotune_batched stored in the handle (or rs_tuning_load read) for the
 * batch's precision and nearest M/N bucket, or
 * defaults (256, 16). */
rs_status rs_resample_batched(rs_handle* h, const void* w, const int64_t* w_off, const int64_t* r_off, int32_t K,
                              const int64_t* h_w_off, const int64_t* h_r_off, uint64_t seed, int32_t* out_idx,
                              const rs_opts* opts, void* stream);

/* Autotuner of rs_resample_batched: runs the call (same arguments, which must
 * be valid; outputs are written) for each candidate CTA size {128, 256, 512}
 * and leaf threshold {4, 16, 64}, times each with CUDA events on `stream`
 * (one warm-up, three timed runs), keeps the fastest in the handle for later
 * calls with zero tile_threads / leaf_L, and writes it to *best (may be NULL):
 * best->tile_threads, best->leaf_L, best->prec.  Synchronises the stream; call
 * it before any stream capture. */
rs_status rs_autotune_batched(rs_handle* h, const void* w, const int64_t* w_off, const int64_t* r_off, int32_t K,
                              const int64_t* h_w_off, const int64_t* h_r_off, uint64_t seed, int32_t* out_idx,
                              const rs_opts* opts, rs_opts* best, void* stream);

/* Autotuner of the divide-and-conquer map given W (Alg. 5, Sec. III; the
 * paper's concluding recommendation ties the best sampler to M/N, and Table
 * I's cost N log2(M/N + 1) to the leaf size).  Draws the N sorted uniforms of
 * the stream (seed, instance 0) into the handle's workspace, then times
 * rs_map with RS_MAP_DAC for every leaf size 1, 2, 4, ..., 256 (one warm-up,
 * three timed runs, CUDA events on `stream`), keeps the fastest in the handle
 * under the key (RS_F64, M/N bucket round(log2(M/N))) for later calls with
 * opts->leaf_L == 0, and writes it to *best (may be NULL): best->algo,
 * best->leaf_L.
 *  W        [M] binary64 cumulative weights (device, read only).
 *  out_idx  [N] int32 device scratch (overwritten).
 * Synchronises the stream; call it before any stream capture. */
rs_status rs_autotune_map(rs_handle* h, const double* W, int64_t M, int64_t N, uint64_t seed, int32_t* out_idx,
                          rs_opts* best, void* stream);

/* Persistence of tuned settings.  rs_tuning_save writes every setting the
 * handle holds (from rs_autotune_map, rs_autotune_batched or an earlier
 * load) to the JSON file at `path`, each keyed by (GPU name, kind "map_dac"
 * or "batched", dtype "f64" or "f32", M/N bucket), keeping the file's entries
 * of other GPUs.  rs_tuning_load adds the file's entries for this handle's
 * GPU (entries of other GPUs are skipped); RS_EINVAL when the file cannot be
 * read or is not a tuning file.  rs_create loads the file named by the
 * environment variable GBRESAMPLE_TUNING, when set (a missing or malformed
 * file leaves the defaults).  Host only; no device work. */
rs_status rs_tuning_save(rs_handle* h, const char* path);
rs_status rs_tuning_load(rs_handle* h, const char* path);

/* The setting the handle would use for an instance (or batch) of M weights
 * and N samples: kind 0 = the DaC map given W, 1 = the batched kernel;
 * precision RS_F64 / RS_F32_COMP.  out->leaf_L and out->tile_threads are 0
 * when nothing is tuned for that kind and precision (the nearest tuned M/N
 * bucket is used otherwise). */
rs_status rs_tuning_get(rs_handle* h, int32_t kind, int32_t precision, int64_t M, int64_t N, rs_opts* out);

/* Synchronise `stream`, return the device status latched since the previous
 * call (RS_OK if none) and clear it. */
rs_status rs_get_status(rs_handle* h, void* stream);

/* Text of the last host-side error on this handle ("" if none). */
const char* rs_last_error(rs_handle* h);

/* Library version string. */
const char* rs_version(void);

/* Tracing (profiling aid).  While enabled, every kernel the handle launches
 * is bracketed by a pair of CUDA events recorded on the launch stream (also
 * inside CUDA-graph capture, where they become event nodes).
 *  rs_trace_enable  on != 0 starts recording; 0 stops and drops pending pairs.
 *  rs_trace_collect synchronises the device, adds the elapsed time of every
 *                   pending pair to per-kernel totals; keep != 0 keeps the
 *                   pairs (a captured graph re-records them on each replay).
 *  rs_trace_report  writes "name launches total_ms" lines into buf (NUL
 *                   terminated, truncated to cap bytes) and returns RS_OK.
 *  rs_trace_reset   clears the totals. */
rs_status rs_trace_enable(rs_handle* h, int on);
rs_status rs_trace_collect(rs_handle* h, int keep);
rs_status rs_trace_report(rs_handle* h, char* buf, int64_t cap);
rs_status rs_trace_reset(rs_handle* h);

#ifdef __cplusplus
}
#endif

#endif /* GBRESAMPLE_H */
