// Internal interface between the host C-ABI layer (api.cu) and the kernel
// translation units.  Not installed; not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gbr {

// One record per 512-element weight segment, written by the reduce pass.  The
// segment's elements are the integers F_j of its fixed-point grid (unit
// 2^(E - bias - shift) of the weight type).
struct SegRec {
  unsigned long long F;  // exact segment sum on the fixed-point grid
  int E;                 // shared exponent of the segment
  int len;               // valid elements (512 except the last segment)
};
static_assert(sizeof(SegRec) == 16, "SegRec layout");

// After the reduce pass every segment sum is put on one global fixed-point
// grid: unit 2^ge with ge = Emax - bias - shift - kGridHead, Emax the largest
// segment exponent.  A segment's sum becomes F * 2^(E - Emax + kGridHead) in
// grid units (truncated below one unit), every prefix is an exact unsigned
// 128-bit integer (the sum of up to 2^22 segments stays below 2^126), and the
// truncation costs at most nseg units = 2^-71 of the total.
constexpr int kGridHead = 41;
constexpr int kSegsPerTile = 8;  // segments per reduce block, per prefix-scan thread

// Exclusive prefix of one segment on the global grid.
struct SegPre {
  unsigned long long lo, hi;
};
static_assert(sizeof(SegPre) == 16, "SegPre layout");

// Prefix of a segment as an xf value (128-bit mantissa, exponent), used only
// when W itself is written, for the leading segments whose prefix is too small
// for the global grid's absolute resolution: the exclusive prefix inside its
// block of the prefix scan (xin) and every block's total (xagg).
struct SegX {
  unsigned long long lo, hi;
  long long e, pad;
};
static_assert(sizeof(SegX) == 32, "SegX layout");

// Search index over segment prefixes: level 0 holds the high 64 bits of every
// segment's prefix, level l every 32^l-th one.  The top level has <= 32
// entries.
constexpr int kMaxLevels = 8;
struct SegIndex {
  long long n;  // segments
  int nlev;
  long long lvl_n[kMaxLevels];
  unsigned long long* lvl[kMaxLevels];
};

// Per-call constants.  S: the total on the global grid (u128) and the grid
// exponent ge; xf values (mantissa lo, hi, exponent): invZ = 1/Z_{N+1}
// (written by the spacing scan), c = S_grid / Z_{N+1} (grid units per spacing
// unit), invS = 1/S_grid (only when W itself is written).
struct PathConsts {
  unsigned long long S[2];
  long long ge;
  long long Emax;
  unsigned long long invS[3];
  unsigned long long c[3];
  unsigned long long invZ[3];
  unsigned long long pad[3];
};
static_assert(sizeof(PathConsts) == 128, "PathConsts layout");

// Weights per segment (one warp, 16 per lane) and look-back descriptor size.
constexpr int kSegLen = 512;
constexpr int kTileDescBytes = 64;

int num_sms();

// --- uniforms (Algorithm 1) ---------------------------------------------
// Draw counts per tile of the spacing scan (256 threads x 4 draws).
constexpr int kUTile = 1024;
cudaError_t init_log_table();
struct LogTab;
void fill_log_table(LogTab& h);  // host copy of the logarithm table
size_t log_table_bytes();
cudaError_t upload_log_table(void* dst);  // synchronous copy into device memory
struct PathConsts;
// scheme: 0 Algorithm 1 (sorted uniforms), 1 stratified, 2 systematic points.
cudaError_t launch_uniform_scan(bool f32, long long ndraw, unsigned long long seed, unsigned long long inst,
                                void* Z, void* Ztot, PathConsts* consts, void* desc, unsigned* ctr, int* status,
                                int spin_limit, bool withhold_first, cudaStream_t st, int scheme = 0);
cudaError_t launch_uniform_norm(long long N, const void* Z, const PathConsts* consts, double* U, cudaStream_t st);
// Up to kUSmallMaxN samples (one step of the CTA's 2048 draws): the spacing
// scan and U = Z / Z_{N+1} by one CTA in one launch (no cleared workspace); Z
// and U identical to the two above.  Beyond one step the multi-tile scan is
// faster.
constexpr long long kUSmallMaxN = 2047;
cudaError_t launch_uniform_small(bool f32, long long ndraw, unsigned long long seed, unsigned long long inst, void* Z,
                                 double* U, cudaStream_t st, int scheme);
cudaError_t launch_philox(unsigned long long seed, unsigned long long inst, unsigned long long first, long long n,
                          unsigned long long* out, cudaStream_t st);

// --- weights (Eq. 3) ------------------------------------------------------
constexpr int kPrefixTilesPerBlock = 256;  // threads (one tile of 8 segments each) per prefix block
cudaError_t launch_w_reduce(bool f32, bool vec, const void* w, long long M, SegRec* seg, int* emax_blk, int* status,
                            cudaStream_t st);
// xin/xagg (nullptr when W is not written) receive the xf prefixes.
cudaError_t launch_seg_prefix(bool f32, long long M, const SegRec* seg, const int* emax_blk, SegPre* pre,
                              SegX* xin, SegX* xagg, const SegIndex& idx, void* desc, unsigned* ctr,
                              PathConsts* consts, bool with_z, bool need_invS, int* status, int spin_limit,
                              bool withhold_first, cudaStream_t st);
cudaError_t launch_w_write(bool f32, bool vec, const void* w, long long M, const SegRec* seg, const SegPre* pre,
                           const SegX* xin, const SegX* xagg, const PathConsts* consts, double* W, cudaStream_t st);

// --- fused single-instance path (one cooperative launch) ----------------
// Exchange area of the fused kernel (owned by the handle, zeroed once): an
// epoch word, then two slots of one 128-byte line per CTA.
constexpr int kFusedMaxCtas = 256;
constexpr int kFusedXchBytes = 256 + 2 * kFusedMaxCtas * 128;
struct LogTab;
struct FusedLaunch {
  const void* w;
  long long M, N;
  unsigned long long seed, inst;
  SegRec* seg;       // [nseg]
  SegPre* rel;       // [nseg]
  void* crel;        // [1024] u128
  void* Z;           // [N] u128
  unsigned* xch;     // kFusedXchBytes, zeroed when allocated
  int* status;
  int spin;
  bool withhold_first;
  const LogTab* tab;  // device copy of the logarithm table
  int* out;
  int scheme;        // uniforms: 0 Algorithm 1, 1 stratified, 2 systematic
};
// Returns cudaErrorCooperativeLaunchTooLarge (nothing launched) when the
// device cannot hold the whole grid at once.
cudaError_t launch_fused(bool f32, bool vec, const FusedLaunch& L, cudaStream_t st);

// --- weights from log-weights: w_j = exp(l_j - max l) ---------------------
// mkey: one 8-byte word of scratch (device).
cudaError_t launch_softmax_weights(const double* l, long long M, double* w, unsigned long long* mkey, int* status,
                                   cudaStream_t st);

// --- the resampled particle set x'_i = x_{r_i} ----------------------------
cudaError_t launch_gather(const void* x, long long M, long long row_bytes, const int* idx, long long N, void* y,
                          int* status, cudaStream_t st);

// --- maps (Eq. 2; Algorithms 3, 4, 5) -------------------------------------
cudaError_t launch_map_seg(bool f32, bool vec, const void* w, long long M, const SegRec* seg, const SegPre* pre,
                           const SegIndex& idx, const PathConsts* consts, const void* Z, long long N, int G, int* out,
                           cudaStream_t st);
// --- batched persistent path (K instances, one CTA per instance) ----------
constexpr int kBMaxSeg = 512;     // segments of the largest instance a CTA takes (M_k <= 262,144)
constexpr int kBMaxN = 2048;      // samples of the largest instance a CTA takes
constexpr int kSortMax = 16384;   // batches up to this size are ordered by M_k on the device
cudaError_t launch_batched_order(const long long* w_off, int K, int* order, cudaStream_t st);
// f32: binary32 weights and draws, else binary64.  w_off == nullptr: the one
// instance (M0, N0); queue == nullptr: CTA b takes instance b (launch K
// CTAs); order == nullptr: identity order.  Instance k draws from the Philox
// stream (seed, inst_base + k).
// leaf_T: segments holding at most this many samples are decided from their
// 32 lane prefixes and one 16-weight block per sample; denser ones from all
// their prefixes.  lpref: scratch of batched_scratch_bytes(f32, threads, K,
// queue != nullptr) bytes (the lane prefixes, kBMaxSeg x 32 per CTA).
size_t batched_scratch_bytes(bool f32, int threads, int K, bool queue);
cudaError_t launch_batched(bool f32, const void* w, const long long* w_off, const long long* r_off, const int* order,
                           int K, unsigned long long seed, unsigned long long inst_base, long long M0, long long N0,
                           int threads, int leaf_T, int* out, unsigned* queue, int* status, cudaStream_t st, int scheme,
                           const LogTab* tab, unsigned long long* lpref);
// --- the whole path of a small instance, weights staged in shared memory
// (512 threads a CTA; N + 1 <= 2048 draws; at most kSmallMaxM weights).
// Indices equal those of every other form of rs_resample_w.
constexpr int kSmThreads = 512;
constexpr long long kSmallMaxN = 2047;
constexpr long long kSmallMaxM = 12288;
// cluster: 1 (one CTA) or 4 (a cluster of four CTAs on four SMs, each
// making a quarter of the draws and mapping those samples).
cudaError_t launch_small(bool f32, const void* w, long long M, long long N, unsigned long long seed,
                         unsigned long long inst, int* out, int* status, cudaStream_t st, int scheme, const LogTab* tab,
                         int cluster);
// The sampling steps (Algorithm 1 + the map named by algo: 0 divide and
// conquer, 1 binary search, 2 linear walk) on one CTA or (cluster 4) a
// cluster of four with W in shared memory: M <= kSmallMaxM, N <= kSmallMaxN; the
// indices equal those of the multi-launch form.
constexpr int kSmallThreadsW = 512;
cudaError_t launch_small_W(bool f32, int algo, const double* W, long long M, long long N, unsigned long long seed,
                           unsigned long long inst, int L, int* out, cudaStream_t st, int scheme, const LogTab* tab,
                           int cluster);
cudaError_t launch_map_binary(const double* W, long long M, const double* U, long long N, int* out, cudaStream_t st);
cudaError_t launch_map_linear(const double* W, long long M, const double* U, long long N, int* out, cudaStream_t st);
cudaError_t launch_map_dac(const double* W, long long M, const double* U, long long N, int L, int stage_max, int* out,
                           cudaStream_t st);

}  // namespace gbr
