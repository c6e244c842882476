// Host side of the C ABI declared in include/gbresample.h: argument checks,
// the grow-only device workspace, launch sequencing and the device status
// word.  Every entry point enqueues on the caller's stream and returns.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/gbresample.h"
#include "internal.h"

struct rs_trace_pair {
  const char* name;
  cudaEvent_t start, stop;
};
struct rs_trace_total {
  const char* name;
  long long launches;
  double ms;
};

// One tuned setting: the kind of call it applies to ("map_dac": the leaf size
// of the divide-and-conquer map given W; "batched": CTA size and leaf
// threshold of the persistent kernel), the weight precision, and the M/N
// bucket round(log2(M/N)) of the instance (or of the whole batch).
struct rs_tune_entry {
  std::string gpu, kind, dtype;
  int bucket = 0, threads = 0, leaf = 0;
};

struct rs_handle {
  int device = 0;
  int* status = nullptr;  // device status word (first device error wins)
  void* logtab = nullptr; // device copy of the spacing logarithm table (fused path)
  unsigned* xch = nullptr; // exchange area of the fused kernel (epoch + slots)
  void* ws = nullptr;     // grow-only workspace
  size_t ws_bytes = 0;
  std::string err;
  cudaStream_t side = nullptr;    // second stream for work independent of the weights pass
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  bool tracing = false;
  std::string gpu;                        // device name (the key of persisted tuning)
  std::vector<rs_tune_entry> tuned;       // tuned settings (autotuners, rs_tuning_load)
  std::vector<rs_trace_pair> pending;
  std::vector<rs_trace_total> totals;
};

namespace gbr {

int num_sms() {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 0 || dev >= 64) dev = 0;
  if (!cached[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    cached[dev] = n > 0 ? n : 1;
  }
  return cached[dev];
}

}  // namespace gbr

namespace {

using namespace gbr;

constexpr long long kMaxLen = (1LL << 31) - 1;
constexpr int kDefaultSpin = 1 << 22;
constexpr int kStageCap = 512;  // shared-memory staging capacity of the DaC leaf (per warp)
// Instances up to this many weights (and at most kBMaxN samples) run on one
// CTA: the persistent kernel's single-instance form, one launch, no
// inter-CTA exchange.
constexpr long long kSmallM = 1LL << 15;
// Default leaf threshold of the persistent kernel (segments with at most
// this many samples are decided from lane prefixes and one weight block).
constexpr int kBatchedLeafDefault = 16;
// From this many samples the shared-memory one-CTA form runs as a cluster of
// four CTAs (the draws, keys and map split four ways).
constexpr long long kSmallClusterN = 384;

rs_status fail(rs_handle* h, rs_status s, const std::string& msg) {
  if (h) h->err = msg;
  return s;
}
rs_status cuda_fail(rs_handle* h, cudaError_t e, const char* where) {
  if (h) h->err = std::string(where) + ": " + cudaGetErrorString(e);
  return RS_ECUDA;
}
#define RS_CK(h, call)                                        \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);  \
  } while (0)

// Event pair around one launch when the handle is tracing.
struct TraceScope {
  rs_handle* h;
  cudaStream_t st;
  rs_trace_pair p{nullptr, nullptr, nullptr};
  TraceScope(rs_handle* h_, const char* name, cudaStream_t st_) : h(h_), st(st_) {
    if (!h->tracing) return;
    p.name = name;
    if (cudaEventCreate(&p.start) != cudaSuccess || cudaEventCreate(&p.stop) != cudaSuccess) {
      cudaGetLastError();
      p.name = nullptr;
      return;
    }
    // While the stream is being captured into a CUDA graph the records must
    // be external (they become event nodes); otherwise they are plain.
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
      cudaGetLastError();
      cs = cudaStreamCaptureStatusNone;
    }
    external = cs == cudaStreamCaptureStatusActive;
    record(p.start);
  }
  void record(cudaEvent_t e) {
    if (external) cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else cudaEventRecord(e, st);
  }
  ~TraceScope() {
    if (!p.name) return;
    record(p.stop);
    h->pending.push_back(p);
  }
  bool external = false;
};
#define RS_TRACE(h, name, st) TraceScope trace_scope_(h, name, st)

struct Opts {
  int algo = RS_MAP_DAC;
  int prec = RS_F64;
  int leaf_L = 0;
  int stage_max = kStageCap;
  int spin = kDefaultSpin;
  int debug = 0;
  int threads = 0;
  int scheme = RS_SCHEME_MULTINOMIAL;
};

rs_status read_opts(rs_handle* h, const rs_opts* o, Opts* out, int default_prec) {
  Opts r;
  r.prec = default_prec;
  if (o) {
    if (o->algo < 0 || o->algo > 2) return fail(h, RS_EINVAL, "opts.algo out of range");
    if (o->prec < 0 || o->prec > 1) return fail(h, RS_EINVAL, "opts.prec out of range");
    if (o->leaf_L < 0 || o->leaf_L > 1024 || (o->leaf_L & (o->leaf_L - 1)))
      return fail(h, RS_EINVAL, "opts.leaf_L must be 0 or a power of two <= 1024");
    if (o->stage_max < 0) return fail(h, RS_EINVAL, "opts.stage_max negative");
    if (o->spin_limit < 0) return fail(h, RS_EINVAL, "opts.spin_limit negative");
    if (o->scheme < RS_SCHEME_MULTINOMIAL || o->scheme > RS_SCHEME_SYSTEMATIC)
      return fail(h, RS_EINVAL, "opts.scheme must be RS_SCHEME_MULTINOMIAL, _STRATIFIED or _SYSTEMATIC");
    r.scheme = o->scheme;
    if (o->tile_threads != 0 && o->tile_threads != 128 && o->tile_threads != 256 && o->tile_threads != 512)
      return fail(h, RS_EINVAL, "opts.tile_threads must be 0, 128, 256 or 512");
    r.threads = o->tile_threads;
    if (o->debug_flags & ~7) return fail(h, RS_EINVAL, "opts.debug_flags: unknown bit");
    r.debug = o->debug_flags;
    r.algo = o->algo;
    r.prec = o->prec;
    r.leaf_L = o->leaf_L;
    if (o->stage_max) r.stage_max = o->stage_max < kStageCap ? o->stage_max : kStageCap;
    if (o->spin_limit) r.spin = o->spin_limit;
  }
  *out = r;
  return RS_OK;
}

// Carves the single workspace allocation into 256-byte aligned regions.
struct Layout {
  size_t off = 0;
  size_t take(size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~size_t(255);
    return o;
  }
};

rs_status ensure_ws(rs_handle* h, size_t bytes) {
  if (bytes <= h->ws_bytes) return RS_OK;
  size_t want = h->ws_bytes ? h->ws_bytes : (size_t)1 << 20;
  while (want < bytes) want *= 2;
  if (h->ws) {
    cudaError_t e = cudaFree(h->ws);  // implicitly waits for work using it
    h->ws = nullptr;
    h->ws_bytes = 0;
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaFree(workspace)");
  }
  cudaError_t e = cudaMalloc(&h->ws, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    h->ws = nullptr;
    return fail(h, RS_ENOMEM, "workspace allocation of " + std::to_string(want) + " bytes failed");
  }
  h->ws_bytes = want;
  return RS_OK;
}

// Regions of one call.  The counters and look-back descriptors sit first so
// that a single memset clears them.
struct Plan {
  // weights side
  long long M = 0, nseg = 0, ntile = 0, pblocks = 0;
  int nlev = 0;
  long long lvl_n[kMaxLevels] = {0};
  int max_blocks = 0;
  size_t o_agg = 0, o_crel = 0;
  size_t o_wdesc = 0, o_seg = 0, o_emax = 0, o_pre = 0, o_xin = 0, o_xagg = 0, o_lvl[kMaxLevels] = {0}, o_consts = 0;
  // uniforms side
  long long N = 0, ndraw = 0, utiles = 0;
  size_t o_udesc = 0, o_Z = 0, o_Ztot = 0, o_U = 0;
  size_t o_ctr = 0, clear_bytes = 0, bytes = 0;
};

Plan make_plan(long long M, long long N, bool need_w, bool need_u, bool need_U, bool need_W = false) {
  Plan p;
  Layout L;
  p.o_ctr = L.take(256);  // [0]: uniform tile counter, [1]: weight tile counter
  if (need_u) {
    p.N = N;
    p.ndraw = N + 1;
    p.utiles = (p.ndraw + kUTile - 1) / kUTile;
    p.o_udesc = L.take((size_t)p.utiles * kTileDescBytes);
  }
  if (need_w) {
    p.M = M;
    p.nseg = (M + kSegLen - 1) / kSegLen;
    p.ntile = (p.nseg + kSegsPerTile - 1) / kSegsPerTile;
    p.pblocks = (p.ntile + kPrefixTilesPerBlock - 1) / kPrefixTilesPerBlock;
    p.o_wdesc = L.take((size_t)p.pblocks * kTileDescBytes);
  }
  p.clear_bytes = L.off;
  if (need_w) {
    p.o_seg = L.take((size_t)p.nseg * sizeof(SegRec));
    // per-block exponent maxima (reduce blocks, or the fused kernel's CTAs),
    // padded to whole 16-byte groups; the fused kernel's CTA totals
    p.max_blocks = num_sms() * 2;
    const long long ne = p.ntile > p.max_blocks ? p.ntile : p.max_blocks;
    p.o_emax = L.take((size_t)((ne + 3) / 4) * 16);
    p.o_agg = L.take((size_t)p.max_blocks * 16);
    p.o_crel = L.take((size_t)2048 * 16);
    p.o_pre = L.take((size_t)p.nseg * sizeof(SegPre));
    if (need_W) {
      p.o_xin = L.take((size_t)p.nseg * sizeof(SegX));
      p.o_xagg = L.take((size_t)p.pblocks * sizeof(SegX));
    }
    long long n = p.nseg;
    p.nlev = 0;
    while (true) {
      p.lvl_n[p.nlev] = n;
      p.o_lvl[p.nlev] = L.take((size_t)n * 8);
      ++p.nlev;
      if (n <= 32 || p.nlev == kMaxLevels) break;
      n = (n + 31) / 32;
    }
    p.o_consts = L.take(sizeof(PathConsts));
  }
  if (need_u) {
    p.o_Z = L.take((size_t)(N > 0 ? N : 1) * 16);
    p.o_Ztot = L.take(16);
    if (need_U) p.o_U = L.take((size_t)(N > 0 ? N : 1) * 8);
  }
  p.bytes = L.off;
  return p;
}

SegIndex index_of(rs_handle* h, const Plan& p) {
  SegIndex idx;
  memset(&idx, 0, sizeof(idx));
  idx.n = p.nseg;
  idx.nlev = p.nlev;
  for (int l = 0; l < p.nlev; ++l) {
    idx.lvl_n[l] = p.lvl_n[l];
    idx.lvl[l] = reinterpret_cast<unsigned long long*>(static_cast<char*>(h->ws) + p.o_lvl[l]);
  }
  return idx;
}

template <typename P>
P* at(rs_handle* h, size_t off) {
  return reinterpret_cast<P*>(static_cast<char*>(h->ws) + off);
}
unsigned* ctr_u(rs_handle* h, const Plan& p) { return at<unsigned>(h, p.o_ctr); }
unsigned* ctr_w(rs_handle* h, const Plan& p) { return at<unsigned>(h, p.o_ctr) + 1; }

rs_status check_handle(rs_handle* h) {
  if (!h) return RS_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return cuda_fail(h, cudaGetLastError(), "cudaGetDevice");
  if (dev != h->device) return fail(h, RS_EINVAL, "handle belongs to another CUDA device than the current one");
  h->err.clear();
  return RS_OK;
}

rs_status check_sizes(rs_handle* h, long long M, long long N) {
  if (M < 1 || M > kMaxLen) return fail(h, RS_EINVAL, "M must satisfy 1 <= M < 2^31");
  if (N < 0 || N > kMaxLen) return fail(h, RS_EINVAL, "N must satisfy 0 <= N < 2^31");
  return RS_OK;
}

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// ---- tuned settings ----------------------------------------------------------
int mn_bucket(long long M, long long N) {
  if (N <= 0 || M <= 0) return 0;
  const double b = std::round(std::log2((double)M / (double)N));
  return (int)(b < -16 ? -16 : (b > 40 ? 40 : b));
}
// The entry for (kind, dtype) with the nearest bucket (ties: the lower), or
// nullptr.
const rs_tune_entry* find_tune(const rs_handle* h, const char* kind, bool f32, int bucket) {
  const rs_tune_entry* best = nullptr;
  for (const auto& t : h->tuned) {
    if (t.kind != kind || t.dtype != (f32 ? "f32" : "f64")) continue;
    if (!best || std::abs(t.bucket - bucket) < std::abs(best->bucket - bucket) ||
        (std::abs(t.bucket - bucket) == std::abs(best->bucket - bucket) && t.bucket < best->bucket))
      best = &t;
  }
  return best;
}
void set_tune(rs_handle* h, const char* kind, bool f32, int bucket, int threads, int leaf) {
  for (auto& t : h->tuned)
    if (t.kind == kind && t.dtype == (f32 ? "f32" : "f64") && t.bucket == bucket) {
      t.threads = threads;
      t.leaf = leaf;
      return;
    }
  rs_tune_entry t;
  t.gpu = h->gpu;
  t.kind = kind;
  t.dtype = f32 ? "f32" : "f64";
  t.bucket = bucket;
  t.threads = threads;
  t.leaf = leaf;
  h->tuned.push_back(t);
}
// Reads the flat JSON written by rs_tuning_save: {"entries": [{"gpu": ...,
// "kind": ..., "dtype": ..., "mn_bucket": n, "tile_threads": n, "leaf_L": n},
// ...]}.  Entries of other GPUs are skipped.  Returns false when the text is
// not of that form.
bool parse_tuning(rs_handle* h, const std::string& text) {
  const size_t e = text.find("\"entries\"");
  if (e == std::string::npos) return false;
  size_t i = text.find('[', e);
  if (i == std::string::npos) return false;
  std::vector<rs_tune_entry> got;
  while (true) {
    const size_t a = text.find('{', i), close = text.find(']', i);
    if (a == std::string::npos || (close != std::string::npos && close < a)) break;
    const size_t b = text.find('}', a);
    if (b == std::string::npos) return false;
    rs_tune_entry t;
    bool ok_kind = false;
    size_t p = a + 1;
    while (p < b) {
      const size_t k0 = text.find('"', p);
      if (k0 == std::string::npos || k0 >= b) break;
      const size_t k1 = text.find('"', k0 + 1);
      const size_t colon = text.find(':', k1);
      if (k1 == std::string::npos || colon == std::string::npos || colon >= b) return false;
      const std::string key = text.substr(k0 + 1, k1 - k0 - 1);
      size_t v = colon + 1;
      while (v < b && (text[v] == ' ' || text[v] == '\n' || text[v] == '\t')) ++v;
      std::string val;
      if (v < b && text[v] == '"') {
        const size_t v1 = text.find('"', v + 1);
        if (v1 == std::string::npos || v1 > b) return false;
        val = text.substr(v + 1, v1 - v - 1);
        p = v1 + 1;
      } else {
        size_t v1 = v;
        while (v1 < b && text[v1] != ',' && text[v1] != '}') ++v1;
        val = text.substr(v, v1 - v);
        p = v1;
      }
      if (key == "gpu") t.gpu = val;
      else if (key == "kind") t.kind = val, ok_kind = true;
      else if (key == "dtype") t.dtype = val;
      else if (key == "mn_bucket") t.bucket = atoi(val.c_str());
      else if (key == "tile_threads") t.threads = atoi(val.c_str());
      else if (key == "leaf_L") t.leaf = atoi(val.c_str());
    }
    if (!ok_kind || (t.dtype != "f32" && t.dtype != "f64")) return false;
    got.push_back(t);
    i = b + 1;
  }
  for (const auto& t : got) {
    if (t.gpu != h->gpu) continue;
    if ((t.kind == "map_dac" && t.leaf >= 1 && t.leaf <= 1024 && !(t.leaf & (t.leaf - 1))) ||
        (t.kind == "batched" && (t.threads == 128 || t.threads == 256 || t.threads == 512) && t.leaf >= 1))
      set_tune(h, t.kind.c_str(), t.dtype == "f32", t.bucket, t.threads, t.leaf);
  }
  return true;
}

// Samples per warp group of the segmented map: about two warps' worth of
// groups per SM slot, at least one sample each.
int group_size(long long N) {
  const long long target = (long long)num_sms() * 64;
  long long G = (N + target - 1) / target;
  if (G < 1) G = 1;
  if (G > (1 << 20)) G = 1 << 20;
  return (int)G;
}

// DaC leaf size: the largest power of two L <= 256 whose expected W range
// (L*M/N elements) fits the staging capacity; 1 when samples are sparse.
int leaf_size(const rs_handle* h, const Opts& o, long long M, long long N) {
  if (o.leaf_L > 0) return o.leaf_L;
  if (const rs_tune_entry* t = find_tune(h, "map_dac", false, mn_bucket(M, N))) return t->leaf;
  double cap = (double)o.stage_max * (double)N / (double)M;
  int L = 1;
  while (L * 2 <= 256 && L * 2 <= cap) L *= 2;
  return L;
}

// Spacing scan (Algorithm 1's Z), plus U = Z / Z_{N+1} when U_out is given.
rs_status enqueue_uniforms(rs_handle* h, const Plan& p, bool f32, uint64_t seed, uint64_t inst, double* U_out,
                           const Opts& o, cudaStream_t st) {
  {
    RS_TRACE(h, "uniform_scan", st);
    RS_CK(h, launch_uniform_scan(f32, p.ndraw, seed, inst, at<void>(h, p.o_Z), at<void>(h, p.o_Ztot),
                                 at<PathConsts>(h, p.o_consts), at<void>(h, p.o_udesc), ctr_u(h, p), h->status,
                                 o.spin, o.debug & 1, st, o.scheme));
  }
  if (U_out) {
    RS_TRACE(h, "uniform_norm", st);
    RS_CK(h, launch_uniform_norm(p.N, at<void>(h, p.o_Z), at<PathConsts>(h, p.o_consts), U_out, st));
  }
  return RS_OK;
}

rs_status enqueue_clear(rs_handle* h, const Plan& p, cudaStream_t st) {
  RS_TRACE(h, "clear", st);
  RS_CK(h, cudaMemsetAsync(h->ws, 0, p.clear_bytes, st));
  return RS_OK;
}

// Segment-prefix scan (also produces S, 1/S and, when the spacing sums exist,
// S/Z_{N+1}).
rs_status enqueue_prefix(rs_handle* h, const Plan& p, const Opts& o, bool f32, bool with_z, bool need_invS,
                         cudaStream_t st) {
  RS_TRACE(h, "seg_prefix", st);
  const SegIndex idx = index_of(h, p);
  RS_CK(h, launch_seg_prefix(f32, p.M, at<SegRec>(h, p.o_seg), at<int>(h, p.o_emax), at<SegPre>(h, p.o_pre),
                             p.o_xin ? at<SegX>(h, p.o_xin) : nullptr, p.o_xagg ? at<SegX>(h, p.o_xagg) : nullptr, idx,
                             at<void>(h, p.o_wdesc), ctr_w(h, p), at<PathConsts>(h, p.o_consts), with_z, need_invS,
                             h->status, o.spin, o.debug & 1, st));
  return RS_OK;
}

// Weights pass: streaming exact segment sums, then the segment-prefix scan.
rs_status enqueue_pass1(rs_handle* h, const Plan& p, const Opts& o, bool f32, bool vec, const void* w,
                        bool with_z, bool need_invS, cudaStream_t st) {
  {
    RS_TRACE(h, "w_reduce", st);
    RS_CK(h, launch_w_reduce(f32, vec, w, p.M, at<SegRec>(h, p.o_seg), at<int>(h, p.o_emax), h->status, st));
  }
  return enqueue_prefix(h, p, o, f32, with_z, need_invS, st);
}

rs_status enqueue_write(rs_handle* h, const Plan& p, bool f32, bool vec, const void* w, double* W_out,
                        cudaStream_t st) {
  RS_TRACE(h, "w_write", st);
  RS_CK(h, launch_w_write(f32, vec, w, p.M, at<SegRec>(h, p.o_seg), at<SegPre>(h, p.o_pre), at<SegX>(h, p.o_xin),
                          at<SegX>(h, p.o_xagg), at<PathConsts>(h, p.o_consts), W_out, st));
  return RS_OK;
}

rs_status enqueue_map(rs_handle* h, const Opts& o, const double* W, long long M, const double* U, long long N,
                      int32_t* out, cudaStream_t st) {
  switch (o.algo) {
    case RS_MAP_BINARY: {
      RS_TRACE(h, "map_binary", st);
      RS_CK(h, launch_map_binary(W, M, U, N, out, st));
      break;
    }
    case RS_MAP_LINEAR: {
      RS_TRACE(h, "map_linear", st);
      RS_CK(h, launch_map_linear(W, M, U, N, out, st));
      break;
    }
    default: {
      RS_TRACE(h, "map_dac", st);
      RS_CK(h, launch_map_dac(W, M, U, N, leaf_size(h, o, M, N), o.stage_max, out, st));
      break;
    }
  }
  return RS_OK;
}

}  // namespace

extern "C" {

const char* rs_version(void) { return "gbresample 0.1 (sm_103a)"; }

rs_status rs_create(rs_handle** out) {
  if (!out) return RS_EINVAL;
  *out = nullptr;
  rs_handle* h = new (std::nothrow) rs_handle();
  if (!h) return RS_ENOMEM;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaMalloc(&h->status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(h->status, 0, sizeof(int));
  if (e == cudaSuccess) e = init_log_table();
  if (e == cudaSuccess) e = cudaMalloc(&h->logtab, log_table_bytes());
  if (e == cudaSuccess) e = upload_log_table(h->logtab);
  if (e == cudaSuccess) e = cudaMalloc(&h->xch, kFusedXchBytes);
  if (e == cudaSuccess) e = cudaMemset(h->xch, 0, kFusedXchBytes);
  int prio_lo = 0, prio_hi = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
  // the side stream carries short work that the weights pass must not starve
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&h->side, cudaStreamNonBlocking, prio_hi);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  cudaDeviceProp prop;
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, h->device);
  if (e == cudaSuccess) h->gpu = prop.name;
  if (e != cudaSuccess) {
    cudaGetLastError();
    if (h->status) cudaFree(h->status);
    if (h->logtab) cudaFree(h->logtab);
    if (h->xch) cudaFree(h->xch);
    if (h->side) cudaStreamDestroy(h->side);
    if (h->ev_fork) cudaEventDestroy(h->ev_fork);
    if (h->ev_join) cudaEventDestroy(h->ev_join);
    delete h;
    return RS_ECUDA;
  }
  // tuned settings persisted by an earlier rs_tuning_save (if any)
  if (const char* path = getenv("GBRESAMPLE_TUNING")) {
    if (*path) rs_tuning_load(h, path);  // a missing or malformed file leaves the defaults
    h->err.clear();
  }
  *out = h;
  return RS_OK;
}

rs_status rs_tuning_save(rs_handle* h, const char* path) {
  if (!h || !path) return RS_EINVAL;
  // keep the file's entries of other GPUs
  std::vector<rs_tune_entry> keep;
  if (FILE* f = fopen(path, "rb")) {
    std::string text;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
    fclose(f);
    rs_handle other;
    for (size_t pos = 0; (pos = text.find("\"gpu\": \"", pos)) != std::string::npos;) {
      const size_t a0 = pos + 8, b0 = text.find('"', a0);
      if (b0 == std::string::npos) break;
      other.gpu = text.substr(a0, b0 - a0);
      pos = b0;
      if (other.gpu == h->gpu) continue;
      other.tuned.clear();
      if (!parse_tuning(&other, text)) break;
      for (const auto& t : other.tuned) {
        bool dup = false;
        for (const auto& k : keep)
          dup |= k.gpu == t.gpu && k.kind == t.kind && k.dtype == t.dtype && k.bucket == t.bucket;
        if (!dup) keep.push_back(t);
      }
    }
  }
  FILE* f = fopen(path, "wb");
  if (!f) return fail(h, RS_EINVAL, std::string("cannot write ") + path);
  fprintf(f, "{\n  \"format\": \"gbresample tuning 1\",\n  \"entries\": [");
  bool first = true;
  auto put = [&](const rs_tune_entry& t) {
    fprintf(f, "%s\n    {\"gpu\": \"%s\", \"kind\": \"%s\", \"dtype\": \"%s\", \"mn_bucket\": %d, "
               "\"tile_threads\": %d, \"leaf_L\": %d}",
            first ? "" : ",", t.gpu.c_str(), t.kind.c_str(), t.dtype.c_str(), t.bucket, t.threads, t.leaf);
    first = false;
  };
  for (const auto& t : keep) put(t);
  for (const auto& t : h->tuned) put(t);
  fprintf(f, "\n  ]\n}\n");
  const bool ok = fclose(f) == 0;
  return ok ? RS_OK : fail(h, RS_EINVAL, std::string("cannot write ") + path);
}

rs_status rs_tuning_load(rs_handle* h, const char* path) {
  if (!h || !path) return RS_EINVAL;
  FILE* f = fopen(path, "rb");
  if (!f) return fail(h, RS_EINVAL, std::string("cannot read ") + path);
  std::string text;
  char buf[4096];
  size_t n;
  while ((n = fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
  fclose(f);
  if (!parse_tuning(h, text)) return fail(h, RS_EINVAL, std::string("not a tuning file: ") + path);
  return RS_OK;
}

rs_status rs_tuning_get(rs_handle* h, int32_t kind, int32_t precision, int64_t M, int64_t N, rs_opts* out) {
  if (!h || !out || (kind != 0 && kind != 1) || (precision != RS_F64 && precision != RS_F32_COMP)) return RS_EINVAL;
  memset(out, 0, sizeof(*out));
  out->prec = precision;
  const rs_tune_entry* t = find_tune(h, kind == 0 ? "map_dac" : "batched", precision == RS_F32_COMP, mn_bucket(M, N));
  if (!t) return RS_OK;
  out->leaf_L = t->leaf;
  out->tile_threads = t->threads;
  return RS_OK;
}

rs_status rs_destroy(rs_handle* h) {
  if (!h) return RS_EINVAL;
  for (auto& p : h->pending) {
    cudaEventDestroy(p.start);
    cudaEventDestroy(p.stop);
  }
  h->pending.clear();
  cudaError_t e1 = cudaSuccess, e2 = cudaSuccess;
  if (h->ws) e1 = cudaFree(h->ws);
  if (h->status) e2 = cudaFree(h->status);
  if (h->logtab) cudaFree(h->logtab);
  if (h->xch) cudaFree(h->xch);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  delete h;
  return (e1 == cudaSuccess && e2 == cudaSuccess) ? RS_OK : RS_ECUDA;
}

const char* rs_last_error(rs_handle* h) { return h ? h->err.c_str() : "null handle"; }

static void drop_pending(rs_handle* h) {
  for (auto& p : h->pending) {
    cudaEventDestroy(p.start);
    cudaEventDestroy(p.stop);
  }
  h->pending.clear();
}

rs_status rs_trace_enable(rs_handle* h, int on) {
  if (!h) return RS_EINVAL;
  h->tracing = on != 0;
  if (!on) drop_pending(h);
  return RS_OK;
}

rs_status rs_trace_collect(rs_handle* h, int keep) {
  if (!h) return RS_EINVAL;
  RS_CK(h, cudaDeviceSynchronize());
  for (auto& p : h->pending) {
    float ms = 0.f;
    RS_CK(h, cudaEventElapsedTime(&ms, p.start, p.stop));
    bool found = false;
    for (auto& t : h->totals)
      if (std::strcmp(t.name, p.name) == 0) {
        t.launches += 1;
        t.ms += ms;
        found = true;
        break;
      }
    if (!found) h->totals.push_back({p.name, 1, (double)ms});
  }
  if (!keep) drop_pending(h);
  return RS_OK;
}

rs_status rs_trace_report(rs_handle* h, char* buf, int64_t cap) {
  if (!h || !buf || cap <= 0) return RS_EINVAL;
  std::string out;
  char line[160];
  for (auto& t : h->totals) {
    std::snprintf(line, sizeof(line), "%s %lld %.6f\n", t.name, t.launches, t.ms);
    out += line;
  }
  const size_t n = out.size() < (size_t)(cap - 1) ? out.size() : (size_t)(cap - 1);
  std::memcpy(buf, out.data(), n);
  buf[n] = 0;
  return RS_OK;
}

rs_status rs_trace_reset(rs_handle* h) {
  if (!h) return RS_EINVAL;
  h->totals.clear();
  return RS_OK;
}

rs_status rs_get_status(rs_handle* h, void* stream) {
  if (!h) return RS_EINVAL;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RS_CK(h, cudaStreamSynchronize(st));
  int v = 0;
  RS_CK(h, cudaMemcpy(&v, h->status, sizeof(int), cudaMemcpyDeviceToHost));
  RS_CK(h, cudaMemset(h->status, 0, sizeof(int)));
  if (v < 0 || v > RS_ETIMEOUT) v = RS_ECUDA;
  return (rs_status)v;
}

rs_status rs_philox(rs_handle* h, uint64_t seed, uint64_t instance, uint64_t first, int64_t n, uint64_t* out,
                    void* stream) {
  rs_status s = check_handle(h);
  if (s) return s;
  if (n < 0) return fail(h, RS_EINVAL, "n must be >= 0");
  if (n == 0) return RS_OK;
  if (!out || !aligned(out, 8)) return fail(h, RS_EINVAL, "out must be a non-NULL 8-byte aligned device pointer");
  RS_TRACE(h, "philox", static_cast<cudaStream_t>(stream));
  RS_CK(h, launch_philox(seed, instance, first, n, reinterpret_cast<unsigned long long*>(out),
                         static_cast<cudaStream_t>(stream)));
  return RS_OK;
}

rs_status rs_sorted_uniform(rs_handle* h, int64_t N, uint64_t seed, uint64_t instance, double* U_out,
                            const rs_opts* opts, void* stream) {
  rs_status s = check_handle(h);
  if (s) return s;
  Opts o;
  if ((s = read_opts(h, opts, &o, RS_F64))) return s;
  if (N < 0 || N > kMaxLen) return fail(h, RS_EINVAL, "N must satisfy 0 <= N < 2^31");
  if (N == 0) return RS_OK;
  if (!U_out || !aligned(U_out, 8)) return fail(h, RS_EINVAL, "U_out must be a non-NULL 8-byte aligned pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Plan p = make_plan(0, N, false, true, false);
  if ((s = ensure_ws(h, p.bytes))) return s;
  if (N <= kUSmallMaxN && !(o.debug & 5)) {  // one CTA, one launch
    RS_TRACE(h, "uniform_small", st);
    RS_CK(h, launch_uniform_small(o.prec == RS_F32_COMP, N + 1, seed, instance, at<void>(h, p.o_Z), U_out, st,
                                  o.scheme));
    return RS_OK;
  }
  if ((s = enqueue_clear(h, p, st))) return s;
  return enqueue_uniforms(h, p, o.prec == RS_F32_COMP, seed, instance, U_out, o, st);
}

rs_status rs_cumulative(rs_handle* h, const void* w, int64_t M, double* W_out, const rs_opts* opts, void* stream) {
  rs_status s = check_handle(h);
  if (s) return s;
  Opts o;
  if ((s = read_opts(h, opts, &o, RS_F64))) return s;
  if ((s = check_sizes(h, M, 0))) return s;
  const bool f32 = o.prec == RS_F32_COMP;
  if (!w || !aligned(w, f32 ? 4 : 8)) return fail(h, RS_EINVAL, "w must be a non-NULL aligned device pointer");
  if (!W_out || !aligned(W_out, 8)) return fail(h, RS_EINVAL, "W_out must be a non-NULL 8-byte aligned pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const Plan p = make_plan(M, 0, true, false, false, true);
  if ((s = ensure_ws(h, p.bytes))) return s;
  const bool vec = aligned(w, 16);
  if ((s = enqueue_clear(h, p, st))) return s;
  if ((s = enqueue_pass1(h, p, o, f32, vec, w, false, true, st))) return s;
  return enqueue_write(h, p, f32, vec, w, W_out, st);
}

rs_status rs_resample_w(rs_handle* h, const void* w, int64_t M, int64_t N, uint64_t seed, uint64_t instance,
                        int32_t* out_idx, double* W_out, const rs_opts* opts, void* stream) {
  rs_status s = check_handle(h);
  if (s) return s;
  Opts o;
  if ((s = read_opts(h, opts, &o, RS_F64))) return s;
  if ((s = check_sizes(h, M, N))) return s;
  const bool f32 = o.prec == RS_F32_COMP;
  if (!w || !aligned(w, f32 ? 4 : 8)) return fail(h, RS_EINVAL, "w must be a non-NULL aligned device pointer");
  if (N > 0 && (!out_idx || !aligned(out_idx, 4))) return fail(h, RS_EINVAL, "out_idx must be a non-NULL pointer");
  if (W_out && !aligned(W_out, 8)) return fail(h, RS_EINVAL, "W_out must be 8-byte aligned");
  if (N == 0 && !W_out) return RS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (N > 0 && !W_out && !(o.debug & 6) && M <= kSmallMaxM && N <= kSmallMaxN) {
    // a small instance: the whole path on one CTA, the weights staged in
    // shared memory
    RS_TRACE(h, "small_smem", st);
    RS_CK(h, launch_small(f32, w, M, N, seed, instance, out_idx, h->status, st, o.scheme,
                          static_cast<const LogTab*>(h->logtab), N >= kSmallClusterN ? 4 : 1));
    return RS_OK;
  }
  if (N > 0 && !W_out && !(o.debug & 6) && M <= kSmallM && N <= kBMaxN) {
    // a small instance: the whole path on one CTA
    Layout L;
    const size_t o_lp = L.take(batched_scratch_bytes(f32, 256, 1, false));
    if ((s = ensure_ws(h, L.off))) return s;
    RS_TRACE(h, "single_cta", st);
    RS_CK(h, launch_batched(f32, w, nullptr, nullptr, nullptr, 1, seed, instance, M, N, 256, kBatchedLeafDefault,
                            out_idx, nullptr, h->status, st, o.scheme, static_cast<const LogTab*>(h->logtab),
                            at<unsigned long long>(h, o_lp)));
    return RS_OK;
  }
  const Plan p = make_plan(M, N, true, N > 0, false, W_out != nullptr);
  if (N > 0 && !W_out && !(o.debug & 2)) {
    // the whole path in one cooperative launch (when the device holds it);
    // it needs no cleared workspace
    if ((s = ensure_ws(h, p.bytes))) return s;
    FusedLaunch F;
    F.w = w;
    F.M = M;
    F.N = N;
    F.seed = seed;
    F.inst = instance;
    F.seg = at<SegRec>(h, p.o_seg);
    F.rel = at<SegPre>(h, p.o_pre);
    F.crel = at<void>(h, p.o_crel);
    F.Z = at<void>(h, p.o_Z);
    F.xch = h->xch;
    F.status = h->status;
    F.spin = o.spin;
    F.withhold_first = o.debug & 1;
    F.tab = static_cast<const LogTab*>(h->logtab);
    F.out = out_idx;
    F.scheme = o.scheme;
    cudaError_t e;
    {
      RS_TRACE(h, "fused", st);
      e = launch_fused(f32, aligned(w, 16), F, st);
    }
    if (e == cudaSuccess) return RS_OK;
    if (e != cudaErrorCooperativeLaunchTooLarge) return cuda_fail(h, e, "launch_fused");
    cudaGetLastError();  // the device cannot hold the grid: multi-kernel path
  }
  if ((s = ensure_ws(h, p.bytes))) return s;
  const bool vec = aligned(w, 16);
  // fork: the workspace clear and the spacing scan (independent of w) run on
  // the handle's side stream while the weights stream through w_reduce; the
  // prefix scan joins them (it needs Z_{N+1} and the cleared counters).
  RS_CK(h, cudaEventRecord(h->ev_fork, st));
  RS_CK(h, cudaStreamWaitEvent(h->side, h->ev_fork, 0));
  if ((s = enqueue_clear(h, p, h->side))) return s;
  if (N > 0) {
    if ((s = enqueue_uniforms(h, p, f32, seed, instance, nullptr, o, h->side))) return s;
  }
  RS_CK(h, cudaEventRecord(h->ev_join, h->side));
  {
    RS_TRACE(h, "w_reduce", st);
    RS_CK(h, launch_w_reduce(f32, vec, w, p.M, at<SegRec>(h, p.o_seg), at<int>(h, p.o_emax), h->status, st));
  }
  RS_CK(h, cudaStreamWaitEvent(st, h->ev_join, 0));
  if ((s = enqueue_prefix(h, p, o, f32, N > 0, W_out != nullptr, st))) return s;
  if (N > 0) {
    RS_TRACE(h, "map_seg", st);
    const SegIndex idx = index_of(h, p);
    RS_CK(h, launch_map_seg(f32, vec, w, M, at<SegRec>(h, p.o_seg), at<SegPre>(h, p.o_pre), idx,
                            at<PathConsts>(h, p.o_consts), at<void>(h, p.o_Z), N, group_size(N), out_idx, st));
  }
  if (W_out) return enqueue_write(h, p, f32, vec, w, W_out, st);
  return RS_OK;
}

rs_status rs_resample_W(rs_handle* h, const double* W, int64_t M, int64_t N, uint64_t seed, uint64_t instance,
                        int32_t* out_idx, const rs_opts* opts, void* stream) {
  rs_status s = check_handle(h);
  if (s) return s;
  Opts o;
  if ((s = read_opts(h, opts, &o, RS_F64))) return s;
  if ((s = check_sizes(h, M, N))) return s;
  if (N == 0) return RS_OK;
  if (!W || !aligned(W, 8)) return fail(h, RS_EINVAL, "W must be a non-NULL 8-byte aligned pointer");
  if (!out_idx || !aligned(out_idx, 4)) return fail(h, RS_EINVAL, "out_idx must be a non-NULL pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (M <= kSmallMaxM && N <= kSmallMaxN && !(o.debug & 5)) {
    // a small instance: the uniforms and the map on one CTA, W in shared
    // memory; the DaC leaves are one per thread unless opts->leaf_L is set
    const int G = N >= kSmallClusterN ? 4 : 1;
    const int L = o.leaf_L > 0 ? o.leaf_L : (int)((N + (long long)kSmallThreadsW * G - 1) / ((long long)kSmallThreadsW * G));
    RS_TRACE(h, "small_W", st);
    RS_CK(h, launch_small_W(o.prec == RS_F32_COMP, o.algo, W, M, N, seed, instance, L, out_idx, st, o.scheme,
                            static_cast<const LogTab*>(h->logtab), G));
    return RS_OK;
  }
  const Plan p = make_plan(0, N, false, true, true);
  if ((s = ensure_ws(h, p.bytes))) return s;
  if (N <= kUSmallMaxN && !(o.debug & 5)) {  // the sorted uniforms by one CTA, one launch
    RS_TRACE(h, "uniform_small", st);
    RS_CK(h, launch_uniform_small(o.prec == RS_F32_COMP, N + 1, seed, instance, at<void>(h, p.o_Z),
                                  at<double>(h, p.o_U), st, o.scheme));
  } else {
    if ((s = enqueue_clear(h, p, st))) return s;
    if ((s = enqueue_uniforms(h, p, o.prec == RS_F32_COMP, seed, instance, at<double>(h, p.o_U), o, st))) return s;
  }
  return enqueue_map(h, o, W, M, at<double>(h, p.o_U), N, out_idx, st);
}

rs_status rs_map(rs_handle* h, const double* W, int64_t M, const double* U, int64_t N, int32_t* out_idx,
                 const rs_opts* opts, void* stream) {
  rs_status s = check_handle(h);
  if (s) return s;
  Opts o;
  if ((s = read_opts(h, opts, &o, RS_F64))) return s;
  if ((s = check_sizes(h, M, N))) return s;
  if (N == 0) return RS_OK;
  if (!W || !aligned(W, 8) || !U || !aligned(U, 8)) return fail(h, RS_EINVAL, "W and U must be 8-byte aligned");
  if (!out_idx || !aligned(out_idx, 4)) return fail(h, RS_EINVAL, "out_idx must be a non-NULL pointer");
  return enqueue_map(h, o, W, M, U, N, out_idx, static_cast<cudaStream_t>(stream));
}

rs_status rs_softmax_weights(rs_handle* h, const double* logw, int64_t M, double* w_out, void* stream) {
  rs_status s = check_handle(h);
  if (s) return s;
  if (M < 1 || M > kMaxLen) return fail(h, RS_EINVAL, "M must satisfy 1 <= M < 2^31");
  if (!logw || !w_out || !aligned(logw, 8) || !aligned(w_out, 8))
    return fail(h, RS_EINVAL, "logw and w_out must be non-NULL 8-byte aligned device pointers");
  if ((s = ensure_ws(h, 256))) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RS_TRACE(h, "softmax", st);
  RS_CK(h, launch_softmax_weights(logw, M, w_out, at<unsigned long long>(h, 0), h->status, st));
  return RS_OK;
}

rs_status rs_resample_logw(rs_handle* h, const double* logw, int64_t M, int64_t N, uint64_t seed, uint64_t instance,
                           int32_t* out_idx, const rs_opts* opts, void* stream) {
  rs_status s = check_handle(h);
  if (s) return s;
  Opts o;
  if ((s = read_opts(h, opts, &o, RS_F64))) return s;
  if (o.prec != RS_F64) return fail(h, RS_EINVAL, "log-weights are binary64 (opts.prec must be RS_F64)");
  if ((s = check_sizes(h, M, N))) return s;
  if (!logw || !aligned(logw, 8)) return fail(h, RS_EINVAL, "logw must be a non-NULL 8-byte aligned pointer");
  if (N > 0 && (!out_idx || !aligned(out_idx, 4))) return fail(h, RS_EINVAL, "out_idx must be a non-NULL pointer");
  if (N == 0) return RS_OK;
  // the weights go to the end of the workspace, beyond the regions of the call
  const Plan p = make_plan(M, N, true, true, false, false);
  const size_t o_w = (p.bytes + 255) & ~size_t(255);
  const size_t o_key = o_w + (((size_t)M * 8 + 255) & ~size_t(255));
  if ((s = ensure_ws(h, o_key + 256))) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* w = at<double>(h, o_w);
  {
    RS_TRACE(h, "softmax", st);
    RS_CK(h, launch_softmax_weights(logw, M, w, at<unsigned long long>(h, o_key), h->status, st));
  }
  return rs_resample_w(h, w, M, N, seed, instance, out_idx, nullptr, opts, stream);
}

rs_status rs_gather(rs_handle* h, const void* x, int64_t M, int64_t row_bytes, const int32_t* idx, int64_t N,
                    void* x_out, void* stream) {
  rs_status s = check_handle(h);
  if (s) return s;
  if (M < 1 || M > kMaxLen) return fail(h, RS_EINVAL, "M must satisfy 1 <= M < 2^31");
  if (N < 0 || N > kMaxLen) return fail(h, RS_EINVAL, "N must satisfy 0 <= N < 2^31");
  if (row_bytes <= 0 || (row_bytes & 3)) return fail(h, RS_EINVAL, "row_bytes must be a positive multiple of 4");
  if (N == 0) return RS_OK;
  if (!x || !idx || !x_out || !aligned(x, 4) || !aligned(idx, 4) || !aligned(x_out, 4))
    return fail(h, RS_EINVAL, "x, idx and x_out must be non-NULL 4-byte aligned device pointers");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  RS_TRACE(h, "gather", st);
  RS_CK(h, launch_gather(x, M, row_bytes, idx, N, x_out, h->status, st));
  return RS_OK;
}

rs_status rs_resample_batched(rs_handle* h, const void* w, const int64_t* w_off, const int64_t* r_off, int32_t K,
                              const int64_t* h_w_off, const int64_t* h_r_off, uint64_t seed, int32_t* out_idx,
                              const rs_opts* opts, void* stream) {
  rs_status s = check_handle(h);
  if (s) return s;
  Opts o;
  if ((s = read_opts(h, opts, &o, RS_F32_COMP))) return s;
  if (K < 0) return fail(h, RS_EINVAL, "K must be >= 0");
  if (K == 0) return RS_OK;
  if (!w || !w_off || !r_off) return fail(h, RS_EINVAL, "w, w_off and r_off must be non-NULL");
  const bool f32 = o.prec == RS_F32_COMP;
  if (!aligned(w, f32 ? 4 : 8)) return fail(h, RS_EINVAL, "w must be aligned to its element size");
  if (!aligned(w_off, 8) || !aligned(r_off, 8)) return fail(h, RS_EINVAL, "w_off and r_off must be 8-byte aligned");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  std::vector<int64_t> wo, ro;
  if (h_w_off && h_r_off) {
    wo.assign(h_w_off, h_w_off + K + 1);
    ro.assign(h_r_off, h_r_off + K + 1);
  } else {
    wo.resize(K + 1);
    ro.resize(K + 1);
    RS_CK(h, cudaMemcpyAsync(wo.data(), w_off, (K + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RS_CK(h, cudaMemcpyAsync(ro.data(), r_off, (K + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    RS_CK(h, cudaStreamSynchronize(st));
  }
  if (wo[0] != 0 || ro[0] != 0) return fail(h, RS_EINVAL, "offsets must start at 0");
  for (int32_t k = 0; k < K; ++k) {
    const long long Mk = wo[k + 1] - wo[k], Nk = ro[k + 1] - ro[k];
    if (Mk < 0 || Nk < 0) return fail(h, RS_EINVAL, "offsets must be non-decreasing");
    if (Nk > 0 && Mk < 1) return fail(h, RS_EINVAL, "an instance with samples needs at least one weight");
    if (Mk > kMaxLen || Nk > kMaxLen) return fail(h, RS_EINVAL, "instance too large");
  }
  if (ro[K] > 0 && (!out_idx || !aligned(out_idx, 4))) return fail(h, RS_EINVAL, "out_idx must be a non-NULL pointer");
  const size_t esz = f32 ? 4 : 8;
  rs_opts one;
  memset(&one, 0, sizeof(one));
  one.prec = o.prec;
  one.spin_limit = o.spin;
  one.scheme = o.scheme;
  one.debug_flags = o.debug & 4;
  const bool per_instance = (o.debug & 4) != 0;  // comparison: every instance on its own
  // instances the persistent kernel does not take (more than kBMaxSeg
  // segments or kBMaxN samples): one single-instance call each
  for (int32_t k = 0; k < K; ++k) {
    const long long Mk = wo[k + 1] - wo[k], Nk = ro[k + 1] - ro[k];
    if (Nk == 0) continue;
    if (!per_instance && (Mk + kSegLen - 1) / kSegLen <= kBMaxSeg && Nk <= kBMaxN) continue;
    const void* wk = static_cast<const char*>(w) + (size_t)wo[k] * esz;
    if ((s = rs_resample_w(h, wk, Mk, Nk, seed, (uint64_t)k, out_idx + ro[k], nullptr, &one, stream))) return s;
  }
  if (per_instance) return RS_OK;
  const rs_tune_entry* tb = find_tune(h, "batched", f32, mn_bucket(wo[K], ro[K]));
  const int threads = o.threads ? o.threads : (tb ? tb->threads : 256);
  const int leaf = o.leaf_L ? o.leaf_L : (tb ? tb->leaf : kBatchedLeafDefault);
  Layout L;
  const size_t o_queue = L.take(256);
  const size_t o_order = L.take((size_t)K * sizeof(int));
  const size_t o_lp = L.take(batched_scratch_bytes(f32, threads, K, true));
  if ((s = ensure_ws(h, L.off))) return s;
  {
    RS_TRACE(h, "batched_order", st);
    RS_CK(h, cudaMemsetAsync(at<unsigned>(h, o_queue), 0, 256, st));
    RS_CK(h, launch_batched_order(reinterpret_cast<const long long*>(w_off), K, at<int>(h, o_order), st));
  }
  {
    RS_TRACE(h, "batched", st);
    RS_CK(h, launch_batched(f32, w, reinterpret_cast<const long long*>(w_off),
                            reinterpret_cast<const long long*>(r_off), at<int>(h, o_order), K, seed, 0ULL, 0, 0,
                            threads, leaf, out_idx, at<unsigned>(h, o_queue), h->status, st, o.scheme,
                            static_cast<const LogTab*>(h->logtab), at<unsigned long long>(h, o_lp)));
  }
  return RS_OK;
}

rs_status rs_autotune_map(rs_handle* h, const double* W, int64_t M, int64_t N, uint64_t seed, int32_t* out_idx,
                          rs_opts* best, void* stream) {
  rs_status s = check_handle(h);
  if (s) return s;
  if ((s = check_sizes(h, M, N))) return s;
  if (N == 0) return fail(h, RS_EINVAL, "N must be positive to tune the map");
  if (!W || !aligned(W, 8)) return fail(h, RS_EINVAL, "W must be a non-NULL 8-byte aligned pointer");
  if (!out_idx || !aligned(out_idx, 4)) return fail(h, RS_EINVAL, "out_idx must be a non-NULL pointer");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Opts o;
  const Plan p = make_plan(0, N, false, true, true);
  if ((s = ensure_ws(h, p.bytes))) return s;
  if ((s = enqueue_clear(h, p, st))) return s;
  if ((s = enqueue_uniforms(h, p, false, seed, 0, at<double>(h, p.o_U), o, st))) return s;
  const double* U = at<double>(h, p.o_U);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RS_CK(h, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(h, cudaGetLastError(), "cudaEventCreate");
  }
  float best_ms = -1.0f;
  int bl = 1;
  o.algo = RS_MAP_DAC;
  for (int L = 1; L <= 256 && !s; L *= 2) {
    o.leaf_L = L;
    if ((s = enqueue_map(h, o, W, M, U, N, out_idx, st))) break;
    cudaEventRecord(e0, st);
    for (int r = 0; r < 3 && !s; ++r) s = enqueue_map(h, o, W, M, U, N, out_idx, st);
    cudaEventRecord(e1, st);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess && !s) s = cuda_fail(h, e, "autotune timing");
    if (!s && (best_ms < 0.0f || ms < best_ms)) {
      best_ms = ms;
      bl = L;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) return s;
  set_tune(h, "map_dac", false, mn_bucket(M, N), 0, bl);
  if (best) {
    memset(best, 0, sizeof(*best));
    best->algo = RS_MAP_DAC;
    best->leaf_L = bl;
  }
  return RS_OK;
}

rs_status rs_autotune_batched(rs_handle* h, const void* w, const int64_t* w_off, const int64_t* r_off, int32_t K,
                              const int64_t* h_w_off, const int64_t* h_r_off, uint64_t seed, int32_t* out_idx,
                              const rs_opts* opts, rs_opts* best, void* stream) {
  rs_status s = check_handle(h);
  if (s) return s;
  Opts o;
  if ((s = read_opts(h, opts, &o, RS_F32_COMP))) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  static const int kThreadsC[3] = {128, 256, 512};
  static const int kLeafC[3] = {4, 16, 64};
  rs_opts c;
  memset(&c, 0, sizeof(c));
  c.prec = o.prec;
  c.scheme = o.scheme;
  c.spin_limit = opts ? opts->spin_limit : 0;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  RS_CK(h, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(h, cudaGetLastError(), "cudaEventCreate");
  }
  float best_ms = -1.0f;
  int bt = 256, bl = 4;
  for (int a = 0; a < 3 && !s; ++a) {
    for (int b = 0; b < 3 && !s; ++b) {
      c.tile_threads = kThreadsC[a];
      c.leaf_L = kLeafC[b];
      if ((s = rs_resample_batched(h, w, w_off, r_off, K, h_w_off, h_r_off, seed, out_idx, &c, stream))) break;
      cudaEventRecord(e0, st);
      for (int r = 0; r < 3 && !s; ++r)
        s = rs_resample_batched(h, w, w_off, r_off, K, h_w_off, h_r_off, seed, out_idx, &c, stream);
      cudaEventRecord(e1, st);
      cudaError_t e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess && !s) s = cuda_fail(h, e, "autotune timing");
      if (!s && (best_ms < 0.0f || ms < best_ms)) {
        best_ms = ms;
        bt = c.tile_threads;
        bl = c.leaf_L;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s) return s;
  {
    long long sM = 0, sN = 0;
    if (h_w_off && h_r_off) {
      sM = h_w_off[K];
      sN = h_r_off[K];
    } else {
      int64_t t[2] = {0, 0};
      RS_CK(h, cudaMemcpy(&t[0], w_off + K, sizeof(int64_t), cudaMemcpyDeviceToHost));
      RS_CK(h, cudaMemcpy(&t[1], r_off + K, sizeof(int64_t), cudaMemcpyDeviceToHost));
      sM = t[0];
      sN = t[1];
    }
    set_tune(h, "batched", o.prec == RS_F32_COMP, mn_bucket(sM, sN), bt, bl);
  }
  if (best) {
    memset(best, 0, sizeof(*best));
    best->prec = o.prec;
    best->tile_threads = bt;
    best->leaf_L = bl;
  }
  return RS_OK;
}

}  // extern "C"
