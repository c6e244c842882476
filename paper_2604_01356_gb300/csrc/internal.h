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

// One record per tile of 8 segments (4096 weights), written by the tile
// prefix scan: P = sum of all earlier tiles as Pm * 2^Pe (128-bit mantissa),
// key = P truncated to binary64 (bit pattern), the search key.
constexpr int kSegsPerTile = 8;
struct TileRec {
  unsigned long long Pm_lo, Pm_hi;
  long long Pe;
  unsigned long long key;
};
static_assert(sizeof(TileRec) == 32, "TileRec layout");

// Search index over tile prefixes: level 0 holds the key of every tile, level
// l every 32^l-th one (non-negative binary64 values order like their
// unsigned bit patterns).  The top level has <= 32 entries.
constexpr int kMaxLevels = 8;
struct SegIndex {
  long long n;  // tiles
  int nlev;
  long long lvl_n[kMaxLevels];
  unsigned long long* lvl[kMaxLevels];
};

// Per-call constants (24-byte xf values: mantissa lo, hi, exponent):
// invZ = 1/Z_{N+1} (written by the spacing scan), S = total weight, invS = 1/S
// (only when W itself is written) and c = S / Z_{N+1} (written by the
// segment-prefix scan).
struct PathConsts {
  unsigned long long S[3];
  unsigned long long invS[3];
  unsigned long long c[3];
  unsigned long long invZ[3];
  unsigned long long pad[4];
};
static_assert(sizeof(PathConsts) == 128, "PathConsts layout");

// Search index over segment prefixes: level 0 holds the bit pattern of P_hi
// of every segment, level l every 32^l-th one (non-negative binary64 values
// order like their unsigned bit patterns).  The top level has <= 32 entries.
constexpr int kMaxLevels = 8;
struct SegIndex {
  long long nseg;
  int nlev;
  long long lvl_n[kMaxLevels];
  unsigned long long* lvl[kMaxLevels];
};

// Weights per segment (one warp, 16 per lane) and look-back descriptor size.
constexpr int kSegLen = 512;
constexpr int kTileDescBytes = 64;

int num_sms();

// --- uniforms (Algorithm 1) ---------------------------------------------
// Draw counts per tile of the spacing scan (256 threads x 1 draw).
constexpr int kUTile = 256;
cudaError_t init_log_table();
struct PathConsts;
cudaError_t launch_uniform_scan(bool f32, long long ndraw, unsigned long long seed, unsigned long long inst,
                                void* Z, void* Ztot, PathConsts* consts, void* desc, unsigned* ctr, int* status,
                                int spin_limit, cudaStream_t st);
cudaError_t launch_uniform_norm(long long N, const void* Z, const PathConsts* consts, double* U, cudaStream_t st);
cudaError_t launch_philox(unsigned long long seed, unsigned long long inst, unsigned long long first, long long n,
                          unsigned long long* out, cudaStream_t st);

// --- weights (Eq. 3) ------------------------------------------------------
// Tile aggregates of the reduce pass: one 24-byte value per 8 segments.
constexpr int kTileAggBytes = 24;
constexpr int kTilePrefixPerBlock = 4096;  // tiles per block of the tile-prefix scan
cudaError_t launch_w_reduce(bool f32, bool vec, const void* w, long long M, SegRec* seg, void* tagg, int* status,
                            cudaStream_t st);
cudaError_t launch_tile_prefix(bool f32, long long M, const void* tagg, TileRec* tiles, const SegIndex& idx,
                               void* desc, unsigned* ctr, PathConsts* consts, bool with_z, bool need_invS,
                               int* status, int spin_limit, bool withhold_first, cudaStream_t st);
cudaError_t launch_w_write(bool f32, bool vec, const void* w, long long M, const SegRec* seg, const TileRec* tiles,
                           const PathConsts* consts, double* W, cudaStream_t st);

// --- maps (Eq. 2; Algorithms 3, 4, 5) -------------------------------------
cudaError_t launch_map_seg(bool f32, bool vec, const void* w, long long M, const SegRec* seg, const TileRec* tiles,
                           const SegIndex& idx, const PathConsts* consts, const void* Z, long long N, int G, int* out,
                           cudaStream_t st);
cudaError_t launch_map_binary(const double* W, long long M, const double* U, long long N, int* out, cudaStream_t st);
cudaError_t launch_map_linear(const double* W, long long M, const double* U, long long N, int* out, cudaStream_t st);
cudaError_t launch_map_dac(const double* W, long long M, const double* U, long long N, int L, int stage_max, int* out,
                           cudaStream_t st);

}  // namespace gbr
