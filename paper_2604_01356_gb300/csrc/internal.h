// Internal interface between the host C-ABI layer (api.cu) and the kernel
// translation units.  Not installed; not part of the public ABI.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace gbr {

// One record per 512-element weight segment, written by the first weights
// pass.  The segment's elements are the integers F_j of the segment's
// fixed-point grid (unit 2^(E - bias - shift) of the weight type); P is the
// exclusive prefix (sum of all earlier segments) as a binary64 pair.
struct SegRec {
  double P_hi, P_lo;
  unsigned long long F;  // exact segment sum on the fixed-point grid
  int E;                 // shared exponent of the segment
  int len;               // valid elements (512 except the last segment)
};
static_assert(sizeof(SegRec) == 32, "SegRec layout");

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
constexpr int kTileDescBytes = 48;

int num_sms();

// --- uniforms (Algorithm 1) ---------------------------------------------
// Draw counts per tile of the spacing scan.
constexpr int kUTile = 4096;
cudaError_t init_log_table();
cudaError_t launch_uniform_scan(bool f32, long long ndraw, unsigned long long seed, unsigned long long inst,
                                void* Z, void* Ztot, void* desc, unsigned* ctr, int* status, int spin_limit,
                                cudaStream_t st);
cudaError_t launch_uniform_norm(bool f32, long long N, const void* Z, const void* Ztot, double* U, cudaStream_t st);
cudaError_t launch_philox(unsigned long long seed, unsigned long long inst, unsigned long long first, long long n,
                          unsigned long long* out, cudaStream_t st);

// --- weights (Eq. 3) ------------------------------------------------------
constexpr int kWTile = 4096;  // weights per look-back tile (8 segments)
cudaError_t launch_w_pass1(bool f32, bool vec, const void* w, long long M, SegRec* seg, const SegIndex& idx,
                           void* desc, unsigned* ctr, void* total, int* status, int spin_limit, bool withhold_first,
                           cudaStream_t st);
cudaError_t launch_w_write(bool f32, bool vec, const void* w, long long M, const SegRec* seg, const void* total,
                           double* W, int* status, cudaStream_t st);

// --- maps (Eq. 2; Algorithms 3, 4, 5) -------------------------------------
cudaError_t launch_map_seg(bool f32, bool vec, const void* w, long long M, const SegRec* seg, const SegIndex& idx,
                           const void* total, const double* U, long long N, int G, int* out, cudaStream_t st);
cudaError_t launch_map_binary(const double* W, long long M, const double* U, long long N, int* out, cudaStream_t st);
cudaError_t launch_map_linear(const double* W, long long M, const double* U, long long N, int* out, cudaStream_t st);
cudaError_t launch_map_dac(const double* W, long long M, const double* U, long long N, int L, int stage_max, int* out,
                           cudaStream_t st);

}  // namespace gbr
