// rs_sorted_uniform_static: the sorted uniforms of Algorithm 1 computed with
// a fixed scratch array instead of a handle's workspace, so that the call
// allocates nothing.  It launches the same spacing-scan and normalisation
// kernels as rs_sorted_uniform; only where their scratch lives differs.
#include <mutex>

#include "../../include/gbresample.h"
#include "internal.h"

namespace gbr {
namespace {

constexpr long long kStaticMaxN = RS_STATIC_MAX_N;
constexpr long long kStaticTiles = (kStaticMaxN + 1 + kUTile - 1) / kUTile;  // look-back tiles for N+1 draws
constexpr int kStaticSpin = 1 << 22;  // polls before a look-back wait gives up (the library default)

// Scratch layout (bytes from the array's start, every region 256-aligned):
//   [0]        tile counter of the scan (cleared by every call)
//   [64]       status word used when the caller passes none
//   [256]      look-back descriptors, 64 B per tile (cleared by every call)
//   kOffConsts per-call constants (1/Z_{N+1})
//   kOffZtot   Z_{N+1}
//   kOffZ      Z_1 .. Z_N, 16 B each
constexpr size_t kOffCtr = 0;
constexpr size_t kOffStatus = 64;
constexpr size_t kOffDesc = 256;
constexpr size_t kRound(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kOffConsts = kRound(kOffDesc + (size_t)kStaticTiles * kTileDescBytes);
constexpr size_t kOffZtot = kRound(kOffConsts + sizeof(PathConsts));
constexpr size_t kOffZ = kRound(kOffZtot + 16);
constexpr size_t kScratchBytes = kRound(kOffZ + (size_t)kStaticMaxN * 16);

static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
unsigned char* g_scratch_ptr[kMaxDevices] = {nullptr};

// Once per device, with that device current: the scratch array's device
// address and the logarithm table of the spacing kernel.
rs_status scratch_for_current_device(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return RS_ECUDA;
  if (dev < 0 || dev >= kMaxDevices) return RS_ECAPACITY;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || !p) return RS_ECUDA;
    if (init_log_table() != cudaSuccess) return RS_ECUDA;
    g_scratch_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_scratch_ptr[dev];
  return RS_OK;
}

}  // namespace
}  // namespace gbr

extern "C" rs_status rs_sorted_uniform_static(int64_t N, uint64_t seed, uint64_t instance, int32_t precision,
                                              double* U_out, int32_t* status, void* stream) {
  using namespace gbr;
  if (N < 0) return RS_EINVAL;
  if (N > kStaticMaxN) return RS_ECAPACITY;
  if (precision != RS_F64 && precision != RS_F32_COMP) return RS_EINVAL;
  if (N == 0) return RS_OK;
  if (!U_out || (reinterpret_cast<uintptr_t>(U_out) % 8) != 0) return RS_EINVAL;
  if (status && (reinterpret_cast<uintptr_t>(status) % 4) != 0) return RS_EINVAL;
  unsigned char* base = nullptr;
  const rs_status s = scratch_for_current_device(&base);
  if (s != RS_OK) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const long long ndraw = N + 1;
  const long long tiles = (ndraw + kUTile - 1) / kUTile;
  unsigned* ctr = reinterpret_cast<unsigned*>(base + kOffCtr);
  int* st_word = status ? reinterpret_cast<int*>(status) : reinterpret_cast<int*>(base + kOffStatus);
  PathConsts* consts = reinterpret_cast<PathConsts*>(base + kOffConsts);
  // the counter and this call's descriptors must start at zero
  if (cudaMemsetAsync(base, 0, kOffDesc + (size_t)tiles * kTileDescBytes, st) != cudaSuccess) return RS_ECUDA;
  if (launch_uniform_scan(precision == RS_F32_COMP, ndraw, seed, instance, base + kOffZ, base + kOffZtot, consts,
                          base + kOffDesc, ctr, st_word, kStaticSpin, false, st) != cudaSuccess)
    return RS_ECUDA;
  if (launch_uniform_norm(N, base + kOffZ, consts, U_out, st) != cudaSuccess) return RS_ECUDA;
  return RS_OK;
}
