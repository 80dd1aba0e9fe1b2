// Systematic resampling for callers that cannot allocate device memory.
//
// ppl_resample needs a caller-supplied workspace.  Some callers have no way
// to provide one: a plugin inside a host application whose device memory is
// owned by that application's pool, or a real-time filtering loop where a
// cudaMalloc could block on device-wide synchronisation.  This variant keeps
// its scratch (scan status words, partial results, prefix sums) in one
// file-scope device array instead, sized for at most kNoAllocMaxParticles
// particles, and calls no allocator.
//
// Host code cannot hand the array's name to a kernel: on the host that name is
// a stand-in, not a device address.  The first call on each device therefore
// looks the address up with cudaGetSymbolAddress, with that device current,
// and caches it; that first call should happen before any stream capture.
// All calls on a device share the one array and it keeps the last call's
// contents, so the parts that must start at zero are cleared on every call,
// and two calls whose work overlaps on the GPU (two streams, or two host
// threads) race on it.
#include <mutex>

#include "kernels.h"

namespace ppl {
namespace {

constexpr int64_t kNoAllocMaxParticles = 1 << 20;
constexpr size_t kNoAllocHeader = 512;
constexpr size_t kNoAllocTiles = ((kNoAllocMaxParticles + kScanTile - 1) / kScanTile) * 8;
constexpr size_t kNoAllocPartials = 4096 * 256;  // >= partials_bytes(), checked at set-up
constexpr size_t kNoAllocPrefix = kNoAllocMaxParticles * 8;
constexpr size_t kNoAllocBounds = 2 * ((kNoAllocMaxParticles + 2047) / 2048) * 8;  // >= bounds count
constexpr size_t kNoAllocBytes =
    kNoAllocHeader + kNoAllocTiles + kNoAllocPartials + kNoAllocPrefix + kNoAllocBounds;

// About 9.4 MB per device, held from module load until the process exits.
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_addr[kMaxDevices] = {nullptr};

ppl_status scratch_for_current_device(char** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return PPL_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_addr[dev]) {
    if (partials_bytes() > kNoAllocPartials) return PPL_EINVAL;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return PPL_ECUDA;
    g_addr[dev] = p;
  }
  *out = static_cast<char*>(g_addr[dev]);
  return PPL_OK;
}

}  // namespace
}  // namespace ppl

using namespace ppl;

extern "C" ppl_status ppl_resample_noalloc(const float* lw, const uint64_t* q_fixed, int64_t n,
                                           int64_t m, uint64_t seed, uint32_t instance,
                                           uint32_t t, int32_t* ancestors, ppl_stream stream) {
  if ((lw == nullptr) == (q_fixed == nullptr)) return PPL_EINVAL;
  if (!ancestors || n < 1 || m < 1) return PPL_EINVAL;
  if (n > kNoAllocMaxParticles || m > kNoAllocMaxParticles) return PPL_EINVAL;  // beyond the static scratch
  if ((size_t)ancestor_bounds_count(m) * 8 > kNoAllocBounds) return PPL_EINVAL;
  char* base = nullptr;
  const ppl_status st = scratch_for_current_device(&base);
  if (st != PPL_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  WsHeader* hdr = reinterpret_cast<WsHeader*>(base);
  uint64_t* tiles = reinterpret_cast<uint64_t*>(base + kNoAllocHeader);
  void* parts = base + kNoAllocHeader + kNoAllocTiles;
  uint64_t* prefix =
      reinterpret_cast<uint64_t*>(base + kNoAllocHeader + kNoAllocTiles + kNoAllocPartials);
  // status, tickets, tile counter and this call's tile status words start at zero
  const size_t clear = kNoAllocHeader + (size_t)scan_tiles(n) * sizeof(uint64_t);
  if (cudaMemsetAsync(base, 0, clear, s) != cudaSuccess) return PPL_ECUDA;
  if (lw && launch_stats(lw, n, hdr, parts, nullptr, s) != cudaSuccess)
    return PPL_ECUDA;
  if (launch_resample_scan(lw, q_fixed, n, m, seed, instance, t, hdr, tiles, prefix, nullptr,
                           s) != cudaSuccess)
    return PPL_ECUDA;
  int64_t* bounds = reinterpret_cast<int64_t*>(base + kNoAllocHeader + kNoAllocTiles +
                                               kNoAllocPartials + kNoAllocPrefix);
  if (launch_ancestors(prefix, n, m, hdr, bounds, ancestors, nullptr, s) != cudaSuccess)
    return PPL_ECUDA;
  return PPL_OK;
}

// Device-side status of the last ppl_resample_noalloc issued on `stream`
// (synchronises the stream).
extern "C" ppl_status ppl_resample_noalloc_status(ppl_stream stream) {
  char* base = nullptr;
  const ppl_status st = scratch_for_current_device(&base);
  if (st != PPL_OK) return st;
  int32_t v = 0;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemcpyAsync(&v, base, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return PPL_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PPL_ECUDA;
  return (ppl_status)v;
}
