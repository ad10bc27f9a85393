// tdgs_scan_noalloc: the exclusive scan of tdgs_scan for callers that
// cannot allocate device memory -- for example code that runs while a CUDA
// graph is being captured, real-time loops that must never hit the device
// allocator (which can block or synchronise), or plugins whose device memory
// belongs to a host application.  Its scratch (look-back status words, the
// tile ticket and the error word) lives in one file-scope device array of
// fixed size instead of context-owned buffers.
#include <mutex>

#include "tdgs_internal.cuh"

namespace tdgs {
namespace {

constexpr uint32_t kNoAllocMaxItems = 1u << 24;                        // 16,777,216 counts
constexpr uint32_t kNoAllocTiles = kNoAllocMaxItems / kScanTileItems;  // 2,048 status words

struct NoAllocScratch {
  uint32_t ticket;                  // tile ticket, starts at 0 on every call
  uint32_t err[3];                  // latched error code and site
  uint64_t status[kNoAllocTiles];   // one look-back word per 8192-count tile
};

// Shared by every call on a device and kept between calls (about 16 KB per
// device, held until the process exits).
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Host code must not use g_noalloc_scratch as an address: the device
// address is looked up once per device with that device current.
std::mutex g_mu;
NoAllocScratch* g_addr[64] = {};

cudaError_t scratch_address(NoAllocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_addr[dev] = static_cast<NoAllocScratch*>(p);
  }
  *out = g_addr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace tdgs

using namespace tdgs;

extern "C" tdgs_status tdgs_scan_noalloc(const uint32_t* counts, uint32_t n, uint32_t* offsets,
                                         uint32_t* total_dev, uint32_t* error_dev, void* stream) {
  if (n > kNoAllocMaxItems) return TDGS_ERR_INVALID_ARGUMENT;
  if (n && (!counts || !offsets)) return TDGS_ERR_INVALID_ARGUMENT;
  auto misaligned = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 3u) != 0; };
  if (misaligned(counts) || misaligned(offsets) || misaligned(total_dev) || misaligned(error_dev))
    return TDGS_ERR_INVALID_ARGUMENT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  NoAllocScratch* sc = nullptr;
  if (scratch_address(&sc) != cudaSuccess) {
    cudaGetLastError();
    return TDGS_ERR_CUDA;
  }
  const uint32_t tiles = (n + kScanTileItems - 1) / kScanTileItems;
  // ticket, error word and the status words this call uses start at zero
  const size_t clear = offsetof(NoAllocScratch, status) + static_cast<size_t>(tiles) * sizeof(uint64_t);
  cudaError_t e = cudaMemsetAsync(sc, 0, clear, s);
  if (e == cudaSuccess && n == 0 && total_dev) e = cudaMemsetAsync(total_dev, 0, 4, s);
  if (e == cudaSuccess && n)
    e = launch_scan(counts, nullptr, nullptr, FrameGeom{}, n, offsets, sc->status, &sc->ticket, 0u,
                    nullptr, total_dev, sc->err, s);
  if (e == cudaSuccess && error_dev)
    e = cudaMemcpyAsync(error_dev, sc->err, 4, cudaMemcpyDeviceToDevice, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return TDGS_ERR_CUDA;
  }
  return TDGS_OK;
}
