// tdgs_scan_noalloc: the exclusive scan of tdgs_scan for callers that
// cannot allocate device memory -- real-time loops that must never reach
// the device allocator (an allocation can block or synchronise the
// device), or plugins whose device memory belongs to a host application
// that does not let them allocate.  Its scratch (look-back status words,
// the tile ticket and the error word) lives in one file-scope device array
// of fixed size instead of context-owned buffers.
#include <cuda.h>

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

// Shared by every call in a context and kept between calls (about 16 KB
// per device, held until the process exits).
static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Host code must not use g_noalloc_scratch as an address: in host code the
// name is a host-side stand-in.  The device address belongs to the CUDA
// context that loaded the module, so it is looked up with cudaGetSymbolAddress
// in the current context and cached by that context's unique id (a context
// made current by a host application, or one created after
// cudaDeviceReset, gets its own lookup).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);

struct DriverFns {
  CtxGetCurrentFn get_current = nullptr;
  CtxGetIdFn get_id = nullptr;
};

const DriverFns& driver_fns() {
  static const DriverFns fns = [] {
    DriverFns f;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f.get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      f.get_id = reinterpret_cast<CtxGetIdFn>(p);
    cudaGetLastError();
    return f;
  }();
  return fns;
}

// The unique id of the current context, or 0 if there is none or it
// cannot be read.
unsigned long long current_context_id() {
  const DriverFns& f = driver_fns();
  if (!f.get_current || !f.get_id) return 0;
  CUcontext c = nullptr;
  if (f.get_current(&c) != CUDA_SUCCESS || !c) return 0;
  unsigned long long id = 0;
  if (f.get_id(c, &id) != CUDA_SUCCESS) return 0;
  return id;
}

struct CacheEntry {
  unsigned long long ctx_id;
  NoAllocScratch* addr;
};
constexpr int kCacheEntries = 64;
std::mutex g_mu;
CacheEntry g_cache[kCacheEntries] = {};
int g_cache_next = 0;

cudaError_t scratch_address(NoAllocScratch** out) {
  const unsigned long long id = current_context_id();
  std::lock_guard<std::mutex> lock(g_mu);
  if (id) {
    for (const CacheEntry& c : g_cache)
      if (c.ctx_id == id) {
        *out = c.addr;
        return cudaSuccess;
      }
  }
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  *out = static_cast<NoAllocScratch*>(p);
  // The lookup may have made the device's primary context current; cache
  // under the id of the context the address was taken in.
  const unsigned long long id_after = id ? id : current_context_id();
  if (id_after) {
    g_cache[g_cache_next] = CacheEntry{id_after, *out};
    g_cache_next = (g_cache_next + 1) % kCacheEntries;
  }
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
