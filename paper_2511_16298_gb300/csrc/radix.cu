// Host side of the radix pass: occupancy-derived grid sizes and the
// cooperative launch.
#include <mutex>
#include <unordered_map>

#include "radix.cuh"

namespace tdgs {
namespace radix {

namespace {
std::mutex g_mu;
std::unordered_map<uint64_t, uint32_t> g_resident;  // (device, fn) -> SMs << 8 | occupancy
}  // namespace

// Occupancy of `k` per SM on the current device (cached per device and kernel).
int occupancy(const Kernel& k, int* sms_out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  const uint64_t key = (static_cast<uint64_t>(dev) << 48) ^ reinterpret_cast<uintptr_t>(k.fn);
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_resident.find(key);
  if (it == g_resident.end()) {
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(k.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(k.smem)) != cudaSuccess)
      return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k.fn, k.threads, k.smem) != cudaSuccess)
      return 0;
    it = g_resident.emplace(key, (static_cast<uint32_t>(sms) << 8) | static_cast<uint32_t>(occ)).first;
  }
  *sms_out = static_cast<int>(it->second >> 8);
  return static_cast<int>(it->second & 0xffu);
}

uint32_t resident_ctas(const Kernel& k, int ctas_per_sm) {
  int sms = 0;
  const int occ = occupancy(k, &sms);
  if (occ <= 0) return 0;
  const int want = ctas_per_sm > 0 ? ctas_per_sm : k.min_blocks;
  return static_cast<uint32_t>(sms * (want < occ ? want : occ));
}

uint32_t grid_for(const Kernel& k, uint32_t m, int ctas_per_sm) {
  const uint32_t resident = resident_ctas(k, ctas_per_sm);
  if (resident == 0) return 0;
  const uint64_t tile = static_cast<uint64_t>(k.threads) * k.items;
  const uint32_t need = static_cast<uint32_t>((static_cast<uint64_t>(m) + tile - 1) / tile);
  uint32_t g = need < resident ? need : resident;
  if (g > kMaxGrid) g = kMaxGrid;
  return g ? g : 1;
}

cudaError_t launch(const Kernel& k, uint32_t grid, const void* kin, const uint32_t* vin, void* kout,
                   uint32_t* vout, PassArgs a, uint32_t* scratch, cudaStream_t s) {
  if (a.m == 0) return cudaSuccess;
  if (grid == 0) return cudaErrorInvalidConfiguration;
  const uint32_t bins = 1u << k.bits;
  a.H = scratch;
  a.P = scratch + static_cast<size_t>(grid) * bins;
  a.tot = a.P + static_cast<size_t>(grid) * bins;
  void* args[] = {(void*)&kin, (void*)&vin, (void*)&kout, (void*)&vout, (void*)&a};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(k.threads);
  cfg.dynamicSmemBytes = k.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, k.fn, args);
}

}  // namespace radix
}  // namespace tdgs
