// Per-frame kernels: tile count, exclusive scan, pair duplication and tile
// ranges (Sec. II-A "Duplication with Tiles"; Table III PrefixSum and
// DuplicateWithTile; Table VI Scan / Duplicate with tiles / Identify Range).
#include "tdgs_internal.cuh"

namespace tdgs {

// ------------------------------------------------------------ tile count
// One Gaussian per thread; one 128-bit load per record (Table IV packs the
// mean, depth and radius into one 16-byte record for exactly this read).
__global__ void __launch_bounds__(256) k_count_tiles(const float4* __restrict__ g, uint32_t n,
                                                     FrameGeom fg, uint32_t* __restrict__ counts,
                                                     uint32_t* err) {
  bool bad = false;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const TileRect q = tile_rect(__ldg(g + i), fg);
    bad |= q.invalid;
    counts[i] = q.count;
  }
  if (__any_sync(0xffffffffu, bad) && lane_id() == 0) latch_error(err, TDGS_ERR_INVALID_ARGUMENT, kSiteCount);
}

cudaError_t launch_count_tiles(const float4* g, uint32_t n, FrameGeom fg, uint32_t* counts,
                               uint32_t* err, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint32_t blocks = (n + 255) / 256;
  const uint32_t grid = blocks < 152u * 16u ? blocks : 152u * 16u;
  k_count_tiles<<<grid, 256, 0, s>>>(g, n, fg, counts, err);
  return cudaGetLastError();
}

// --------------------------------------------------------- exclusive scan
// Single-pass scan with decoupled look-back (Merrill & Garland, 2016).
// Each block takes the next tile of 8192 items from a ticket counter (so
// every predecessor tile is already running or done), publishes its
// aggregate, then walks back over its predecessors' status words 32 at a
// time until it meets an inclusive prefix.  Status word: bits 63-62 flag
// (1 = aggregate, 2 = inclusive prefix), bits 61-0 value.  Sums are 64-bit
// so that an overflow of the 32-bit offsets is detected, not wrapped.
namespace {
constexpr int kScanThreads = 256;
constexpr int kScanItems = kScanTileItems / kScanThreads;  // 32
constexpr uint64_t kFlagA = 1ull << 62;
constexpr uint64_t kFlagP = 2ull << 62;
constexpr uint64_t kValMask = (1ull << 62) - 1;

__host__ __device__ constexpr uint32_t spad(uint32_t p) { return p + (p >> 5); }

__device__ __forceinline__ uint64_t warp_incl_scan64(uint64_t v) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint64_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane_id() >= static_cast<uint32_t>(d)) v += o;
  }
  return v;
}
}  // namespace

// kMode 0: counts[i]; 1: counts computed from recs[i]; 2: counts[gather[i]].
template <int kMode>
__global__ void __launch_bounds__(kScanThreads)
    k_scan(const uint32_t* __restrict__ counts, const float4* __restrict__ recs,
           const uint32_t* __restrict__ gather, FrameGeom fg, uint32_t n,
           uint32_t* __restrict__ offsets, uint64_t* status, uint32_t* ticket,
           uint32_t ticket_base, uint64_t* total64, uint32_t* total32, uint32_t* err) {
  constexpr bool kFromRecords = kMode == 1;
  __shared__ uint32_t s_items[spad(kScanTileItems) + 1];
  __shared__ uint64_t s_warp[kScanThreads / 32];
  __shared__ uint64_t s_excl;
  __shared__ uint32_t s_tile;
  const uint32_t t = threadIdx.x;
  const uint32_t lane = lane_id();
  const uint32_t warp = t >> 5;
  if (t == 0) s_tile = atomicAdd(ticket, 1u) - ticket_base;
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint64_t base = static_cast<uint64_t>(tile) * kScanTileItems;

  // Coalesced (striped) load of the tile's counts, transposed through
  // shared memory to a blocked layout for the per-thread serial scan.
  bool bad = false;
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const uint32_t p = j * kScanThreads + t;
    const uint64_t idx = base + p;
    uint32_t v = 0;
    if (idx < n) {
      if constexpr (kMode == 1) {
        const TileRect q = tile_rect(__ldg(recs + idx), fg);
        bad |= q.invalid;
        v = q.count;
      } else if constexpr (kMode == 2) {
        v = __ldg(counts + __ldg(gather + idx));
      } else {
        v = __ldg(counts + idx);
      }
    }
    s_items[spad(p)] = v;
  }
  if (kFromRecords && __any_sync(0xffffffffu, bad) && lane == 0)
    latch_error(err, TDGS_ERR_INVALID_ARGUMENT, kSiteScan);
  __syncthreads();
  uint32_t mine[kScanItems];
  uint64_t tsum = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    mine[k] = s_items[spad(t * kScanItems + k)];
    tsum += mine[k];
  }
  const uint64_t winc = warp_incl_scan64(tsum);
  if (lane == 31) s_warp[warp] = winc;
  __syncthreads();
  if (warp == 0) {
    uint64_t w = lane < kScanThreads / 32 ? s_warp[lane] : 0;
    w = warp_incl_scan64(w);
    if (lane < kScanThreads / 32) s_warp[lane] = w;  // inclusive warp totals
  }
  __syncthreads();
  const uint64_t agg = s_warp[kScanThreads / 32 - 1];
  const uint64_t texcl = winc - tsum + (warp ? s_warp[warp - 1] : 0);

  // Look-back by warp 0.
  if (warp == 0) {
    uint64_t excl = 0;
    if (tile == 0) {
      if (lane == 0) st_release(status, kFlagP | (agg & kValMask));
    } else {
      if (lane == 0) st_release(status + tile, kFlagA | (agg & kValMask));
      int64_t k = static_cast<int64_t>(tile) - 1;
      uint32_t spins = 0;
      while (true) {
        const int64_t kk = k - lane;
        uint64_t s = kk >= 0 ? ld_acquire(status + kk) : kFlagP;
        while (__any_sync(0xffffffffu, (s >> 62) == 0)) {
          if (++spins > kSpinLimit) break;
          if ((s >> 62) == 0) {
            __nanosleep(32);
            s = ld_acquire(status + kk);
          }
        }
        if (spins > kSpinLimit) {
          if (lane == 0) latch_error(err, TDGS_ERR_TIMEOUT, kSiteScanTimeout);
          break;
        }
        const uint32_t pmask = __ballot_sync(0xffffffffu, (s >> 62) == 2);
        const uint32_t stop = pmask ? __ffs(pmask) - 1 : 31;
        uint64_t v = lane <= stop ? (s & kValMask) : 0;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(0xffffffffu, v, d);
        excl += v;
        if (pmask) break;
        k -= 32;
      }
      if (lane == 0) st_release(status + tile, kFlagP | ((excl + agg) & kValMask));
    }
    if (lane == 0) s_excl = excl;
  }
  __syncthreads();
  const uint64_t tile_excl = s_excl;
  const uint64_t incl_end = tile_excl + agg;
  if (incl_end > 0xffffffffull && t == 0) latch_error(err, TDGS_ERR_OVERFLOW, kSiteScan);
  uint64_t run = tile_excl + texcl;
#pragma unroll
  for (int k = 0; k < kScanItems; ++k) {
    s_items[spad(t * kScanItems + k)] = static_cast<uint32_t>(run);
    run += mine[k];
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kScanItems; ++j) {
    const uint32_t p = j * kScanThreads + t;
    const uint64_t idx = base + p;
    if (idx < n) offsets[idx] = s_items[spad(p)];
  }
  if (t == 0 && base + kScanTileItems >= n) {  // last tile writes the total
    if (total64) *total64 = incl_end;
    if (total32) *total32 = incl_end > 0xffffffffull ? 0xffffffffu : static_cast<uint32_t>(incl_end);
  }
}

cudaError_t launch_scan(const uint32_t* counts, const float4* recs, const uint32_t* gather,
                        FrameGeom fg, uint32_t n, uint32_t* offsets, uint64_t* status,
                        uint32_t* ticket, uint32_t ticket_base, uint64_t* total64,
                        uint32_t* total32, uint32_t* err, cudaStream_t s) {
  const uint32_t tiles = (n + kScanTileItems - 1) / kScanTileItems;
  if (tiles == 0) return cudaSuccess;
  if (recs)
    k_scan<1><<<tiles, kScanThreads, 0, s>>>(counts, recs, gather, fg, n, offsets, status, ticket,
                                             ticket_base, total64, total32, err);
  else if (gather)
    k_scan<2><<<tiles, kScanThreads, 0, s>>>(counts, recs, gather, fg, n, offsets, status, ticket,
                                             ticket_base, total64, total32, err);
  else
    k_scan<0><<<tiles, kScanThreads, 0, s>>>(counts, recs, gather, fg, n, offsets, status, ticket,
                                             ticket_base, total64, total32, err);
  return cudaGetLastError();
}

// ------------------------------------------------------------- duplicate
// Load-balanced expansion.  A warp owns 32 consecutive Gaussians; their
// pairs occupy one contiguous output range (their offsets are consecutive
// in the scan).  The warp walks that range 32 pairs at a time: lane l takes
// pair q = chunk + l, finds the owning Gaussian by a 5-step binary search
// over the lanes' start offsets (shuffles), and derives (ty, tx) from the
// local index (row-major within the Gaussian's tile rectangle).  Every
// store is a fully coalesced 256-byte (keys) / 128-byte (values) run.
// kNorm: the paper's 32-bit key (Sec. IV-B), tile << 10 | q with q the
// depth normalised to 2^10 over the visible range norm[0..1] (float bits):
// scale = 1024 / (dmax - dmin) (0 if equal), q = min(1023, floor((depth -
// dmin) * scale)), in float32 in this order.
template <bool kNorm>
__global__ void __launch_bounds__(256)
    k_duplicate(const float4* __restrict__ g, const uint32_t* __restrict__ offsets, uint32_t n,
                FrameGeom fg, void* __restrict__ keys_raw, uint32_t* __restrict__ values,
                uint32_t cap, const uint32_t* __restrict__ norm, uint32_t* err) {
  float dmin = 0.0f, scale = 0.0f;
  if constexpr (kNorm) {
    dmin = __uint_as_float(norm[0]);
    const float dmax = __uint_as_float(norm[1]);
    scale = dmax > dmin ? __fdiv_rn(1024.0f, __fsub_rn(dmax, dmin)) : 0.0f;
  }
  const uint32_t lane = lane_id();
  const uint32_t warps_total = (gridDim.x * blockDim.x) >> 5;
  bool bad = false, over = false;
  for (uint32_t wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
       static_cast<uint64_t>(wg) * 32u < n; wg += warps_total) {
    const uint32_t i = wg * 32u + lane;
    TileRect q;
    uint64_t start = 0;
    if (i < n) {
      q = tile_rect(__ldg(g + i), fg);
      start = __ldg(offsets + i);
      bad |= q.invalid;
    } else {
      q.x0 = q.y0 = q.x1 = q.y1 = 0;
      q.count = 0;
    }
    uint32_t depth_bits = i < n ? __float_as_uint(__ldg(&g[i].z)) : 0u;
    if constexpr (kNorm) {
      const float f = floorf(__fmul_rn(__fsub_rn(__uint_as_float(depth_bits), dmin), scale));
      depth_bits = f >= 1023.0f ? 1023u : static_cast<uint32_t>(f);
    }
    uint64_t end = start + q.count;
    // warp range [begin, end_max)
    uint64_t end_max = end;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, end_max, d);
      end_max = o > end_max ? o : end_max;
    }
    if (i >= n) start = end_max;  // never selected by the owner search
    const uint64_t begin = __shfl_sync(0xffffffffu, start, 0);
    const int32_t w = q.x1 - q.x0;
    for (uint64_t c = begin; c < end_max; c += 32) {
      const uint64_t p = c + lane;
      uint32_t lo = 0;
#pragma unroll
      for (uint32_t step = 16; step > 0; step >>= 1) {
        const uint64_t sc = __shfl_sync(0xffffffffu, start, lo + step);
        if (sc <= p) lo += step;
      }
      const uint64_t s0 = __shfl_sync(0xffffffffu, start, lo);
      const int32_t ow = __shfl_sync(0xffffffffu, w, lo);
      const int32_t ox0 = __shfl_sync(0xffffffffu, q.x0, lo);
      const int32_t oy0 = __shfl_sync(0xffffffffu, q.y0, lo);
      const uint32_t od = __shfl_sync(0xffffffffu, depth_bits, lo);
      if (p < end_max && ow > 0) {
        const uint32_t j = static_cast<uint32_t>(p - s0);
        const uint32_t ry = j / static_cast<uint32_t>(ow);
        const uint32_t rx = j - ry * static_cast<uint32_t>(ow);
        const uint64_t tile = static_cast<uint64_t>(oy0 + ry) * static_cast<uint64_t>(fg.gx) +
                              static_cast<uint64_t>(ox0 + rx);
        if (p < cap) {
          if constexpr (kNorm)
            static_cast<uint32_t*>(keys_raw)[p] = (static_cast<uint32_t>(tile) << 10) | od;
          else
            static_cast<uint64_t*>(keys_raw)[p] = (tile << 32) | od;
          values[p] = wg * 32u + lo;
        } else {
          over = true;
        }
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) latch_error(err, TDGS_ERR_INVALID_ARGUMENT, kSiteDuplicate);
  if (__any_sync(0xffffffffu, over) && lane == 0) latch_error(err, TDGS_ERR_CAPACITY, kSiteDuplicate);
}

cudaError_t launch_duplicate(const float4* g, const uint32_t* offsets, uint32_t n,
                             FrameGeom fg, uint64_t* keys, uint32_t* values, uint32_t cap,
                             uint32_t* err, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint32_t warps = (n + 31) / 32;
  const uint32_t blocks = (warps + 7) / 8;
  const uint32_t grid = blocks < 152u * 32u ? blocks : 152u * 32u;
  k_duplicate<false><<<grid, 256, 0, s>>>(g, offsets, n, fg, keys, values, cap, nullptr, err);
  return cudaGetLastError();
}

cudaError_t launch_duplicate_norm(const float4* g, const uint32_t* offsets, uint32_t n, FrameGeom fg,
                                  uint32_t* keys, uint32_t* values, uint32_t cap, const uint32_t* norm,
                                  uint32_t* err, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint32_t warps = (n + 31) / 32;
  const uint32_t blocks = (warps + 7) / 8;
  const uint32_t grid = blocks < 152u * 32u ? blocks : 152u * 32u;
  k_duplicate<true><<<grid, 256, 0, s>>>(g, offsets, n, fg, keys, values, cap, norm, err);
  return cudaGetLastError();
}

// Smallest and largest depth (float bits; positive finite depths order as
// unsigned integers) of the Gaussians with pairs: norm[0] min, norm[1] max
// (all ones / zero on entry).
__global__ void __launch_bounds__(256) k_norm_range(const float4* __restrict__ g, const uint32_t* __restrict__ counts,
                                                    uint32_t n, uint32_t* norm) {
  uint32_t lo = 0xffffffffu, hi = 0u;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (__ldg(counts + i)) {
      const uint32_t b = __float_as_uint(__ldg(&g[i].z));
      lo = min(lo, b);
      hi = max(hi, b);
    }
  }
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if (lane_id() == 0) {
    if (lo != 0xffffffffu) atomicMin(norm, lo);
    if (hi != 0u) atomicMax(norm + 1, hi);
  }
}

cudaError_t launch_norm_range(const float4* g, const uint32_t* counts, uint32_t n, uint32_t* norm, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const uint32_t blocks = (n + 255) / 256;
  const uint32_t grid = blocks < 152u * 8u ? blocks : 152u * 8u;
  k_norm_range<<<grid, 256, 0, s>>>(g, counts, n, norm);
  return cudaGetLastError();
}

// ---------------------------------------------------------- tile ranges
// Identify Range: a tile's range starts where its id differs from the
// previous key's and ends where it differs from the next key's.  ranges is
// zeroed beforehand, so tiles without pairs stay {0, 0}.
// K, kShift: 64-bit keys with the tile above bit 32, or the 32-bit
// normalised keys with the tile above bit 10.
template <typename K, int kShift>
__global__ void __launch_bounds__(256) k_tile_ranges(const K* __restrict__ keys, uint32_t m,
                                                     uint32_t num_tiles, uint2* ranges,
                                                     uint32_t* err) {
  bool bad = false;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < m; k += gridDim.x * blockDim.x) {
    const uint64_t t = static_cast<uint64_t>(__ldg(keys + k)) >> kShift;
    if (t >= num_tiles) {
      bad = true;
      continue;
    }
    const uint64_t prev = k > 0 ? (static_cast<uint64_t>(__ldg(keys + k - 1)) >> kShift) : ~0ull;
    const uint64_t next = k + 1 < m ? (static_cast<uint64_t>(__ldg(keys + k + 1)) >> kShift) : ~0ull;
    if (t != prev) ranges[t].x = k;
    if (t != next) ranges[t].y = k + 1;
  }
  if (__any_sync(0xffffffffu, bad) && lane_id() == 0) latch_error(err, TDGS_ERR_INVALID_ARGUMENT, kSiteRanges);
}

cudaError_t launch_tile_ranges(const uint64_t* keys, uint32_t m, uint32_t num_tiles,
                               uint2* ranges, uint32_t* err, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  const uint32_t blocks = (m + 255) / 256;
  const uint32_t grid = blocks < 152u * 16u ? blocks : 152u * 16u;
  k_tile_ranges<uint64_t, 32><<<grid, 256, 0, s>>>(keys, m, num_tiles, ranges, err);
  return cudaGetLastError();
}

cudaError_t launch_tile_ranges_norm(const uint32_t* keys, uint32_t m, uint32_t num_tiles, uint2* ranges,
                                    uint32_t* err, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  const uint32_t blocks = (m + 255) / 256;
  const uint32_t grid = blocks < 152u * 16u ? blocks : 152u * 16u;
  k_tile_ranges<uint32_t, 10><<<grid, 256, 0, s>>>(keys, m, num_tiles, ranges, err);
  return cudaGetLastError();
}

}  // namespace tdgs
