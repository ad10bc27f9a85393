// Stable LSD radix pass shared by every sort in the library (the Sorting
// step of Sec. II-A orders instances by tile, then by depth).
//
// One digit pass is one persistent, cooperatively launched kernel whose
// grid is the number of CTAs resident on the GPU (a multiple of the SM
// count).  CTA c owns one contiguous chunk of the input:
//   phase 1  histogram of the chunk's digits (keys read with an L2
//            evict-last policy so phase 3 finds most of them in L2);
//   barrier
//   phase 2  one warp per digit scans the chunk histograms over chunks
//            -> each chunk's exclusive prefix per digit, and digit totals;
//   barrier
//            every CTA scans the totals over digits; its running output
//            base per digit = digit start + chunk prefix;
//   phase 3  the chunk is processed tile by tile: warp-level match.any
//            ranking into per-warp shared counters, exchange through shared
//            memory into digit order, coalesced scatter at base + rank.
// Two bounded grid barriers replace a decoupled look-back, whose walk
// depth grows with the number of resident tiles when digits are wide.
//
// Template knobs: key type K (uint32/uint64), whether a uint32 value
// travels with the key, and "expand" (the last pass of the frame path: the
// key is a packed (tile, depth rank) element and the scatter writes the
// final 64-bit key and the Gaussian index instead).
#pragma once

#include "tdgs_internal.cuh"

namespace tdgs {
namespace radix {

constexpr uint32_t kNoDigit = 0xffffffffu;
constexpr uint32_t kMaxGrid = 512;  // chunks per pass (the column scan holds 16 per lane)

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t ld_hint(const uint64_t* a, uint64_t pol) {
  uint64_t v;
  asm volatile("ld.global.L2::cache_hint.u64 %0, [%1], %2;" : "=l"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ uint32_t ld_hint(const uint32_t* a, uint64_t pol) {
  uint32_t v;
  asm volatile("ld.global.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ uint32_t ld_acquire32(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release32(uint32_t* p, uint32_t v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Self-resetting grid barrier for a cooperatively launched grid (all CTAs
// resident).  bar[0] counts arrivals, bar[1] is the generation.  The wait is
// bounded: on timeout the error is latched and the CTA moves on (every
// scatter stays bounds-checked).
__device__ __forceinline__ void grid_barrier(uint32_t* bar, uint32_t* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t gen = ld_acquire32(bar + 1);
    __threadfence();
    const uint32_t arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      st_release32(bar + 1, gen + 1);
    } else {
      uint32_t spins = 0;
      while (ld_acquire32(bar + 1) == gen) {
        if (++spins > kSpinLimit) {
          latch_error(err, TDGS_ERR_TIMEOUT, kSiteBarrier);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
}

template <int kWarps>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t x = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t o = __shfl_up_sync(0xffffffffu, x, d);
    if (lane >= static_cast<uint32_t>(d)) x += o;
  }
  if (lane == 31) s_warp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    uint32_t w = lane < kWarps ? s_warp[lane] : 0;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= static_cast<uint32_t>(d)) w += o;
    }
    if (lane < kWarps) s_warp[lane] = w;
  }
  __syncthreads();
  const uint32_t r = x - v + (warp ? s_warp[warp - 1] : 0);
  __syncthreads();
  return r;
}

// Digit of a key.  With drop31 (64-bit keys only) bit 31 of every key is
// known to be zero and is squeezed out: (tile bits : depth bits 30..0).
template <typename K>
__device__ __forceinline__ uint32_t digit_of(K k, uint32_t shift, uint32_t mask, bool drop31) {
  if constexpr (sizeof(K) == 8) {
    const uint64_t e = drop31 ? ((k & 0x7fffffffull) | ((k >> 32) << 31)) : k;
    return static_cast<uint32_t>(e >> shift) & mask;
  } else {
    return (k >> shift) & mask;
  }
}

struct PassArgs {
  uint32_t m;
  uint32_t shift, mask;
  int drop31;
  uint64_t bad_mask;     // key bits that must be zero (checked in phase 1)
  uint32_t* H;           // [grid][bins] chunk histograms
  uint32_t* P;           // [grid][bins] chunk prefixes
  uint32_t* tot;         // [bins] digit totals
  uint32_t* bar;         // grid barrier words
  uint32_t* err;
  // expansion (frame path, last pass): element = (global tile << rbits) | rank
  uint32_t rbits;
  const uint32_t* sdepth;      // depth bits by rank
  const uint32_t* sorder;      // global record index by rank
  const uint32_t* vrec_begin;  // [nv+1] first record of each view
  const uint32_t* vtile_begin; // [nv+1] first global tile of each view
  uint32_t nv;
  uint32_t* rmin;              // per global tile: first sorted position (atomicMin)
  uint32_t* rmax;              // per global tile: one past the last (atomicMax)
  const uint64_t* m_dev;       // optional device element count, capped at m
};

template <typename K, bool kVals, bool kExpand, int kBits, int kThreads, int kItems>
struct PassShape {
  static constexpr int kBins = 1 << kBits;
  static constexpr int kWarps = kThreads / 32;
  static constexpr int kTileKeys = kThreads * kItems;
  static constexpr int kBpt = (kBins + kThreads - 1) / kThreads;
  static constexpr size_t kWhBytes = static_cast<size_t>(kWarps) * kBins * 2;
  static constexpr size_t kXBytes = static_cast<size_t>(kTileKeys) * sizeof(K);
  static constexpr size_t kUBytes = kWhBytes > kXBytes ? kWhBytes : kXBytes;
  static constexpr size_t kSmem = kUBytes + static_cast<size_t>(kBins) * 8;
  static constexpr int kMinBlocks = kThreads >= 512 ? 1 : ((sizeof(K) == 4 && !kVals) ? 3 : 2);
};

template <typename K, bool kVals, bool kExpand, int kBits, int kThreads, int kItems>
__global__ void __launch_bounds__(kThreads, (PassShape<K, kVals, kExpand, kBits, kThreads, kItems>::kMinBlocks))
    k_radix_pass(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                 void* __restrict__ kout_raw, uint32_t* __restrict__ vout, PassArgs a) {
  using S = PassShape<K, kVals, kExpand, kBits, kThreads, kItems>;
  constexpr int kBins = S::kBins;
  constexpr int kWarps = S::kWarps;
  constexpr int kTileKeys = S::kTileKeys;
  constexpr int kBpt = S::kBpt;
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t* wh = reinterpret_cast<uint16_t*>(smem);  // [kWarps][kBins] while ranking
  K* xk = reinterpret_cast<K*>(smem);                 // key exchange afterwards
  uint32_t* xv = reinterpret_cast<uint32_t*>(smem);   // value exchange afterwards
  uint32_t* base = reinterpret_cast<uint32_t*>(smem + S::kUBytes);  // running output base
  uint32_t* lstart = base + kBins;                                   // tile-local digit start
  __shared__ uint32_t s_warp[kWarps];
  __shared__ uint32_t s_vrec[kExpand ? kMaxViews + 1 : 1];
  __shared__ uint32_t s_vtile[kExpand ? kMaxViews + 1 : 1];

  const uint32_t t = threadIdx.x;
  const uint32_t lane = lane_id();
  const uint32_t warp = t >> 5;
  const bool d31 = a.drop31 != 0;
  uint32_t m = a.m;
  if (a.m_dev) {
    const uint64_t md = *a.m_dev;
    if (md > a.m && t == 0 && blockIdx.x == 0) latch_error(a.err, TDGS_ERR_CAPACITY, kSiteRadixCapacity);
    m = md < a.m ? static_cast<uint32_t>(md) : a.m;
  }
  const uint32_t G = gridDim.x;
  const uint32_t c = blockIdx.x;
  // chunks are multiples of 4 keys so that every chunk starts 16-byte aligned
  const uint64_t Sz = ((static_cast<uint64_t>(m) + G - 1) / G + 3) & ~3ull;
  const uint64_t b64 = c * Sz, e64 = c * Sz + Sz;
  const uint32_t beg = static_cast<uint32_t>(b64 < m ? b64 : m);
  const uint32_t end = static_cast<uint32_t>(e64 < m ? e64 : m);

  if constexpr (kExpand) {
    for (uint32_t v = t; v <= a.nv; v += kThreads) {
      s_vrec[v] = a.vrec_begin[v];
      s_vtile[v] = a.vtile_begin[v];
    }
  }
  // ---- phase 1: chunk histogram (lstart doubles as the counter array)
  for (uint32_t b = t; b < kBins; b += kThreads) lstart[b] = 0;
  __syncthreads();
  {
    const uint64_t keep = policy_evict_last();
    bool bad = false;
    constexpr int kU = 8;
    for (uint64_t i0 = beg + warp * 32 * kU; i0 < end; i0 += kThreads * kU) {
      K k8[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const uint64_t i = i0 + u * 32 + lane;
        k8[u] = i < end ? ld_hint(kin + i, keep) : K(0);
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const uint64_t i = i0 + u * 32 + lane;
        if (i < end) {
          bad |= (static_cast<uint64_t>(k8[u]) & a.bad_mask) != 0;
          atomicAdd(&lstart[digit_of<K>(k8[u], a.shift, a.mask, d31)], 1u);
        }
      }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) latch_error(a.err, TDGS_ERR_INVALID_ARGUMENT, kSiteRadixKeys);
  }
  __syncthreads();
  for (uint32_t b = t; b < kBins; b += kThreads) a.H[static_cast<size_t>(c) * kBins + b] = lstart[b];
  grid_barrier(a.bar, a.err);

  // ---- phase 2: column scans over chunks, one warp per digit
  // Lane l holds chunks l*kCol .. l*kCol+kCol-1 of one digit column; all
  // loads are issued before the scan so the column costs one L2 round trip.
  constexpr uint32_t kCol = kMaxGrid / 32;
  for (uint32_t b = c * kWarps + warp; b < static_cast<uint32_t>(kBins); b += G * kWarps) {
    uint32_t h[kCol];
#pragma unroll
    for (uint32_t q = 0; q < kCol; ++q) {
      const uint32_t cc = lane * kCol + q;
      h[q] = cc < G ? __ldcg(a.H + static_cast<size_t>(cc) * kBins + b) : 0u;
    }
    uint32_t sum = 0;
#pragma unroll
    for (uint32_t q = 0; q < kCol; ++q) sum += h[q];
    uint32_t x = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, x, d);
      if (lane >= static_cast<uint32_t>(d)) x += o;
    }
    uint32_t run = x - sum;
#pragma unroll
    for (uint32_t q = 0; q < kCol; ++q) {
      const uint32_t cc = lane * kCol + q;
      if (cc < G) a.P[static_cast<size_t>(cc) * kBins + b] = run;
      run += h[q];
    }
    if (lane == 31) a.tot[b] = x;
  }
  grid_barrier(a.bar, a.err);
  {
    uint32_t seg[kBpt];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kBpt; ++i) {
      const uint32_t b = t * kBpt + i;
      seg[i] = b < kBins ? __ldcg(a.tot + b) : 0;
      sum += seg[i];
    }
    uint32_t run = block_excl_scan<kWarps>(sum, s_warp);
#pragma unroll
    for (int i = 0; i < kBpt; ++i) {
      const uint32_t b = t * kBpt + i;
      if (b < kBins) base[b] = run + __ldcg(a.P + static_cast<size_t>(c) * kBins + b);
      run += seg[i];
    }
  }
  __syncthreads();

  // ---- phase 3: stable rank + scatter, tile by tile
  const uint64_t drop = policy_evict_first();
  bool out_of_range = false;
  for (uint64_t tb64 = beg; tb64 < end; tb64 += kTileKeys) {
    const uint32_t tb = static_cast<uint32_t>(tb64);
    const uint32_t valid = min(static_cast<uint32_t>(kTileKeys), end - tb);
    for (uint32_t i = t; i < kWarps * kBins / 2; i += kThreads) reinterpret_cast<uint32_t*>(wh)[i] = 0;
    K k[kItems];
    uint32_t v[kVals ? kItems : 1];
    uint32_t r[kItems];
    const uint32_t wbase = warp * 32 * kItems;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      const uint32_t idx = wbase + j * 32 + lane;
      k[j] = idx < valid ? ld_hint(kin + tb + idx, drop) : K(0);
      if constexpr (kVals) v[j] = idx < valid ? ld_hint(vin + tb + idx, drop) : 0u;
    }
    __syncthreads();
    // rank within the warp: the lowest lane of each equal-digit group reads
    // and bumps the warp's counter of that digit
    uint16_t* my_wh = wh + warp * kBins;
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      const uint32_t idx = wbase + j * 32 + lane;
      const uint32_t d = idx < valid ? digit_of<K>(k[j], a.shift, a.mask, d31) : kNoDigit;
      uint32_t peers;
      if constexpr (kBits <= 8) {
        // lanes with equal digits: AND of one ballot per digit bit
        peers = __ballot_sync(0xffffffffu, d != kNoDigit);
        if (d == kNoDigit) peers = ~peers;
#pragma unroll
        for (int bit = 0; bit < kBits; ++bit) {
          const uint32_t bal = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
          peers &= ((d >> bit) & 1u) ? bal : ~bal;
        }
      } else {
        peers = __match_any_sync(0xffffffffu, d);
      }
      const uint32_t leader = __ffs(peers) - 1;
      uint32_t before = 0;
      if (lane == leader && d != kNoDigit) before = my_wh[d];
      before = __shfl_sync(0xffffffffu, before, leader);
      if (lane == leader && d != kNoDigit) my_wh[d] = static_cast<uint16_t>(before + __popc(peers));
      r[j] = before + __popc(peers & lanemask_lt());
      __syncwarp();
    }
    __syncthreads();
    // exclusive prefix over warps per digit; tile count per digit
    uint32_t cnt[kBpt];
#pragma unroll
    for (int i = 0; i < kBpt; ++i) {
      const uint32_t b = t + i * kThreads;
      cnt[i] = 0;
      if (b < kBins) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
          const uint32_t x = wh[w * kBins + b];
          wh[w * kBins + b] = static_cast<uint16_t>(run);
          run += x;
        }
        cnt[i] = run;
        lstart[b] = run;
      }
    }
    __syncthreads();
    {
      uint32_t seg[kBpt];
      uint32_t sum = 0;
#pragma unroll
      for (int i = 0; i < kBpt; ++i) {
        const uint32_t b = t * kBpt + i;
        seg[i] = b < kBins ? lstart[b] : 0;
        sum += seg[i];
      }
      uint32_t run = block_excl_scan<kWarps>(sum, s_warp);
#pragma unroll
      for (int i = 0; i < kBpt; ++i) {
        const uint32_t b = t * kBpt + i;
        if (b < kBins) lstart[b] = run;
        run += seg[i];
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      const uint32_t idx = wbase + j * 32 + lane;
      if (idx < valid) {
        const uint32_t d = digit_of<K>(k[j], a.shift, a.mask, d31);
        r[j] += lstart[d] + my_wh[d];
      }
    }
    __syncthreads();  // wh is overwritten by the exchange below; lstart becomes the offset
#pragma unroll
    for (int i = 0; i < kBpt; ++i) {
      const uint32_t b = t + i * kThreads;
      if (b < kBins) lstart[b] = base[b] - lstart[b];
    }
#pragma unroll
    for (int j = 0; j < kItems; ++j)
      if (wbase + j * 32 + lane < valid) xk[r[j]] = k[j];
    __syncthreads();
    // Scatter in digit order.  A destination outside [0, m) can only come
    // from a timed-out barrier or keys changed underneath the sort: it is
    // dropped and reported instead of written.
    uint32_t dst[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const uint32_t p = i * kThreads + t;
      dst[i] = 0xffffffffu;
      if (p < valid) {
        const K key = xk[p];
        const uint32_t d = digit_of<K>(key, a.shift, a.mask, d31);
        dst[i] = lstart[d] + p;
        if (dst[i] < m) {
          if constexpr (kExpand) {
            const uint32_t rk = static_cast<uint32_t>(key & ((static_cast<K>(1) << a.rbits) - 1));
            const uint64_t gt = static_cast<uint64_t>(key >> a.rbits);
            const uint32_t gi = __ldg(a.sorder + rk);
            const uint32_t v = a.nv == 1 ? 0u : find_view(s_vrec, a.nv, gi);
            static_cast<uint64_t*>(kout_raw)[dst[i]] = ((gt - s_vtile[v]) << 32) | __ldg(a.sdepth + rk);
            vout[dst[i]] = gi - s_vrec[v];
            if (a.rmin) {  // first / last element of a tile run in this tile's exchange
              if (p == 0 || static_cast<uint64_t>(xk[p - 1] >> a.rbits) != gt)
                atomicMin(a.rmin + gt, dst[i]);
              if (p + 1 == valid || static_cast<uint64_t>(xk[p + 1] >> a.rbits) != gt)
                atomicMax(a.rmax + gt, dst[i] + 1);
            }
          } else {
            static_cast<K*>(kout_raw)[dst[i]] = key;
          }
        } else {
          out_of_range = true;
        }
      }
    }
    if constexpr (kVals) {
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kItems; ++j)
        if (wbase + j * 32 + lane < valid) xv[r[j]] = v[j];
      __syncthreads();
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        const uint32_t p = i * kThreads + t;
        if (p < valid && dst[i] < m) vout[dst[i]] = xv[p];
      }
    }
    __syncthreads();  // every scatter has read base[] before it moves on
#pragma unroll
    for (int i = 0; i < kBpt; ++i) {
      const uint32_t b = t + i * kThreads;
      if (b < kBins) base[b] += cnt[i];
    }
    __syncthreads();
  }
  if (out_of_range) latch_error(a.err, TDGS_ERR_CAPACITY, kSiteRadixRange);
}

// --------------------------------------------------------------- host side
using PassFn = void (*)(const void*, const uint32_t*, void*, uint32_t*, PassArgs);

struct Kernel {
  const void* fn;     // the __global__ function
  int bits, threads, items;
  size_t smem;
  int min_blocks;
};

template <typename K, bool kVals, bool kExpand, int kBits, int kThreads, int kItems>
Kernel make_kernel() {
  using S = PassShape<K, kVals, kExpand, kBits, kThreads, kItems>;
  return Kernel{reinterpret_cast<const void*>(&k_radix_pass<K, kVals, kExpand, kBits, kThreads, kItems>),
                kBits, kThreads, kItems, S::kSmem, S::kMinBlocks};
}

// Resident CTAs of `k` on the current device (0 on failure); caches the
// occupancy query per device and kernel.
uint32_t resident_ctas(const Kernel& k);

// Grid for m keys: every CTA gets at least one tile, at most all resident.
uint32_t grid_for(const Kernel& k, uint32_t m);

// Scratch words a pass with this kernel and grid needs.
inline size_t scratch_words(const Kernel& k, uint32_t grid) {
  return static_cast<size_t>(grid) * (1u << k.bits) * 2 + (1u << k.bits);
}

// Launch one pass (cooperative).  scratch: scratch_words() uint32 words.
cudaError_t launch(const Kernel& k, uint32_t grid, const void* kin, const uint32_t* vin, void* kout,
                   uint32_t* vout, PassArgs a, uint32_t* scratch, cudaStream_t s);

}  // namespace radix
}  // namespace tdgs
