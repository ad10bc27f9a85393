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

// Chunk of the input owned by this CTA (chunks are multiples of 4 keys so
// every chunk starts 16-byte aligned); m may come from device memory.
struct Chunk {
  uint32_t m, beg, end;
};
__device__ __forceinline__ Chunk chunk_of(const PassArgs& a) {
  Chunk ch;
  ch.m = a.m;
  if (a.m_dev) {
    const uint64_t md = *a.m_dev;
    if (md > a.m && threadIdx.x == 0 && blockIdx.x == 0)
      latch_error(a.err, TDGS_ERR_CAPACITY, kSiteRadixCapacity);
    ch.m = md < a.m ? static_cast<uint32_t>(md) : a.m;
  }
  const uint32_t G = gridDim.x;
  const uint64_t Sz = ((static_cast<uint64_t>(ch.m) + G - 1) / G + 3) & ~3ull;
  const uint64_t b64 = blockIdx.x * Sz, e64 = blockIdx.x * Sz + Sz;
  ch.beg = static_cast<uint32_t>(b64 < ch.m ? b64 : ch.m);
  ch.end = static_cast<uint32_t>(e64 < ch.m ? e64 : ch.m);
  return ch;
}

// Phases 1-2: histogram of this chunk's digits, column scans over chunks
// between two grid barriers, then base[b] = first output position of this
// chunk's keys with digit b.  hist: kBins words of shared scratch.
template <typename K, int kBins, int kThreads>
__device__ __forceinline__ void chunk_bases(const K* __restrict__ kin, const PassArgs& a,
                                            uint32_t beg, uint32_t end, bool d31, uint32_t* base,
                                            uint32_t* hist, uint32_t* s_warp) {
  constexpr int kWarps = kThreads / 32;
  constexpr int kBpt = (kBins + kThreads - 1) / kThreads;
  const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;
  const uint32_t G = gridDim.x, c = blockIdx.x;
  for (uint32_t b = t; b < kBins; b += kThreads) hist[b] = 0;
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
          atomicAdd(&hist[digit_of<K>(k8[u], a.shift, a.mask, d31)], 1u);
        }
      }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) latch_error(a.err, TDGS_ERR_INVALID_ARGUMENT, kSiteRadixKeys);
  }
  __syncthreads();
  for (uint32_t b = t; b < kBins; b += kThreads) a.H[static_cast<size_t>(c) * kBins + b] = hist[b];
  grid_barrier(a.bar, a.err);
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
  __syncthreads();
}

// Output of one key at its sorted position dst.  Plain passes store the
// key; the expanding pass stores (local tile << 32 | depth bits) and the
// view-local Gaussian index, and records the first/last position of each
// global tile run seen in this tile's exchange buffer xk.
template <typename K, bool kExpand>
__device__ __forceinline__ void emit_key(const PassArgs& a, K key, uint32_t dst, const K* xk,
                                         uint32_t p, uint32_t valid, const uint32_t* s_vrec,
                                         const uint32_t* s_vtile, void* kout_raw, uint32_t* vout) {
  if constexpr (kExpand) {
    const uint32_t rk = static_cast<uint32_t>(key & ((static_cast<K>(1) << a.rbits) - 1));
    const uint64_t gt = static_cast<uint64_t>(key >> a.rbits);
    const uint32_t gi = __ldg(a.sorder + rk);
    const uint32_t v = a.nv == 1 ? 0u : find_view(s_vrec, a.nv, gi);
    static_cast<uint64_t*>(kout_raw)[dst] = ((gt - s_vtile[v]) << 32) | __ldg(a.sdepth + rk);
    vout[dst] = gi - s_vrec[v];
    if (a.rmin) {
      if (p == 0 || static_cast<uint64_t>(xk[p - 1] >> a.rbits) != gt) atomicMin(a.rmin + gt, dst);
      if (p + 1 == valid || static_cast<uint64_t>(xk[p + 1] >> a.rbits) != gt) atomicMax(a.rmax + gt, dst + 1);
    }
  } else {
    static_cast<K*>(kout_raw)[dst] = key;
  }
}

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
  const Chunk ch = chunk_of(a);
  const uint32_t m = ch.m, beg = ch.beg, end = ch.end;
  if constexpr (kExpand) {
    for (uint32_t v = t; v <= a.nv; v += kThreads) {
      s_vrec[v] = a.vrec_begin[v];
      s_vtile[v] = a.vtile_begin[v];
    }
  }
  chunk_bases<K, kBins, kThreads>(kin, a, beg, end, d31, base, lstart, s_warp);
  // bins and bits this pass's digit actually uses (<= kBins, kBits)
  const uint32_t nb = a.mask + 1 < static_cast<uint32_t>(kBins) ? a.mask + 1 : static_cast<uint32_t>(kBins);
  const int nbits = 32 - __clz(nb - 1);

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
        // lanes with equal digits: AND of one ballot per digit bit (only
        // the bits this pass's digit actually has)
        peers = __ballot_sync(0xffffffffu, d != kNoDigit);
        if (d == kNoDigit) peers = ~peers;
#pragma unroll
        for (int bit = 0; bit < kBits; ++bit) {
          if (bit < nbits) {
            const uint32_t bal = __ballot_sync(0xffffffffu, (d >> bit) & 1u);
            peers &= ((d >> bit) & 1u) ? bal : ~bal;
          }
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
      if (b < nb) {
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
          emit_key<K, kExpand>(a, key, dst[i], xk, p, valid, s_vrec, s_vtile, kout_raw, vout);
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

// ------------------------------------------------- bulk copies (TMA)
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// One thread: expect `bytes` on `bar`, then copy them global -> shared.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar,
                                          uint64_t policy) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}
// Wait for phase `parity` of `bar`, bounded; returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t spin = 0; spin < kSpinLimit; ++spin) {
    uint32_t ok;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(ok) : "r"(smem_u32(bar)), "r"(parity) : "memory");
    if (ok) return true;
  }
  return false;
}

// ------------------------------------------------ counter-table ranking
// Keys-only pass for digits of at most 6 bits (the tile passes of the fused
// frame).  Thread t owns 16 consecutive keys of a 4096-key tile (blocked,
// loaded as 16-byte vectors).  Ranking needs no cross-lane operation:
//   1. every thread bumps its own column of a [64 digits][256 threads]
//      counter table (the count before the bump is the key's rank among
//      its own earlier keys with that digit);
//   2. one exclusive scan over the table in digit-major, thread-minor order
//      turns each counter into "keys of the tile with a smaller digit, plus
//      keys with this digit in earlier threads";
//   3. rank = scanned counter + own-column rank: the stable position of
//      the key in the tile sorted by digit.
// The table is padded (row stride 260 words, quarter-row stride 65) so the
// bumps and the per-thread scan segments hit distinct banks.
namespace ct {
constexpr int kThreads = 256, kItems = 16, kBins = 64, kTileKeys = kThreads * kItems;
constexpr int kRow = 260, kQuarter = 65;
constexpr size_t kTableWords = static_cast<size_t>(kBins) * kRow;
constexpr size_t kTableBytes = kTableWords * 4;       // 66,560 B
constexpr int kRing = 4;                               // phase-1 copy blocks in flight
constexpr uint32_t kBlockBytes = 16384;                // bytes per phase-1 block
// layout: table | stage (one tile of keys) | base, off | 5 mbarriers
template <typename K>
__host__ __device__ constexpr size_t stage_bytes() { return static_cast<size_t>(kTileKeys) * sizeof(K); }
template <typename K>
__host__ __device__ constexpr size_t smem_bytes() { return kTableBytes + stage_bytes<K>() + kBins * 8 + 64; }
__device__ __forceinline__ uint32_t cell(uint32_t d, uint32_t t) {
  return d * kRow + (t >> 6) * kQuarter + (t & 63);
}
}  // namespace ct

__device__ __forceinline__ uint4 ld_hint_v4(const void* a, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(a), "l"(pol));
  return v;
}

// Keys are fetched with bulk copies into shared memory: in phase 1 the
// chunk streams through a ring of kRing 16 KB blocks held in the (not yet
// used) counter table; in phase 3 the next tile is copied into the stage
// buffer while the current one (already in registers) is ranked and
// scattered.  A copy may read up to 15 bytes past the last key: every
// buffer this kernel reads carries 16 bytes of slack.  Waits are bounded.
template <typename K, bool kExpand>
__global__ void __launch_bounds__(ct::kThreads, 2)
    k_radix_pass_ct(const K* __restrict__ kin, const uint32_t* __restrict__ vin_unused,
                    void* __restrict__ kout_raw, uint32_t* __restrict__ vout, PassArgs a) {
  using namespace ct;
  extern __shared__ __align__(128) unsigned char smem[];
  uint32_t* C = reinterpret_cast<uint32_t*>(smem);  // counter table, then the key exchange
  K* xk = reinterpret_cast<K*>(smem);
  K* stage = reinterpret_cast<K*>(smem + kTableBytes);
  uint32_t* base = reinterpret_cast<uint32_t*>(smem + kTableBytes + stage_bytes<K>());
  uint32_t* off = base + kBins;  // phase-1 histogram, then base - tile-local start
  uint64_t* mbar = reinterpret_cast<uint64_t*>(off + kBins);  // [0..kRing-1] ring, [kRing] stage
  __shared__ uint32_t s_warp[kThreads / 32];
  __shared__ uint32_t s_vrec[kExpand ? kMaxViews + 1 : 1];
  __shared__ uint32_t s_vtile[kExpand ? kMaxViews + 1 : 1];
  const uint32_t t = threadIdx.x;
  const Chunk ch = chunk_of(a);
  const uint32_t m = ch.m, beg = ch.beg, end = ch.end;
  if (t == 0) {
    for (int i = 0; i <= kRing; ++i) mbar_init(mbar + i, 1);
    fence_mbar_init();
  }
  if constexpr (kExpand) {
    for (uint32_t v = t; v <= a.nv; v += kThreads) {
      s_vrec[v] = a.vrec_begin[v];
      s_vtile[v] = a.vtile_begin[v];
    }
  }
  for (uint32_t b = t; b < kBins; b += kThreads) off[b] = 0;
  __syncthreads();
  const uint64_t keep = policy_evict_last();
  const uint64_t drop = policy_evict_first();
  bool timed_out = false;

  // ---- phase 1: histogram, keys streamed through the ring
  {
    constexpr uint32_t kPerBlock = kBlockBytes / sizeof(K);
    const uint32_t nblk = (end - beg + kPerBlock - 1) / kPerBlock;
    unsigned char* ring = smem;  // kRing * kBlockBytes <= kTableBytes
    auto issue = [&](uint32_t blk) {
      const uint32_t kb = beg + blk * kPerBlock;
      const uint32_t cnt = min(kPerBlock, end - kb);
      const uint32_t bytes = (cnt * static_cast<uint32_t>(sizeof(K)) + 15u) & ~15u;
      bulk_load(ring + (blk % kRing) * kBlockBytes, kin + kb, bytes, mbar + (blk % kRing), keep);
    };
    if (t == 0)
      for (uint32_t blk = 0; blk < nblk && blk < kRing; ++blk) issue(blk);
    uint32_t issued = nblk < kRing ? nblk : kRing;  // same value in every thread
    bool bad = false;
    for (uint32_t blk = 0; blk < nblk; ++blk) {
      // block-uniform decision: every thread leaves together or not at all
      if (__syncthreads_or(!mbar_wait(mbar + (blk % kRing), (blk / kRing) & 1u))) {
        timed_out = true;
        if (t == 0)  // let the copies still in flight land (bounded)
          for (uint32_t q = blk; q < issued; ++q) mbar_wait(mbar + (q % kRing), (q / kRing) & 1u);
        break;
      }
      const K* kb = reinterpret_cast<const K*>(ring + (blk % kRing) * kBlockBytes);
      const uint32_t cnt = min(kPerBlock, end - (beg + blk * kPerBlock));
      for (uint32_t i = t; i < cnt; i += kThreads) {
        const K key = kb[i];
        bad |= (static_cast<uint64_t>(key) & a.bad_mask) != 0;
        atomicAdd(&off[digit_of<K>(key, a.shift, a.mask, false)], 1u);
      }
      __syncthreads();  // every thread is done with this block before it is refilled
      if (blk + kRing < nblk) {
        if (t == 0) {
          fence_proxy_async();
          issue(blk + kRing);
        }
        ++issued;
      }
    }
    if (__any_sync(0xffffffffu, bad) && lane_id() == 0)
      latch_error(a.err, TDGS_ERR_INVALID_ARGUMENT, kSiteRadixKeys);
  }
  __syncthreads();
  // ---- phase 2: offsets over chunks (the histogram is in off[])
  for (uint32_t b = t; b < kBins; b += kThreads) a.H[static_cast<size_t>(blockIdx.x) * kBins + b] = off[b];
  grid_barrier(a.bar, a.err);
  {
    const uint32_t lane = lane_id(), warp = t >> 5, G = gridDim.x, c = blockIdx.x;
    constexpr uint32_t kCol = kMaxGrid / 32;
    for (uint32_t b = c * (kThreads / 32) + warp; b < static_cast<uint32_t>(kBins); b += G * (kThreads / 32)) {
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
  }
  grid_barrier(a.bar, a.err);
  {
    const uint32_t v = t < kBins ? __ldcg(a.tot + t) : 0u;
    const uint32_t run = block_excl_scan<kThreads / 32>(v, s_warp);
    if (t < kBins) base[t] = run + __ldcg(a.P + static_cast<size_t>(blockIdx.x) * kBins + t);
  }
  __syncthreads();

  // ---- phase 3: tiles; the next tile is copied while this one is processed
  bool out_of_range = false;
  const uint32_t ntile = (end - beg + kTileKeys - 1) / kTileKeys;
  auto issue_tile = [&](uint32_t i) {
    const uint32_t tb = beg + i * kTileKeys;
    const uint32_t cnt = min(static_cast<uint32_t>(kTileKeys), end - tb);
    const uint32_t bytes = (cnt * static_cast<uint32_t>(sizeof(K)) + 15u) & ~15u;
    bulk_load(stage, kin + tb, bytes, mbar + kRing, drop);
  };
  if (t == 0 && ntile > 0 && !timed_out) {
    fence_proxy_async();
    issue_tile(0);
  }
  for (uint32_t i = 0; i < ntile && !timed_out; ++i) {
    const uint32_t tb = beg + i * kTileKeys;
    const uint32_t valid = min(static_cast<uint32_t>(kTileKeys), end - tb);
    for (uint32_t z = t; z < kTableWords / 4; z += kThreads) reinterpret_cast<uint4*>(C)[z] = make_uint4(0, 0, 0, 0);
    if (__syncthreads_or(!mbar_wait(mbar + kRing, i & 1u))) {
      timed_out = true;
      if (t == 0) mbar_wait(mbar + kRing, i & 1u);  // the pending copy, bounded
      break;
    }
    K k[kItems];
    const uint32_t first = t * kItems;
#pragma unroll
    for (int j = 0; j < kItems; ++j) k[j] = first + j < valid ? stage[first + j] : K(0);
    __syncthreads();  // stage fully read; table zeroed
    if (t == 0 && i + 1 < ntile) {
      fence_proxy_async();
      issue_tile(i + 1);
    }
    // 1. own-column counts
    uint32_t r[kItems];
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      if (first + j < valid) {
        uint32_t* cp = C + cell(digit_of<K>(k[j], a.shift, a.mask, false), t);
        const uint32_t o = *cp;
        *cp = o + 1;
        r[j] = o;
      }
    }
    __syncthreads();
    // 2. exclusive scan in (digit, thread) order: thread t owns the 64
    //    counters of digit t/4, threads 64*(t%4) .. 64*(t%4)+63
    {
      uint32_t* seg = C + (t >> 2) * kRow + (t & 3) * kQuarter;
      uint32_t sum = 0;
#pragma unroll 16
      for (int q = 0; q < 64; ++q) sum += seg[q];
      uint32_t run = block_excl_scan<kThreads / 32>(sum, s_warp);
#pragma unroll 16
      for (int q = 0; q < 64; ++q) {
        const uint32_t x = seg[q];
        seg[q] = run;
        run += x;
      }
    }
    __syncthreads();
    // 3. ranks; per-digit tile start and count
#pragma unroll
    for (int j = 0; j < kItems; ++j)
      if (first + j < valid) r[j] += C[cell(digit_of<K>(k[j], a.shift, a.mask, false), t)];
    uint32_t cnt = 0;
    if (t < kBins) {
      const uint32_t s0 = C[cell(t, 0)];
      const uint32_t s1 = t + 1 < kBins ? C[cell(t + 1, 0)] : valid;
      cnt = s1 - s0;
      off[t] = base[t] - s0;
    }
    __syncthreads();  // the table is overwritten by the exchange below
#pragma unroll
    for (int j = 0; j < kItems; ++j)
      if (first + j < valid) xk[r[j]] = k[j];
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kItems; ++q) {
      const uint32_t p = q * kThreads + t;
      if (p < valid) {
        const K key = xk[p];
        const uint32_t dst = off[digit_of<K>(key, a.shift, a.mask, false)] + p;
        if (dst < m) emit_key<K, kExpand>(a, key, dst, xk, p, valid, s_vrec, s_vtile, kout_raw, vout);
        else out_of_range = true;
      }
    }
    __syncthreads();
    if (t < kBins) base[t] += cnt;
    __syncthreads();
  }
  if (timed_out && t == 0) latch_error(a.err, TDGS_ERR_TIMEOUT, kSiteCopyWait);
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

template <typename K, bool kExpand>
Kernel make_ct_kernel() {
  return Kernel{reinterpret_cast<const void*>(&k_radix_pass_ct<K, kExpand>), 6, ct::kThreads, ct::kItems,
                ct::smem_bytes<K>(), 2};
}

template <typename K, bool kVals, bool kExpand, int kBits, int kThreads, int kItems>
Kernel make_kernel() {
  using S = PassShape<K, kVals, kExpand, kBits, kThreads, kItems>;
  return Kernel{reinterpret_cast<const void*>(&k_radix_pass<K, kVals, kExpand, kBits, kThreads, kItems>),
                kBits, kThreads, kItems, S::kSmem, S::kMinBlocks};
}

// Resident CTAs of `k` on the current device (0 on failure); caches the
// occupancy query per device and kernel.
uint32_t resident_ctas(const Kernel& k, int ctas_per_sm = 0);

// Grid for m keys: every CTA gets at least one tile, at most all resident.
uint32_t grid_for(const Kernel& k, uint32_t m, int ctas_per_sm = 0);

// Scratch words a pass with this kernel and grid needs.
inline size_t scratch_words(const Kernel& k, uint32_t grid) {
  return static_cast<size_t>(grid) * (1u << k.bits) * 2 + (1u << k.bits);
}

// Launch one pass (cooperative).  scratch: scratch_words() uint32 words.
cudaError_t launch(const Kernel& k, uint32_t grid, const void* kin, const uint32_t* vin, void* kout,
                   uint32_t* vout, PassArgs a, uint32_t* scratch, cudaStream_t s);

}  // namespace radix
}  // namespace tdgs
