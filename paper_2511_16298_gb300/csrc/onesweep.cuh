// Pieces of the onesweep radix passes (onesweep.cu, tdgs_sort_pairs) that
// do not depend on the element type or digit width: tiles copied into
// shared memory by bulk copies with bounded mbarrier waits, per-digit
// status words (flag + 30-bit count), the scan CTAs that turn the tiles'
// digit counts into prefixes, and the bounded wait for a tile's prefix.
#pragma once

#include "radix.cuh"

namespace tdgs {
namespace osw {

constexpr int kThreads = 256;                      // threads of a pass CTA
constexpr int kWarps = kThreads / 32;
constexpr uint32_t kFlagA = 1u << 30;              // status: this tile's own count
constexpr uint32_t kFlagP = 2u << 30;              // status: inclusive prefix over tiles <= this one
constexpr uint32_t kCountMask = (1u << 30) - 1u;
constexpr uint32_t kMaxPairs = 1u << 30;           // counts in a status word have 30 bits

// ------------------------------------------------------ shared-memory TMA
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
}
// The one arrival of a phase, expecting `bytes` of bulk-copy data (0: the
// phase completes at once).
__device__ __forceinline__ void mbar_arrive(uint64_t* bar, uint32_t bytes) {
  if (bytes == 0) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(bar))
                 : "memory");
  } else {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(
                     smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
  }
}
// Bulk copy global -> shared completing on `bar` (both addresses 16-byte
// aligned, bytes a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
// Bounded wait for phase `parity` of `bar`; false (error latched) if the
// copy did not arrive.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint32_t* err) {
  for (uint32_t i = 0; i < kSpinLimit; ++i) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  latch_error(err, TDGS_ERR_TIMEOUT, kSiteBarrier);
  return false;
}

__device__ __forceinline__ uint2 ld_relaxed_v2(const uint32_t* p) {
  uint2 v;
  asm volatile("ld.relaxed.gpu.global.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_v2(uint32_t* p, uint32_t x, uint32_t y) {
  asm volatile("st.relaxed.gpu.global.v2.u32 [%0], {%1, %2};" ::"l"(p), "r"(x), "r"(y) : "memory");
}

// Exclusive sum of v over the CTA (kThreads threads).
__device__ __forceinline__ uint32_t cta_excl_scan(uint32_t v, uint32_t* s_warp) {
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
    uint32_t w = lane < kWarps ? s_warp[lane] : 0u;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, w, d);
      if (lane >= static_cast<uint32_t>(d)) w += o;
    }
    if (lane < kWarps) s_warp[lane] = w;
  }
  __syncthreads();
  const uint32_t r = x - v + (warp ? s_warp[warp - 1] : 0u);
  __syncthreads();
  return r;
}

// The scan CTAs: the last scan_ctas<kBins>() CTAs of the grid take no tiles; scan
// CTA c owns digits [64 c, 64 c + 64).  Lane l of every warp owns digit
// pair 64 c + 2 l, +1; warp w reads rows (tiles) k + 8 w .. k + 8 w + 7 of
// it, so one round reads 64 rows per pair at once (one L2 round trip).
// Per pair, the rows up to the first tile whose counts are not out yet are
// consumed in order: running sums plus the sums of the warps before give
// each row its inclusive prefix, which overwrites its counts.  The next
// round starts at the first row not consumed (after a short sleep when no
// pair moved).  The scan waits only on counts, which every tile publishes
// without waiting on anything, so it always finishes (the wait is
// bounded).  Spreading the digits over several CTAs spreads the status
// traffic (about 4 KB per tile) over several SMs.
constexpr uint32_t kSegRows = 8;  // rows per warp and round
static_assert(kWarps * kSegRows == 64, "scan layout");
template <uint32_t kBins>
constexpr uint32_t scan_ctas() {
  static_assert(kBins % 64 == 0, "scan CTAs own 64 digits each");
  return kBins / 64;
}
template <uint32_t kBins>
__device__ __forceinline__ void scan_tiles(uint32_t* __restrict__ status, uint32_t ntiles, uint32_t c,
                                           uint32_t* err, uint32_t* sm) {
  uint32_t(*s_stop)[32] = reinterpret_cast<uint32_t(*)[32]>(sm);
  uint32_t(*s_sum0)[32] = reinterpret_cast<uint32_t(*)[32]>(sm + kWarps * 32);
  uint32_t(*s_sum1)[32] = reinterpret_cast<uint32_t(*)[32]>(sm + 2 * kWarps * 32);
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t* col = status + 64 * c + 2 * lane;
  uint32_t k = 0, run0 = 0, run1 = 0, idle = 0;  // per pair: first row not consumed, its sums
  while (__syncthreads_or(k < ntiles)) {
    const uint32_t r0 = k + kSegRows * warp;
    uint2 w[kSegRows];
#pragma unroll
    for (uint32_t q = 0; q < kSegRows; ++q)
      w[q] = r0 + q < ntiles ? ld_relaxed_v2(col + static_cast<size_t>(r0 + q) * kBins) : make_uint2(0u, 0u);
    uint32_t stop = kSegRows, t0 = 0, t1 = 0;  // first unusable row of the segment; sums before it
#pragma unroll
    for (uint32_t q = 0; q < kSegRows; ++q) {
      const bool ready = r0 + q < ntiles && (w[q].x & ~kCountMask) != 0 && (w[q].y & ~kCountMask) != 0;
      if (!ready && stop == kSegRows) stop = q;
      if (stop == kSegRows) {
        t0 += w[q].x & kCountMask;
        t1 += w[q].y & kCountMask;
      }
    }
    s_stop[warp][lane] = stop;
    s_sum0[warp][lane] = t0;
    s_sum1[warp][lane] = t1;
    __syncthreads();
    // this pair's rows consumed in this round: every warp's segment up to
    // the first one that stops early
    uint32_t before0 = 0, before1 = 0, all0 = 0, all1 = 0, used = 0;
    bool open = true;  // segments so far were complete
#pragma unroll
    for (uint32_t v = 0; v < kWarps; ++v) {
      if (open) {
        if (v < warp) {
          before0 += s_sum0[v][lane];
          before1 += s_sum1[v][lane];
        }
        all0 += s_sum0[v][lane];
        all1 += s_sum1[v][lane];
        used += s_stop[v][lane];
        open = s_stop[v][lane] == kSegRows;
      }
    }
    // this warp's segment lies inside the consumed rows if every earlier
    // segment was complete
    bool mine = true;
#pragma unroll
    for (uint32_t v = 0; v < kWarps; ++v)
      if (v < warp && s_stop[v][lane] != kSegRows) mine = false;
    if (mine) {
      uint32_t p0 = run0 + before0, p1 = run1 + before1;
#pragma unroll
      for (uint32_t q = 0; q < kSegRows; ++q) {
        if (q < stop) {
          p0 += w[q].x & kCountMask;
          p1 += w[q].y & kCountMask;
          st_relaxed_v2(col + static_cast<size_t>(r0 + q) * kBins, kFlagP | (p0 & kCountMask),
                        kFlagP | (p1 & kCountMask));
        }
      }
    }
    k += used;
    run0 += all0;
    run1 += all1;
    // no pair of the CTA moved: wait a little (bounded)
    if (!__syncthreads_or(used != 0 || k >= ntiles)) {
      if (++idle > kSpinLimit) {
        latch_error(err, TDGS_ERR_TIMEOUT, kSiteBarrier);
        return;
      }
      __nanosleep(64);
    }
  }
}

// Exclusive prefix of digits 2t and 2t+1 for tile `tile` > 0: the inclusive
// prefix the scan CTAs wrote for tile - 1 (bounded wait).
template <uint32_t kBins>
__device__ __forceinline__ void wait_prefix(const uint32_t* __restrict__ status, uint32_t tile, uint32_t t,
                                            uint32_t& e0, uint32_t& e1, uint32_t* err) {
  const uint32_t* row = status + static_cast<size_t>(tile - 1) * kBins + 2 * t;
  uint2 w = ld_relaxed_v2(row);
  uint32_t spins = 0;
  while ((w.x & ~kCountMask) != kFlagP || (w.y & ~kCountMask) != kFlagP) {
    if (++spins > kSpinLimit) {
      latch_error(err, TDGS_ERR_TIMEOUT, kSiteBarrier);
      break;
    }
    __nanosleep(32);
    w = ld_relaxed_v2(row);
  }
  e0 = w.x & kCountMask;
  e1 = w.y & kCountMask;
}

}  // namespace osw
}  // namespace tdgs
