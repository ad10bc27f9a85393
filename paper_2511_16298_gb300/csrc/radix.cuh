// Stable LSD radix pass shared by every sort in the library (the Sorting
// step of Sec. II-A orders instances by tile, then by depth).
//
// One digit pass is one persistent, cooperatively launched kernel whose
// grid is the number of CTAs resident on the GPU (a multiple of the SM
// count).  CTA c owns one contiguous chunk of the input:
//   phase 1  histogram of the chunk's digits (16-byte loads with an L2
//            evict-last policy, so phase 3 finds most keys in L2);
//   barrier
//   phase 2  one warp per digit scans the chunk histograms over chunks
//            -> each chunk's exclusive prefix per digit, and digit totals;
//   barrier
//            every CTA scans the totals over digits; its running output
//            base per digit = digit start + chunk prefix;
//   phase 3  the chunk is processed tile by tile (kThreads x kItems keys):
//            stable ranking inside each warp from one ballot per digit bit,
//            per-warp digit counters in shared memory, a prefix over warps
//            and digits, exchange through shared memory into digit order,
//            coalesced scatter at base + rank.
// Two bounded grid barriers replace a decoupled look-back, whose walk
// depth grows with the number of resident tiles when digits are wide.
//
// Ranking uses ballots for every digit width: on this GPU one match.any
// costs about as much as eight ballot rounds, so the ballot chain wins up
// to 12-bit digits.
//
// Template knobs: key type K (uint32/uint64), whether a uint32 value
// travels with the key, and "expand" (the last pass of the frame path: the
// key is a packed (tile, depth rank) element and the scatter writes the
// final 64-bit key and the Gaussian index instead).
#pragma once

#include "tdgs_internal.cuh"

namespace tdgs {
namespace radix {

constexpr uint32_t kMaxGrid = 512;  // chunks per pass (the column scan holds 16 per lane)

__device__ __forceinline__ uint64_t policy_evict_last() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint4 ld_hint_v4(const void* a, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(a), "l"(pol));
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

// Hint: bring [p, p + bytes) into L2 with one bulk prefetch (the 16-byte
// aligned part of it; nothing is read into registers or shared memory).
__device__ __forceinline__ void prefetch_l2(const void* p, uint64_t bytes) {
  const uint64_t a = reinterpret_cast<uint64_t>(p);
  const uint64_t lo = (a + 15) & ~15ull, hi = (a + bytes) & ~15ull;
  if (hi > lo)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"(static_cast<uint32_t>(hi - lo))
                 : "memory");
}

__device__ __forceinline__ uint32_t atom_add_acq_rel32(uint32_t* p, uint32_t v) {
  uint32_t old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

// Self-resetting grid barrier for a cooperatively launched grid (all CTAs
// resident).  bar[0] counts arrivals, bar[1] is the generation.  After the
// block barrier, thread 0 arrives with an acquire-release add (publishing
// its block's writes); the last arrival resets the count and releases the
// next generation, which the others acquire.  The wait is bounded: on
// timeout the error is latched and the CTA moves on (every scatter stays
// bounds-checked).
__device__ __forceinline__ void grid_barrier(uint32_t* bar, uint32_t* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t gen = ld_acquire32(bar + 1);
    const uint32_t arrived = atom_add_acq_rel32(bar, 1u);
    if (arrived == gridDim.x - 1) {
      bar[0] = 0u;  // ordered before the release below
      st_release32(bar + 1, gen + 1);
    } else {
      uint32_t spins = 0;
      while (ld_acquire32(bar + 1) == gen) {
        if (++spins > kSpinLimit) {
          latch_error(err, TDGS_ERR_TIMEOUT, kSiteBarrier);
          break;
        }
        __nanosleep(32);
      }
    }
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

// Lanes of the warp whose digit equals this lane's, from one ballot per
// digit bit: a lane keeps the ballot where its own bit is set and the
// complement where it is clear.  Digits must be < 2^kBits.
template <int kBits>
__device__ __forceinline__ uint32_t equal_digit_lanes(uint32_t d) {
  uint32_t peers = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < kBits; ++b) {
    asm("{\n\t.reg .pred p;\n\t.reg .u32 t;\n\t"
        "and.b32 t, %1, %2;\n\t"
        "setp.ne.u32 p, t, 0;\n\t"
        "vote.sync.ballot.b32 t, p, 0xffffffff;\n\t"
        "@!p not.b32 t, t;\n\t"
        "and.b32 %0, %0, t;\n\t}"
        : "+r"(peers)
        : "r"(d), "r"(1u << b));
  }
  return peers;
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
  const uint2* sdo;            // by rank: {depth bits, global record index}
  const uint32_t* vrec_begin;  // [nv+1] first record of each view
  const uint32_t* vtile_begin; // [nv+1] first global tile of each view
  uint32_t nv;
  uint32_t* rmin;              // per global tile: first sorted position (atomicMin)
  uint32_t* rmax;              // per global tile: one past the last (atomicMax)
  // view-local tile ranges [start, end) (t_all entries), or null: a single
  // pass over the whole tile id writes them from its digit totals; the last
  // of several passes, after a grid barrier, from rmin/rmax (which it then
  // resets to all ones / zero)
  uint2* ranges;
  const uint32_t* pbeg;        // [nv+1] first pair of each view
  uint32_t t_all;
  const uint64_t* m_dev;       // optional device element count, capped at m
};

// kOcc: CTAs per SM the register budget is sized for (launch bounds); 0
// picks 2 for 64-bit keys, wide digits and expanding passes, 3 otherwise.
template <typename K, bool kVals, bool kExpand, int kBits, int kThreads, int kItems, int kOcc>
struct PassShape {
  static constexpr int kBins = 1 << kBits;
  static constexpr int kWarps = kThreads / 32;
  static constexpr int kTileKeys = kThreads * kItems;
  static constexpr int kBpt = (kBins + kThreads - 1) / kThreads;
  static constexpr int kCols = kBins / 2;  // counter words: two 16-bit digits each
  static constexpr int kCpt = (kCols + kThreads - 1) / kThreads;
  // shared memory, no aliasing: per-warp counters | key exchange |
  // value exchange |
  // base, lstart, off per digit
  static constexpr size_t kWhBytes = static_cast<size_t>(kWarps) * kBins * 2;
  static constexpr size_t kXkBytes = static_cast<size_t>(kTileKeys) * sizeof(K);
  static constexpr size_t kXvBytes = kVals ? static_cast<size_t>(kTileKeys) * 4 : 0;
  static constexpr size_t kSmem = kWhBytes + kXkBytes + kXvBytes + static_cast<size_t>(kBins) * 12;
  static constexpr int kMinBlocks =
      kOcc > 0 ? kOcc : (kThreads >= 512 ? 1 : ((kBits > 10 || sizeof(K) == 8) ? 2 : 3));
  static_assert(kBits >= 6 && kBits <= 12, "digits of 6..12 bits");
  static_assert(kTileKeys <= 32768, "per-warp counters and their prefixes are 16-bit");
  static_assert(kWhBytes % 16 == 0, "counters are cleared with 16-byte stores");
};

// Chunk of the input owned by this CTA (chunks are multiples of 4 keys so
// every chunk starts 16-byte aligned when the array does); m may come from
// device memory.
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

// Phase 1 body for one key.
template <typename K>
__device__ __forceinline__ void count_key(K k, const PassArgs& a, bool d31, uint32_t* hist, bool& bad) {
  if constexpr (sizeof(K) == 8) bad |= (k & a.bad_mask) != 0;
  atomicAdd(&hist[digit_of<K>(k, a.shift, a.mask, d31)], 1u);
}

// Phase 2, after every chunk has written its histogram row H[c][*]: a
// grid barrier, one warp per digit scans the column over chunks (chunk
// prefixes P, digit totals tot), a grid barrier, then base[b] = first
// output position of this chunk's keys with digit b.  With kRowSum (at
// most 64 digits, or 512-thread CTAs: one per SM, so at most 152 chunks)
// each CTA sums the rows itself after the first barrier.  With a.ranges set,
// the tile ranges are written from the digit totals.
template <int kBins, int kThreads, bool kRowSum = (kBins <= 64 || (kThreads >= 512 && kBins <= kThreads))>
__device__ __forceinline__ void scan_chunks(const PassArgs& a, uint32_t* base, uint32_t* s_warp,
                                            const uint32_t* s_vtile) {
  constexpr int kWarps = kThreads / 32;
  constexpr int kBpt = (kBins + kThreads - 1) / kThreads;
  const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;
  const uint32_t G = gridDim.x, c = blockIdx.x;
  if constexpr (kRowSum) {
    // Few digits or few chunks: after one grid barrier every CTA sums the
    // histogram rows itself (16-byte loads, kRows row groups in parallel):
    // the rows of the chunks before it and all rows.  No second barrier, no
    // P or tot.
    constexpr int kQ = kBins / 4;          // 16-byte words per row
    constexpr int kRows = kThreads / kQ;   // row groups
    static_assert(kBins <= kThreads && kThreads % kQ == 0, "one digit per thread in the row sums");
    __shared__ uint4 s_pre[kRows][kQ];
    __shared__ uint4 s_all[kRows][kQ];
    grid_barrier(a.bar, a.err);
    const uint32_t q = t % kQ, r = t / kQ;
    uint4 pre = make_uint4(0, 0, 0, 0), all = make_uint4(0, 0, 0, 0);
#pragma unroll 8
    for (uint32_t cc = r; cc < G; cc += kRows) {
      const uint4 h = __ldcg(reinterpret_cast<const uint4*>(a.H + static_cast<size_t>(cc) * kBins) + q);
      all.x += h.x; all.y += h.y; all.z += h.z; all.w += h.w;
      if (cc < c) {
        pre.x += h.x; pre.y += h.y; pre.z += h.z; pre.w += h.w;
      }
    }
    s_pre[r][q] = pre;
    s_all[r][q] = all;
    __syncthreads();
    uint32_t seg = 0, before = 0;
    if (t < static_cast<uint32_t>(kBins)) {
      const uint32_t* sp = reinterpret_cast<const uint32_t*>(&s_pre[0][0]);
      const uint32_t* sa = reinterpret_cast<const uint32_t*>(&s_all[0][0]);
#pragma unroll
      for (int rr = 0; rr < kRows; ++rr) {
        seg += sa[rr * kBins + t];
        before += sp[rr * kBins + t];
      }
    }
    const uint32_t run = block_excl_scan<kWarps>(seg, s_warp);
    if (t < static_cast<uint32_t>(kBins)) {
      const uint32_t b = t;
      base[b] = run + before;
      if (a.ranges && !a.rmin && b < a.t_all && b % G == c) {
        uint2 rg = make_uint2(0u, 0u);
        if (seg) {
          const uint32_t pb = a.pbeg[a.nv == 1 ? 0u : find_view(s_vtile, a.nv, b)];
          rg = make_uint2(run - pb, run + seg - pb);
        }
        a.ranges[b] = rg;
      }
    }
    __syncthreads();
    return;
  }
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
    if (b < kBins) {
      base[b] = run + __ldcg(a.P + static_cast<size_t>(c) * kBins + b);
      // every tile's range, spread over the CTAs; positions are relative
      // to the view's first pair
      if (a.ranges && !a.rmin && b < a.t_all && b % G == c) {
        uint2 rg = make_uint2(0u, 0u);
        if (seg[i]) {
          const uint32_t pb = a.pbeg[a.nv == 1 ? 0u : find_view(s_vtile, a.nv, b)];
          rg = make_uint2(run - pb, run + seg[i] - pb);
        }
        a.ranges[b] = rg;
      }
    }
    run += seg[i];
  }
  __syncthreads();
}

// Phases 1-2: histogram of this chunk's digits, column scans over chunks
// between two grid barriers, then base[b] = first output position of this
// chunk's keys with digit b.  hist: kBins words of shared scratch.  With
// a.ranges set, the tile ranges are written from the digit totals.
template <typename K, int kBins, int kThreads, uint32_t kU = 8>
__device__ __forceinline__ void chunk_bases(const K* __restrict__ kin, const PassArgs& a,
                                            uint32_t beg, uint32_t end, bool d31, uint32_t* base,
                                            uint32_t* hist, uint32_t* s_warp, const uint32_t* s_vtile) {
  const uint32_t t = threadIdx.x, lane = lane_id(), c = blockIdx.x;
  for (uint32_t b = t; b < kBins; b += kThreads) hist[b] = 0;
  __syncthreads();
  {
    const uint64_t keep = policy_evict_last();
    bool bad = false;
    const K* kc = kin + beg;
    const uint32_t len = end - beg;
    uint32_t done = 0;
    if ((reinterpret_cast<uintptr_t>(kc) & 15u) == 0) {
      constexpr uint32_t kPer = 16 / sizeof(K);  // keys per 16-byte vector; kU vectors in flight per thread
      const uint32_t nvec = len / kPer;
      for (uint32_t q0 = t; q0 < nvec; q0 += kThreads * kU) {
        uint4 w[kU];
#pragma unroll
        for (uint32_t u = 0; u < kU; ++u) {
          const uint32_t q = q0 + u * kThreads;
          w[u] = q < nvec ? ld_hint_v4(kc + q * kPer, keep) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (uint32_t u = 0; u < kU; ++u) {
          if (q0 + u * kThreads < nvec) {
            const K* e = reinterpret_cast<const K*>(&w[u]);
#pragma unroll
            for (uint32_t i = 0; i < kPer; ++i) count_key<K>(e[i], a, d31, hist, bad);
          }
        }
      }
      done = nvec * kPer;
    }
    for (uint32_t i = done + t; i < len; i += kThreads) count_key<K>(kc[i], a, d31, hist, bad);
    if (__any_sync(0xffffffffu, bad) && lane == 0) latch_error(a.err, TDGS_ERR_INVALID_ARGUMENT, kSiteRadixKeys);
  }
  __syncthreads();
  for (uint32_t b = t; b < kBins; b += kThreads) a.H[static_cast<size_t>(c) * kBins + b] = hist[b];
  scan_chunks<kBins, kThreads>(a, base, s_warp, s_vtile);
}

// Output of one key at its sorted position dst.  Plain passes store the
// key; the expanding pass stores (local tile << 32 | depth bits dep) and
// the view-local Gaussian index (gi is the global record index, gathered
// when the tile was loaded), and (multi-pass tile sorts) records the
// first/last position of each global tile run seen in this tile's exchange
// buffer xk (run_ends: this element's own test; false when the tile's runs
// were recorded per digit).
template <typename K, bool kExpand>
__device__ __forceinline__ void emit_key(const PassArgs& a, K key, uint32_t gi, uint32_t dep, uint32_t dst,
                                         const K* xk, uint32_t p, uint32_t valid, const uint32_t* s_vrec,
                                         const uint32_t* s_vtile, void* kout_raw, uint32_t* vout,
                                         bool run_ends = true) {
  if constexpr (kExpand) {
    const uint32_t gt = static_cast<uint32_t>(key >> a.rbits);
    uint32_t tb = 0, rb = 0;  // first global tile and record of the view (0 for one view)
    if (a.nv != 1) {
      const uint32_t v = find_view(s_vrec, a.nv, gi);
      tb = s_vtile[v];
      rb = s_vrec[v];
    }
    static_cast<uint64_t*>(kout_raw)[dst] = (static_cast<uint64_t>(gt - tb) << 32) | dep;
    vout[dst] = gi - rb;
    if (a.rmin && run_ends) {
      if (p == 0 || static_cast<uint32_t>(xk[p - 1] >> a.rbits) != gt) atomicMin(a.rmin + gt, dst);
      if (p + 1 == valid || static_cast<uint32_t>(xk[p + 1] >> a.rbits) != gt) atomicMax(a.rmax + gt, dst + 1);
    }
  } else {
    static_cast<K*>(kout_raw)[dst] = key;
  }
}

// Shared-memory layout of one pass CTA.
template <typename K>
struct Smem {
  uint16_t* wh;     // [kWarps][kBins] per-warp digit counters, then exclusive prefixes over warps
  K* xk;            // key exchange
  uint32_t* xv;     // value exchange
  uint32_t* base;   // [kBins] running output base of this chunk per digit
  uint32_t* lstart; // [kBins] tile count per digit, then tile-local digit start
  uint32_t* off;    // [kBins] base - tile-local start: output position = off[digit] + p
};

// Tile-local digit starts from the per-digit tile counts in lstart (one
// warp when the digits fit 16 per lane, else the whole block), and per
// digit: off = base - start, base += count.
template <typename S, typename K>
__device__ __forceinline__ void digit_starts(const Smem<K>& sm, uint32_t* s_warp) {
  constexpr int kBins = S::kBins;
  constexpr int kWarps = S::kWarps;
  constexpr int kThreads = kWarps * 32;
  const uint32_t t = threadIdx.x;
  if constexpr (kBins <= 512) {
    constexpr int kPer = kBins / 32;
    if (t < 32) {
      uint32_t c[kPer];
      uint32_t sum = 0;
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        c[i] = sm.lstart[t * kPer + i];
        sum += c[i];
      }
      uint32_t x = sum;
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, x, dd);
        if (t >= static_cast<uint32_t>(dd)) x += o;
      }
      uint32_t run = x - sum;
#pragma unroll
      for (int i = 0; i < kPer; ++i) {
        const uint32_t b = t * kPer + i;
        const uint32_t bs = sm.base[b];
        sm.lstart[b] = run;
        sm.off[b] = bs - run;
        sm.base[b] = bs + c[i];
        run += c[i];
      }
    }
  } else {
    constexpr int kBpt = S::kBpt;
    uint32_t c[kBpt];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kBpt; ++i) {
      const uint32_t b = t * kBpt + i;
      c[i] = b < kBins ? sm.lstart[b] : 0u;
      sum += c[i];
    }
    uint32_t run = block_excl_scan<kWarps>(sum, s_warp);
#pragma unroll
    for (int i = 0; i < kBpt; ++i) {
      const uint32_t b = t * kBpt + i;
      if (b < kBins) {
        const uint32_t bs = sm.base[b];
        sm.lstart[b] = run;
        sm.off[b] = bs - run;
        sm.base[b] = bs + c[i];
      }
      run += c[i];
    }
    (void)kThreads;
  }
}

// Registers of one tile between its ranking and its scatter.
template <typename K, bool kExpand, int kItems>
struct TileRegs {
  K k[kItems];
  uint32_t d[kItems];  // digits
  uint32_t r[kItems];  // ranks: within the warp, then within the tile
};

// Phase 3, first half, for one tile of `valid` keys starting at kt
// (kFull: valid == kTileKeys, no bounds checks): load, stable rank within
// each warp, exclusive prefix over warps; on return (after a block
// barrier) lstart holds the tile's count per digit -- with more than 64
// digits; with at most 64 the per-warp counts are left for scatter_tile,
// which folds the prefix into its one-warp digit starts.  Each warp's
// counter row is zero on entry.
// rank_keys is the same after the load, for keys and digits already in
// R.k / R.d (item j of lane l of warp w is tile item w * 32 * kItems +
// j * 32 + l).
template <bool kFull, typename S, typename K, bool kExpand, int kBits, int kItems>
__device__ __forceinline__ void rank_keys(uint32_t valid, const Smem<K>& sm, TileRegs<K, kExpand, kItems>& R);

template <bool kFull, typename S, typename K, bool kExpand, int kBits, int kItems>
__device__ __forceinline__ void rank_tile(const K* __restrict__ kt, uint32_t valid, const PassArgs& a, bool d31,
                                          const Smem<K>& sm, TileRegs<K, kExpand, kItems>& R) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t wbase = warp * 32 * kItems;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t idx = wbase + j * 32 + lane;
    R.k[j] = (kFull || idx < valid) ? __ldcs(kt + idx) : K(0);
    R.d[j] = digit_of<K>(R.k[j], a.shift, a.mask, d31);
  }
  rank_keys<kFull, S, K, kExpand, kBits, kItems>(valid, sm, R);
}

template <bool kFull, typename S, typename K, bool kExpand, int kBits, int kItems>
__device__ __forceinline__ void rank_keys(uint32_t valid, const Smem<K>& sm, TileRegs<K, kExpand, kItems>& R) {
  constexpr int kBins = S::kBins;
  constexpr int kWarps = S::kWarps;
  constexpr int kThreads = kWarps * 32;
  constexpr int kCols = S::kCols;
  constexpr int kCpt = S::kCpt;
  const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;
  const uint32_t wbase = warp * 32 * kItems;
  // rank within the warp, kGroup items at a time: the equal-digit lane
  // sets of the group first (independent ballot chains), then every lane
  // of a set reads the warp's counter and the set's highest lane writes it
  // back bumped
  constexpr int kGroup = sizeof(K) == 8 ? 4 : 8;
  static_assert(kItems % kGroup == 0, "items per thread: a multiple of the ranking group");
  uint16_t* my_wh = sm.wh + warp * kBins;
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int j0 = 0; j0 < kItems; j0 += kGroup) {
#pragma unroll
    for (int j = j0; j < j0 + kGroup; ++j) {
      R.r[j] = equal_digit_lanes<kBits>(R.d[j]);
      if constexpr (!kFull) {
        const uint32_t first = wbase + j * 32;
        const uint32_t nlive = valid > first ? min(valid - first, 32u) : 0u;
        R.r[j] &= nlive >= 32 ? 0xffffffffu : ((1u << nlive) - 1u);
      }
    }
#pragma unroll
    for (int j = j0; j < j0 + kGroup; ++j) {
      const uint32_t peers = R.r[j];
      const bool live = kFull || wbase + j * 32 + lane < valid;
      const uint32_t before = my_wh[R.d[j]];
      __syncwarp();
      const uint32_t cnt = __popc(peers);
      const uint32_t below = __popc(peers & lt);
      if (live && below + 1 == cnt) my_wh[R.d[j]] = static_cast<uint16_t>(before + cnt);
      __syncwarp();
      R.r[j] = before + below;
    }
  }
  __syncthreads();
  // exclusive prefix over warps per digit (two digits per 32-bit word);
  // tile count per digit into lstart.  With at most 64 digits scatter_tile
  // does this together with the digit starts in one warp (one block
  // barrier less per tile).
  if constexpr (S::kBins > 64) {
    uint32_t* wh32 = reinterpret_cast<uint32_t*>(sm.wh);
#pragma unroll
    for (int i = 0; i < kCpt; ++i) {
      const uint32_t c = t + i * kThreads;
      if (c < static_cast<uint32_t>(kCols)) {
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
          const uint32_t x = wh32[w * kCols + c];
          wh32[w * kCols + c] = run;
          run += x;  // halves stay below 2^16: no carry between digits
        }
        sm.lstart[2 * c] = run & 0xffffu;
        sm.lstart[2 * c + 1] = run >> 16;
      }
    }
    __syncthreads();
  }
}

// Phase 3, second half: digit starts (with base[] = this chunk's running
// output base per digit), exchange into digit order, coalesced scatter.
// Returns false if a destination fell outside [0, m).  Block barriers:
// after the digit starts and after the exchange (and one more for values);
// this warp's counter row is zeroed again.
template <bool kFull, typename S, typename K, bool kVals, bool kExpand, int kBits, int kItems>
__device__ __forceinline__ bool scatter_tile(const uint32_t* __restrict__ vt, uint32_t valid, uint32_t m,
                                             const PassArgs& a, bool d31, const Smem<K>& sm, uint32_t* s_warp,
                                             const uint32_t* s_vrec, const uint32_t* s_vtile, void* kout_raw,
                                             uint32_t* vout, TileRegs<K, kExpand, kItems>& R) {
  constexpr int kBins = S::kBins;
  constexpr int kWarps = S::kWarps;
  constexpr int kThreads = kWarps * 32;
  const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;
  const uint32_t wbase = warp * 32 * kItems;
  uint16_t* my_wh = sm.wh + warp * kBins;
  bool ok = true;
  __shared__ uint32_t s_low;  // expanding pass: tile item 0's tile bits below this pass's digit
  if constexpr (kExpand)
    if (t == 0) s_low = static_cast<uint32_t>(R.k[0] >> a.rbits) & ((1u << (a.shift - a.rbits)) - 1u);
  if constexpr (kBins <= 64) {
    // one warp: prefix over warps of each counter column (two digits per
    // word, lane = column), the tile's count per digit, the digit starts
    constexpr int kCols = S::kCols;
    if (t < 32) {
      uint32_t* wh32 = reinterpret_cast<uint32_t*>(sm.wh);
      uint32_t run = 0;
      if (lane < static_cast<uint32_t>(kCols)) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
          const uint32_t x = wh32[w * kCols + lane];
          wh32[w * kCols + lane] = run;
          run += x;  // halves stay below 2^16: no carry between digits
        }
      }
      const uint32_t c0 = run & 0xffffu, c1 = run >> 16;
      const uint32_t sum = c0 + c1;
      uint32_t x = sum;
#pragma unroll
      for (int dd = 1; dd < 32; dd <<= 1) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, x, dd);
        if (lane >= static_cast<uint32_t>(dd)) x += o;
      }
      if (lane < static_cast<uint32_t>(kCols)) {
        const uint32_t st0 = x - sum, st1 = st0 + c0;
        const uint32_t b0 = 2 * lane, b1 = b0 + 1;
        const uint32_t bs0 = sm.base[b0], bs1 = sm.base[b1];
        sm.lstart[b0] = st0;
        sm.lstart[b1] = st1;
        sm.off[b0] = bs0 - st0;
        sm.off[b1] = bs1 - st1;
        sm.base[b0] = bs0 + c0;
        sm.base[b1] = bs1 + c1;
      }
    }
  } else {
    digit_starts<S, K>(sm, s_warp);
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kItems; ++j) R.r[j] += sm.lstart[R.d[j]] + my_wh[R.d[j]];
  __syncwarp();
  {  // this warp's counter row is read: zero it for the next tile
    uint4* z = reinterpret_cast<uint4*>(my_wh);
    for (uint32_t i = lane; i < static_cast<uint32_t>(kBins) / 8; i += 32) z[i] = make_uint4(0, 0, 0, 0);
  }
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    if (kFull || wbase + j * 32 + lane < valid) {
      sm.xk[R.r[j]] = R.k[j];
    }
  }
  // values are fetched only now (fewer registers live while ranking);
  // the key scatter below hides their latency
  uint32_t v[kVals ? kItems : 1];
  if constexpr (kVals) {
#pragma unroll
    for (int j = 0; j < kItems; ++j) {
      const uint32_t idx = wbase + j * 32 + lane;
      v[j] = (kFull || idx < valid) ? __ldcs(vt + idx) : 0u;
    }
  }
  // The expanding pass of a multi-pass tile sort records each tile run's
  // first and last position.  When the tile's elements share the tile bits
  // the earlier passes sorted by (its first and last element do: the input
  // is sorted by them), each digit run is one tile: one thread per digit
  // records its ends.  Otherwise every element tests its neighbours.
  bool per_digit = false;
  if constexpr (kExpand) {
    if (a.rmin) {
      const uint32_t lb = a.shift - a.rbits;  // tile bits sorted by the earlier passes
      const uint32_t lmask = (1u << lb) - 1u;
      const uint32_t lo0 = s_low;  // written before the digit-start barrier
      bool same = true;
#pragma unroll
      for (int j = 0; j < kItems; ++j)
        if (kFull || wbase + j * 32 + lane < valid) same &= (static_cast<uint32_t>(R.k[j] >> a.rbits) & lmask) == lo0;
      per_digit = __syncthreads_and(same) != 0;
      if (per_digit) {
        for (uint32_t d = t; d < static_cast<uint32_t>(kBins); d += kThreads) {
          const uint32_t st = sm.lstart[d];
          const uint32_t en = d + 1 < static_cast<uint32_t>(kBins) ? sm.lstart[d + 1] : valid;
          if (en > st) {
            const uint32_t gt = (d << lb) | lo0, first = sm.off[d] + st;
            if (first < m && first + (en - st) <= m) {
              atomicMin(a.rmin + gt, first);
              atomicMax(a.rmax + gt, first + (en - st));
            }
          }
        }
      }
    } else {
      __syncthreads();
    }
  } else {
    __syncthreads();
  }
  // Scatter in digit order.  A destination outside [0, m) can only come
  // from a timed-out barrier or keys changed underneath the sort: it is
  // dropped and reported instead of written.
  uint32_t dst[kItems];
  if constexpr (kExpand) {
    // the expanding pass gathers {depth key, record index} of each
    // element's depth position now, kHalf loads in flight before the stores
    constexpr int kHalf = kItems >= 16 ? kItems / 2 : kItems;
#pragma unroll
    for (int i0 = 0; i0 < kItems; i0 += kHalf) {
      K key[kHalf];
      uint32_t at[kHalf];
      uint2 dg[kHalf];
#pragma unroll
      for (int h = 0; h < kHalf; ++h) {
        const uint32_t p = (i0 + h) * kThreads + t;
        at[h] = 0xffffffffu;
        key[h] = K(0);
        dg[h] = make_uint2(0u, 0u);
        if (kFull || p < valid) {
          key[h] = sm.xk[p];
          at[h] = sm.off[digit_of<K>(key[h], a.shift, a.mask, d31)] + p;
          if (at[h] < m) dg[h] = __ldg(a.sdo + static_cast<uint32_t>(key[h] & ((static_cast<K>(1) << a.rbits) - 1)));
        }
      }
#pragma unroll
      for (int h = 0; h < kHalf; ++h) {
        const uint32_t p = (i0 + h) * kThreads + t;
        if (kFull || p < valid) {
          if (at[h] < m)
            emit_key<K, true>(a, key[h], dg[h].y, dg[h].x, at[h], sm.xk, p, valid, s_vrec, s_vtile, kout_raw, vout,
                              !per_digit);
          else
            ok = false;
        }
      }
    }
  } else {
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const uint32_t p = i * kThreads + t;
      dst[i] = 0xffffffffu;
      if (kFull || p < valid) {
        const K key = sm.xk[p];
        dst[i] = sm.off[digit_of<K>(key, a.shift, a.mask, d31)] + p;
        if (dst[i] < m)
          emit_key<K, false>(a, key, 0u, 0u, dst[i], sm.xk, p, valid, s_vrec, s_vtile, kout_raw, vout);
        else
          ok = false;
      }
    }
  }
  if constexpr (kVals) {
#pragma unroll
    for (int j = 0; j < kItems; ++j)
      if (kFull || wbase + j * 32 + lane < valid) sm.xv[R.r[j]] = v[j];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const uint32_t p = i * kThreads + t;
      if ((kFull || p < valid) && dst[i] < m) vout[dst[i]] = sm.xv[p];
    }
  }
  return ok;
}

// Phase 3 for one tile: both halves.
template <bool kFull, typename S, typename K, bool kVals, bool kExpand, int kBits, int kItems>
__device__ __forceinline__ bool rank_and_scatter(const K* __restrict__ kt, const uint32_t* __restrict__ vt,
                                                 uint32_t valid, uint32_t m, const PassArgs& a, bool d31,
                                                 const Smem<K>& sm, uint32_t* s_warp,
                                                 const uint32_t* s_vrec, const uint32_t* s_vtile,
                                                 void* kout_raw, uint32_t* vout) {
  TileRegs<K, kExpand, kItems> R;
  rank_tile<kFull, S, K, kExpand, kBits, kItems>(kt, valid, a, d31, sm, R);
  return scatter_tile<kFull, S, K, kVals, kExpand, kBits, kItems>(vt, valid, m, a, d31, sm, s_warp, s_vrec,
                                                                  s_vtile, kout_raw, vout, R);
}

template <typename K, bool kVals, bool kExpand, int kBits, int kThreads, int kItems, int kOcc>
__global__ void __launch_bounds__(kThreads, (PassShape<K, kVals, kExpand, kBits, kThreads, kItems, kOcc>::kMinBlocks))
    k_radix_pass(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                 void* __restrict__ kout_raw, uint32_t* __restrict__ vout, PassArgs a) {
  using S = PassShape<K, kVals, kExpand, kBits, kThreads, kItems, kOcc>;
  constexpr uint32_t kTileKeys = S::kTileKeys;
  extern __shared__ __align__(16) unsigned char smem[];
  Smem<K> sm;
  {
    unsigned char* q = smem;
    sm.wh = reinterpret_cast<uint16_t*>(q);
    q += S::kWhBytes;
    sm.xk = reinterpret_cast<K*>(q);
    q += S::kXkBytes;
    sm.xv = reinterpret_cast<uint32_t*>(q);
    q += S::kXvBytes;
    sm.base = reinterpret_cast<uint32_t*>(q);
    sm.lstart = sm.base + S::kBins;
    sm.off = sm.lstart + S::kBins;
  }
  __shared__ uint32_t s_warp[S::kWarps];
  __shared__ uint32_t s_vrec[kExpand ? kMaxViews + 1 : 1];
  __shared__ uint32_t s_vtile[kExpand ? kMaxViews + 1 : 1];

  const uint32_t t = threadIdx.x;
  const bool d31 = a.drop31 != 0;
  const Chunk ch = chunk_of(a);
  const uint32_t m = ch.m, beg = ch.beg, end = ch.end;
  if constexpr (kExpand) {
    for (uint32_t v = t; v <= a.nv; v += kThreads) {
      s_vrec[v] = a.vrec_begin[v];
      s_vtile[v] = a.vtile_begin[v];
    }
  }
  {
    uint4* z = reinterpret_cast<uint4*>(sm.wh);
    for (uint32_t i = t; i < S::kWhBytes / 16; i += kThreads) z[i] = make_uint4(0, 0, 0, 0);
  }
  // (chunk_bases starts and ends with a block barrier)
  if constexpr (kVals)  // the first tile's values, while the histogram is built
    if (t == 0 && end > beg) prefetch_l2(vin + beg, static_cast<uint64_t>(min(kTileKeys, end - beg)) * 4);
  chunk_bases<K, S::kBins, kThreads>(kin, a, beg, end, d31, sm.base, sm.lstart, s_warp, s_vtile);
  if (t == 0 && end > beg)  // the first tile's keys again: phase 1 read the whole chunk since
    prefetch_l2(kin + beg, static_cast<uint64_t>(min(kTileKeys, end - beg)) * sizeof(K));

  // ---- phase 3: stable rank + scatter, tile by tile; while a tile is
  // processed, the next one's keys and values are prefetched into L2
  bool ok = true;
  const uint32_t len = end - beg;
  const uint32_t full = len / kTileKeys;
  for (uint32_t i = 0; i < full; ++i) {
    const uint32_t tb = beg + i * kTileKeys;
    if (t == 0 && tb + kTileKeys < end) {
      const uint32_t cnt = min(kTileKeys, end - (tb + kTileKeys));
      prefetch_l2(kin + tb + kTileKeys, static_cast<uint64_t>(cnt) * sizeof(K));
      if constexpr (kVals) prefetch_l2(vin + tb + kTileKeys, static_cast<uint64_t>(cnt) * 4);
    }
    ok &= rank_and_scatter<true, S, K, kVals, kExpand, kBits, kItems>(
        kin + tb, kVals ? vin + tb : nullptr, kTileKeys, m, a, d31, sm, s_warp, s_vrec, s_vtile, kout_raw, vout);
  }
  const uint32_t rest = len - full * kTileKeys;
  if (rest) {
    const uint32_t tb = beg + full * kTileKeys;
    ok &= rank_and_scatter<false, S, K, kVals, kExpand, kBits, kItems>(
        kin + tb, kVals ? vin + tb : nullptr, rest, m, a, d31, sm, s_warp, s_vrec, s_vtile, kout_raw, vout);
  }
  if (!ok) latch_error(a.err, TDGS_ERR_CAPACITY, kSiteRadixRange);
  if constexpr (kExpand) {
    if (a.rmin && a.ranges) {
      grid_barrier(a.bar, a.err);  // every tile's first and last position is recorded
      for (uint32_t tt = blockIdx.x * kThreads + t; tt < a.t_all; tt += gridDim.x * kThreads) {
        const uint32_t lo = __ldcg(a.rmin + tt);
        if (lo == 0xffffffffu) {
          a.ranges[tt] = make_uint2(0u, 0u);
        } else {
          const uint32_t pb = a.pbeg[a.nv == 1 ? 0u : find_view(s_vtile, a.nv, tt)];
          a.ranges[tt] = make_uint2(lo - pb, __ldcg(a.rmax + tt) - pb);
          a.rmin[tt] = 0xffffffffu;  // back to the empty state for the next frame
          a.rmax[tt] = 0u;
        }
      }
    }
  }
}

// --------------------------------------------------------------- host side
struct Kernel {
  const void* fn;     // the __global__ function
  int bits, threads, items;
  size_t smem;
  int min_blocks;
};

template <typename K, bool kVals, bool kExpand, int kBits, int kThreads, int kItems, int kOcc = 0>
Kernel make_kernel() {
  using S = PassShape<K, kVals, kExpand, kBits, kThreads, kItems, kOcc>;
  return Kernel{reinterpret_cast<const void*>(&k_radix_pass<K, kVals, kExpand, kBits, kThreads, kItems, kOcc>),
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
