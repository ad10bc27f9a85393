// Depth sort of the frame path in one cooperative launch (Sec. II-A,
// Sorting: a frame's Gaussians ordered by depth before their pairs are
// emitted), followed by the exclusive scan of their tile counts in that
// order (the first pair of every Gaussian).
//
// The N depth keys (raw float bits; all ones for a Gaussian without pairs)
// are compressed to key - smallest (all ones -> one past the largest) and
// sorted stably, least significant digit first, with as many digits of at
// most 9 bits as the compressed range needs.  One CTA of 512 threads per SM
// owns one chunk of at most 8192 keys and ranks it in shared memory in
// every pass (radix::rank_tile).
//
// A chunk's output base per digit = the keys of smaller digits (all
// chunks) + the keys of that digit in the chunks before it.  Neither needs
// a column scan between two grid barriers here:
//  * Digit totals.  Pass 0 adds each chunk's counts of every pass's digit
//    into per-pass totals (global atomics) before the launch's one extra
//    grid barrier; later passes find their totals ready.
//  * Chunk counts.  Each chunk publishes its 512 digit counts as one 1 KB
//    row of 16-bit words (14-bit count, 2-bit launch tag).  Chunk c reads
//    rows 0..c-1 if it lies in the first half of the grid, else rows
//    c+1..G-1, which it subtracts with its own counts from the totals: no
//    CTA reads more than half of the rows, and it waits for those rows
//    only (their tags), not for a barrier.
//  * One grid barrier ends each pass: the next pass reads what every CTA
//    wrote.
// The value that travels with a key is the record index (22 bits) with the
// Gaussian's tile count in the top 10 bits (1023: at least that many, the
// count is read again at the end), loaded in order in pass 0.  The last
// pass writes the sorted record indices and, at each sorted position, the
// tile count (the sorted keys are not needed later): no gather of the
// counts in depth order.  After the final barrier each chunk sums its counts, publishes
// the sum tagged with the launch number and adds the sums of the chunks
// before it: the pair offsets, with no further barrier.
//
// A barrier is an arrival counter of its own: a CTA adds one with release
// semantics and waits (acquire, bounded) until the count reaches the grid
// size.  The counters used mid-launch are reset after the final barrier,
// the final one at the start of the next launch.  State kept between
// launches (counters, totals, rows, launch number) lives in a dedicated
// zero-initialised buffer, which the host clears again after an error was
// latched on the device.
#include "radix.cuh"

namespace tdgs {
namespace depth {

constexpr int kThreads = 512, kItems = 16, kBits = 9;
constexpr uint32_t kBins = 1u << kBits;
constexpr uint32_t kWarps = kThreads / 32;
constexpr uint32_t kMaxPasses = 4;  // 32 key bits in digits of at most 9
constexpr uint32_t kMaxGrid = radix::kMaxGrid;  // chunks (CTAs) at most
constexpr uint32_t kValueBits = 22; // record indices below 2^22 (N <= kMaxGrid * 8192)
constexpr uint32_t kRecMask = (1u << kValueBits) - 1u;
constexpr uint32_t kCntEscape = (1u << (32 - kValueBits)) - 1u;  // 1023: the count is gathered again
using S = radix::PassShape<uint32_t, true, false, kBits, kThreads, kItems, 1>;
constexpr uint32_t kTileKeys = S::kTileKeys;
static_assert(kTileKeys == 8192, "one 8192-key chunk per CTA");
static_assert(kTileKeys < (1u << 14), "a chunk's count of one digit fits 14 bits");
static_assert(static_cast<uint64_t>(kMaxGrid) * kTileKeys <= (1ull << kValueBits), "record index bits");
static_assert(kThreads == static_cast<int>(kBins), "one digit per thread in the base computation");

// Scratch layout (uint32 words).
constexpr uint32_t kLine = 32;                      // one 128-byte line
constexpr uint32_t kSlots = 8;                      // barrier counters, one line each
constexpr uint32_t kFinalSlot = kSlots - 1;         // before the offsets
constexpr uint32_t kSeqWord = kSlots * kLine;       // launch number
constexpr uint32_t kHistWord = kSeqWord + kLine;    // [kMaxPasses][kBins] digit totals
constexpr uint32_t kSumWord = kHistWord + kMaxPasses * kBins;  // [kMaxGrid] u64 tagged chunk sums
constexpr uint32_t kRowWord = kSumWord + 2 * kMaxGrid;         // [kMaxPasses][G][kBins / 2] rows
constexpr uint32_t kRowWords = kBins / 2;
constexpr uint32_t kRowGroups = kThreads / (kBins / 8);        // rows read in parallel (8)
constexpr uint32_t kRowBatch = 10;                             // rows per thread in flight
static_assert(kSlots >= kMaxPasses + 1, "pass 0's barrier, the ends of passes 0..P-2 and the final one");
static_assert(kRowWord % 4 == 0 && kSumWord % 2 == 0, "aligned rows and sums");

__device__ __forceinline__ void red_release_add(uint32_t* p, uint32_t v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint4 ld_relaxed_v4(const uint32_t* p) {
  uint4 v;
  asm volatile("ld.relaxed.gpu.global.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p)
               : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_v4(uint32_t* p, uint4 v) {
  asm volatile("st.relaxed.gpu.global.v4.u32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w)
               : "memory");
}
__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(uint64_t* p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Grid barrier on a counter used once per launch (bounded wait).
__device__ __forceinline__ void arrive_and_wait(uint32_t* slot, uint32_t grid, uint32_t* err) {
  __syncthreads();
  if (threadIdx.x == 0) {
    red_release_add(slot, 1u);
    uint32_t spins = 0;
    while (radix::ld_acquire32(slot) < grid) {
      if (++spins > kSpinLimit) {
        latch_error(err, TDGS_ERR_TIMEOUT, kSiteBarrier);
        break;
      }
      __nanosleep(20);
    }
  }
  __syncthreads();
}

// A row word holds two 16-bit counts, each tagged in its top two bits.
__device__ __forceinline__ bool row_ready(const uint4& w, uint32_t tag2) {
  return ((w.x & 0xc000c000u) == tag2) & ((w.y & 0xc000c000u) == tag2) & ((w.z & 0xc000c000u) == tag2) &
         ((w.w & 0xc000c000u) == tag2);
}

// Sum of bins 8q..8q+7 over rows r_lo + g, r_lo + g + kRowGroups, ... < r_hi
// of one pass, waiting (bounded) until each row carries this launch's tag.
__device__ __forceinline__ void sum_rows(const uint32_t* __restrict__ rows, uint32_t r_lo, uint32_t r_hi,
                                         uint32_t g, uint32_t q, uint32_t tag2, uint32_t acc[8], uint32_t* err) {
  for (uint32_t r0 = r_lo + g; r0 < r_hi; r0 += kRowGroups * kRowBatch) {
    uint4 w[kRowBatch];
    uint32_t pend = 0;
#pragma unroll
    for (uint32_t i = 0; i < kRowBatch; ++i) {
      const uint32_t r = r0 + i * kRowGroups;
      w[i] = make_uint4(tag2, tag2, tag2, tag2);  // rows past the range count zero
      if (r < r_hi) w[i] = ld_relaxed_v4(rows + static_cast<size_t>(r) * kRowWords + 4 * q);
      if (!row_ready(w[i], tag2)) pend |= 1u << i;
    }
    uint32_t spins = 0;
    while (pend) {
      if (++spins > kSpinLimit) {
        latch_error(err, TDGS_ERR_TIMEOUT, kSiteBarrier);
        break;
      }
      __nanosleep(32);
#pragma unroll
      for (uint32_t i = 0; i < kRowBatch; ++i) {
        if (pend & (1u << i)) {
          w[i] = ld_relaxed_v4(rows + static_cast<size_t>(r0 + i * kRowGroups) * kRowWords + 4 * q);
          if (row_ready(w[i], tag2)) pend &= ~(1u << i);
        }
      }
    }
#pragma unroll
    for (uint32_t i = 0; i < kRowBatch; ++i) {
      const uint32_t x[4] = {w[i].x, w[i].y, w[i].z, w[i].w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc[2 * u] += x[u] & 0x3fffu;
        acc[2 * u + 1] += (x[u] >> 16) & 0x3fffu;
      }
    }
  }
}

__global__ void __launch_bounds__(kThreads, 1)
    k_depth_sort(const uint32_t* __restrict__ key0, uint32_t* __restrict__ k1, uint32_t* __restrict__ v1,
                 uint32_t* __restrict__ k2, uint32_t* __restrict__ v2, const uint32_t* __restrict__ counts,
                 uint32_t* __restrict__ offsets, uint32_t* __restrict__ range, uint32_t n,
                 uint32_t* __restrict__ scratch, uint32_t* __restrict__ err) {
  extern __shared__ __align__(16) unsigned char smem[];
  radix::Smem<uint32_t> sm;
  {
    unsigned char* p = smem;
    sm.wh = reinterpret_cast<uint16_t*>(p);
    p += S::kWhBytes;
    sm.xk = reinterpret_cast<uint32_t*>(p);
    p += S::kXkBytes;
    sm.xv = reinterpret_cast<uint32_t*>(p);
    p += S::kXvBytes;
    sm.base = reinterpret_cast<uint32_t*>(p);
    sm.lstart = sm.base + kBins;
    sm.off = sm.lstart + kBins;
  }
  // the row sums of the groups share the value exchange buffer (not live then)
  uint32_t* s_part = sm.xv;
  static_assert(S::kXvBytes >= kRowGroups * kBins * 4, "row-sum partials fit the value exchange");
  __shared__ uint32_t s_hx[kMaxPasses - 1][kBins];  // pass 0: this chunk's counts of the later digits
  __shared__ uint32_t s_warp[kWarps];
  __shared__ unsigned long long s_sum[kWarps];
  __shared__ unsigned long long s_base;
  const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5, c = blockIdx.x, G = gridDim.x;
  const uint32_t Sz = ((n + G - 1) / G + 3) & ~3u;
  const uint32_t beg = min(c * Sz, n), end = min(beg + Sz, n);
  uint32_t valid = end - beg;
  bool ok = valid <= kTileKeys;  // guaranteed by the host
  if (!ok) valid = kTileKeys;
  {
    uint4* z = reinterpret_cast<uint4*>(sm.wh);
    for (uint32_t i = t; i < S::kWhBytes / 16; i += kThreads) z[i] = make_uint4(0, 0, 0, 0);
    for (uint32_t i = t; i < (kMaxPasses - 1) * kBins; i += kThreads) (&s_hx[0][0])[i] = 0u;
  }
  uint32_t* hist = scratch + kHistWord;
  uint64_t* sums = reinterpret_cast<uint64_t*>(scratch + kSumWord);
  uint32_t* rows = scratch + kRowWord;
  const uint32_t seq = __ldcg(scratch + kSeqWord);
  const uint32_t tag2 = (seq % 3u + 1u) * 0x40004000u;
  const uint32_t tag16 = (seq % 3u + 1u) << 14;
  const uint64_t tag32 = static_cast<uint64_t>((seq & 0x7fffffffu) + 1u) << 32;
  // digits from the compressed range
  const uint32_t lo = __ldcg(range), hi = __ldcg(range + 1);
  const uint32_t cull = hi >= lo ? hi - lo + 1u : 0u;  // compressed keys are 0 .. cull
  const uint32_t bits = cull ? 32u - static_cast<uint32_t>(__clz(cull)) : 0u;
  const uint32_t passes = bits ? (bits + kBits - 1) / kBits : 1u;
  const uint32_t width = (bits + passes - 1) / passes;
  const uint32_t mask = width ? (1u << width) - 1u : 0u;
  if (c == 0 && t == 0) {
    range[2] = passes;
    scratch[kFinalSlot * kLine] = 0u;  // the previous launch's final barrier
  }
  radix::PassArgs a{};
  a.m = n;
  a.sub = lo;
  a.cull = cull;
  a.mask = mask;
  a.err = err;
  __syncthreads();
  const uint32_t g = t / (kBins / 8), q = t % (kBins / 8);  // row group, column of 8 bins
  const bool low_half = c < G / 2;
  for (uint32_t p = 0; p < passes; ++p) {
    const bool last = p + 1 == passes;
    // pass p reads pair (p - 1) and writes pair p; the last pass writes (k1, v1)
    const bool to_one = ((passes - 1 - p) & 1u) == 0;
    const uint32_t* kin = p == 0 ? key0 : (to_one ? k2 : k1);
    const uint32_t* vin = to_one ? v2 : v1;
    uint32_t* kout = to_one ? k1 : k2;
    uint32_t* vout = to_one ? v1 : v2;
    a.shift = p * width;
    a.xform_in = p == 0;
    radix::TileRegs<uint32_t, false, kItems> R;
    radix::rank_tile<false, S, uint32_t, false, kBits, kItems, true>(kin + beg, valid, a, false, sm, R);
    // publish this chunk's digit counts (lstart) as a tagged row
    if (t < kBins / 8) {
      const uint32_t* ls = sm.lstart + 8 * t;
      uint4 w;
      w.x = (ls[0] | tag16) | ((ls[1] | tag16) << 16);
      w.y = (ls[2] | tag16) | ((ls[3] | tag16) << 16);
      w.z = (ls[4] | tag16) | ((ls[5] | tag16) << 16);
      w.w = (ls[6] | tag16) | ((ls[7] | tag16) << 16);
      st_relaxed_v4(rows + (static_cast<size_t>(p) * G + c) * kRowWords + 4 * t, w);
    }
    if (p == 0) {
      // every pass's digit totals, ready after one grid barrier
      const uint32_t wbase = warp * 32 * kItems;
      for (uint32_t pp = 1; pp < passes; ++pp) {
#pragma unroll
        for (int j = 0; j < kItems; ++j)
          if (wbase + j * 32 + lane < valid) atomicAdd(&s_hx[pp - 1][(R.k[j] >> (pp * width)) & mask], 1u);
      }
      __syncthreads();
      if (sm.lstart[t]) atomicAdd(hist + t, sm.lstart[t]);
      for (uint32_t pp = 1; pp < passes; ++pp)
        if (s_hx[pp - 1][t]) atomicAdd(hist + pp * kBins + t, s_hx[pp - 1][t]);
      arrive_and_wait(scratch, G, err);
    }
    // output base per digit: keys of smaller digits + this digit's keys in
    // the chunks before this one
    {
      const uint32_t tot = __ldcg(hist + p * kBins + t);
      const uint32_t own = sm.lstart[t];
      uint32_t acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      sum_rows(rows + static_cast<size_t>(p) * G * kRowWords, low_half ? 0u : c + 1, low_half ? c : G, g, q,
               tag2, acc, err);
#pragma unroll
      for (int i = 0; i < 8; ++i) s_part[g * kBins + 8 * q + i] = acc[i];
      __syncthreads();
      uint32_t sum = 0;
#pragma unroll
      for (uint32_t gg = 0; gg < kRowGroups; ++gg) sum += s_part[gg * kBins + t];
      const uint32_t before = low_half ? sum : tot - own - sum;
      const uint32_t start = radix::block_excl_scan<kWarps>(tot, s_warp);
      sm.base[t] = start + before;
      __syncthreads();
    }
    // tile-local digit starts, exchange into digit order, coalesced scatter
    radix::digit_starts<S, uint32_t>(sm, s_warp);
    __syncthreads();
    const uint32_t wbase = warp * 32 * kItems;
    uint16_t* my_wh = sm.wh + warp * kBins;
#pragma unroll
    for (int j = 0; j < kItems; ++j) R.r[j] += sm.lstart[R.d[j]] + my_wh[R.d[j]];
    __syncwarp();
    {
      uint4* z = reinterpret_cast<uint4*>(my_wh);
      for (uint32_t i = lane; i < kBins / 8; i += 32) z[i] = make_uint4(0, 0, 0, 0);
    }
    if (!last) {
#pragma unroll
      for (int j = 0; j < kItems; ++j)
        if (wbase + j * 32 + lane < valid) sm.xk[R.r[j]] = R.k[j];
      uint32_t v[kItems];
#pragma unroll
      for (int j = 0; j < kItems; ++j) {
        const uint32_t idx = wbase + j * 32 + lane;
        v[j] = 0u;
        if (idx < valid) {
          if (p == 0)
            v[j] = (beg + idx) | (min(__ldg(counts + beg + idx), kCntEscape) << kValueBits);
          else
            v[j] = __ldcs(vin + beg + idx);
        }
      }
      __syncthreads();
      uint32_t dst[kItems];
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        const uint32_t pos = i * kThreads + t;
        dst[i] = 0xffffffffu;
        if (pos < valid) {
          const uint32_t key = sm.xk[pos];
          dst[i] = sm.off[(key >> a.shift) & mask] + pos;
          if (dst[i] < n)
            kout[dst[i]] = key;
          else
            ok = false;
        }
      }
#pragma unroll
      for (int j = 0; j < kItems; ++j)
        if (wbase + j * 32 + lane < valid) sm.xv[R.r[j]] = v[j];
      __syncthreads();
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        const uint32_t pos = i * kThreads + t;
        if (pos < valid && dst[i] < n) vout[dst[i]] = sm.xv[pos];
      }
      arrive_and_wait(scratch + (1 + p) * kLine, G, err);
    } else {
      // (digit, value) in one 8-byte exchange over both exchange buffers;
      // each sorted position gets its record index (v1) and that
      // Gaussian's tile count (k1)
      uint32_t v[kItems];
#pragma unroll
      for (int j = 0; j < kItems; ++j) {
        const uint32_t idx = wbase + j * 32 + lane;
        v[j] = 0u;
        if (idx < valid) {
          if (p == 0)
            v[j] = (beg + idx) | (min(__ldg(counts + beg + idx), kCntEscape) << kValueBits);
          else
            v[j] = __ldcs(vin + beg + idx);
        }
      }
      uint64_t* x64 = reinterpret_cast<uint64_t*>(sm.xk);
      static_assert(S::kXkBytes + S::kXvBytes >= kTileKeys * 8, "the 8-byte exchange spans both buffers");
#pragma unroll
      for (int j = 0; j < kItems; ++j)
        if (wbase + j * 32 + lane < valid) x64[R.r[j]] = (static_cast<uint64_t>(R.d[j]) << 32) | v[j];
      __syncthreads();
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        const uint32_t pos = i * kThreads + t;
        if (pos < valid) {
          const uint64_t x = x64[pos];
          const uint32_t w = static_cast<uint32_t>(x), rec = w & kRecMask;
          const uint32_t dst = sm.off[static_cast<uint32_t>(x >> 32)] + pos;
          if (dst < n && rec < n) {
            uint32_t cnt = w >> kValueBits;
            if (cnt == kCntEscape) cnt = __ldg(counts + rec);
            v1[dst] = rec;
            k1[dst] = cnt;
          } else {
            ok = false;
          }
        }
      }
      arrive_and_wait(scratch + kFinalSlot * kLine, G, err);
    }
  }
  if (!ok) latch_error(err, TDGS_ERR_CAPACITY, kSiteRadixRange);
  // The pair offsets: counts in depth order (k1) scanned; kItems consecutive
  // positions per thread, chunk sums by a tagged look-back.
  {
    static_assert(kItems % 4 == 0, "16-byte loads of the counts");
    const uint32_t pos0 = beg + t * kItems;
    uint32_t cnt[kItems];
    uint64_t sum = 0;
#pragma unroll
    for (int j = 0; j < kItems; j += 4) {
      uint4 x = make_uint4(0, 0, 0, 0);
      if (pos0 + j + 4 <= end) {
        x = __ldcg(reinterpret_cast<const uint4*>(k1 + pos0 + j));
      } else {
        if (pos0 + j < end) x.x = __ldcg(k1 + pos0 + j);
        if (pos0 + j + 1 < end) x.y = __ldcg(k1 + pos0 + j + 1);
        if (pos0 + j + 2 < end) x.z = __ldcg(k1 + pos0 + j + 2);
      }
      cnt[j] = x.x;
      cnt[j + 1] = x.y;
      cnt[j + 2] = x.z;
      cnt[j + 3] = x.w;
      sum += static_cast<uint64_t>(x.x) + x.y + x.z + x.w;
    }
    unsigned long long xs = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const unsigned long long o = __shfl_up_sync(0xffffffffu, xs, d);
      if (lane >= static_cast<uint32_t>(d)) xs += o;
    }
    if (lane == 31) s_sum[warp] = xs;
    __syncthreads();
    if (t == 0) {
      unsigned long long run = 0;
      for (uint32_t w = 0; w < kWarps; ++w) {
        const unsigned long long v = s_sum[w];
        s_sum[w] = run;
        run += v;
      }
      // this chunk's sum for the chunks after it (saturated: an overflow
      // is latched below)
      st_relaxed_u64(sums + c, tag32 | (run > 0xffffffffull ? 0xffffffffull : run));
      s_base = run;
    }
    __syncthreads();
    const uint64_t csum = s_base;
    uint64_t run = xs - sum + s_sum[warp];
    __syncthreads();
    if (warp == 0) {
      // all sums of the chunks before this one in flight at once, then the
      // ones not yet published again (bounded)
      constexpr uint32_t kPer = kMaxGrid / 32;
      uint64_t w[kPer];
      uint32_t pend = 0;
#pragma unroll
      for (uint32_t i = 0; i < kPer; ++i) {
        const uint32_t cc = lane + 32 * i;
        w[i] = tag32;
        if (cc < c) {
          w[i] = ld_relaxed_u64(sums + cc);
          if ((w[i] & 0xffffffff00000000ull) != tag32) pend |= 1u << i;
        }
      }
      uint32_t spins = 0;
      while (pend) {
        if (++spins > kSpinLimit) {
          latch_error(err, TDGS_ERR_TIMEOUT, kSiteBarrier);
          break;
        }
        __nanosleep(32);
#pragma unroll
        for (uint32_t i = 0; i < kPer; ++i) {
          if (pend & (1u << i)) {
            w[i] = ld_relaxed_u64(sums + lane + 32 * i);
            if ((w[i] & 0xffffffff00000000ull) == tag32) pend &= ~(1u << i);
          }
        }
      }
      unsigned long long before = 0;
#pragma unroll
      for (uint32_t i = 0; i < kPer; ++i) before += w[i] & 0xffffffffull;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) before += __shfl_xor_sync(0xffffffffu, before, d);
      if (lane == 0) s_base = before;
    }
    __syncthreads();
    run += s_base;
    if (t == 0 && s_base + csum > 0xffffffffull) latch_error(err, TDGS_ERR_OVERFLOW, kSiteScan);
#pragma unroll
    for (int j = 0; j < kItems; j += 4) {
      uint32_t o[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        o[u] = static_cast<uint32_t>(run);
        run += cnt[j + u];
      }
      if (pos0 + j + 4 <= end) {
        *reinterpret_cast<uint4*>(offsets + pos0 + j) = make_uint4(o[0], o[1], o[2], o[3]);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (pos0 + j + u < end) offsets[pos0 + j + u] = o[u];
      }
    }
  }
  // Reset for the next launch (every reader of these is past the final
  // barrier): this chunk's rows; CTA 0 the totals, the mid-launch counters
  // and the launch number.
  for (uint32_t i = t; i < passes * (kRowWords / 4); i += kThreads) {
    const uint32_t pp = i / (kRowWords / 4), w = i % (kRowWords / 4);
    reinterpret_cast<uint4*>(rows + (static_cast<size_t>(pp) * G + c) * kRowWords)[w] = make_uint4(0, 0, 0, 0);
  }
  if (c == 0) {
    for (uint32_t i = t; i < passes * kBins; i += kThreads) hist[i] = 0u;
    if (t < passes) scratch[t * kLine] = 0u;  // slots 0 .. passes-1
    if (t == 0) scratch[kSeqWord] = seq + 1u;
  }
}

}  // namespace depth

// ------------------------------------------------------------- host side
uint32_t depth_sort_grid() {
  static const radix::Kernel k{reinterpret_cast<const void*>(&depth::k_depth_sort), depth::kBits, depth::kThreads,
                               depth::kItems, depth::S::kSmem, 1};
  uint32_t g = radix::resident_ctas(k, 1);
  return g > radix::kMaxGrid ? radix::kMaxGrid : g;
}

uint32_t depth_sort_capacity(uint32_t grid) {
  // chunks of ceil(n / G) keys rounded up to a multiple of 4 fit one tile
  // (8192, itself a multiple of 4) exactly when n <= G * 8192
  return grid * depth::kTileKeys;
}

size_t depth_sort_scratch_words(uint32_t grid) {
  return depth::kRowWord + static_cast<size_t>(depth::kMaxPasses) * grid * depth::kRowWords;
}

cudaError_t launch_depth_sort(uint32_t grid, const uint32_t* key0, uint32_t* k1, uint32_t* v1, uint32_t* k2,
                              uint32_t* v2, uint32_t* range, const uint32_t* counts, uint32_t* offsets, uint32_t n,
                              uint32_t* scratch, uint32_t* err, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  if (grid == 0 || grid > radix::kMaxGrid || n > depth_sort_capacity(grid)) return cudaErrorInvalidConfiguration;
  void* args[] = {(void*)&key0, (void*)&k1, (void*)&v1, (void*)&k2, (void*)&v2, (void*)&counts,
                  (void*)&offsets, (void*)&range, (void*)&n, (void*)&scratch, (void*)&err};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(depth::kThreads);
  cfg.dynamicSmemBytes = depth::S::kSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(&depth::k_depth_sort), args);
}

}  // namespace tdgs
