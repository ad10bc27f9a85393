// Depth sort of the frame path in one cooperative launch (Sec. II-A,
// Sorting: a frame's Gaussians ordered by depth before their pairs are
// emitted), followed by the exclusive scan of their tile counts in that
// order (the first pair of every Gaussian).  Two forms, both with one
// 8192-key tile per CTA (larger frames take the onesweep passes over the
// same compressed keys, onesweep.cu):
//  * k_depth_sort<true>: the tile count step first (records in, keys kept
//    in registers), then the sort.
//  * k_depth_sort<false>: keys and counts from the count kernel.
//
// The N depth keys (raw float bits; all ones for a Gaussian without pairs)
// are compressed to key - smallest (all ones -> one past the largest) and
// sorted stably, least significant digit first, with as many digits of at
// most 9 bits as the compressed range needs.  One CTA of 512 threads per SM
// owns one chunk (one tile) and ranks it in shared memory in every pass
// (radix::rank_keys).
//
// A chunk's output base per digit = the keys of smaller digits (all
// chunks) + the keys of that digit in the chunks before it.  Neither needs
// a column scan between two grid barriers here:
//  * Digit totals.  Pass 0 adds each chunk's counts of every later pass's
//    digit into per-pass totals (global atomics); they are complete at pass
//    0's end.  Pass 0's own totals come from the count step's histogram of
//    the keys' low 9 bits (digit 0 of key - smallest is a rotation of it),
//    or, without the count step, from the same atomics and one extra grid
//    barrier.
//  * Chunk counts.  Each chunk publishes its 512 digit counts as one 1 KB
//    row of 16-bit words holding count + 1 (rows are zero between
//    launches, so 0 means "not written yet").  Chunk c reads rows 0..c-1 if
//    it lies in the first half of the grid, else rows c+1..G-1, which it
//    subtracts with its own counts from the totals: no CTA reads more than
//    half of the rows, and it waits for those rows only, not for a barrier.
//  * One grid barrier ends each pass: the next pass reads what every CTA
//    wrote.
// The value that travels with a key is the record index (22 bits) with the
// Gaussian's tile count in the top 10 bits (1023: at least that many, the
// count is read again at the end), made in pass 0.  The last pass writes
// the sorted record indices and, at each sorted position, the tile count
// (the sorted keys are not needed later): no gather of the counts in depth
// order.  Output positions grow with the exchange position, so each warp
// adds the counts it writes into per-chunk sums by runs of equal chunk (a
// lane scan; a run's last lane adds, its first lane subtracts); the sums
// reach global memory by atomics before the final barrier, after which
// each chunk scans its counts from the sum of the chunks before it: the
// pair offsets.
//
// Each tile's values (pass 0: the tile counts) come into shared memory by
// one bulk copy issued before the tile is ranked, so their latency hides
// behind the ranking; keys and values cross the exchange as one 8-byte
// word.
//
// A barrier is an arrival counter of its own: a CTA adds one with release
// semantics and waits (acquire, bounded) until the count reaches the grid
// size.  The counters used mid-launch are reset after the final barrier,
// the final one at the start of the next launch.  State kept between
// launches (counters, totals, rows, histogram) lives in a dedicated
// zero-initialised buffer, which the host clears again after an error was
// latched on the device.
#include "onesweep.cuh"

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
constexpr size_t kSmem = S::kSmem + kTileKeys * 4;  // + the staged values
static_assert(S::kSmem % 16 == 0, "the staged values start 16-byte aligned");
static_assert(kTileKeys == 8192, "one 8192-key chunk per CTA");
static_assert(4 * kTileKeys + 1 < (1u << 16), "a chunk's count of one digit, plus one, fits a 16-bit row field");
static_assert(static_cast<uint64_t>(kMaxGrid) * kTileKeys <= (1ull << kValueBits), "record index bits");
static_assert(kThreads == static_cast<int>(kBins), "one digit per thread in the base computation");

// Scratch layout (uint32 words).
constexpr uint32_t kLine = 32;                      // one 128-byte line
constexpr uint32_t kSlots = 8;                      // barrier counters, one line each
constexpr uint32_t kFinalSlot = kSlots - 1;         // before the offsets
constexpr uint32_t kHistWord = kSlots * kLine;      // [kMaxPasses][kBins] digit totals
constexpr uint32_t kRawWord = kHistWord + kMaxPasses * kBins;  // fused count: [kBins] keys by low 9 bits, culled
constexpr uint32_t kSumWord = kRawWord + kBins + kLine;          // [kMaxGrid] counts per output chunk
constexpr uint32_t kRowWord = kSumWord + kMaxGrid;             // [kMaxPasses][G][kBins / 2] rows
constexpr uint32_t kRowWords = kBins / 2;
constexpr uint32_t kRowGroups = kThreads / (kBins / 8);        // rows read in parallel (8)
constexpr uint32_t kRowBatch = 10;                             // rows per thread in flight
static_assert(kSlots >= kMaxPasses + 1, "pass 0's barrier, the ends of passes 0..P-2 and the final one");
static_assert(kRowWord % 4 == 0, "16-byte aligned rows");

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

// Exclusive sums of (a, b) over the CTA, both at once (the caller
// synchronises before s_w2 is used again).
__device__ __forceinline__ uint2 excl_scan2(uint32_t a, uint32_t b, uint2* s_w2) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  uint32_t x = a, y = b;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const uint32_t xo = __shfl_up_sync(0xffffffffu, x, d), yo = __shfl_up_sync(0xffffffffu, y, d);
    if (lane >= static_cast<uint32_t>(d)) {
      x += xo;
      y += yo;
    }
  }
  if (lane == 31) s_w2[warp] = make_uint2(x, y);
  __syncthreads();
  if (warp == 0) {
    uint2 w = lane < kWarps ? s_w2[lane] : make_uint2(0u, 0u);
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t xo = __shfl_up_sync(0xffffffffu, w.x, d), yo = __shfl_up_sync(0xffffffffu, w.y, d);
      if (lane >= static_cast<uint32_t>(d)) {
        w.x += xo;
        w.y += yo;
      }
    }
    if (lane < kWarps) s_w2[lane] = w;
  }
  __syncthreads();
  const uint2 before = warp ? s_w2[warp - 1] : make_uint2(0u, 0u);
  return make_uint2(x - a + before.x, y - b + before.y);
}

// A row word holds two 16-bit fields, count + 1 each (0: not written yet;
// rows are zero between launches).
__device__ __forceinline__ bool row_ready(const uint4& w) {
  return (__vcmpeq2(w.x, 0u) | __vcmpeq2(w.y, 0u) | __vcmpeq2(w.z, 0u) | __vcmpeq2(w.w, 0u)) == 0u;
}

// Sum of bins 8q..8q+7 over rows r_lo + g, r_lo + g + kRowGroups, ... < r_hi
// of one pass, waiting (bounded) until each row is written.
__device__ __forceinline__ void sum_rows(const uint32_t* __restrict__ rows, uint32_t r_lo, uint32_t r_hi,
                                         uint32_t g, uint32_t q, uint32_t acc[8], uint32_t* err) {
  for (uint32_t r0 = r_lo + g; r0 < r_hi; r0 += kRowGroups * kRowBatch) {
    uint4 w[kRowBatch];
    uint32_t pend = 0;
#pragma unroll
    for (uint32_t i = 0; i < kRowBatch; ++i) {
      const uint32_t r = r0 + i * kRowGroups;
      w[i] = make_uint4(0x10001u, 0x10001u, 0x10001u, 0x10001u);  // rows past the range count zero
      if (r < r_hi) w[i] = ld_relaxed_v4(rows + static_cast<size_t>(r) * kRowWords + 4 * q);
      if (!row_ready(w[i])) pend |= 1u << i;
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
          if (row_ready(w[i])) pend &= ~(1u << i);
        }
      }
    }
#pragma unroll
    for (uint32_t i = 0; i < kRowBatch; ++i) {
      const uint32_t x[4] = {w[i].x, w[i].y, w[i].z, w[i].w};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        acc[2 * u] += (x[u] & 0xffffu) - 1u;
        acc[2 * u + 1] += (x[u] >> 16) - 1u;
      }
    }
  }
}

// One ranked tile of `valid` keys (tile items start at record tb; item j of
// this thread goes to tile position pos[j]): the (key, value) -- in the
// last pass (digit, value); hi[j] is the key or the digit -- exchange
// through shared memory, and the scatter to off[digit] + tile position.
// Values come from vstage (items below nstaged) or vsrc + tb;
// pass 0 (first) makes each value the record index with the tile count in
// its top bits.  The last pass writes v1 (record index) and k1 (count) and
// adds the counts it writes into the per-output-chunk sums csum (chunks of
// Sz positions; vstage is free by then and holds per-warp sums).  Returns
// false if a destination fell outside [0, n).  Ends with a block barrier.
__device__ __forceinline__ bool exchange_scatter(const radix::Smem<uint32_t>& sm, uint32_t* vstage,
                                                 const uint32_t (&hi)[kItems], const uint32_t (&pos)[kItems],
                                                 uint32_t valid,
                                                 uint32_t tb, uint32_t nstaged, const uint32_t* vsrc, bool first,
                                                 bool last, uint32_t shift, uint32_t mask, uint32_t n,
                                                 uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                                                 uint32_t* __restrict__ k1, uint32_t* __restrict__ v1,
                                                 const uint32_t* __restrict__ counts, uint32_t Sz, uint32_t G,
                                                 uint32_t* __restrict__ csum) {
  const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;
  bool ok = true;
  const uint32_t wbase = warp * 32 * kItems;
  // (key, value) -- in the last pass (digit, value) -- in one 8-byte
  // exchange over both exchange buffers
  uint32_t v[kItems];
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t idx = wbase + j * 32 + lane;
    v[j] = 0u;
    if (idx < valid) {
      const uint32_t x = idx < nstaged ? vstage[idx] : __ldg(vsrc + tb + idx);
      v[j] = first ? (tb + idx) | (min(x, kCntEscape) << kValueBits) : x;
    }
  }
  uint64_t* x64 = reinterpret_cast<uint64_t*>(sm.xk);
  static_assert(S::kXkBytes + S::kXvBytes >= kTileKeys * 8, "the 8-byte exchange spans both buffers");
#pragma unroll
  for (int j = 0; j < kItems; ++j)
    if (wbase + j * 32 + lane < valid) x64[pos[j]] = (static_cast<uint64_t>(hi[j]) << 32) | v[j];
  __syncthreads();
  if (!last) {
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const uint32_t xp = i * kThreads + t;
      if (xp < valid) {
        const uint64_t x = x64[xp];
        const uint32_t key = static_cast<uint32_t>(x >> 32);
        const uint32_t dst = sm.off[(key >> shift) & mask] + xp;
        if (dst < n) {
          kout[dst] = key;
          vout[dst] = static_cast<uint32_t>(x);
        } else {
          ok = false;
        }
      }
    }
  } else {
    // each sorted position gets its record index (v1) and that
    // Gaussian's tile count (k1); the counts are summed per output chunk
    // per-warp rows of counts per output chunk, over the staged values
    // (read before the exchange barrier above)
    static_assert(kWarps * kMaxGrid * 4 <= kTileKeys * 4, "per-warp chunk sums fit the staging buffer");
    uint32_t* w_csum = vstage + warp * kMaxGrid;
    for (uint32_t k = lane; k < G; k += 32) w_csum[k] = 0u;
    __syncwarp();
    const float inv_sz = 1.0f / static_cast<float>(Sz);
    uint32_t q[kItems], cnt[kItems];  // output chunk (all ones: none) and count per item
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const uint32_t xp = i * kThreads + t;
      q[i] = 0xffffffffu;
      cnt[i] = 0u;
      if (xp < valid) {
        const uint64_t x = x64[xp];
        const uint32_t w = static_cast<uint32_t>(x), rec = w & kRecMask;
        const uint32_t dst = sm.off[static_cast<uint32_t>(x >> 32)] + xp;
        if (dst < n && rec < n) {
          uint32_t c1 = w >> kValueBits;
          if (c1 == kCntEscape) c1 = __ldg(counts + rec);
          cnt[i] = c1;
          v1[dst] = rec;
          k1[dst] = c1;
          // dst / Sz: a float estimate (dst < 2^22 is exact) corrected by one
          uint32_t qq = static_cast<uint32_t>(static_cast<float>(dst) * inv_sz);
          if (qq * Sz > dst) --qq;
          else if ((qq + 1u) * Sz <= dst) ++qq;
          q[i] = qq;
        } else {
          ok = false;
        }
      }
    }
    // q never decreases from lane to lane, so equal chunks are runs: an
    // inclusive scan of the counts over the lanes (all items at once),
    // then a run's last lane adds its scan and its first lane subtracts
    // the scan before it (modulo 2^32, exact for every chunk sum)
    uint32_t incl[kItems];
#pragma unroll
    for (int i = 0; i < kItems; ++i) incl[i] = cnt[i];
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        const uint32_t o = __shfl_up_sync(0xffffffffu, incl[i], d);
        if (lane >= static_cast<uint32_t>(d)) incl[i] += o;
      }
    }
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      const uint32_t qp = __shfl_up_sync(0xffffffffu, q[i], 1), qn = __shfl_down_sync(0xffffffffu, q[i], 1);
      if (q[i] != 0xffffffffu) {
        if (lane == 31 || qn != q[i]) atomicAdd(&w_csum[q[i]], incl[i]);
        if (lane != 0 && qp != q[i]) atomicAdd(&w_csum[q[i]], cnt[i] - incl[i]);
      }
    }
    __syncthreads();
    for (uint32_t k = t; k < G; k += kThreads) {
      uint32_t sum = 0;
#pragma unroll
      for (uint32_t w = 0; w < kWarps; ++w) sum += vstage[w * kMaxGrid + k];
      if (sum) atomicAdd(csum + k, sum);
    }
  }
  __syncthreads();
  return ok;
}

// Sum of the chunk sums csum[0 .. c) (one warp; every lane returns it).
__device__ __forceinline__ uint64_t chunks_before(const uint32_t* csum, uint32_t c) {
  constexpr uint32_t kPer = kMaxGrid / 32;
  const uint32_t lane = lane_id();
  uint64_t before = 0;
#pragma unroll
  for (uint32_t i = 0; i < kPer; ++i) {
    const uint32_t cc = lane + 32 * i;
    if (cc < c) before += __ldcg(csum + cc);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) before += __shfl_xor_sync(0xffffffffu, before, d);
  return before;
}

// Pair offsets of positions [b, e) (at most kTileKeys; b a multiple of 4):
// the exclusive scan of the counts k1 from `base`, kItems consecutive
// positions per thread.  Returns base + their sum; a sum above 2^32 - 1
// latches TDGS_ERR_OVERFLOW.  Block barriers inside.
__device__ __forceinline__ uint64_t scan_offsets(const uint32_t* __restrict__ k1, uint32_t* __restrict__ offsets,
                                                 uint32_t b, uint32_t e, uint64_t base, unsigned long long* s_sum,
                                                 uint32_t* err) {
  static_assert(kItems % 4 == 0, "16-byte loads of the counts");
  const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;
  const uint32_t pos0 = b + t * kItems;
  uint32_t cnt[kItems];
  uint64_t sum = 0;
#pragma unroll
  for (int j = 0; j < kItems; j += 4) {
    uint4 x = make_uint4(0, 0, 0, 0);
    if (pos0 + j + 4 <= e) {
      x = __ldcg(reinterpret_cast<const uint4*>(k1 + pos0 + j));
    } else {
      if (pos0 + j < e) x.x = __ldcg(k1 + pos0 + j);
      if (pos0 + j + 1 < e) x.y = __ldcg(k1 + pos0 + j + 1);
      if (pos0 + j + 2 < e) x.z = __ldcg(k1 + pos0 + j + 2);
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
    unsigned long long run = base;
    for (uint32_t w = 0; w < kWarps; ++w) {
      const unsigned long long v = s_sum[w];
      s_sum[w] = run;
      run += v;
    }
    s_sum[kWarps] = run;
    if (run > 0xffffffffull) latch_error(err, TDGS_ERR_OVERFLOW, kSiteScan);
  }
  __syncthreads();
  uint64_t run = xs - sum + s_sum[warp];
  const uint64_t total = s_sum[kWarps];
#pragma unroll
  for (int j = 0; j < kItems; j += 4) {
    uint32_t o[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      o[u] = static_cast<uint32_t>(run);
      run += cnt[j + u];
    }
    if (pos0 + j + 4 <= e) {
      *reinterpret_cast<uint4*>(offsets + pos0 + j) = make_uint4(o[0], o[1], o[2], o[3]);
    } else {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (pos0 + j + u < e) offsets[pos0 + j + u] = o[u];
    }
  }
  __syncthreads();  // s_sum is free again
  return total;
}

// kCount: the tile count step runs first in the same launch (records of
// the view table in, keys kept in registers); else the keys come from the
// count kernel (key0) with the range it published.
template <bool kCount>
__global__ void __launch_bounds__(kThreads, 1) k_depth_sort(DepthSortArgs A) {
  const uint32_t* __restrict__ key0 = A.key0;
  uint32_t* __restrict__ k1 = A.k1;
  uint32_t* __restrict__ v1 = A.v1;
  uint32_t* __restrict__ k2 = A.k2;
  uint32_t* __restrict__ v2 = A.v2;
  uint32_t* __restrict__ counts = A.counts;
  uint32_t* __restrict__ offsets = A.offsets;
  uint32_t* __restrict__ range = A.range;
  uint32_t* __restrict__ scratch = A.scratch;
  uint32_t* __restrict__ err = A.err;
  const uint32_t n = A.n;
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
  uint32_t* vstage = reinterpret_cast<uint32_t*>(smem + S::kSmem);  // this pass's values, in chunk order
  // the row sums of the groups share the value exchange buffer (not live then)
  uint32_t* s_part = sm.xv;
  static_assert(S::kXvBytes >= kRowGroups * kBins * 4, "row-sum partials fit the value exchange");
  __shared__ uint32_t s_hx[kMaxPasses - 1][kBins];  // pass 0: this chunk's counts of the later digits
  __shared__ uint2 s_warp2[kWarps];
  __shared__ unsigned long long s_sum[kWarps + 1];
  __shared__ unsigned long long s_base;
  __shared__ __align__(8) uint64_t s_mbar;
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
  uint32_t* csum = scratch + kSumWord;
  uint32_t* rows = scratch + kRowWord;
  uint32_t* raw = scratch + kRawWord;
  radix::TileRegs<uint32_t, false, kItems> R;
  __shared__ uint32_t s_h0[kCount ? kBins : 1];  // fused count: pass 0's digit totals
  uint32_t lo, hi;
  if constexpr (kCount) {
    // ---- the tile count step (Sec. II-A): per record its tile count and
    // depth key (raw depth bits; all ones without pairs), kept in R.k and,
    // for the counts, in the staging buffer; per view its pair total; the
    // smallest / largest key with pairs; the keys' low 9 bits counted
    __shared__ uint32_t s_begin[kMaxViews + 1];
    __shared__ const float4* s_g[kMaxViews];
    __shared__ FrameGeom s_geom[kMaxViews];
    __shared__ unsigned long long s_tot[kMaxViews];
    __shared__ uint32_t s_raw[kBins];
    __shared__ uint32_t s_lo, s_hi, s_cull;
    const ViewTable& vt = A.vt;
    const uint32_t nv = vt.nv;
    for (uint32_t v = t; v <= nv; v += kThreads) s_begin[v] = vt.rec_begin[v];
    for (uint32_t v = t; v < nv; v += kThreads) {
      s_g[v] = vt.g[v];
      s_geom[v] = vt.geom[v];
      s_tot[v] = 0ull;
    }
    s_raw[t] = 0u;
    s_h0[t] = 0u;
    if (t == 0) {
      s_lo = 0xffffffffu;
      s_hi = 0u;
      s_cull = 0u;
    }
    __syncthreads();
    const uint32_t wbase = warp * 32 * kItems;
    uint32_t klo = 0xffffffffu, khi = 0u, nculled = 0u;
    unsigned long long tsum = 0;  // one view: this thread's pairs
    bool bad = false;
    constexpr int kGroup = 16;  // records in flight per thread
#pragma unroll
    for (int j0 = 0; j0 < kItems; j0 += kGroup) {
      float4 rec[kGroup];
      uint32_t vv[kGroup];
#pragma unroll
      for (int u = 0; u < kGroup; ++u) {
        const uint32_t idx = wbase + (j0 + u) * 32 + lane, i = beg + idx;
        vv[u] = 0u;
        rec[u] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < valid) {
          vv[u] = nv == 1 ? 0u : find_view(s_begin, nv, i);
          rec[u] = __ldg(s_g[vv[u]] + (i - s_begin[vv[u]]));
        }
      }
#pragma unroll
      for (int u = 0; u < kGroup; ++u) {
        const int j = j0 + u;
        const uint32_t idx = wbase + j * 32 + lane;
        R.k[j] = 0xffffffffu;
        if (idx < valid) {
          const TileRect tr = tile_rect(rec[u], s_geom[vv[u]]);
          bad |= tr.invalid;
          const uint32_t cnt = tr.count;
          vstage[idx] = cnt;
          if (cnt >= kCntEscape) counts[beg + idx] = cnt;
          if (cnt) {
            const uint32_t key = __float_as_uint(rec[u].z);
            R.k[j] = key;
            klo = min(klo, key);
            khi = max(khi, key);
            atomicAdd(&s_raw[key & (kBins - 1)], 1u);
            if (nv == 1)
              tsum += cnt;
            else
              atomicAdd(&s_tot[vv[u]], static_cast<unsigned long long>(cnt));
          } else {
            ++nculled;
          }
        }
      }
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) latch_error(err, TDGS_ERR_INVALID_ARGUMENT, kSiteViewsCount);
    klo = __reduce_min_sync(0xffffffffu, klo);
    khi = __reduce_max_sync(0xffffffffu, khi);
    nculled = __reduce_add_sync(0xffffffffu, nculled);
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) tsum += __shfl_xor_sync(0xffffffffu, tsum, d);
    if (lane == 0) {
      atomicMin(&s_lo, klo);
      atomicMax(&s_hi, khi);
      if (nculled) atomicAdd(&s_cull, nculled);
      if (nv == 1 && tsum) atomicAdd(&s_tot[0], tsum);
    }
    __syncthreads();
    if (s_raw[t]) atomicAdd(raw + t, s_raw[t]);
    for (uint32_t v = t; v < nv; v += kThreads)
      if (s_tot[v]) atomicAdd(reinterpret_cast<unsigned long long*>(vt.vtot + v), s_tot[v]);
    if (t == 0) {
      if (s_lo != 0xffffffffu) atomicMin(range, s_lo);
      if (s_hi != 0u) atomicMax(range + 1, s_hi);
      if (s_cull) atomicAdd(raw + kBins, s_cull);
    }
    arrive_and_wait(scratch, G, err);  // every record counted
    lo = __ldcg(range);
    hi = __ldcg(range + 1);
    if (c == 0 && t == 0) {
      // each view's first pair in the sorted list and M, also for the host
      uint64_t run = 0;
      for (uint32_t v = 0; v < nv; ++v) {
        vt.pbeg[v] = static_cast<uint32_t>(run);
        run += __ldcg(reinterpret_cast<const unsigned long long*>(vt.vtot + v));
      }
      vt.pbeg[nv] = static_cast<uint32_t>(run);
      *A.total = run;
      range[2] = lo;
      range[3] = hi;
      if (A.host_status) {
        // one 8-byte store (no fence: nothing else needs ordering with it)
        const uint64_t m40 = run < (1ull << 40) ? run : (1ull << 40) - 1;
        const uint64_t e8 = min(__ldcg(err), 255u);
        *reinterpret_cast<volatile uint64_t*>(A.host_status) =
            (static_cast<uint64_t>(A.host_seq) << 48) | (e8 << 40) | m40;
      }
    }
  } else {
    lo = __ldcg(range + 2);
    hi = __ldcg(range + 3);
  }
  // digits from the compressed range
  const uint32_t cull = hi >= lo ? hi - lo + 1u : 0u;  // compressed keys are 0 .. cull
  const uint32_t bits = cull ? 32u - static_cast<uint32_t>(__clz(cull)) : 0u;
  const uint32_t passes = bits ? (bits + kBits - 1) / kBits : 1u;
  const uint32_t width = (bits + passes - 1) / passes;
  const uint32_t mask = width ? (1u << width) - 1u : 0u;
  if (c == 0 && t == 0) {
    range[4] = passes;
    scratch[kFinalSlot * kLine] = 0u;  // the previous launch's final barrier
  }
  if (c == 0)  // this launch's chunk sums (added to after the first barrier)
    for (uint32_t i = t; i < G; i += kThreads) csum[i] = 0u;
  const uint32_t nbulk = valid & ~3u;  // values by bulk copy; the last 1-3 by plain loads
  if (t == 0) {
    osw::mbar_init(&s_mbar);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if constexpr (kCount) {
    // pass 0's digit totals: digit 0 of key - lo is (low 9 bits - lo) & mask
    // (width <= 9); the culled keys all have cull & mask
    const uint32_t r = __ldcg(raw + t);
    if (r) atomicAdd(&s_h0[(t - lo) & mask], r);
    if (t == 0) {
      const uint32_t nc = __ldcg(raw + kBins);
      if (nc) atomicAdd(&s_h0[cull & mask], nc);
    }
  }
  radix::PassArgs a{};
  a.m = n;
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
    const uint32_t* vsrc = p == 0 ? counts : vin;
    const bool counted = kCount && p == 0;  // values (the counts) already staged by the count step
    const uint32_t nstaged = counted ? valid : nbulk;
    if (t == 0) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      osw::mbar_arrive(&s_mbar, counted ? 0u : nbulk * 4);
      if (!counted && nbulk) osw::bulk_g2s(vstage, vsrc + beg, nbulk * 4, &s_mbar);
    }
    {
      // this pass's keys: pass 0 compresses them (from the count step's
      // registers or from key0), later passes read them as written
      const uint32_t wbase = warp * 32 * kItems;
      if (counted) {
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
          const uint32_t idx = wbase + j * 32 + lane;
          R.k[j] = idx < valid ? (R.k[j] == 0xffffffffu ? cull : R.k[j] - lo) : 0u;
        }
      } else {
#pragma unroll
        for (int j = 0; j < kItems; ++j) {
          const uint32_t idx = wbase + j * 32 + lane;
          R.k[j] = idx < valid ? __ldcs(kin + beg + idx) : 0u;
        }
        if (p == 0) {
#pragma unroll
          for (int j = 0; j < kItems; ++j)
            if (wbase + j * 32 + lane < valid) R.k[j] = R.k[j] == 0xffffffffu ? cull : R.k[j] - lo;
        }
      }
#pragma unroll
      for (int j = 0; j < kItems; ++j) R.d[j] = (R.k[j] >> a.shift) & mask;
      radix::rank_keys<false, S, uint32_t, false, kBits, kItems>(valid, sm, R);
    }
    // publish this chunk's digit counts (lstart) as its row (count + 1)
    if (t < kBins / 8) {
      const uint32_t* ls = sm.lstart + 8 * t;
      uint4 w;
      w.x = (ls[0] + 1u) | ((ls[1] + 1u) << 16);
      w.y = (ls[2] + 1u) | ((ls[3] + 1u) << 16);
      w.z = (ls[4] + 1u) | ((ls[5] + 1u) << 16);
      w.w = (ls[6] + 1u) | ((ls[7] + 1u) << 16);
      st_relaxed_v4(rows + (static_cast<size_t>(p) * G + c) * kRowWords + 4 * t, w);
    }
    if (p == 0) {
      // every later pass's digit totals (ready at this pass's end barrier);
      // pass 0's own after one more barrier, unless the count step gave them
      const uint32_t wbase = warp * 32 * kItems;
      for (uint32_t pp = 1; pp < passes; ++pp) {
#pragma unroll
        for (int j = 0; j < kItems; ++j)
          if (wbase + j * 32 + lane < valid) atomicAdd(&s_hx[pp - 1][(R.k[j] >> (pp * width)) & mask], 1u);
      }
      __syncthreads();
      for (uint32_t pp = 1; pp < passes; ++pp)
        if (s_hx[pp - 1][t]) atomicAdd(hist + pp * kBins + t, s_hx[pp - 1][t]);
      if constexpr (!kCount) {
        if (sm.lstart[t]) atomicAdd(hist + t, sm.lstart[t]);
        arrive_and_wait(scratch, G, err);
      }
    }
    // output base per digit: keys of smaller digits + this digit's keys in
    // the chunks before this one
    {
      const uint32_t tot = (kCount && p == 0) ? s_h0[t] : __ldcg(hist + p * kBins + t);
      const uint32_t own = sm.lstart[t];
      uint32_t acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
      sum_rows(rows + static_cast<size_t>(p) * G * kRowWords, low_half ? 0u : c + 1, low_half ? c : G, g, q,
               acc, err);
#pragma unroll
      for (int i = 0; i < 8; ++i) s_part[g * kBins + 8 * q + i] = acc[i];
      __syncthreads();
      uint32_t sum = 0;
#pragma unroll
      for (uint32_t gg = 0; gg < kRowGroups; ++gg) sum += s_part[gg * kBins + t];
      const uint32_t before = low_half ? sum : tot - own - sum;
      // digit starts over all keys and inside this chunk in one scan;
      // output position of the chunk's p-th key in digit order = off[digit] + p
      const uint2 st = excl_scan2(tot, own, s_warp2);
      sm.lstart[t] = st.y;
      sm.off[t] = st.x + before - st.y;
    }
    if (!osw::mbar_wait(&s_mbar, p & 1u, err) && t == 0) (void)osw::mbar_wait(&s_mbar, p & 1u, err);
    __syncthreads();
    {
      // ranks into tile positions; this warp's counter row back to zero
      uint16_t* my_wh = sm.wh + warp * kBins;
#pragma unroll
      for (int j = 0; j < kItems; ++j) R.r[j] += sm.lstart[R.d[j]] + my_wh[R.d[j]];
      __syncwarp();
      uint4* z = reinterpret_cast<uint4*>(my_wh);
      for (uint32_t i = lane; i < kBins / 8; i += 32) z[i] = make_uint4(0, 0, 0, 0);
    }
    uint32_t hk[kItems];  // exchanged with each value: the key, in the last pass its digit
#pragma unroll
    for (int j = 0; j < kItems; ++j) hk[j] = last ? R.d[j] : R.k[j];
    ok &= exchange_scatter(sm, vstage, hk, R.r, valid, beg, nstaged, vsrc, p == 0, last, a.shift, mask, n, kout,
                           vout, k1, v1, counts, Sz, G, csum);
    arrive_and_wait(scratch + (last ? kFinalSlot : 1 + p) * kLine, G, err);
  }
  if (!ok) latch_error(err, TDGS_ERR_CAPACITY, kSiteRadixRange);
  // The pair offsets: counts in depth order (k1) scanned from the sum of
  // the chunks before this one.
  if (warp == 0) {
    uint64_t before = chunks_before(csum, c);
    if (lane == 0) s_base = before;
  }
  __syncthreads();
  scan_offsets(k1, offsets, beg, end, s_base, s_sum, err);
  // Reset for the next launch (every reader of these is past the final
  // barrier): this chunk's rows; CTA 0 the totals, the histogram of the
  // count step, the key range and the mid-launch counters.
  for (uint32_t i = t; i < passes * (kRowWords / 4); i += kThreads) {
    const uint32_t pp = i / (kRowWords / 4), w = i % (kRowWords / 4);
    reinterpret_cast<uint4*>(rows + (static_cast<size_t>(pp) * G + c) * kRowWords)[w] = make_uint4(0, 0, 0, 0);
  }
  if (c == 0) {
    for (uint32_t i = t; i < passes * kBins; i += kThreads) hist[i] = 0u;
    if constexpr (kCount) {
      raw[t] = 0u;
      if (t == 0) {
        raw[kBins] = 0u;
        range[0] = 0xffffffffu;
        range[1] = 0u;
      }
    }
    if (t < passes) scratch[t * kLine] = 0u;  // slots 0 .. passes-1
  }
}

}  // namespace depth

// ------------------------------------------------------------- host side
namespace {
enum class Form { kCount, kOne };
radix::Kernel depth_kernel(Form f) {
  const void* fn = f == Form::kCount ? reinterpret_cast<const void*>(&depth::k_depth_sort<true>)
                                     : reinterpret_cast<const void*>(&depth::k_depth_sort<false>);
  return radix::Kernel{fn, depth::kBits, depth::kThreads, depth::kItems, depth::kSmem, 1};
}

cudaError_t launch_depth(Form f, uint32_t grid, const DepthSortArgs& a, cudaStream_t s) {
  if (a.n == 0) return cudaSuccess;
  if (grid == 0 || grid > radix::kMaxGrid || a.n > depth_sort_count_capacity(grid))
    return cudaErrorInvalidConfiguration;
  if (f == Form::kCount && a.vt.nv > kMaxViews) return cudaErrorInvalidValue;
  DepthSortArgs args = a;
  void* params[] = {(void*)&args};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(depth::kThreads);
  cfg.dynamicSmemBytes = depth::kSmem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelExC(&cfg, depth_kernel(f).fn, params);
}
}  // namespace

uint32_t depth_sort_grid() {
  // every form: one CTA per SM (the occupancy query also sets their shared
  // memory limit on this device)
  uint32_t g = radix::kMaxGrid;
  for (Form f : {Form::kCount, Form::kOne}) {
    const uint32_t r = radix::resident_ctas(depth_kernel(f), 1);
    if (r < g) g = r;
  }
  return g;
}

uint32_t depth_sort_count_capacity(uint32_t grid) {
  // chunks of ceil(n / G) keys rounded up to a multiple of 4 fit one tile
  // (8192, itself a multiple of 4) exactly when n <= G * 8192
  return grid * depth::kTileKeys;
}

size_t depth_sort_scratch_words(uint32_t grid) {
  return depth::kRowWord + static_cast<size_t>(depth::kMaxPasses) * grid * depth::kRowWords;
}

cudaError_t launch_depth_sort(uint32_t grid, const DepthSortArgs& a, cudaStream_t s) {
  return launch_depth(Form::kOne, grid, a, s);
}

cudaError_t launch_count_depth_sort(uint32_t grid, const DepthSortArgs& a, cudaStream_t s) {
  return launch_depth(Form::kCount, grid, a, s);
}

}  // namespace tdgs
