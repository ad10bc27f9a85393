// tdgs_sort_pairs as a onesweep LSD radix sort (the Sorting step of
// Sec. II-A: instances ordered by tile, then by depth; sorting is 86-89 % of
// the frame in Table VI), and the same passes over the depth keys of large
// frames.
//
//   k_onesweep_hist  reads every key once and counts the first pass's
//                    digits (shared-memory counters per CTA, then global
//                    atomics); the last CTA scans them into the first
//                    pass's digit starts.  It also clears the first pass's
//                    status words, the later passes' counters and the tile
//                    tickets.
//   k_onesweep_pass  one cooperative launch per digit.  Compute CTAs take
//                    tiles of 4096 pairs in ticket order; a tile arrives in
//                    shared memory by bulk copies (double buffered: the
//                    next tile is in flight while this one is ranked), is
//                    ranked stably with one ballot per digit bit, publishes
//                    its per-digit counts at once, counts the next pass's
//                    digits and is exchanged into digit order in place.
//                    The last CTAs of the grid are scan CTAs that turn the
//                    published counts into per-tile prefixes; a compute CTA
//                    takes tile k's prefix one iteration after publishing
//                    it (while it ranked the next tile) and writes tile k
//                    out with coalesced stores.  Every key and value is
//                    read once and written once per pass.
//
// Key forms: 64-bit keys with the digit a bit field of the low word, of the
// high word, or spanning both (tdgs_sort_pairs), and 32-bit depth keys
// compressed to their range, whose pass plan each launch reads from the
// range on the device.  Tickets keep the waits deadlock-free: a tile only
// waits on tiles with smaller tickets, and ranking (which publishes the
// counts) never waits on another CTA.  Every wait is bounded and latches
// TDGS_ERR_TIMEOUT when it runs out; every scatter is checked against the
// pair count.
#include <mutex>
#include <type_traits>

#include "onesweep.cuh"

namespace tdgs {
namespace onesweep {

using namespace osw;

constexpr int kBits = 9;
constexpr uint32_t kBins = 1u << kBits;
constexpr int kItems = 16;
constexpr uint32_t kTileKeys = kThreads * kItems;  // 4096
constexpr int kGroup = 4;                          // items ranked together (independent ballot chains)
constexpr uint32_t kScanCtas = scan_ctas<kBins>();

static_assert(kBins == 2 * kThreads, "two digits per thread in the look-back and the digit scan");

template <typename K>
struct TileBuf {
  K k[kTileKeys];
  uint32_t v[kTileKeys];
};
constexpr size_t kWhBytes = static_cast<size_t>(kWarps) * kBins * 2;  // per-warp 16-bit counters
template <typename K>
constexpr size_t smem_bytes() {
  return 2 * sizeof(TileBuf<K>) + kWhBytes + 3 * kBins * 4;
}

// Digit of one key for one pass.  64-bit keys (tdgs_sort_pairs): bits
// [shift, shift + width) of the key, or of (tile bits : depth bits 30..0)
// when bit 31 is dropped (the keys then have bit 31 clear), in three forms
// chosen on the host (make_digit) and compiled separately: a bit field of
// the low word, a bit field of the high word, or a field spanning both,
// (lo >> msh) | (hi << hsh).  32-bit depth keys (the depth sort of
// Sec. II-A's frame; form kDigitDepth): bits [msh, msh + width) of the key
// less the smallest visible key lo, culled Gaussians' keys (all ones)
// becoming cull, one more than the largest; the device derives the pass
// plan from the key range the count kernel published (depth_digits).
struct Digit {
  uint32_t mode;  // kDigitLo, kDigitHi, kDigitSpan or kDigitDepth
  uint32_t msh;   // right shift of the word holding the field (the low word for a span)
  uint32_t hsh;   // span: left shift of the high word
  uint32_t mask;
  uint32_t lo, cull;  // depth keys: the compression
};
constexpr int kDigitLo = 0, kDigitHi = 1, kDigitSpan = 2, kDigitDepth = 3, kDigitNone = 4;
template <int kMode>
using KeyOf = std::conditional_t<kMode == kDigitDepth, uint32_t, uint64_t>;
template <int kMode, typename K>
__device__ __forceinline__ uint32_t digit_m(K k, const Digit& g) {
  if constexpr (kMode == kDigitDepth) {
    const uint32_t x = static_cast<uint32_t>(k) == 0xffffffffu ? g.cull : static_cast<uint32_t>(k) - g.lo;
    return (x >> g.msh) & g.mask;
  } else {
    const uint32_t lo = static_cast<uint32_t>(k), hi = static_cast<uint32_t>(static_cast<uint64_t>(k) >> 32);
    if constexpr (kMode == kDigitLo) return (lo >> g.msh) & g.mask;
    if constexpr (kMode == kDigitHi) return (hi >> g.msh) & g.mask;
    return ((lo >> g.msh) | (hi << g.hsh)) & g.mask;
  }
}

// Shared-memory slot of digit d in the per-digit tables of a pass (the
// warps' 16-bit counters, the tile-local starts, the output offsets, the
// next pass's counts).  A digit spanning the two key words is (tile bits :
// top depth bits), whose low bits take few values, so a warp's digits would
// crowd a few banks; the slot d ^ ((d >> 6) << 1) spreads them and keeps
// each digit pair 2t, 2t + 1 in one 32-bit word of the 16-bit counters
// (word t ^ (t >> 5)).  A bijection on [0, 512): ranks, counts and starts
// are unchanged.
template <bool kSwz>
__device__ __forceinline__ uint32_t slot(uint32_t d) {
  if constexpr (kSwz) return d ^ ((d >> 6) << 1);
  return d;
}

// Pass plan of the depth keys from their range (range[2..3]: the smallest
// and largest visible key): the compressed keys 0 .. cull need `bits` bits,
// split evenly over the fewest passes of at most kBits.
struct DepthDigits {
  uint32_t lo, cull, passes, width, mask;
};
__device__ __forceinline__ DepthDigits depth_digits(const uint32_t* range) {
  DepthDigits d;
  d.lo = __ldcg(range + 2);
  const uint32_t hi = __ldcg(range + 3);
  d.cull = hi >= d.lo ? hi - d.lo + 1u : 0u;
  const uint32_t bits = d.cull ? 32u - static_cast<uint32_t>(__clz(d.cull)) : 0u;
  d.passes = bits ? (bits + kBits - 1) / kBits : 1u;
  d.width = (bits + d.passes - 1) / d.passes;
  d.mask = d.width ? (1u << d.width) - 1u : 0u;
  return d;
}

struct HistArgs {
  uint32_t m, passes, ntiles;
  Digit dg[kMaxPasses];
  uint64_t bad_mask;   // key bits that must be zero
  uint32_t* hist;      // [kMaxPasses][kBins], zero on entry, left zero
  uint32_t* gstart;    // [kMaxPasses][kBins] digit starts (exclusive scan of hist)
  uint32_t* done;      // block counter, zero on entry, left zero
  uint32_t* tickets;   // [kMaxPasses] tile tickets, cleared here
  uint32_t* status0;   // [ntiles][kBins] look-back status of pass 0, cleared here
  uint32_t* range;     // depth keys: the key range (range[2..3]); the pass count goes to range[4]
  uint32_t* err;
};

struct PassArgs {
  uint32_t m, ntiles;
  Digit dg;
  Digit dgn;               // the next pass's digit (counted while ranking)
  const uint32_t* gstart;  // [kBins] this pass's digit starts (pass 0), or null
  const uint32_t* hist;    // [kBins] this pass's digit counts (later passes; gstart is null)
  uint32_t* hist_next;     // [kBins] the next pass's digit counts, accumulated here (or null)
  uint32_t* status;        // [ntiles][kBins] this pass's status (all zero on entry)
  uint32_t* status_next;   // [ntiles][kBins] the next pass's, cleared here (or null)
  uint32_t* ticket;        // zero on entry
  // depth keys: the pass number, the key range and the three key and value
  // buffers (0: input; the last pass that runs writes buffer 1)
  uint32_t pass;
  const uint32_t* range;
  uint32_t* dk[3];
  uint32_t* dv[3];
  uint32_t* err;
};

// ----------------------------------------------------------- histograms
// Digit counts of the first pass (each pass counts the next one's digits
// while it ranks).  Thread t of a block reads 8 consecutive keys (64
// bytes; a warp reads 2 KB contiguously) and adds runs of equal digits with
// one shared-memory atomic each: duplicated keys come in runs (one
// Gaussian's tiles share its depth).  The block's next chunk is prefetched
// into L2 while it counts.  Few blocks (4 per SM) keep the final global
// atomics on the counters few.
constexpr int kHistThreads = 512;
template <int kMode>
__global__ void __launch_bounds__(kHistThreads) k_onesweep_hist(const KeyOf<kMode>* __restrict__ keys, HistArgs a) {
  using K = KeyOf<kMode>;
  __shared__ uint32_t h[kBins];
  __shared__ uint32_t s_warp[kHistThreads / 32];
  __shared__ bool s_last;
  const uint32_t t = threadIdx.x;
  for (uint32_t i = t; i < kBins; i += kHistThreads) h[i] = 0;
  // housekeeping for the passes: tile tickets, later passes' counters,
  // pass 0's look-back status
  if (blockIdx.x == 0) {
    if (t < kMaxPasses) a.tickets[t] = 0;
    for (uint32_t i = kBins + t; i < kMaxPasses * kBins; i += kHistThreads) a.hist[i] = 0;
  }
  {
    uint4* z = reinterpret_cast<uint4*>(a.status0);
    const size_t nz = static_cast<size_t>(a.ntiles) * kBins / 4;
    for (size_t i = static_cast<size_t>(blockIdx.x) * kHistThreads + t; i < nz;
         i += static_cast<size_t>(gridDim.x) * kHistThreads)
      z[i] = make_uint4(0, 0, 0, 0);
  }
  __syncthreads();
  const uint32_t m = a.m;
  Digit dg0 = a.dg[0];  // 64-bit keys: the first digit is bits [0, width) of the low word
  if constexpr (kMode == kDigitDepth) {
    const DepthDigits dd = depth_digits(a.range);
    dg0 = Digit{kDigitDepth, 0u, 0u, dd.mask, dd.lo, dd.cull};
    if (blockIdx.x == 0 && t == 0) a.range[4] = dd.passes;  // for the host's diagnostics
  }
  const bool vec = (reinterpret_cast<uintptr_t>(keys) & 15u) == 0;
  constexpr uint32_t kStep = 8 * kHistThreads;  // keys per block and step: 8 consecutive per thread
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * kStep;
  bool bad = false;
  for (uint64_t base = static_cast<uint64_t>(blockIdx.x) * kStep; base < m; base += stride) {
    if (t == 0 && base + stride < m)  // the next step's keys into L2 while this step counts
      radix::prefetch_l2(keys + base + stride, (min(static_cast<uint64_t>(kStep), m - (base + stride))) * 8);
    const uint64_t i0 = base + 8 * t;
    K k[8];
    if (vec && i0 + 8 <= m) {
      if constexpr (sizeof(K) == 8) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const uint4 w = __ldcs(reinterpret_cast<const uint4*>(keys + i0) + u);
          k[2 * u] = (static_cast<uint64_t>(w.y) << 32) | w.x;
          k[2 * u + 1] = (static_cast<uint64_t>(w.w) << 32) | w.z;
        }
      } else {
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const uint4 w = __ldcs(reinterpret_cast<const uint4*>(keys + i0) + u);
          k[4 * u] = w.x;
          k[4 * u + 1] = w.y;
          k[4 * u + 2] = w.z;
          k[4 * u + 3] = w.w;
        }
      }
    } else {
#pragma unroll
      for (int j = 0; j < 8; ++j) k[j] = i0 + j < m ? keys[i0 + j] : K(0);
    }
    uint32_t run_d = 0, run_n = 0;  // runs of equal digits: one atomic each
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if (i0 + j < m) {
        if constexpr (kMode != kDigitDepth) bad |= (k[j] & a.bad_mask) != 0;
        const uint32_t d = digit_m<kMode>(k[j], dg0);
        if (run_n && d != run_d) {
          atomicAdd(&h[run_d], run_n);
          run_n = 0;
        }
        run_d = d;
        ++run_n;
      }
    }
    if (run_n) atomicAdd(&h[run_d], run_n);
  }
  if (__any_sync(0xffffffffu, bad) && lane_id() == 0) latch_error(a.err, TDGS_ERR_INVALID_ARGUMENT, kSiteRadixKeys);
  __syncthreads();
  for (uint32_t q = t; q < kBins; q += kHistThreads)
    if (h[q]) atomicAdd(a.hist + q, h[q]);
  __threadfence();
  __syncthreads();
  if (t == 0) s_last = atomicAdd(a.done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last block: the first pass's digit starts; leave its counters and the
  // block counter zero
  const uint32_t c = __ldcg(a.hist + t);
  a.gstart[t] = radix::block_excl_scan<kHistThreads / 32>(c, s_warp);
  a.hist[t] = 0;
  if (t == 0) *a.done = 0;
}

// One tile's keys and values (first `nbulk` pairs, a multiple of 4) by bulk
// copies completing on `bar`.
template <typename K>
__device__ __forceinline__ void load_tile(TileBuf<K>* b, uint64_t* bar, const K* kin, const uint32_t* vin,
                                          uint32_t first, uint32_t nbulk) {
  const uint32_t kb = nbulk * static_cast<uint32_t>(sizeof(K)), vb = nbulk * 4;
  mbar_arrive(bar, kb + vb);
  if (nbulk) {
    bulk_g2s(b->k, kin + first, kb, bar);
    bulk_g2s(b->v, vin + first, vb, bar);
  }
}

// ------------------------------------------------------------- one pass
// Stable rank of one tile held in shared memory (tile order: warp, item,
// lane): r[j] = number of earlier items of this warp with the same digit;
// the warp's counter row (zero on entry) ends holding its count per digit.
template <int kMode, int kModeN>
__device__ __forceinline__ void rank_in_warps(const TileBuf<KeyOf<kMode>>& tb, uint32_t valid, const Digit& dg, uint16_t* my_wh,
                                              uint32_t (&r)[kItems], const Digit& dgn, uint32_t* hn) {
  const uint32_t lane = lane_id(), warp = threadIdx.x >> 5;
  const uint32_t wbase = warp * 32 * kItems;
  const uint32_t lt = lanemask_lt();
#pragma unroll
  for (int j0 = 0; j0 < kItems; j0 += kGroup) {
    uint32_t d[kGroup];
#pragma unroll
    for (int g = 0; g < kGroup; ++g) {
      const uint32_t idx = wbase + (j0 + g) * 32 + lane;
      const KeyOf<kMode> key = idx < valid ? tb.k[idx] : KeyOf<kMode>(0);
      d[g] = slot<kMode == kDigitSpan>(digit_m<kMode>(key, dg));  // equal slots <=> equal digits
      if constexpr (kModeN != kDigitNone)  // (depth keys: hn is null in the last pass)
        if (idx < valid && (kMode != kDigitDepth || hn))
          atomicAdd(&hn[slot<kModeN == kDigitSpan>(digit_m<kModeN>(key, dgn))], 1u);
      r[j0 + g] = radix::equal_digit_lanes<kBits>(d[g]);
      const uint32_t fi = wbase + (j0 + g) * 32;
      const uint32_t nlive = valid > fi ? min(valid - fi, 32u) : 0u;
      r[j0 + g] &= nlive >= 32 ? 0xffffffffu : ((1u << nlive) - 1u);
    }
#pragma unroll
    for (int g = 0; g < kGroup; ++g) {
      const uint32_t peers = r[j0 + g];
      const bool live = wbase + (j0 + g) * 32 + lane < valid;
      const uint32_t before = my_wh[d[g]];
      __syncwarp();
      const uint32_t cnt = __popc(peers), below = __popc(peers & lt);
      if (live && below + 1 == cnt) my_wh[d[g]] = static_cast<uint16_t>(before + cnt);
      __syncwarp();
      r[j0 + g] = before + below;
    }
  }
}

// The compute warps of a CTA are software-pipelined over its tiles:
// iteration i ranks tile k_i, publishes its per-digit counts and exchanges
// it into digit order in shared memory; then it takes the prefix of tile
// k_(i-1) (ranked one iteration earlier) from the scan CTAs and scatters
// that tile.  The prefix is needed a whole ranking phase after the counts
// went out, so the scan has (nearly always) produced it.  Ranking never
// waits for another CTA, so every tile with a ticket publishes its counts
// and the scan always completes.  Launched cooperatively: the scan CTAs
// must run alongside every other CTA.  While ranking, the CTA also counts
// the next pass's digits; the counts reach hist_next when it finishes.
template <int kMode, int kModeN>
__global__ void __launch_bounds__(kThreads, 2)
    k_onesweep_pass(const KeyOf<kMode>* __restrict__ kin, const uint32_t* __restrict__ vin,
                    KeyOf<kMode>* __restrict__ kout, uint32_t* __restrict__ vout, PassArgs a) {
  using K = KeyOf<kMode>;
  constexpr bool kSwz = kMode == kDigitSpan;  // per-digit tables in swizzled slots
  extern __shared__ __align__(128) unsigned char smem[];
  TileBuf<K>* buf = reinterpret_cast<TileBuf<K>*>(smem);
  uint16_t* wh = reinterpret_cast<uint16_t*>(smem + 2 * sizeof(TileBuf<K>));
  uint32_t* lstart = reinterpret_cast<uint32_t*>(smem + 2 * sizeof(TileBuf<K>) + kWhBytes);
  uint32_t* off = lstart + kBins;
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t s_tile[2];
  __shared__ uint32_t s_warp[kWarps];

  Digit dg = a.dg, dgn = a.dgn;
  uint32_t* hist_next = a.hist_next;
  uint32_t* status_next = a.status_next;
  if constexpr (kMode == kDigitDepth) {
    // The pass plan from the key range: a pass beyond it ends at once on
    // every CTA (scan CTAs included); the buffers alternate so that the
    // last pass that runs writes buffer 1.
    const DepthDigits dd = depth_digits(a.range);
    if (a.pass >= dd.passes) return;
    dg = Digit{kDigitDepth, a.pass * dd.width, 0u, dd.mask, dd.lo, dd.cull};
    dgn = dg;
    dgn.msh += dd.width;
    if (a.pass + 1 >= dd.passes) {
      hist_next = nullptr;
      status_next = nullptr;
    }
    const uint32_t out = ((dd.passes - 1 - a.pass) & 1u) ? 2u : 1u;
    const uint32_t in = a.pass == 0 ? 0u : (((dd.passes - a.pass) & 1u) ? 2u : 1u);
    kin = a.dk[in];
    vin = a.dv[in];
    kout = a.dk[out];
    vout = a.dv[out];
  }
  uint32_t* hn = kModeN != kDigitNone && hist_next ? off + kBins : nullptr;  // next pass's digit counts of this CTA

  const uint32_t t = threadIdx.x, lane = lane_id(), warp = t >> 5;
  const uint32_t m = a.m, ntiles = a.ntiles;
  if (blockIdx.x >= gridDim.x - kScanCtas) {  // a scan CTA
    scan_tiles<kBins>(a.status, ntiles, blockIdx.x - (gridDim.x - kScanCtas), a.err, reinterpret_cast<uint32_t*>(smem));
    return;
  }
  uint16_t* my_wh = wh + warp * kBins;
  {
    uint4* z = reinterpret_cast<uint4*>(wh);
    for (uint32_t i = t; i < kWhBytes / 16; i += kThreads) z[i] = make_uint4(0, 0, 0, 0);
  }
  if (hn) {
    hn[2 * t] = 0;
    hn[2 * t + 1] = 0;
  }
  uint32_t g0, g1;  // this pass's first output position of digits 2t and 2t+1
  if (a.gstart) {
    g0 = __ldg(a.gstart + 2 * t);
    g1 = __ldg(a.gstart + 2 * t + 1);
  } else {
    const uint32_t h0 = __ldcg(a.hist + 2 * t), h1 = __ldcg(a.hist + 2 * t + 1);
    g0 = cta_excl_scan(h0 + h1, s_warp);
    g1 = g0 + h0;
  }
  auto bulk_items = [&](uint32_t tile) {
    const uint32_t first = tile * kTileKeys;
    const uint32_t valid = min(kTileKeys, m - first);
    return valid & ~3u;  // the last 1-3 items of a ragged tile are read by threads
  };
  if (t == 0) {
    mbar_init(&mbar[0]);
    mbar_init(&mbar[1]);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const uint32_t first = atomicAdd(a.ticket, 1u);
    s_tile[1] = first;
    if (first < ntiles) load_tile(&buf[0], &mbar[0], kin, vin, first * kTileKeys, bulk_items(first));
  }
  __syncthreads();
  uint32_t cur = s_tile[1];
  uint32_t phase = 0;  // bit b: parity of the next wait on mbar[b]
  bool ok = true;
  bool have_prev = false;
  uint32_t prev = 0, pc0 = 0, ps0 = 0, pvalid = 0;  // the tile waiting for its scatter
  for (uint32_t it = 0;; ++it) {
    const bool have_cur = cur < ntiles;
    if (!have_cur && !have_prev) break;
    const uint32_t b = it & 1u;  // cur is in buf[b], prev in buf[b ^ 1]
    uint32_t c0 = 0, c1 = 0, s0 = 0, valid = 0;
    // The next tile's ticket is taken at the start of the iteration and its
    // data prefetched into L2 once the ticket returns; the copy into shared
    // memory goes out at the end of the iteration (when its buffer is free)
    // and then comes from L2.  Its counts are published in the next
    // iteration, and the tiles after it look back one more iteration later,
    // so taking it here costs them no waiting.
    uint32_t nxt = ntiles;
    if (t == 0 && have_cur) nxt = atomicAdd(a.ticket, 1u);
    if (have_cur) {
      TileBuf<K>& tb = buf[b];
      const uint32_t first = cur * kTileKeys;
      valid = min(kTileKeys, m - first);
      const bool arrived = mbar_wait(&mbar[b], (phase >> b) & 1u, a.err);
      if (__syncthreads_or(!arrived)) {
        // A copy that never arrived (error latched): the whole CTA stops
        // together.  Thread 0 waits once more, bounded, for that copy (the
        // only one in flight), so nothing lands in shared memory after the
        // CTA exits.
        if (t == 0) (void)mbar_wait(&mbar[b], (phase >> b) & 1u, a.err);
        break;
      }
      phase ^= 1u << b;
      if (valid != kTileKeys) {  // ragged last tile: its last 1-3 items by plain loads
        const uint32_t nb = valid & ~3u;
        if (t < valid - nb) {
          tb.k[nb + t] = kin[first + nb + t];
          tb.v[nb + t] = vin[first + nb + t];
        }
        __syncthreads();
      }
      // ---- stable rank within each warp
      uint32_t r[kItems];
      rank_in_warps<kMode, kModeN>(tb, valid, dg, my_wh, r, dgn, hn);
      if (t == 0 && nxt < ntiles) {
        const uint32_t nf = nxt * kTileKeys, nv = min(kTileKeys, m - nf);
        radix::prefetch_l2(kin + nf, static_cast<uint64_t>(nv) * 8);
        radix::prefetch_l2(vin + nf, static_cast<uint64_t>(nv) * 4);
      }
      __syncthreads();
      // ---- per-digit counts (column t holds digits 2t and 2t+1), prefixes over warps
      {
        uint32_t* wh32 = reinterpret_cast<uint32_t*>(wh);
        uint32_t run = 0;
        const uint32_t pw = slot<kSwz>(2 * t) >> 1;  // the word of digits 2t, 2t+1
#pragma unroll
        for (int w = 0; w < kWarps; ++w) {
          const uint32_t x = wh32[w * (kBins / 2) + pw];
          wh32[w * (kBins / 2) + pw] = run;
          run += x;  // halves stay below 2^16: no carry between digits
        }
        c0 = run & 0xffffu;
        c1 = run >> 16;
      }
      // ---- publish the counts (tile 0: its counts are its inclusive prefix)
      st_relaxed_v2(a.status + static_cast<size_t>(cur) * kBins + 2 * t, kFlagA | c0, kFlagA | c1);
      // ---- tile-local digit starts, positions, exchange into digit order
      s0 = cta_excl_scan(c0 + c1, s_warp);
      lstart[slot<kSwz>(2 * t)] = s0;
      lstart[slot<kSwz>(2 * t + 1)] = s0 + c0;
      __syncthreads();
      const uint32_t wbase = warp * 32 * kItems;
      K kr[kItems];
      uint32_t vr[kItems];
#pragma unroll
      for (int j = 0; j < kItems; ++j) {
        const uint32_t idx = wbase + j * 32 + lane;
        if (idx < valid) {
          kr[j] = tb.k[idx];
          vr[j] = tb.v[idx];
          const uint32_t dd = digit_m<kMode>(kr[j], dg);
          const uint32_t sd = slot<kSwz>(dd);
          r[j] += lstart[sd] + my_wh[sd];
        }
      }
      __syncwarp();
      {  // this warp's counter row is read: zero it for the next tile
        uint4* z = reinterpret_cast<uint4*>(my_wh);
        for (uint32_t i = lane; i < kBins / 8; i += 32) z[i] = make_uint4(0, 0, 0, 0);
      }
      __syncthreads();
#pragma unroll
      for (int j = 0; j < kItems; ++j) {
        if (wbase + j * 32 + lane < valid && r[j] < kTileKeys) {
          tb.k[r[j]] = kr[j];
          tb.v[r[j]] = vr[j];
        }
      }
    }
    // ---- the previous tile: its prefix, output positions
    if (have_prev) {
      uint32_t e0 = 0, e1 = 0;
      if (prev != 0) wait_prefix<kBins>(a.status, prev, t, e0, e1, a.err);
      if (status_next)
        *reinterpret_cast<uint2*>(status_next + static_cast<size_t>(prev) * kBins + 2 * t) = make_uint2(0u, 0u);
      off[slot<kSwz>(2 * t)] = g0 + e0 - ps0;
      off[slot<kSwz>(2 * t + 1)] = g1 + e1 - (ps0 + pc0);
    }
    __syncthreads();  // cur is in digit order; off[] of prev is complete
    // ---- coalesced scatter of the previous tile in digit order
    if (have_prev) {
      const TileBuf<K>& pb = buf[b ^ 1u];
#pragma unroll
      for (int i = 0; i < kItems; ++i) {
        const uint32_t p = i * kThreads + t;
        if (p < pvalid) {
          const K key = pb.k[p];
          const uint32_t dst = off[slot<kSwz>(digit_m<kMode>(key, dg))] + p;
          if (dst < m) {
            kout[dst] = key;
            vout[dst] = pb.v[p];
          } else {
            ok = false;
          }
        }
      }
    }
    if (t == 0) s_tile[b] = nxt;
    __syncthreads();  // buf[b ^ 1] is free; the next tile's number is visible
    if (t == 0 && nxt < ntiles) {
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      load_tile(&buf[b ^ 1u], &mbar[b ^ 1u], kin, vin, nxt * kTileKeys, bulk_items(nxt));
    }
    have_prev = have_cur;
    if (have_cur) {
      prev = cur;
      pc0 = c0;
      ps0 = s0;
      pvalid = valid;
    }
    cur = s_tile[b];
  }
  if (!ok) latch_error(a.err, TDGS_ERR_CAPACITY, kSiteRadixRange);
  if (hn) {  // this CTA's counts of the next pass's digits
    __syncthreads();
    for (uint32_t i = t; i < kBins; i += kThreads)
      if (const uint32_t c = hn[slot<kModeN == kDigitSpan>(i)]) atomicAdd(hist_next + i, c);
  }
}


}  // namespace onesweep

// ------------------------------------------------------------ host side
namespace {
std::mutex g_mu;
uint32_t g_grid[2][64] = {};  // resident pass CTAs per key width and device (0: not queried)

const void* depth_pass_kernel() {
  return reinterpret_cast<const void*>(&onesweep::k_onesweep_pass<onesweep::kDigitDepth, onesweep::kDigitDepth>);
}
size_t pass_smem(bool depth) {
  return depth ? onesweep::smem_bytes<uint32_t>() : onesweep::smem_bytes<uint64_t>();
}

// Resident CTAs of the pass kernel (64-bit keys, or the 32-bit depth keys);
// every form of one key width has the same launch bounds and shared memory.
uint32_t pass_grid(bool depth) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
  std::lock_guard<std::mutex> lock(g_mu);
  uint32_t& g = g_grid[depth ? 1 : 0][dev];
  if (!g) {
    const void* fn =
        depth ? depth_pass_kernel()
              : reinterpret_cast<const void*>(&onesweep::k_onesweep_pass<onesweep::kDigitLo, onesweep::kDigitNone>);
    const size_t smem = pass_smem(depth);
    int sms = 0, occ = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
      return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, onesweep::kThreads, smem) != cudaSuccess || occ <= 0)
      return 0;
    g = static_cast<uint32_t>(sms * occ);
  }
  return g;
}

// Scratch layout shared by both key widths: hist | gstart | done, tickets
// | status rows of two passes.
void scratch_layout(onesweep::HistArgs& a, uint32_t* scratch) {
  using namespace onesweep;
  a.hist = scratch;
  a.gstart = scratch + kMaxPasses * kBins;
  a.done = scratch + 2 * kMaxPasses * kBins;
  a.tickets = a.done + 4;
  a.status0 = scratch + onesweep_header_words();
}
void pass_layout(onesweep::PassArgs& a, uint32_t pass, bool has_next, uint32_t* scratch) {
  using namespace onesweep;
  if (has_next) a.hist_next = scratch + (pass + 1) * kBins;
  if (pass == 0)
    a.gstart = scratch + kMaxPasses * kBins;
  else
    a.hist = scratch + pass * kBins;
  a.ticket = scratch + 2 * kMaxPasses * kBins + 4 + pass;
  uint32_t* st = scratch + onesweep_header_words();
  const size_t rows = static_cast<size_t>(a.ntiles) * kBins;
  a.status = st + (pass & 1u) * rows;
  a.status_next = has_next ? st + ((pass + 1) & 1u) * rows : nullptr;
}

// 4096 keys per block and step, at least 4 steps per block (fewer blocks:
// fewer global atomics on the 512 counters), at most 4 blocks per SM
uint32_t hist_grid(uint32_t m) {
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  constexpr uint32_t kPerBlock = 4 * 8 * onesweep::kHistThreads;
  uint32_t grid = static_cast<uint32_t>((static_cast<uint64_t>(m) + kPerBlock - 1) / kPerBlock);
  const uint32_t cap = static_cast<uint32_t>(sms) * 4;
  if (grid > cap) grid = cap;
  return grid ? grid : 1;
}

// One cooperative launch of a pass: CTAs that take tiles while they last,
// plus the scan CTAs (all resident).
cudaError_t launch_pass(const void* fn, bool depth, const void* kin, const uint32_t* vin, void* kout, uint32_t* vout,
                        onesweep::PassArgs& a, cudaStream_t s) {
  using namespace onesweep;
  const uint32_t resident = pass_grid(depth);
  if (resident < 2 * kScanCtas) return cudaErrorInvalidConfiguration;
  const uint32_t grid = (a.ntiles < resident - kScanCtas ? a.ntiles : resident - kScanCtas) + kScanCtas;
  void* args[] = {(void*)&kin, (void*)&vin, (void*)&kout, (void*)&vout, (void*)&a};
  const size_t smem = pass_smem(depth);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem)) != cudaSuccess)
    return cudaErrorInvalidConfiguration;
  return cudaLaunchKernelExC(&cfg, fn, args);
}

onesweep::Digit make_digit(uint32_t shift, uint32_t mask, bool drop31) {
  onesweep::Digit d{};
  d.mask = mask;
  // bits [0, 31) (or [0, 32) without the drop) are the low word's; bits
  // from 31 on (32 on) are the high word's
  const uint32_t width = static_cast<uint32_t>(__builtin_popcount(mask));
  const uint32_t split = drop31 ? 31u : 32u;
  if (shift + width <= split) {
    d.mode = onesweep::kDigitLo;
    d.msh = shift;
  } else if (shift >= split) {
    d.mode = onesweep::kDigitHi;
    d.msh = shift - split;
  } else {  // 0 < split - shift < width <= 9: both shifts stay below 32
    d.mode = onesweep::kDigitSpan;
    d.msh = shift;
    d.hsh = split - shift;
  }
  return d;
}

// The pass kernel for a digit form and the next pass's digit form.
template <int kMode>
const void* pass_kernel(uint32_t next) {
  using namespace onesweep;
  switch (next) {
    case kDigitLo: return reinterpret_cast<const void*>(&k_onesweep_pass<kMode, kDigitLo>);
    case kDigitHi: return reinterpret_cast<const void*>(&k_onesweep_pass<kMode, kDigitHi>);
    case kDigitSpan: return reinterpret_cast<const void*>(&k_onesweep_pass<kMode, kDigitSpan>);
    default: return reinterpret_cast<const void*>(&k_onesweep_pass<kMode, kDigitNone>);
  }
}
}  // namespace

bool onesweep_eligible(uint32_t m, const void* keys, const void* values, const void* keys_alt,
                       const void* values_alt) {
  auto a16 = [](const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; };
  return m > 0 && m < onesweep::kMaxPairs && a16(keys) && a16(values) && a16(keys_alt) && a16(values_alt);
}

size_t onesweep_scratch_words(uint32_t m) {
  const size_t ntiles = (static_cast<size_t>(m) + onesweep::kTileKeys - 1) / onesweep::kTileKeys;
  return onesweep_header_words() + 2 * ntiles * onesweep::kBins;
}

size_t onesweep_header_words() {
  // hist | gstart | done + tickets (padded to 16 bytes)
  return 2 * static_cast<size_t>(kMaxPasses) * onesweep::kBins + 4 + kMaxPasses;
}

uint32_t onesweep_tile_keys() { return onesweep::kTileKeys; }

cudaError_t launch_onesweep_hist(const SortPlan& plan, const uint64_t* keys, uint32_t m, uint32_t* scratch,
                                 uint32_t* err, cudaStream_t s) {
  using namespace onesweep;
  HistArgs a{};
  a.m = m;
  a.passes = 1;  // the first pass's digits; each pass counts the next one's
  a.ntiles = (m + kTileKeys - 1) / kTileKeys;
  a.dg[0] = make_digit(plan.shift[0], plan.mask[0], plan.drop31);
  a.bad_mask = plan.bad_mask;
  scratch_layout(a, scratch);
  a.err = err;
  const uint32_t grid = hist_grid(m);
  if (grid == 0) return cudaErrorInvalidDevice;
  k_onesweep_hist<kDigitLo><<<grid, kHistThreads, 0, s>>>(keys, a);
  return cudaGetLastError();
}

cudaError_t launch_onesweep_pass(const SortPlan& plan, uint32_t pass, const uint64_t* kin, const uint32_t* vin,
                                 uint64_t* kout, uint32_t* vout, uint32_t m, uint32_t* scratch, uint32_t* err,
                                 cudaStream_t s) {
  using namespace onesweep;
  PassArgs a{};
  a.m = m;
  a.ntiles = (m + kTileKeys - 1) / kTileKeys;
  a.dg = make_digit(plan.shift[pass], plan.mask[pass], plan.drop31);
  const bool has_next = pass + 1 < plan.passes;
  if (has_next) a.dgn = make_digit(plan.shift[pass + 1], plan.mask[pass + 1], plan.drop31);
  pass_layout(a, pass, has_next, scratch);
  a.err = err;
  const uint32_t next = has_next ? a.dgn.mode : static_cast<uint32_t>(kDigitNone);
  const void* fn = a.dg.mode == kDigitLo   ? pass_kernel<kDigitLo>(next)
                   : a.dg.mode == kDigitHi ? pass_kernel<kDigitHi>(next)
                                           : pass_kernel<kDigitSpan>(next);
  return launch_pass(fn, false, kin, vin, kout, vout, a, s);
}

cudaError_t launch_depth_onesweep_hist(const uint32_t* keys, uint32_t n, uint32_t* range, uint32_t* scratch,
                                       uint32_t* err, cudaStream_t s) {
  using namespace onesweep;
  HistArgs a{};
  a.m = n;
  a.passes = 1;
  a.ntiles = (n + kTileKeys - 1) / kTileKeys;
  a.range = range;
  scratch_layout(a, scratch);
  a.err = err;
  const uint32_t grid = hist_grid(n);
  if (grid == 0) return cudaErrorInvalidDevice;
  k_onesweep_hist<kDigitDepth><<<grid, kHistThreads, 0, s>>>(keys, a);
  return cudaGetLastError();
}

cudaError_t launch_depth_onesweep_pass(uint32_t pass, uint32_t* const dk[3], uint32_t* const dv[3], uint32_t n,
                                       const uint32_t* range, uint32_t* scratch, uint32_t* err, cudaStream_t s) {
  using namespace onesweep;
  if (pass >= kDepthOnesweepPasses) return cudaErrorInvalidValue;
  PassArgs a{};
  a.m = n;
  a.ntiles = (n + kTileKeys - 1) / kTileKeys;
  // the device drops the next pass's counts and status when this pass is
  // the last that the key range needs
  pass_layout(a, pass, pass + 1 < kDepthOnesweepPasses, scratch);
  a.pass = pass;
  a.range = range;
  for (int i = 0; i < 3; ++i) {
    a.dk[i] = dk[i];
    a.dv[i] = dv[i];
  }
  a.err = err;
  return launch_pass(depth_pass_kernel(), true, nullptr, nullptr, nullptr, nullptr, a, s);
}

}  // namespace tdgs
