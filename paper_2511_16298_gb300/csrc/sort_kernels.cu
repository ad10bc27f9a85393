// Stable LSD radix sort of (uint64 key, uint32 value) pairs -- the Sorting
// step of Sec. II-A (by tile, then by depth).  Onesweep structure (Adinets &
// Merrill, 2022): one upfront read of the keys builds the histograms of
// every digit, then each digit pass is a single kernel that ranks a tile of
// keys, resolves its global offsets with a decoupled look-back across
// tiles, and scatters.  Only the key bits that can be non-zero take part
// (32 depth bits plus the tile bits; bit 31 is skipped when every depth is
// positive).
#include "tdgs_internal.cuh"

namespace tdgs {

namespace {

// Look-back status word of one (tile, digit): flag (bits 31-30: 1 =
// aggregate of this tile only, 2 = inclusive prefix over tiles 0..k), an
// epoch tag (bits 29-27) that tells this pass's words from stale ones left
// by earlier passes, and the count (bits 26-0).
constexpr uint32_t kFlagAgg = 1u << 30;
constexpr uint32_t kFlagPre = 2u << 30;
constexpr uint32_t kEpochShift = 27;
constexpr uint32_t kCountMask = (1u << 27) - 1;
constexpr uint32_t kNoDigit = 0xffffffffu;

struct DigitShifts {
  uint32_t shift[kMaxPasses];
  uint32_t mask[kMaxPasses];
};

// With drop31 the sorted key is (tile bits : depth bits 30..0): bit 31 of
// every key is known to be zero and is squeezed out.
__device__ __forceinline__ uint64_t sort_key(uint64_t k, bool drop31) {
  return drop31 ? ((k & 0x7fffffffull) | ((k >> 32) << 31)) : k;
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

}  // namespace

// ------------------------------------------------------ upfront histogram
// grid = (blocks per portion, portions).  Histograms of every pass's digit
// over all keys are counted with shared-memory atomics and added to the
// global histograms hist[pass][bin].  Also checks that no key sets a bit
// outside the sorted range.
__global__ void __launch_bounds__(512)
    k_upfront_hist(const uint64_t* __restrict__ keys, uint32_t m, uint32_t portion,
                   uint32_t passes, uint32_t bins, DigitShifts ds, int drop31, uint64_t bad_mask,
                   uint32_t* __restrict__ hist, uint32_t* err) {
  extern __shared__ uint32_t sh[];
  const uint32_t t = threadIdx.x;
  for (uint32_t i = t; i < passes * bins; i += blockDim.x) sh[i] = 0;
  __syncthreads();
  const uint32_t q = blockIdx.y;
  const uint64_t pbeg = static_cast<uint64_t>(q) * portion;
  const uint64_t pend = pbeg + portion < m ? pbeg + portion : m;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  bool bad = false;
  uint64_t i = pbeg + static_cast<uint64_t>(blockIdx.x) * blockDim.x + t;
  for (; i + 3 * stride < pend; i += 4 * stride) {
    uint64_t k[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) k[u] = __ldcs(keys + i + u * stride);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      bad |= (k[u] & bad_mask) != 0;
      const uint64_t e = sort_key(k[u], drop31);
#pragma unroll
      for (uint32_t p = 0; p < kMaxPasses; ++p)
        if (p < passes) atomicAdd(&sh[p * bins + ((e >> ds.shift[p]) & ds.mask[p])], 1u);
    }
  }
  for (; i < pend; i += stride) {
    const uint64_t k = __ldcs(keys + i);
    bad |= (k & bad_mask) != 0;
    const uint64_t e = sort_key(k, drop31);
#pragma unroll
    for (uint32_t p = 0; p < kMaxPasses; ++p)
      if (p < passes) atomicAdd(&sh[p * bins + ((e >> ds.shift[p]) & ds.mask[p])], 1u);
  }
  __syncthreads();
  for (uint32_t j = t; j < passes * bins; j += blockDim.x)
    if (sh[j]) atomicAdd(hist + j, sh[j]);
  if (__any_sync(0xffffffffu, bad) && lane_id() == 0) latch_error(err, TDGS_ERR_INVALID_ARGUMENT);
}

// ---------------------------------------------------------- digit offsets
// One block per pass: offs[p][b] = number of keys whose digit p is < b,
// i.e. where the keys with digit b start after pass p.
__global__ void __launch_bounds__(1024)
    k_digit_offsets(const uint32_t* __restrict__ hist, uint32_t bins, uint32_t* __restrict__ offs) {
  __shared__ uint32_t s_warp[32];
  const size_t p = blockIdx.x;
  const uint32_t per = (bins + 1023) / 1024;  // 1 or 2
  uint32_t tot[2] = {0, 0};
  uint32_t sum = 0;
  for (uint32_t i = 0; i < per; ++i) {
    const uint32_t b = threadIdx.x * per + i;
    if (b < bins) tot[i] = hist[p * bins + b];
    sum += tot[i];
  }
  uint32_t run = block_excl_scan<32>(sum, s_warp);
  for (uint32_t i = 0; i < per; ++i) {
    const uint32_t b = threadIdx.x * per + i;
    if (b < bins) offs[p * bins + b] = run;
    run += tot[i];
  }
}

// ------------------------------------------------------------ one pass
// A block sorts one tile of kThreads*kItems consecutive keys of a portion.
//  1. Ranking: warp w owns keys [w*32*kItems, (w+1)*32*kItems) of the tile,
//     loaded warp-striped (item j of lane l is key w*32*kItems + j*32 + l,
//     so every load is one coalesced 256-byte access).  For item j the warp
//     groups equal digits with match.any; the group's lowest lane reads
//     and bumps the warp's private 16-bit counter of that digit, so a key's
//     rank is the number of earlier keys of the warp with the same digit.
//  2. Per digit: exclusive prefix over warps -> tile-local start; the tile
//     total is published for the look-back.
//  3. Look-back: per digit, sum predecessor tiles' aggregates back to the
//     first inclusive prefix; publish this tile's inclusive prefix.
//  4. Exchange: keys are placed in shared memory in digit order, then
//     written out by consecutive threads, so every digit's keys leave as a
//     contiguous run; values follow through the same exchange.
// Stability: ranks follow key order within a warp (item-major, lane-minor),
// warps follow key order within a tile, tiles follow key order through the
// ticket counter and the look-back.
template <int kBits, int kThreads, int kItems>
__global__ void __launch_bounds__(kThreads, (kThreads <= 256 ? 2 : 1))
    k_onesweep(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin,
               uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, uint32_t total,
               uint32_t begin, uint32_t count, uint32_t shift, uint32_t mask, int drop31,
               const uint32_t* __restrict__ digit_off, uint32_t* __restrict__ next_off,
               uint32_t* status, uint32_t epoch, uint32_t* ticket, uint32_t ticket_base,
               uint32_t* err) {
  constexpr int kBins = 1 << kBits;
  constexpr int kWarps = kThreads / 32;
  constexpr int kTileKeys = kThreads * kItems;
  constexpr int kBpt = (kBins + kThreads - 1) / kThreads;  // bins per thread
  constexpr int kWhBytes = kWarps * kBins * 2;
  constexpr int kXBytes = kTileKeys * 8;
  constexpr int kUBytes = kWhBytes > kXBytes ? kWhBytes : kXBytes;
  extern __shared__ __align__(16) unsigned char smem[];
  uint16_t* wh = reinterpret_cast<uint16_t*>(smem);   // [kWarps][kBins] during ranking
  uint64_t* xk = reinterpret_cast<uint64_t*>(smem);   // key exchange afterwards
  uint32_t* xv = reinterpret_cast<uint32_t*>(smem);   // value exchange afterwards
  uint32_t* bin_a = reinterpret_cast<uint32_t*>(smem + kUBytes);
  __shared__ uint32_t s_warp[kWarps];
  __shared__ uint32_t s_tile;

  const uint32_t t = threadIdx.x;
  const uint32_t lane = lane_id();
  const uint32_t warp = t >> 5;
  const bool d31 = drop31 != 0;

  for (uint32_t i = t; i < kWarps * kBins / 2; i += kThreads) reinterpret_cast<uint32_t*>(wh)[i] = 0;
  if (t == 0) s_tile = atomicAdd(ticket, 1u) - ticket_base;
  __syncthreads();
  const uint32_t tile = s_tile;
  const uint32_t tile_base = begin + tile * kTileKeys;
  const uint32_t left = count - tile * kTileKeys;
  const uint32_t valid = left < static_cast<uint32_t>(kTileKeys) ? left : kTileKeys;

  uint64_t k[kItems];
  uint32_t v[kItems];
  uint32_t r[kItems];
  const uint32_t wbase = warp * 32 * kItems;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t idx = wbase + j * 32 + lane;
    if (idx < valid) {
      k[j] = __ldcs(kin + tile_base + idx);
      v[j] = __ldcs(vin + tile_base + idx);
    } else {
      k[j] = 0;
      v[j] = 0;
    }
  }

  // 1. rank within the warp
  uint16_t* my_wh = wh + warp * kBins;
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t idx = wbase + j * 32 + lane;
    const uint32_t d = idx < valid ? static_cast<uint32_t>((sort_key(k[j], d31) >> shift) & mask) : kNoDigit;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t leader = __ffs(peers) - 1;
    uint32_t before = 0;
    if (lane == leader && d != kNoDigit) before = my_wh[d];
    before = __shfl_sync(0xffffffffu, before, leader);
    if (lane == leader && d != kNoDigit) my_wh[d] = static_cast<uint16_t>(before + __popc(peers));
    r[j] = before + __popc(peers & lanemask_lt());
    __syncwarp();
  }
  __syncthreads();

  // 2. exclusive prefix over warps; tile totals; publish aggregates
  uint32_t tot[kBpt];
#pragma unroll
  for (int i = 0; i < kBpt; ++i) {
    const uint32_t b = t + i * kThreads;
    tot[i] = 0;
    if (b < kBins) {
      uint32_t run = 0;
#pragma unroll 4
      for (int w = 0; w < kWarps; ++w) {
        const uint32_t c = wh[w * kBins + b];
        wh[w * kBins + b] = static_cast<uint16_t>(run);
        run += c;
      }
      tot[i] = run;
      bin_a[b] = run;
      st_relaxed(status + static_cast<size_t>(tile) * kBins + b,
                 (tile == 0 ? kFlagPre : kFlagAgg) | (epoch << kEpochShift) | run);
    }
  }
  __syncthreads();
  // tile-local digit starts: exclusive scan of the totals over digits
  {
    uint32_t seg[kBpt];
    uint32_t sum = 0;
#pragma unroll
    for (int i = 0; i < kBpt; ++i) {
      const uint32_t b = t * kBpt + i;
      seg[i] = b < kBins ? bin_a[b] : 0;
      sum += seg[i];
    }
    uint32_t run = block_excl_scan<kWarps>(sum, s_warp);
#pragma unroll
    for (int i = 0; i < kBpt; ++i) {
      const uint32_t b = t * kBpt + i;
      if (b < kBins) bin_a[b] = run;
      run += seg[i];
    }
  }

  // 3. decoupled look-back, all of this thread's digits in flight together
  uint32_t excl[kBpt];
  {
    int32_t kk[kBpt];
    bool done[kBpt];
#pragma unroll
    for (int i = 0; i < kBpt; ++i) {
      excl[i] = 0;
      kk[i] = static_cast<int32_t>(tile) - 1;
      done[i] = tile == 0 || (t + i * kThreads) >= static_cast<uint32_t>(kBins);
    }
    uint32_t spins = 0;
    while (true) {
      uint32_t s[kBpt];
#pragma unroll
      for (int i = 0; i < kBpt; ++i)
        s[i] = done[i] ? 0u : ld_relaxed(status + static_cast<size_t>(kk[i]) * kBins + t + i * kThreads);
      bool all = true, waiting = false;
#pragma unroll
      for (int i = 0; i < kBpt; ++i) {
        if (done[i]) continue;
        const uint32_t fl = s[i] >> 30;
        if (fl == 0 || ((s[i] >> kEpochShift) & 7u) != epoch) {
          waiting = true;
          all = false;
          continue;
        }
        excl[i] += s[i] & kCountMask;
        if (fl == 2) {
          done[i] = true;
        } else {
          --kk[i];
          all = false;
        }
      }
      if (all) break;
      if (waiting) {
        if (++spins > kSpinLimit) {
          latch_error(err, TDGS_ERR_TIMEOUT);
          break;
        }
        __nanosleep(20);
      }
    }
    if (tile > 0) {
#pragma unroll
      for (int i = 0; i < kBpt; ++i) {
        const uint32_t b = t + i * kThreads;
        if (b < static_cast<uint32_t>(kBins))
          st_relaxed(status + static_cast<size_t>(tile) * kBins + b,
                     kFlagPre | (epoch << kEpochShift) | ((excl[i] + tot[i]) & kCountMask));
      }
    }
    // The last tile of a portion hands the running digit offsets to the
    // next portion of the same pass (launched after this one).
    if (next_off && tile == gridDim.x - 1) {
#pragma unroll
      for (int i = 0; i < kBpt; ++i) {
        const uint32_t b = t + i * kThreads;
        if (b < static_cast<uint32_t>(kBins)) next_off[b] = __ldg(digit_off + b) + excl[i] + tot[i];
      }
    }
  }
  __syncthreads();

  // 4. exchange through shared memory in digit order
#pragma unroll
  for (int j = 0; j < kItems; ++j) {
    const uint32_t idx = wbase + j * 32 + lane;
    if (idx < valid) {
      const uint32_t d = static_cast<uint32_t>((sort_key(k[j], d31) >> shift) & mask);
      r[j] += bin_a[d] + my_wh[d];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kBpt; ++i) {
    const uint32_t b = t + i * kThreads;
    if (b < static_cast<uint32_t>(kBins)) bin_a[b] = __ldg(digit_off + b) + excl[i] - bin_a[b];
  }
#pragma unroll
  for (int j = 0; j < kItems; ++j)
    if (wbase + j * 32 + lane < valid) xk[r[j]] = k[j];
  __syncthreads();
  // Destinations come from the histograms; a destination outside [0,
  // total) can only follow a timed-out look-back or inconsistent inputs and
  // is dropped (and reported) instead of written.
  uint32_t dst[kItems];
  bool out_of_range = false;
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t p = i * kThreads + t;
    dst[i] = 0xffffffffu;
    if (p < valid) {
      const uint64_t key = xk[p];
      const uint32_t d = static_cast<uint32_t>((sort_key(key, d31) >> shift) & mask);
      dst[i] = bin_a[d] + p;
      if (dst[i] < total) {
        kout[dst[i]] = key;
      } else {
        out_of_range = true;
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < kItems; ++j)
    if (wbase + j * 32 + lane < valid) xv[r[j]] = v[j];
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    const uint32_t p = i * kThreads + t;
    if (p < valid && dst[i] < total) vout[dst[i]] = xv[p];
  }
  if (out_of_range) latch_error(err, TDGS_ERR_CAPACITY);
}

// ------------------------------------------------------------ variants
namespace {
using PassFn = void (*)(const uint64_t*, const uint32_t*, uint64_t*, uint32_t*, uint32_t, uint32_t,
                        uint32_t, uint32_t, uint32_t, int, const uint32_t*, uint32_t*, uint32_t*,
                        uint32_t, uint32_t*, uint32_t, uint32_t*);

template <int B, int T, int I>
constexpr size_t pass_smem() {
  constexpr size_t wh = static_cast<size_t>(T / 32) * (1u << B) * 2;
  constexpr size_t x = static_cast<size_t>(T) * I * 8;
  return (wh > x ? wh : x) + (static_cast<size_t>(1) << B) * 4;
}

struct VariantEntry {
  PassVariant v;
  PassFn fn;
  size_t smem;
};

#define TDGS_VARIANT(B, T, I) {{B, T, I}, k_onesweep<B, T, I>, pass_smem<B, T, I>()}
const VariantEntry kVariants[] = {
    TDGS_VARIANT(8, 256, 16),  TDGS_VARIANT(8, 512, 16),
    TDGS_VARIANT(10, 256, 16), TDGS_VARIANT(10, 512, 16),
    TDGS_VARIANT(11, 256, 16), TDGS_VARIANT(11, 512, 16), TDGS_VARIANT(11, 1024, 8),
};
#undef TDGS_VARIANT
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);
bool g_smem_set[kNumVariants] = {};
}  // namespace

int num_pass_variants() { return kNumVariants; }
PassVariant pass_variant(int i) { return kVariants[i].v; }

int default_pass_variant(uint32_t digit_bits) {
  if (digit_bits <= 8) return 0;
  if (digit_bits <= 10) return 2;
  return 4;
}

SortPlan make_sort_plan(uint32_t m, uint32_t tile_bits, uint32_t flags, int variant_override) {
  SortPlan p{};
  p.drop31 = (flags & TDGS_SORT_DEPTH_POSITIVE) != 0;
  p.key_bits = 32 + tile_bits - (p.drop31 ? 1 : 0);
  p.bad_mask = tile_bits >= 32 ? 0ull : ~((1ull << (32 + tile_bits)) - 1);
  if (p.drop31) p.bad_mask |= 1ull << 31;
  uint32_t max_bits = 11;
  if (variant_override >= 0 && variant_override < kNumVariants) {
    max_bits = static_cast<uint32_t>(kVariants[variant_override].v.bits);
    p.variant = static_cast<uint32_t>(variant_override);
  }
  p.passes = (p.key_bits + max_bits - 1) / max_bits;
  p.digit_bits = (p.key_bits + p.passes - 1) / p.passes;
  if (!(variant_override >= 0 && variant_override < kNumVariants))
    p.variant = static_cast<uint32_t>(default_pass_variant(p.digit_bits));
  for (uint32_t i = 0; i < p.passes; ++i) {
    p.shift[i] = i * p.digit_bits;
    const uint32_t w = p.key_bits - p.shift[i] < p.digit_bits ? p.key_bits - p.shift[i] : p.digit_bits;
    p.mask[i] = (1u << w) - 1;
  }
  const PassVariant& v = kVariants[p.variant].v;
  p.tile_keys = static_cast<uint32_t>(v.threads * v.items);
  p.portion = kPortionMax;  // a multiple of every (power-of-two) tile size
  p.portions = m == 0 ? 0 : static_cast<uint32_t>((static_cast<uint64_t>(m) + p.portion - 1) / p.portion);
  return p;
}

size_t onesweep_status_bytes(const SortPlan& plan) {
  const uint32_t tiles = (plan.portion + plan.tile_keys - 1) / plan.tile_keys;
  return static_cast<size_t>(tiles) * (1u << kVariants[plan.variant].v.bits) * 4;
}

cudaError_t launch_upfront_hist(const uint64_t* keys, uint32_t m, const SortPlan& plan,
                                uint32_t* hist, uint32_t* err, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  DigitShifts ds{};
  for (uint32_t i = 0; i < plan.passes; ++i) {
    ds.shift[i] = plan.shift[i];
    ds.mask[i] = plan.mask[i];
  }
  const uint32_t bins = 1u << kVariants[plan.variant].v.bits;
  const size_t smem = static_cast<size_t>(plan.passes) * bins * 4;
  static bool attr_set = false;
  if (!attr_set) {
    cudaFuncSetAttribute(k_upfront_hist, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    attr_set = true;
  }
  const uint32_t per_portion = plan.portions > 1 ? plan.portion : m;
  uint32_t bx = (per_portion + 512 * 16 - 1) / (512 * 16);
  const uint32_t cap = (152u * 3u + plan.portions - 1) / plan.portions;
  if (bx > cap) bx = cap;
  if (bx == 0) bx = 1;
  k_upfront_hist<<<dim3(bx, plan.portions), 512, smem, s>>>(keys, m, plan.portion, plan.passes, bins,
                                                             ds, plan.drop31 ? 1 : 0, plan.bad_mask,
                                                             hist, err);
  return cudaGetLastError();
}

cudaError_t launch_digit_offsets(const uint32_t* hist, const SortPlan& plan, uint32_t* offs,
                                 cudaStream_t s) {
  if (plan.portions == 0) return cudaSuccess;
  const uint32_t bins = 1u << kVariants[plan.variant].v.bits;
  k_digit_offsets<<<plan.passes, 1024, 0, s>>>(hist, bins, offs);
  return cudaGetLastError();
}

cudaError_t launch_onesweep_pass(const SortPlan& plan, uint32_t pass, uint32_t portion,
                                 const uint64_t* kin, const uint32_t* vin, uint64_t* kout,
                                 uint32_t* vout, uint32_t m, const uint32_t* digit_off,
                                 uint32_t* next_off, uint32_t* status, uint32_t epoch,
                                 uint32_t* ticket, uint32_t ticket_base, uint32_t* err,
                                 uint32_t* grid_out, cudaStream_t s) {
  const VariantEntry& e = kVariants[plan.variant];
  if (!g_smem_set[plan.variant]) {
    cudaError_t ce = cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          static_cast<int>(e.smem));
    if (ce != cudaSuccess) return ce;
    g_smem_set[plan.variant] = true;
  }
  const uint64_t beg = static_cast<uint64_t>(portion) * plan.portion;
  const uint64_t end = beg + plan.portion < m ? beg + plan.portion : m;
  const uint32_t count = static_cast<uint32_t>(end - beg);
  const uint32_t grid = (count + plan.tile_keys - 1) / plan.tile_keys;
  *grid_out = grid;
  if (grid == 0) return cudaSuccess;
  e.fn<<<grid, e.v.threads, e.smem, s>>>(kin, vin, kout, vout, m, static_cast<uint32_t>(beg), count,
                                         plan.shift[pass], plan.mask[pass], plan.drop31 ? 1 : 0,
                                         digit_off, next_off, status, epoch, ticket, ticket_base,
                                         err);
  return cudaGetLastError();
}

}  // namespace tdgs
