// C ABI of libtdgs: argument checks, scratch management and launch order.
// Every call maps one step (or the fused frame) of the 3DGS sort step
// described in Sec. II-A to the kernels of frame_kernels.cu and
// sort_kernels.cu.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <new>
#include <cstring>
#include <string>
#include <vector>

#include "tdgs_internal.cuh"

using namespace tdgs;

namespace {

// Device words read back by the host: the pair count of the fused frame and
// the latched error, adjacent so one 16-byte copy fetches both.
struct DevStatus {
  uint64_t total;
  uint32_t err;
  uint32_t pad;
};

struct Buffer {
  void* p = nullptr;
  size_t bytes = 0;
};

enum KernelId {
  kKCount, kKScan, kKDuplicate, kKRanges, kKRadixPass,
  kKFrameCount, kKDepthSort, kKDupDepth, kKTilePass, kKRangesDiff, kKNum
};
const char* const kKernelNames[kKNum] = {
    "count_tiles",  "scan",       "duplicate_keys",     "tile_ranges",    "radix_pass",
    "frame_count",  "depth_sort", "duplicate_by_depth", "tile_sort_pass", "ranges_from_diff"};

struct PendingTime {
  int id;
  cudaEvent_t a, b;
  uint64_t items;
};

}  // namespace

struct tdgs_context {
  int device = 0;
  DevStatus* d_status = nullptr;
  DevStatus* h_status = nullptr;  // pinned
  uint32_t* d_tickets = nullptr;  // [0] scan tiles, [2..3] radix grid barrier
  uint32_t ticket_base[2] = {0, 0};
  Buffer scan_status, sort_scratch;
  // fused-frame buffers
  Buffer f_counts, f_dkey[2], f_dval[2], f_soff, f_diff, f_stream[2], f_keys, f_values, f_ranges;
  int variant_override = -1;
  std::string last_error;
  // tracing
  uint64_t launches = 0;
  bool timing = false;
  std::vector<PendingTime> pending;
  std::vector<cudaEvent_t> free_events;
  uint64_t k_launches[kKNum] = {};
  uint64_t k_items[kKNum] = {};
  double k_ms[kKNum] = {};
};

namespace {

class DeviceGuard {
 public:
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev_) != cudaSuccess) prev_ = -1;
    if (prev_ != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev_ >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev_) cudaSetDevice(prev_);
  }

 private:
  int prev_ = -1;
};

tdgs_status fail(tdgs_context* ctx, tdgs_status st, const std::string& msg) {
  if (ctx) ctx->last_error = msg;
  return st;
}

tdgs_status cuda_fail(tdgs_context* ctx, cudaError_t e, const char* where) {
  std::string msg = std::string(where) + ": " + cudaGetErrorString(e);
  cudaGetLastError();  // clear a sticky launch error so later calls start clean
  return fail(ctx, e == cudaErrorMemoryAllocation ? TDGS_ERR_OUT_OF_MEMORY : TDGS_ERR_CUDA, msg);
}

#define TDGS_CUDA(ctx, expr)                              \
  do {                                                    \
    cudaError_t _e = (expr);                              \
    if (_e != cudaSuccess) return cuda_fail(ctx, _e, #expr); \
  } while (0)

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Grow `b` to at least `bytes`.  The stream is drained first so nothing in
// flight still uses the old allocation.
tdgs_status ensure(tdgs_context* ctx, Buffer& b, size_t bytes, cudaStream_t s,
                   bool* grown = nullptr) {
  if (grown) *grown = false;
  if (b.bytes >= bytes && b.p) return TDGS_OK;
  const size_t want = std::max<size_t>(bytes + bytes / 4, 256);
  TDGS_CUDA(ctx, cudaStreamSynchronize(s));
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  TDGS_CUDA(ctx, cudaMalloc(&b.p, want));
  b.bytes = want;
  if (grown) *grown = true;
  return TDGS_OK;
}

uint32_t* err_word(tdgs_context* ctx) { return &ctx->d_status->err; }

cudaEvent_t take_event(tdgs_context* ctx) {
  if (!ctx->free_events.empty()) {
    cudaEvent_t e = ctx->free_events.back();
    ctx->free_events.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Resolve recorded event pairs into the per-kernel totals.
void drain_timings(tdgs_context* ctx) {
  for (const PendingTime& t : ctx->pending) {
    float ms = 0.f;
    if (cudaEventSynchronize(t.b) == cudaSuccess && cudaEventElapsedTime(&ms, t.a, t.b) == cudaSuccess) {
      ctx->k_ms[t.id] += ms;
      ctx->k_launches[t.id] += 1;
      ctx->k_items[t.id] += t.items;
    } else {
      cudaGetLastError();
    }
    ctx->free_events.push_back(t.a);
    ctx->free_events.push_back(t.b);
  }
  ctx->pending.clear();
}

void clear_timings(tdgs_context* ctx) {
  drain_timings(ctx);
  for (int i = 0; i < kKNum; ++i) {
    ctx->k_ms[i] = 0;
    ctx->k_launches[i] = 0;
    ctx->k_items[i] = 0;
  }
}

// Launch one kernel through `fn` (returns cudaError_t); counts it and, with
// timing on, brackets it with events on `s`.  items == 0 means the launcher
// has nothing to do and launches nothing.
template <class Fn>
tdgs_status traced(tdgs_context* ctx, KernelId id, uint64_t items, cudaStream_t s, const char* what,
                   Fn&& fn) {
  if (items == 0) return TDGS_OK;
  cudaEvent_t a = nullptr, b = nullptr;
  if (ctx->timing) {
    a = take_event(ctx);
    b = take_event(ctx);
    if (a && b) cudaEventRecord(a, s);
  }
  const cudaError_t e = fn();
  if (e != cudaSuccess) {
    if (a) ctx->free_events.push_back(a);
    if (b) ctx->free_events.push_back(b);
    return cuda_fail(ctx, e, what);
  }
  ctx->launches += 1;
  if (a && b) {
    cudaEventRecord(b, s);
    ctx->pending.push_back({static_cast<int>(id), a, b, items});
  }
  return TDGS_OK;
}

#define TDGS_TRACED(ctx, id, items, s, expr)                                      \
  do {                                                                           \
    tdgs_status _st = traced(ctx, id, items, s, #expr, [&]() { return (expr); }); \
    if (_st != TDGS_OK) return _st;                                              \
  } while (0)

tdgs_status do_scan(tdgs_context* ctx, const uint32_t* counts, const float4* recs,
                    const uint32_t* gather, FrameGeom fg, uint32_t n, uint32_t* offsets,
                    uint64_t* total64, uint32_t* total32, cudaStream_t s) {
  const uint32_t tiles = (n + kScanTileItems - 1) / kScanTileItems;
  tdgs_status st = ensure(ctx, ctx->scan_status, static_cast<size_t>(tiles) * 8, s);
  if (st != TDGS_OK) return st;
  TDGS_CUDA(ctx, cudaMemsetAsync(ctx->scan_status.p, 0, static_cast<size_t>(tiles) * 8, s));
  TDGS_TRACED(ctx, kKScan, n, s,
              launch_scan(counts, recs, gather, fg, n, offsets,
                          static_cast<uint64_t*>(ctx->scan_status.p), ctx->d_tickets + 0,
                          ctx->ticket_base[0], total64, total32, err_word(ctx), s));
  ctx->ticket_base[0] += tiles;
  return TDGS_OK;
}

tdgs_status do_sort(tdgs_context* ctx, uint64_t* keys, uint32_t* values, uint64_t* keys_alt,
                    uint32_t* values_alt, uint32_t m, uint32_t tile_bits, uint32_t flags,
                    int* result_in_alt, cudaStream_t s) {
  *result_in_alt = 0;
  if (m == 0) return TDGS_OK;
  const SortPlan plan = make_sort_plan(m, tile_bits, flags, ctx->variant_override);
  if (plan.grid == 0) return fail(ctx, TDGS_ERR_CUDA, "device query for the sort plan failed");
  tdgs_status st = ensure(ctx, ctx->sort_scratch, radix_scratch_words(plan) * 4, s);
  if (st != TDGS_OK) return st;
  uint64_t* kin = keys;
  uint32_t* vin = values;
  uint64_t* kout = keys_alt;
  uint32_t* vout = values_alt;
  for (uint32_t p = 0; p < plan.passes; ++p) {
    TDGS_TRACED(ctx, kKRadixPass, m, s,
                launch_radix_pass(plan, p, kin, vin, kout, vout, m,
                                  static_cast<uint32_t*>(ctx->sort_scratch.p), ctx->d_tickets + 2,
                                  err_word(ctx), s));
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  *result_in_alt = static_cast<int>(plan.passes & 1u);
  return TDGS_OK;
}

tdgs_status read_and_clear_error(tdgs_context* ctx, cudaStream_t s) {
  TDGS_CUDA(ctx, cudaMemcpyAsync(&ctx->h_status->err, &ctx->d_status->err, 4,
                                 cudaMemcpyDeviceToHost, s));
  TDGS_CUDA(ctx, cudaStreamSynchronize(s));
  const uint32_t e = ctx->h_status->err;
  if (e != 0) {
    TDGS_CUDA(ctx, cudaMemsetAsync(&ctx->d_status->err, 0, 4, s));
    TDGS_CUDA(ctx, cudaStreamSynchronize(s));
    return fail(ctx, static_cast<tdgs_status>(e), "error latched on the device");
  }
  return TDGS_OK;
}

}  // namespace

// ====================================================================== ABI
extern "C" {

const char* tdgs_status_string(tdgs_status s) {
  switch (s) {
    case TDGS_OK: return "ok";
    case TDGS_ERR_INVALID_ARGUMENT: return "invalid argument";
    case TDGS_ERR_OUT_OF_MEMORY: return "out of device memory";
    case TDGS_ERR_OVERFLOW: return "pair count overflows 32 bits";
    case TDGS_ERR_CUDA: return "CUDA error";
    case TDGS_ERR_TIMEOUT: return "cross-block wait timed out";
    case TDGS_ERR_CAPACITY: return "output capacity too small";
  }
  return "unknown status";
}

const char* tdgs_last_error(const tdgs_context* ctx) {
  return ctx ? ctx->last_error.c_str() : "";
}

uint32_t tdgs_num_tiles(tdgs_frame f) {
  return ((f.width + 15u) / 16u) * ((f.height + 15u) / 16u);
}

uint32_t tdgs_tile_bits(tdgs_frame f) {
  const uint32_t t = tdgs_num_tiles(f);
  uint32_t b = 0;
  while (b < 32 && (1ull << b) < t) ++b;
  return b;
}

int tdgs_sort_variant_count(void) { return num_pass_variants(); }

tdgs_status tdgs_sort_variant_info(int i, int* bits, int* threads, int* items) {
  if (i < 0 || i >= num_pass_variants()) return TDGS_ERR_INVALID_ARGUMENT;
  const PassVariant v = pass_variant(i);
  if (bits) *bits = v.bits;
  if (threads) *threads = v.threads;
  if (items) *items = v.items;
  return TDGS_OK;
}

tdgs_status tdgs_context_set_sort_variant(tdgs_context* ctx, int variant) {
  if (!ctx || variant < -1 || variant >= num_pass_variants()) return TDGS_ERR_INVALID_ARGUMENT;
  ctx->variant_override = variant;
  return TDGS_OK;
}

tdgs_status tdgs_context_create(tdgs_context** out, int device) {
  if (!out) return TDGS_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    return TDGS_ERR_INVALID_ARGUMENT;
  }
  DeviceGuard g(device);
  tdgs_context* ctx = new (std::nothrow) tdgs_context();
  if (!ctx) return TDGS_ERR_OUT_OF_MEMORY;
  ctx->device = device;
  if (cudaMalloc(&ctx->d_status, sizeof(DevStatus)) != cudaSuccess ||
      cudaMalloc(&ctx->d_tickets, 4 * sizeof(uint32_t)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_status, sizeof(DevStatus)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(DevStatus)) != cudaSuccess ||
      cudaMemset(ctx->d_tickets, 0, 4 * sizeof(uint32_t)) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    tdgs_context_destroy(ctx);
    return TDGS_ERR_OUT_OF_MEMORY;
  }
  *out = ctx;
  return TDGS_OK;
}

uint64_t tdgs_context_launch_count(const tdgs_context* ctx) { return ctx ? ctx->launches : 0; }

tdgs_status tdgs_context_enable_timing(tdgs_context* ctx, int enable) {
  if (!ctx) return TDGS_ERR_INVALID_ARGUMENT;
  DeviceGuard g(ctx->device);
  clear_timings(ctx);
  ctx->timing = enable != 0;
  return TDGS_OK;
}

int tdgs_context_kernel_times(tdgs_context* ctx, tdgs_kernel_time* out, int max) {
  if (!ctx || (max > 0 && !out)) return -1;
  DeviceGuard g(ctx->device);
  drain_timings(ctx);
  int n = 0;
  for (int i = 0; i < kKNum; ++i) {
    if (!ctx->k_launches[i]) continue;
    if (n < max) {
      out[n].name = kKernelNames[i];
      out[n].launches = ctx->k_launches[i];
      out[n].items = ctx->k_items[i];
      out[n].total_ms = ctx->k_ms[i];
    }
    ++n;
  }
  for (int i = 0; i < kKNum; ++i) {
    ctx->k_ms[i] = 0;
    ctx->k_launches[i] = 0;
    ctx->k_items[i] = 0;
  }
  return n;
}

void tdgs_context_destroy(tdgs_context* ctx) {
  if (!ctx) return;
  DeviceGuard g(ctx->device);
  drain_timings(ctx);
  for (cudaEvent_t e : ctx->free_events) cudaEventDestroy(e);
  Buffer* bufs[] = {&ctx->scan_status, &ctx->sort_scratch, &ctx->f_counts,    &ctx->f_dkey[0],
                    &ctx->f_dkey[1],    &ctx->f_dval[0],     &ctx->f_dval[1],    &ctx->f_soff,
                    &ctx->f_diff,       &ctx->f_stream[0],   &ctx->f_stream[1],  &ctx->f_keys,
                    &ctx->f_values,     &ctx->f_ranges};
  for (Buffer* b : bufs)
    if (b->p) cudaFree(b->p);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_tickets) cudaFree(ctx->d_tickets);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  delete ctx;
}

tdgs_status tdgs_context_sync(tdgs_context* ctx, void* stream) {
  if (!ctx) return TDGS_ERR_INVALID_ARGUMENT;
  DeviceGuard g(ctx->device);
  return read_and_clear_error(ctx, static_cast<cudaStream_t>(stream));
}

tdgs_status tdgs_count_tiles(tdgs_context* ctx, const tdgs_gaussian2d* g, uint32_t n,
                             tdgs_frame f, uint32_t* tiles_touched, void* stream) {
  if (!ctx) return TDGS_ERR_INVALID_ARGUMENT;
  if (f.width == 0 || f.height == 0) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "empty image");
  if (n == 0) return TDGS_OK;
  if (!g || !tiles_touched) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null pointer");
  if (!aligned(g, 16) || !aligned(tiles_touched, 4))
    return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "misaligned pointer");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TDGS_TRACED(ctx, kKCount, n, s,
              launch_count_tiles(reinterpret_cast<const float4*>(g), n, make_geom(f),
                                 tiles_touched, err_word(ctx), s));
  return TDGS_OK;
}

tdgs_status tdgs_scan(tdgs_context* ctx, const uint32_t* counts, uint32_t n, uint32_t* offsets,
                      uint32_t* total_dev, void* stream) {
  if (!ctx) return TDGS_ERR_INVALID_ARGUMENT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  DeviceGuard dg(ctx->device);
  if (n == 0) {
    if (total_dev) TDGS_CUDA(ctx, cudaMemsetAsync(total_dev, 0, 4, s));
    return TDGS_OK;
  }
  if (!counts || !offsets) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null pointer");
  if (!aligned(counts, 4) || !aligned(offsets, 4) || (total_dev && !aligned(total_dev, 4)))
    return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "misaligned pointer");
  return do_scan(ctx, counts, nullptr, nullptr, FrameGeom{}, n, offsets, nullptr, total_dev, s);
}

tdgs_status tdgs_duplicate_keys(tdgs_context* ctx, const tdgs_gaussian2d* g,
                                const uint32_t* offsets, uint32_t n, tdgs_frame f,
                                uint64_t* keys, uint32_t* values, uint32_t m_capacity,
                                void* stream) {
  if (!ctx) return TDGS_ERR_INVALID_ARGUMENT;
  if (f.width == 0 || f.height == 0) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "empty image");
  if (n == 0) return TDGS_OK;
  if (!g || !offsets || (m_capacity && (!keys || !values)))
    return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null pointer");
  if (!aligned(g, 16) || !aligned(offsets, 4) || !aligned(keys, 8) || !aligned(values, 4))
    return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "misaligned pointer");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TDGS_TRACED(ctx, kKDuplicate, n, s,
              launch_duplicate(reinterpret_cast<const float4*>(g), offsets, n, make_geom(f),
                               keys, values, m_capacity, err_word(ctx), s));
  return TDGS_OK;
}

tdgs_status tdgs_sort_pairs(tdgs_context* ctx, uint64_t* keys, uint32_t* values,
                            uint64_t* keys_alt, uint32_t* values_alt, uint32_t m,
                            uint32_t tile_bits, uint32_t flags, int* result_in_alt,
                            void* stream) {
  if (!ctx || !result_in_alt) return TDGS_ERR_INVALID_ARGUMENT;
  *result_in_alt = 0;
  if (tile_bits > 32) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "tile_bits > 32");
  if (flags & ~TDGS_SORT_DEPTH_POSITIVE) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "unknown flag");
  if (m == 0) return TDGS_OK;
  if (!keys || !values || !keys_alt || !values_alt)
    return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null pointer");
  if (!aligned(keys, 8) || !aligned(keys_alt, 8) || !aligned(values, 4) || !aligned(values_alt, 4))
    return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "misaligned pointer");
  if (keys == keys_alt || values == values_alt)
    return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "alternate buffers must differ");
  DeviceGuard dg(ctx->device);
  return do_sort(ctx, keys, values, keys_alt, values_alt, m, tile_bits, flags, result_in_alt,
                 static_cast<cudaStream_t>(stream));
}

tdgs_status tdgs_tile_ranges(tdgs_context* ctx, const uint64_t* sorted_keys, uint32_t m,
                             uint32_t num_tiles, tdgs_range* ranges, void* stream) {
  if (!ctx) return TDGS_ERR_INVALID_ARGUMENT;
  if (num_tiles == 0) return m ? fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "no tiles") : TDGS_OK;
  if (!ranges || (m && !sorted_keys)) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null pointer");
  if (!aligned(ranges, 8) || !aligned(sorted_keys, 8))
    return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "misaligned pointer");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TDGS_CUDA(ctx, cudaMemsetAsync(ranges, 0, static_cast<size_t>(num_tiles) * sizeof(tdgs_range), s));
  TDGS_TRACED(ctx, kKRanges, m, s,
              launch_tile_ranges(sorted_keys, m, num_tiles, reinterpret_cast<uint2*>(ranges),
                                 err_word(ctx), s));
  return TDGS_OK;
}

// Fused frame, depth first.  Steps (all on `stream`):
//   1. frame_count: tile counts, depth keys, per-CTA tile difference grids
//   2. depth_sort: the N Gaussians by (depth bits, index)  -> depth order
//   3. scan of the counts in depth order -> pair offsets, pair count M
//   4. (host) read M and the error word; size the pair buffers
//   5. duplicate_by_depth: element (tile << rbits | depth position) per pair
//   6. tile_sort_pass x1-2: stable passes on the tile bits; the last one
//      writes the final keys (tile << 32 | depth bits) and indices
//   7. ranges_from_diff: per-tile counts from the difference grids, scanned
// The result equals the stable sort of the 64-bit keys of steps 1-4 of the
// per-step calls: ties of the 64-bit key are pairs of distinct Gaussians in
// the same tile with equal depth, which both orders put in index order.
tdgs_status tdgs_sort_frame(tdgs_context* ctx, const tdgs_gaussian2d* g, uint32_t n,
                            tdgs_frame f, const uint64_t** sorted_keys,
                            const uint32_t** sorted_values, const tdgs_range** ranges,
                            uint32_t* m_out, void* stream) {
  if (!ctx || !sorted_keys || !sorted_values || !ranges || !m_out)
    return TDGS_ERR_INVALID_ARGUMENT;
  *m_out = 0;
  if (f.width == 0 || f.height == 0) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "empty image");
  if (n && !g) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null pointer");
  if (!aligned(g, 16)) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "misaligned pointer");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const FrameGeom fg = make_geom(f);
  const uint32_t T = tdgs_num_tiles(f);
  const uint32_t tb = tdgs_tile_bits(f);
  const float4* rec = reinterpret_cast<const float4*>(g);
  uint32_t rbits = 0;
  while (rbits < 32 && (1ull << rbits) < n) ++rbits;
  const bool wide = tb + rbits > 32 || rbits >= 32;
  const uint64_t cells = static_cast<uint64_t>(fg.gx + 1) * (fg.gy + 1);
  const bool use_diff = cells <= kMaxDiffCells;
  const uint32_t count_grid = use_diff ? 152u * 2u : 152u * 8u;

  tdgs_status st = TDGS_OK;
  const size_t n4 = static_cast<size_t>(n) * 4 + 16;
  for (Buffer* b : {&ctx->f_counts, &ctx->f_dkey[0], &ctx->f_dkey[1], &ctx->f_dval[0],
                    &ctx->f_dval[1], &ctx->f_soff})
    if (st == TDGS_OK) st = ensure(ctx, *b, n4, s);
  if (st == TDGS_OK && use_diff) st = ensure(ctx, ctx->f_diff, (count_grid + 1) * cells * 4, s);
  if (st == TDGS_OK) st = ensure(ctx, ctx->f_ranges, static_cast<size_t>(T) * 8, s);
  const uint32_t dgrid = depth_sort_grid(n ? n : 1);
  if (dgrid == 0) return fail(ctx, TDGS_ERR_CUDA, "device query for the depth sort failed");
  if (st == TDGS_OK) st = ensure(ctx, ctx->sort_scratch, depth_sort_scratch_words(dgrid) * 4, s);
  if (st != TDGS_OK) return st;
  uint32_t* counts = static_cast<uint32_t*>(ctx->f_counts.p);
  uint32_t* dk[2] = {static_cast<uint32_t*>(ctx->f_dkey[0].p), static_cast<uint32_t*>(ctx->f_dkey[1].p)};
  uint32_t* dv[2] = {static_cast<uint32_t*>(ctx->f_dval[0].p), static_cast<uint32_t*>(ctx->f_dval[1].p)};
  uint32_t* soff = static_cast<uint32_t*>(ctx->f_soff.p);
  int32_t* diff = use_diff ? static_cast<int32_t*>(ctx->f_diff.p) : nullptr;
  uint32_t* scratch = static_cast<uint32_t*>(ctx->sort_scratch.p);
  uint32_t* bar = ctx->d_tickets + 2;

  // 1-3
  TDGS_TRACED(ctx, kKFrameCount, n, s,
              launch_frame_count(rec, n, fg, counts, dk[0], dv[0], diff, count_grid, err_word(ctx), s));
  for (uint32_t p = 0; p < kDepthPasses; ++p) {
    TDGS_TRACED(ctx, kKDepthSort, n, s,
                launch_depth_pass(dgrid, p, dk[p & 1], dv[p & 1], dk[(p + 1) & 1], dv[(p + 1) & 1], n,
                                  scratch, bar, err_word(ctx), s));
  }
  const uint32_t* sdepth = dk[kDepthPasses & 1];
  const uint32_t* sorder = dv[kDepthPasses & 1];
  if (n) {
    st = do_scan(ctx, counts, nullptr, sorder, fg, n, soff, &ctx->d_status->total, nullptr, s);
    if (st != TDGS_OK) return st;
  } else {
    TDGS_CUDA(ctx, cudaMemsetAsync(&ctx->d_status->total, 0, 8, s));
  }
  // 4
  TDGS_CUDA(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(DevStatus),
                                 cudaMemcpyDeviceToHost, s));
  TDGS_CUDA(ctx, cudaStreamSynchronize(s));
  if (ctx->h_status->err) {
    const tdgs_status e = static_cast<tdgs_status>(ctx->h_status->err);
    TDGS_CUDA(ctx, cudaMemsetAsync(&ctx->d_status->err, 0, 4, s));
    return fail(ctx, e, "error latched on the device");
  }
  const uint64_t total = ctx->h_status->total;
  if (total > 0xffffffffull) return fail(ctx, TDGS_ERR_OVERFLOW, "pair count above 2^32-1");
  const uint32_t m = static_cast<uint32_t>(total);
  const size_t esz = wide ? 8 : 4;
  for (int b = 0; b < 2 && st == TDGS_OK; ++b)
    st = ensure(ctx, ctx->f_stream[b], static_cast<size_t>(m) * esz + 16, s);
  if (st == TDGS_OK) st = ensure(ctx, ctx->f_keys, static_cast<size_t>(m) * 8 + 16, s);
  if (st == TDGS_OK) st = ensure(ctx, ctx->f_values, static_cast<size_t>(m) * 4 + 16, s);
  // 5-6
  const uint32_t npass = tb <= 8 ? 1u : 2u;
  const uint32_t w0 = npass == 1 ? tb : (tb + 1) / 2;
  const uint32_t sgrid = stream_grid(wide, npass == 1, m ? m : 1);
  const uint32_t sgrid_x = stream_grid(wide, true, m ? m : 1);
  if (sgrid == 0 || sgrid_x == 0) return fail(ctx, TDGS_ERR_CUDA, "device query for the tile sort failed");
  if (st == TDGS_OK)
    st = ensure(ctx, ctx->sort_scratch,
                std::max(stream_scratch_words(wide, false, sgrid), stream_scratch_words(wide, true, sgrid_x)) * 4,
                s);
  if (st != TDGS_OK) return st;
  scratch = static_cast<uint32_t*>(ctx->sort_scratch.p);
  void* s0 = ctx->f_stream[0].p;
  void* s1 = ctx->f_stream[1].p;
  uint64_t* okeys = static_cast<uint64_t*>(ctx->f_keys.p);
  uint32_t* ovals = static_cast<uint32_t*>(ctx->f_values.p);
  TDGS_TRACED(ctx, kKDupDepth, m ? n : 0, s,
              launch_dup_depth(rec, sorder, soff, n, fg, rbits, s0, wide, m, err_word(ctx), s));
  if (npass == 1) {
    TDGS_TRACED(ctx, kKTilePass, m, s,
                launch_stream_pass(wide, true, sgrid_x, s0, okeys, ovals, m, rbits, tb, rbits, sdepth,
                                   sorder, scratch, bar, err_word(ctx), s));
  } else {
    TDGS_TRACED(ctx, kKTilePass, m, s,
                launch_stream_pass(wide, false, sgrid, s0, s1, nullptr, m, rbits, w0, rbits, sdepth,
                                   sorder, scratch, bar, err_word(ctx), s));
    TDGS_TRACED(ctx, kKTilePass, m, s,
                launch_stream_pass(wide, true, sgrid_x, s1, okeys, ovals, m, rbits + w0, tb - w0, rbits,
                                   sdepth, sorder, scratch, bar, err_word(ctx), s));
  }
  // 7
  uint2* rg = static_cast<uint2*>(ctx->f_ranges.p);
  if (use_diff && n) {
    TDGS_TRACED(ctx, kKRangesDiff, T, s,
                launch_ranges_from_diff(diff, count_grid, fg, diff + count_grid * cells, rg,
                                        err_word(ctx), s));
  } else {
    TDGS_CUDA(ctx, cudaMemsetAsync(rg, 0, static_cast<size_t>(T) * 8, s));
    TDGS_TRACED(ctx, kKRanges, m, s, launch_tile_ranges(okeys, m, T, rg, err_word(ctx), s));
  }
  *sorted_keys = okeys;
  *sorted_values = ovals;
  *ranges = reinterpret_cast<const tdgs_range*>(rg);
  *m_out = m;
  return TDGS_OK;
}

}  // extern "C"
