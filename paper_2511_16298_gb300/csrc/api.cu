// C ABI of libtdgs: argument checks, scratch management and launch order.
// Every call maps one step (or the fused frame) of the 3DGS sort step
// described in Sec. II-A to the kernels of frame_kernels.cu and
// sort_kernels.cu.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <new>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "render.cuh"
#include "tdgs_internal.cuh"

using namespace tdgs;

namespace {

// Device words read back by the host: the pair count of the fused frame and
// the latched error, adjacent so one 16-byte copy fetches both.
struct DevStatus {
  uint64_t total;
  uint32_t err;
  uint32_t site;  // which kernel latched err (ErrorSite)
};

const char* site_name(uint32_t site) {
  switch (site) {
    case kSiteCount: return "tile count";
    case kSiteScan: return "scan";
    case kSiteScanTimeout: return "scan look-back wait";
    case kSiteDuplicate: return "duplicate_keys";
    case kSiteRanges: return "tile_ranges";
    case kSiteRadixKeys: return "radix pass key check";
    case kSiteRadixRange: return "radix pass destination out of range";
    case kSiteRadixCapacity: return "radix pass count above reserved capacity";
    case kSiteBarrier: return "radix pass grid barrier wait";
    case kSiteViewsCount: return "frame count";
    case kSiteViewsDup: return "duplicate by depth";
    case kSiteRender: return "render (a sorted value is not a Gaussian index)";
  }
  return "device";
}

// The early pair count in mapped host memory: the count kernel writes
// {total, err, site}; the single launch that counts and sorts writes the
// tagged word seq (16 bits) << 48 | min(error, 255) << 40 | min(M, 2^40 - 1).
struct EarlyStatus {
  uint64_t total;
  uint32_t err;
  uint32_t site;
  uint64_t tagged;
  uint64_t pad;
};

struct Buffer {
  void* p = nullptr;
  size_t bytes = 0;
};

enum KernelId {
  kKCount, kKScan, kKDuplicate, kKRanges, kKRadixPass,
  kKFrameCount, kKDepthSort, kKFrameScan, kKDupDepth, kKTilePass, kKTileExpand, kKPreprocess, kKBitonic, kKRender, kKPreCount, kKNormRange, kKNormDup, kKNormPass,
  kKNormRanges, kKRenderOrder, kKSortHist, kKOnesweep, kKCountDepth, kKNum
};
const char* const kKernelNames[kKNum] = {
    "count_tiles",  "scan",       "duplicate_keys",     "tile_ranges",    "radix_pass",
    "frame_count",  "depth_sort", "scan_by_depth", "duplicate_by_depth", "tile_sort_pass",
    "tile_expand_pass", "preprocess", "bitonic_sort", "render", "preprocess_count", "norm_range",
    "norm_duplicate", "norm_sort_pass", "norm_ranges", "render_order", "sort_histogram", "onesweep_pass",
    "count_depth_sort"};

// View table as stored in device memory (SoA, fixed maximum size).
struct ViewBlob {
  const float4* g[kMaxViews];
  uint64_t vtot[kMaxViews];
  FrameGeom geom[kMaxViews];
  uint32_t rec_begin[kMaxViews + 1];
  uint32_t tile_begin[kMaxViews + 1];
  uint32_t pbeg[kMaxViews + 1];
  uint32_t nt[kMaxViews];
};

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
  // Pinned and mapped: the count kernel writes the pair count and the error
  // word here itself, so reading them back needs no copy (a copy would
  // queue behind other streams' large downloads on the copy engine).
  EarlyStatus* h_early = nullptr;
  EarlyStatus* d_early = nullptr;  // its device address
  cudaEvent_t ev_count = nullptr;  // recorded after the count kernel (or the launch that counts and sorts)
  uint32_t early_seq = 0;          // the last seq asked of the launch that counts and sorts
  bool early_fused = false;        // the last front half counted inside the depth sort
  uint32_t* d_tickets = nullptr;  // [1] count blocks (reset by the kernel), [2..3] radix grid barrier
  uint32_t ticket_base[2] = {0, 0};
  Buffer scan_status, sort_scratch;
  Buffer os_scratch;  // onesweep sort: histograms, digit starts, tickets, look-back status
  Buffer f_dsort;     // single-launch depth sort: barrier counters, totals, rows (kept zero between launches)
  Buffer f_dos;       // onesweep depth sort (large N): histograms, digit starts, tickets, look-back status
  // State that kernels keep between launches, to be cleared before its next
  // use after an error was latched on the device (a bounded wait may have
  // given up mid-launch): the depth sort's buffers, the onesweep header, the
  // radix grid barrier words.
  bool dsort_dirty = true, dos_dirty = true, os_dirty = false, bar_dirty = false;
  // fused-frame / multi-view buffers
  Buffer f_rec3, f_conic;  // projected records and conics of tdgs_sort_frame_3d
  Buffer d_cams;           // cameras of the 3D calls (device)
  Buffer diag;             // barrier words of tdgs_diag_barrier_timeout
  Buffer r_order;          // tile order of tdgs_render (heaviest first)
  uint32_t render_wave = 0;  // rendering blocks resident at once (0: not queried yet)
  Proj3D proj{};           // 3D calls: the count kernel projects first
  bool proj_on = false;
  Buffer b_keys, b_vals;   // padded scratch of tdgs_sort_pairs_bitonic
  Buffer n_counts, n_offs, n_norm, n_keys[2], n_vals[2], n_ranges;  // tdgs_sort_frame_normalized
  Buffer f_counts, f_dkey[3], f_dval[3], f_soff, f_sdo, f_rminmax, f_stream[2], f_keys, f_values, f_ranges;
  // depth-key range: accumulators [0..1], result [2..3], passes of the last
  // resident depth sort [4]
  uint32_t* d_range = nullptr;
  // f_rminmax holds first positions in its first half and one-past-last
  // positions in its second half, kept at (all ones, zero) between frames:
  // the ranges kernel resets what the last tile pass recorded
  bool rminmax_dirty = true;
  ViewBlob* d_views = nullptr;  // device view table
  ViewBlob* h_views = nullptr;  // pinned staging of the table
  uint32_t nv = 0, n_all = 0, t_all = 0;
  uint64_t capacity = 0;        // pair capacity reserved for the asynchronous path
  bool reserved = false;
  Tuning tuning;
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

void note_device_error(tdgs_context* ctx) {
  ctx->dsort_dirty = ctx->dos_dirty = ctx->os_dirty = ctx->bar_dirty = true;
}

// The radix grid barrier words back to zero if an error was latched since
// their last use.
tdgs_status clear_barrier_if_dirty(tdgs_context* ctx, cudaStream_t s) {
  if (ctx->bar_dirty) {
    TDGS_CUDA(ctx, cudaMemsetAsync(ctx->d_tickets + 2, 0, 2 * sizeof(uint32_t), s));
    ctx->bar_dirty = false;
  }
  return TDGS_OK;
}

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

tdgs_status do_scan(tdgs_context* ctx, KernelId id, const uint32_t* counts, const float4* recs,
                    const uint32_t* gather, FrameGeom fg, uint32_t n, uint32_t* offsets,
                    uint64_t* total64, uint32_t* total32, cudaStream_t s) {
  // scan_status: the tile ticket in word 0, then one status word per tile;
  // one memset clears both
  const uint32_t tiles = (n + kScanTileItems - 1) / kScanTileItems;
  tdgs_status st = ensure(ctx, ctx->scan_status, static_cast<size_t>(tiles) * 8 + 8, s);
  if (st != TDGS_OK) return st;
  TDGS_CUDA(ctx, cudaMemsetAsync(ctx->scan_status.p, 0, static_cast<size_t>(tiles) * 8 + 8, s));
  uint64_t* words = static_cast<uint64_t*>(ctx->scan_status.p);
  TDGS_TRACED(ctx, id, n, s,
              launch_scan(counts, recs, gather, fg, n, offsets, words + 1, reinterpret_cast<uint32_t*>(words), 0u,
                          total64, total32, err_word(ctx), s));
  return TDGS_OK;
}

tdgs_status do_sort(tdgs_context* ctx, uint64_t* keys, uint32_t* values, uint64_t* keys_alt,
                    uint32_t* values_alt, uint32_t m, uint32_t tile_bits, uint32_t flags,
                    int* result_in_alt, cudaStream_t s) {
  *result_in_alt = 0;
  if (m == 0) return TDGS_OK;
  if (tdgs_status st0 = clear_barrier_if_dirty(ctx, s); st0 != TDGS_OK) return st0;
  const SortPlan plan = make_sort_plan(m, tile_bits, flags, ctx->tuning);
  if (ctx->tuning.sort_variant < 0 && onesweep_eligible(m, keys, values, keys_alt, values_alt)) {
    bool grown = false;
    tdgs_status st = ensure(ctx, ctx->os_scratch, onesweep_scratch_words(m) * 4, s, &grown);
    if (st != TDGS_OK) return st;
    uint32_t* scratch = static_cast<uint32_t*>(ctx->os_scratch.p);
    if (grown || ctx->os_dirty) TDGS_CUDA(ctx, cudaMemsetAsync(scratch, 0, onesweep_header_words() * 4, s));
    ctx->os_dirty = false;
    TDGS_TRACED(ctx, kKSortHist, m, s, launch_onesweep_hist(plan, keys, m, scratch, err_word(ctx), s));
    uint64_t* kin = keys;
    uint32_t* vin = values;
    uint64_t* kout = keys_alt;
    uint32_t* vout = values_alt;
    for (uint32_t p = 0; p < plan.passes; ++p) {
      TDGS_TRACED(ctx, kKOnesweep, m, s,
                  launch_onesweep_pass(plan, p, kin, vin, kout, vout, m, scratch, err_word(ctx), s));
      std::swap(kin, kout);
      std::swap(vin, vout);
    }
    *result_in_alt = static_cast<int>(plan.passes & 1u);
    return TDGS_OK;
  }
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
  TDGS_CUDA(ctx, cudaMemcpyAsync(&ctx->h_status->err, &ctx->d_status->err, 8,
                                 cudaMemcpyDeviceToHost, s));
  TDGS_CUDA(ctx, cudaStreamSynchronize(s));
  const uint32_t e = ctx->h_status->err;
  if (e != 0) {
    note_device_error(ctx);
    TDGS_CUDA(ctx, cudaMemsetAsync(&ctx->d_status->err, 0, 8, s));
    TDGS_CUDA(ctx, cudaStreamSynchronize(s));
    return fail(ctx, static_cast<tdgs_status>(e),
                std::string("error latched on the device by ") + site_name(ctx->h_status->site));
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

tdgs_status tdgs_sort_variant_info(int i, int* bits, int* threads, int* items, int* blocks_per_sm) {
  if (i < 0 || i >= num_pass_variants()) return TDGS_ERR_INVALID_ARGUMENT;
  const PassVariant v = pass_variant(i);
  if (bits) *bits = v.bits;
  if (threads) *threads = v.threads;
  if (items) *items = v.items;
  if (blocks_per_sm) *blocks_per_sm = v.blocks_per_sm;
  return TDGS_OK;
}

tdgs_status tdgs_context_set_tuning(tdgs_context* ctx, int key, int value) {
  if (!ctx) return TDGS_ERR_INVALID_ARGUMENT;
  switch (key) {
    case TDGS_TUNE_SORT_VARIANT:
      if (value < -1 || value >= num_pass_variants()) return TDGS_ERR_INVALID_ARGUMENT;
      ctx->tuning.sort_variant = value;
      return TDGS_OK;
    case TDGS_TUNE_TILE_DIGIT_BITS:
      if (value != 0 && (value < 4 || value > 12)) return TDGS_ERR_INVALID_ARGUMENT;
      ctx->tuning.tile_digit_bits = value;
      return TDGS_OK;
    case TDGS_TUNE_CTAS_PER_SM:
      if (value < 0 || value > 8) return TDGS_ERR_INVALID_ARGUMENT;
      ctx->tuning.ctas_per_sm = value;
      return TDGS_OK;
    case TDGS_TUNE_DEPTH_DIGIT_BITS:
      if (value != 0 && value != 8 && value != 11) return TDGS_ERR_INVALID_ARGUMENT;
      ctx->tuning.depth_digit_bits = value;
      return TDGS_OK;
  }
  return TDGS_ERR_INVALID_ARGUMENT;
}

tdgs_status tdgs_context_get_tuning(const tdgs_context* ctx, int key, int* value) {
  if (!ctx || !value) return TDGS_ERR_INVALID_ARGUMENT;
  switch (key) {
    case TDGS_TUNE_SORT_VARIANT: *value = ctx->tuning.sort_variant; return TDGS_OK;
    case TDGS_TUNE_TILE_DIGIT_BITS: *value = ctx->tuning.tile_digit_bits; return TDGS_OK;
    case TDGS_TUNE_CTAS_PER_SM: *value = ctx->tuning.ctas_per_sm; return TDGS_OK;
    case TDGS_TUNE_DEPTH_DIGIT_BITS: *value = ctx->tuning.depth_digit_bits; return TDGS_OK;
  }
  return TDGS_ERR_INVALID_ARGUMENT;
}

tdgs_status tdgs_context_set_sort_variant(tdgs_context* ctx, int variant) {
  if (!ctx || variant < -1 || variant >= num_pass_variants()) return TDGS_ERR_INVALID_ARGUMENT;
  ctx->tuning.sort_variant = variant;
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
      cudaMalloc(&ctx->d_range, 8 * sizeof(uint32_t)) != cudaSuccess ||
      cudaMemset(ctx->d_range, 0, 8 * sizeof(uint32_t)) != cudaSuccess ||
      cudaMemset(ctx->d_range, 0xff, sizeof(uint32_t)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_status, sizeof(DevStatus)) != cudaSuccess ||
      cudaHostAlloc(&ctx->h_early, sizeof(EarlyStatus), cudaHostAllocMapped) != cudaSuccess ||
      cudaHostGetDevicePointer(reinterpret_cast<void**>(&ctx->d_early), ctx->h_early, 0) != cudaSuccess ||
      cudaMalloc(&ctx->d_views, sizeof(ViewBlob)) != cudaSuccess ||
      cudaMallocHost(&ctx->h_views, sizeof(ViewBlob)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(DevStatus)) != cudaSuccess ||
      cudaMemset(ctx->d_tickets, 0, 4 * sizeof(uint32_t)) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->ev_count, cudaEventDisableTiming) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    tdgs_context_destroy(ctx);
    return TDGS_ERR_OUT_OF_MEMORY;
  }
  // pinned memory may come back from an earlier allocation: no stale seq
  std::memset(ctx->h_early, 0, sizeof(EarlyStatus));
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

tdgs_status tdgs_context_depth_passes(tdgs_context* ctx, int* passes, void* stream) {
  if (!ctx || !passes) return TDGS_ERR_INVALID_ARGUMENT;
  DeviceGuard g(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t v = 0;
  TDGS_CUDA(ctx, cudaMemcpyAsync(&v, ctx->d_range + 4, 4, cudaMemcpyDeviceToHost, s));
  TDGS_CUDA(ctx, cudaStreamSynchronize(s));
  *passes = static_cast<int>(v);
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
  Buffer* bufs[] = {&ctx->scan_status, &ctx->sort_scratch, &ctx->os_scratch, &ctx->f_dsort, &ctx->f_dos, &ctx->f_counts, &ctx->f_dkey[0],
                    &ctx->f_dkey[1],    &ctx->f_dkey[2],     &ctx->f_dval[0],    &ctx->f_dval[1],
                    &ctx->f_dval[2],    &ctx->f_soff,       &ctx->f_sdo,        &ctx->f_rec3,
                    &ctx->f_conic,      &ctx->d_cams,       &ctx->diag,       &ctx->b_keys,       &ctx->b_vals,       &ctx->n_counts,
                    &ctx->n_offs,       &ctx->n_norm,       &ctx->n_keys[0],    &ctx->n_keys[1],
                    &ctx->n_vals[0],    &ctx->n_vals[1],    &ctx->n_ranges,
                    &ctx->f_rminmax,    &ctx->f_stream[0],   &ctx->f_stream[1],  &ctx->f_keys,
                    &ctx->f_values,     &ctx->f_ranges,     &ctx->r_order};
  if (ctx->d_views) cudaFree(ctx->d_views);
  if (ctx->h_views) cudaFreeHost(ctx->h_views);
  for (Buffer* b : bufs)
    if (b->p) cudaFree(b->p);
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->d_tickets) cudaFree(ctx->d_tickets);
  if (ctx->d_range) cudaFree(ctx->d_range);
  if (ctx->h_status) cudaFreeHost(ctx->h_status);
  if (ctx->h_early) cudaFreeHost(ctx->h_early);
  if (ctx->ev_count) cudaEventDestroy(ctx->ev_count);
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
  return do_scan(ctx, kKScan, counts, nullptr, nullptr, FrameGeom{}, n, offsets, nullptr, total_dev, s);
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

tdgs_status tdgs_sort_pairs_bitonic(tdgs_context* ctx, const uint64_t* keys_in, const uint32_t* values_in,
                                    uint64_t* keys_out, uint32_t* values_out, uint32_t m, void* stream) {
  if (!ctx) return TDGS_ERR_INVALID_ARGUMENT;
  if (m == 0) return TDGS_OK;
  if (m > (1u << 31)) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "at most 2^31 pairs");
  if (!keys_in || !values_in || !keys_out || !values_out) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null pointer");
  if (!aligned(keys_in, 8) || !aligned(keys_out, 8) || !aligned(values_in, 4) || !aligned(values_out, 4))
    return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "misaligned pointer");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n2 = bitonic_padded(m);
  tdgs_status st = ensure(ctx, ctx->b_keys, n2 * 8, s);
  if (st == TDGS_OK) st = ensure(ctx, ctx->b_vals, n2 * 4, s);
  if (st != TDGS_OK) return st;
  TDGS_TRACED(ctx, kKBitonic, m, s,
              launch_bitonic(keys_in, values_in, m, keys_out, values_out, static_cast<uint64_t*>(ctx->b_keys.p),
                             static_cast<uint32_t*>(ctx->b_vals.p), s));
  return TDGS_OK;
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

}  // extern "C"

namespace {

uint32_t bits_for(uint64_t count) {  // smallest b with count <= 2^b
  uint32_t b = 0;
  while (b < 64 && (1ull << b) < count) ++b;
  return b;
}

// Validate the views, fill the pinned staging table and the totals.
tdgs_status stage_views(tdgs_context* ctx, const tdgs_view* views, uint32_t nv) {
  if (nv == 0 || nv > kMaxViews) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "view count out of range");
  if (!views) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null views");
  ViewBlob* h = ctx->h_views;
  uint64_t n_all = 0, t_all = 0;
  for (uint32_t v = 0; v < nv; ++v) {
    const tdgs_view& w = views[v];
    if (w.f.width == 0 || w.f.height == 0) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "empty image");
    if (w.n && !w.g) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null pointer");
    if (!aligned(w.g, 16)) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "misaligned pointer");
    h->g[v] = reinterpret_cast<const float4*>(w.g);
    h->geom[v] = make_geom(w.f);
    h->rec_begin[v] = static_cast<uint32_t>(n_all);
    h->tile_begin[v] = static_cast<uint32_t>(t_all);
    h->nt[v] = tdgs_num_tiles(w.f);
    h->vtot[v] = 0;
    n_all += w.n;
    t_all += h->nt[v];
  }
  if (n_all > 0xffffffffull || t_all > 0xffffffffull)
    return fail(ctx, TDGS_ERR_OVERFLOW, "too many Gaussians or tiles in one batch");
  h->rec_begin[nv] = static_cast<uint32_t>(n_all);
  h->tile_begin[nv] = static_cast<uint32_t>(t_all);
  ctx->nv = nv;
  ctx->n_all = static_cast<uint32_t>(n_all);
  ctx->t_all = static_cast<uint32_t>(t_all);
  return TDGS_OK;
}

ViewTable device_table(tdgs_context* ctx) {
  ViewBlob* d = ctx->d_views;
  ViewTable vt;
  vt.g = d->g;
  vt.rec_begin = d->rec_begin;
  vt.tile_begin = d->tile_begin;
  vt.geom = d->geom;
  vt.vtot = d->vtot;
  vt.pbeg = d->pbeg;
  vt.nv = ctx->nv;
  return vt;
}

struct Shape {
  uint32_t rbits, tbits;
  bool wide;
  uint32_t npass, w0;
  uint32_t kbits;  // compiled digit width of the tile passes before the last
  uint32_t klast;  // compiled digit width of the last (expanding) pass, for its own width
};

Shape shape_of(const tdgs_context* ctx) {
  Shape sh;
  sh.rbits = bits_for(ctx->n_all);
  sh.tbits = bits_for(ctx->t_all);
  sh.wide = sh.tbits + sh.rbits > 32 || sh.rbits >= 32;
  // digit width of the tile passes: at most 8 bits by default (12 if
  // tuned: one pass, but its scatter writes runs of about one element per
  // digit, which costs more than a second pass); the bits are split evenly
  // over the passes
  const uint32_t dmax = ctx->tuning.tile_digit_bits > 0 ? static_cast<uint32_t>(ctx->tuning.tile_digit_bits) : 8u;
  sh.npass = sh.tbits <= dmax ? 1u : (sh.tbits + dmax - 1) / dmax;
  sh.w0 = (sh.tbits + sh.npass - 1) / std::max(1u, sh.npass);
  sh.kbits = stream_kernel_bits(sh.w0);
  sh.klast = stream_kernel_bits(sh.tbits - (sh.npass - 1) * sh.w0);  // e.g. 13 tile bits: 7 + 6
  return sh;
}

// Buffers that depend only on the record and tile counts.
tdgs_status ensure_record_buffers(tdgs_context* ctx, cudaStream_t s) {
  const size_t n4 = static_cast<size_t>(ctx->n_all) * 4 + 16;
  tdgs_status st = TDGS_OK;
  for (Buffer* b : {&ctx->f_counts, &ctx->f_dkey[0], &ctx->f_dkey[1], &ctx->f_dkey[2], &ctx->f_dval[0],
                    &ctx->f_dval[1], &ctx->f_dval[2], &ctx->f_soff})
    if (st == TDGS_OK) st = ensure(ctx, *b, n4, s);
  if (st == TDGS_OK) st = ensure(ctx, ctx->f_sdo, static_cast<size_t>(ctx->n_all) * 8 + 16, s);
  bool grown = false;
  if (st == TDGS_OK) st = ensure(ctx, ctx->f_rminmax, static_cast<size_t>(ctx->t_all) * 8 + 16, s, &grown);
  if (grown) ctx->rminmax_dirty = true;
  if (st == TDGS_OK) st = ensure(ctx, ctx->f_ranges, static_cast<size_t>(ctx->t_all) * 8 + 16, s);
  const uint32_t n_all = ctx->n_all;
  const uint32_t tiles = (n_all + kScanTileItems - 1) / kScanTileItems;
  if (st == TDGS_OK) st = ensure(ctx, ctx->scan_status, static_cast<size_t>(tiles) * 8 + 8, s);
  const DepthPlan dp = plan_depth_sort(n_all, ctx->tuning.depth_digit_bits, ctx->tuning.ctas_per_sm);
  if (dp.grid == 0) return fail(ctx, TDGS_ERR_CUDA, "device query for the depth sort failed");
  if (st == TDGS_OK) st = ensure(ctx, ctx->sort_scratch, dp.scratch_words * 4, s);
  if (st == TDGS_OK && dp.resident) {
    grown = false;
    st = ensure(ctx, ctx->f_dsort, depth_sort_scratch_words(dp.grid) * 4, s, &grown);
    if (st == TDGS_OK && (grown || ctx->dsort_dirty)) {
      TDGS_CUDA(ctx, cudaMemsetAsync(ctx->f_dsort.p, 0, ctx->f_dsort.bytes, s));
      ctx->dsort_dirty = false;
    }
  }
  if (st == TDGS_OK && dp.onesweep) {
    grown = false;
    st = ensure(ctx, ctx->f_dos, onesweep_scratch_words(n_all ? n_all : 1) * 4, s, &grown);
    if (st == TDGS_OK && (grown || ctx->dos_dirty)) {
      TDGS_CUDA(ctx, cudaMemsetAsync(ctx->f_dos.p, 0, onesweep_header_words() * 4, s));
      ctx->dos_dirty = false;
    }
  }
  return st;
}

// Buffers that depend on the pair count (or capacity) m.
tdgs_status ensure_pair_buffers(tdgs_context* ctx, uint64_t m, cudaStream_t s) {
  const Shape sh = shape_of(ctx);
  const size_t esz = sh.wide ? 8 : 4;
  tdgs_status st = TDGS_OK;
  for (int b = 0; b < 2 && st == TDGS_OK; ++b) st = ensure(ctx, ctx->f_stream[b], m * esz + 16, s);
  if (st == TDGS_OK) st = ensure(ctx, ctx->f_keys, m * 8 + 16, s);
  if (st == TDGS_OK) st = ensure(ctx, ctx->f_values, m * 4 + 16, s);
  const uint32_t mm = static_cast<uint32_t>(m ? m : 1);
  const int cps = ctx->tuning.ctas_per_sm;
  const uint32_t g0 = stream_grid(sh.wide, false, sh.kbits, mm, cps), g1 = stream_grid(sh.wide, true, sh.klast, mm, cps);
  if (g0 == 0 || g1 == 0) return fail(ctx, TDGS_ERR_CUDA, "device query for the tile sort failed");
  if (st == TDGS_OK)
    st = ensure(ctx, ctx->sort_scratch,
                std::max(stream_scratch_words(sh.wide, false, sh.kbits, g0),
                         stream_scratch_words(sh.wide, true, sh.klast, g1)) * 4,
                s);
  return st;
}

// Steps before the pair count is known: view table upload, counts, depth
// sort, scan in depth order (total -> d_status->total).
tdgs_status run_front(tdgs_context* ctx, cudaStream_t s, bool early_total = false) {
  const ViewTable vt = device_table(ctx);
  const uint32_t n_all = ctx->n_all;
  if (tdgs_status st0 = clear_barrier_if_dirty(ctx, s); st0 != TDGS_OK) return st0;
  TDGS_CUDA(ctx, cudaMemcpyAsync(ctx->d_views, ctx->h_views, sizeof(ViewBlob), cudaMemcpyHostToDevice, s));
  uint32_t* counts = static_cast<uint32_t*>(ctx->f_counts.p);
  uint32_t* dk[3] = {static_cast<uint32_t*>(ctx->f_dkey[0].p), static_cast<uint32_t*>(ctx->f_dkey[1].p),
                     static_cast<uint32_t*>(ctx->f_dkey[2].p)};
  uint32_t* dv[3] = {static_cast<uint32_t*>(ctx->f_dval[0].p), static_cast<uint32_t*>(ctx->f_dval[1].p),
                     static_cast<uint32_t*>(ctx->f_dval[2].p)};
  const DepthPlan dp = plan_depth_sort(n_all, ctx->tuning.depth_digit_bits, ctx->tuning.ctas_per_sm);
  DepthSortArgs da{};
  da.vt = vt;
  da.total = &ctx->d_status->total;
  da.k1 = dk[1];
  da.v1 = dv[1];
  da.k2 = dk[2];
  da.v2 = dv[2];
  da.counts = counts;
  da.offsets = static_cast<uint32_t*>(ctx->f_soff.p);
  da.range = ctx->d_range;
  da.n = n_all;
  da.scratch = static_cast<uint32_t*>(ctx->f_dsort.p);
  da.err = err_word(ctx);
  ctx->early_fused = dp.resident && n_all > 0 && n_all <= depth_sort_count_capacity(dp.grid) && !ctx->proj_on;
  if (ctx->early_fused) {
    // one launch: counts, M (also to the mapped host status, tagged with a
    // fresh seq), the depth sort and the offsets
    if (early_total) {
      da.host_status = reinterpret_cast<uint32_t*>(&ctx->d_early->tagged);
      ctx->early_seq = (ctx->early_seq + 1) & 0xffffu;
      if (ctx->early_seq == 0) ctx->early_seq = 1;  // 0: never written
      da.host_seq = ctx->early_seq;
    }
    TDGS_TRACED(ctx, kKCountDepth, n_all, s, launch_count_depth_sort(dp.grid, da, s));
    if (early_total) TDGS_CUDA(ctx, cudaEventRecord(ctx->ev_count, s));
    return TDGS_OK;
  }
  // launched even for zero Gaussians: it writes the view starts and M = 0
  TDGS_TRACED(ctx, ctx->proj_on ? kKPreCount : kKFrameCount, n_all ? n_all : 1, s,
              launch_views_count(vt, n_all, counts, dk[0], dv[0], err_word(ctx), ctx->d_tickets + 1,
                                 &ctx->d_status->total, ctx->d_range, early_total ? ctx->d_early : nullptr, s,
                                 ctx->proj_on ? &ctx->proj : nullptr));
  if (early_total) {
    // M (and any latched error) as soon as the count kernel is done: the
    // kernel wrote them to the mapped host status (h_early)
    TDGS_CUDA(ctx, cudaEventRecord(ctx->ev_count, s));
  }
  const uint32_t dpasses = dp.passes;
  uint32_t* scratch = static_cast<uint32_t*>(ctx->sort_scratch.p);
  if (dp.resident) {  // one launch: the sort (pass count from the depth range) and the offsets
    da.key0 = dk[0];
    TDGS_TRACED(ctx, kKDepthSort, n_all, s, launch_depth_sort(dp.grid, da, s));
  } else if (dp.onesweep) {  // histogram, then the passes the key range needs (result in pair 1)
    if (n_all) {
      uint32_t* dos = static_cast<uint32_t*>(ctx->f_dos.p);
      TDGS_TRACED(ctx, kKDepthSort, n_all, s,
                  launch_depth_onesweep_hist(dk[0], n_all, ctx->d_range, dos, err_word(ctx), s));
      for (uint32_t p = 0; p < dpasses; ++p)
        TDGS_TRACED(ctx, kKDepthSort, n_all, s,
                    launch_depth_onesweep_pass(p, dk, dv, n_all, ctx->d_range, dos, err_word(ctx), s));
    }
  } else {
    for (uint32_t p = 0; p < dpasses; ++p) {
      TDGS_TRACED(ctx, kKDepthSort, n_all, s,
                  launch_depth_pass(dp, p, dk[p & 1], dv[p & 1], dk[(p + 1) & 1], dv[(p + 1) & 1], n_all, scratch,
                                    ctx->d_tickets + 2, err_word(ctx), s));
    }
  }
  if (n_all && !dp.resident) {
    tdgs_status st = do_scan(ctx, kKFrameScan, counts, nullptr, dv[dp.result], FrameGeom{}, n_all,
                             static_cast<uint32_t*>(ctx->f_soff.p), &ctx->d_status->total, nullptr, s);
    if (st != TDGS_OK) return st;
  } else if (n_all == 0) {
    TDGS_CUDA(ctx, cudaMemsetAsync(&ctx->d_status->total, 0, 8, s));
  }
  return TDGS_OK;
}

// Steps after: duplication, tile passes, ranges.  m = exact pair count, or
// the reserved capacity with m_dev pointing at the device count.
tdgs_status run_back(tdgs_context* ctx, uint32_t m, const uint64_t* m_dev, cudaStream_t s) {
  const ViewTable vt = device_table(ctx);
  const Shape sh = shape_of(ctx);
  const uint32_t n_all = ctx->n_all;
  const uint32_t dres = plan_depth_sort(n_all, ctx->tuning.depth_digit_bits, ctx->tuning.ctas_per_sm).result;
  const uint32_t* sorder = static_cast<uint32_t*>(ctx->f_dval[dres].p);
  uint2* sdo = static_cast<uint2*>(ctx->f_sdo.p);
  uint32_t* scratch = static_cast<uint32_t*>(ctx->sort_scratch.p);
  uint32_t* bar = ctx->d_tickets + 2;
  void* st[2] = {ctx->f_stream[0].p, ctx->f_stream[1].p};
  const size_t half = ctx->f_rminmax.bytes / 8;  // tiles the buffer holds
  uint32_t* rmin = static_cast<uint32_t*>(ctx->f_rminmax.p);
  uint32_t* rmax = rmin + half;
  TDGS_TRACED(ctx, kKDupDepth, m ? n_all : 0, s,
              launch_views_dup(vt, sorder, static_cast<uint32_t*>(ctx->f_soff.p), n_all, sh.rbits, st[0],
                               sh.wide, m, sdo, err_word(ctx), s));
  // One pass over the whole tile id writes the ranges from its digit
  // totals; with several passes the last one records each tile's first and
  // last position and a small kernel turns them into ranges.
  const bool single = sh.npass == 1;
  uint2* ranges = static_cast<uint2*>(ctx->f_ranges.p);
  if (m == 0) {
    TDGS_CUDA(ctx, cudaMemsetAsync(ranges, 0, static_cast<size_t>(ctx->t_all) * 8, s));
    return TDGS_OK;
  }
  if (!single) {
    if (ctx->rminmax_dirty) {
      TDGS_CUDA(ctx, cudaMemsetAsync(rmin, 0xff, half * 4, s));
      TDGS_CUDA(ctx, cudaMemsetAsync(rmax, 0, half * 4, s));
    }
    ctx->rminmax_dirty = true;  // until the last pass below is enqueued
  }
  uint32_t shift = sh.rbits;
  for (uint32_t p = 0; p < sh.npass; ++p) {
    const bool last = p + 1 == sh.npass;
    const uint32_t width = last ? sh.tbits - (shift - sh.rbits) : sh.w0;
    StreamPass sp{};
    sp.wide = sh.wide;
    sp.expand = last;
    sp.bits = last ? sh.klast : sh.kbits;
    sp.grid = stream_grid(sh.wide, last, sp.bits, m, ctx->tuning.ctas_per_sm);
    sp.kin = st[p & 1];
    sp.kout = last ? ctx->f_keys.p : st[(p + 1) & 1];
    sp.vout = last ? static_cast<uint32_t*>(ctx->f_values.p) : nullptr;
    sp.m = m;
    sp.m_dev = m_dev;
    sp.shift = shift;
    sp.width = width;
    sp.rbits = sh.rbits;
    sp.sdo = sdo;
    sp.views = &vt;
    sp.rmin = last && !single ? rmin : nullptr;
    sp.rmax = last && !single ? rmax : nullptr;
    sp.ranges = last ? ranges : nullptr;
    sp.t_all = ctx->t_all;
    TDGS_TRACED(ctx, last ? kKTileExpand : kKTilePass, m, s, launch_stream_pass(sp, scratch, bar, err_word(ctx), s));
    shift += width;
  }
  if (!single) ctx->rminmax_dirty = false;  // the last pass turned them into ranges and reset them
  return TDGS_OK;
}

// Exact mode.  The count kernel already sums the pairs (M), so the host
// copies M right after it and waits on that copy alone, while the depth
// sort and the scan run; the back half is then enqueued with the exact M
// before the GPU runs out of work.
tdgs_status sort_views_exact(tdgs_context* ctx, cudaStream_t s, uint32_t* m_out) {
  tdgs_status st = ensure_record_buffers(ctx, s);
  if (st != TDGS_OK) return st;
  st = run_front(ctx, s, true);
  if (st != TDGS_OK) return st;
  uint32_t early_err = 0;
  uint64_t early_total = 0;
  if (ctx->early_fused) {
    // the launch that counts and sorts writes M early and keeps running:
    // wait for the word with its seq
    uint64_t* tp = &ctx->h_early->tagged;
    uint64_t w = __atomic_load_n(tp, __ATOMIC_ACQUIRE);
    while ((w >> 48) != ctx->early_seq) {
      const cudaError_t q = cudaEventQuery(ctx->ev_count);
      if (q == cudaSuccess) {
        w = __atomic_load_n(tp, __ATOMIC_ACQUIRE);
        if ((w >> 48) == ctx->early_seq) break;
        return fail(ctx, TDGS_ERR_CUDA, "the depth sort ended without reporting the pair count");
      }
      if (q != cudaErrorNotReady) return cuda_fail(ctx, q, "cudaEventQuery");
      w = __atomic_load_n(tp, __ATOMIC_ACQUIRE);
    }
    early_err = static_cast<uint32_t>((w >> 40) & 0xffu);
    early_total = w & ((1ull << 40) - 1);
  } else {
    TDGS_CUDA(ctx, cudaEventSynchronize(ctx->ev_count));
    const volatile EarlyStatus* early = ctx->h_early;
    early_err = early->err;
    early_total = early->total;
  }
  if (early_err) {
    note_device_error(ctx);
    TDGS_CUDA(ctx, cudaStreamSynchronize(s));
    TDGS_CUDA(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    TDGS_CUDA(ctx, cudaStreamSynchronize(s));
    const tdgs_status e = static_cast<tdgs_status>(ctx->h_status->err);
    TDGS_CUDA(ctx, cudaMemsetAsync(&ctx->d_status->err, 0, 8, s));
    return fail(ctx, e, std::string("error latched on the device by ") + site_name(ctx->h_status->site));
  }
  const uint64_t total = early_total;
  if (total > 0xffffffffull) {  // the scan latches the same overflow: clear it
    TDGS_CUDA(ctx, cudaStreamSynchronize(s));
    TDGS_CUDA(ctx, cudaMemsetAsync(&ctx->d_status->err, 0, 8, s));
    return fail(ctx, TDGS_ERR_OVERFLOW, "pair count above 2^32-1");
  }
  const uint32_t m = static_cast<uint32_t>(total);
  st = ensure_pair_buffers(ctx, m, s);
  if (st != TDGS_OK) return st;
  st = run_back(ctx, m, nullptr, s);
  if (st != TDGS_OK) return st;
  *m_out = m;
  return TDGS_OK;
}

// Per-view results, read after the work on `s` is complete.
tdgs_status fill_results(tdgs_context* ctx, tdgs_view_result* results, uint32_t nv, cudaStream_t s) {
  tdgs_status st = read_and_clear_error(ctx, s);
  if (st != TDGS_OK) return st;
  TDGS_CUDA(ctx, cudaMemcpyAsync(ctx->h_views->pbeg, ctx->d_views->pbeg, sizeof(uint32_t) * (nv + 1),
                                 cudaMemcpyDeviceToHost, s));
  TDGS_CUDA(ctx, cudaStreamSynchronize(s));
  const uint64_t* k = static_cast<const uint64_t*>(ctx->f_keys.p);
  const uint32_t* v = static_cast<const uint32_t*>(ctx->f_values.p);
  const tdgs_range* r = static_cast<const tdgs_range*>(ctx->f_ranges.p);
  for (uint32_t i = 0; i < nv; ++i) {
    const uint32_t b = ctx->h_views->pbeg[i], e = ctx->h_views->pbeg[i + 1];
    results[i].keys = k + b;
    results[i].values = v + b;
    results[i].ranges = r + ctx->h_views->tile_begin[i];
    results[i].m = e - b;
    results[i].num_tiles = ctx->h_views->nt[i];
  }
  return TDGS_OK;
}

// Camera validation for the preprocessing calls (host pointer).
tdgs_status check_camera(tdgs_context* ctx, const tdgs_camera* cam, CameraDev* out) {
  if (!cam) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null camera");
  if (!(cam->fx > 0.0f) || !(cam->fy > 0.0f) || !std::isfinite(cam->fx) || !std::isfinite(cam->fy))
    return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "focal length must be finite and > 0");
  if (cam->width == 0 || cam->height == 0) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "empty image");
  static_assert(sizeof(tdgs_camera) == sizeof(CameraDev), "camera layout");
  std::memcpy(out, cam, sizeof(CameraDev));
  return TDGS_OK;
}

// Preprocessing fused into the count kernel for nv cameras of the same n
// 3D Gaussians, then the rest of the fused frame over the nv views.
tdgs_status sort_views_3d(tdgs_context* ctx, const tdgs_gaussian3d* g, const tdgs_cov3d* cov, uint32_t n,
                          const tdgs_camera* cams, uint32_t nv, cudaStream_t s, uint32_t* m_out) {
  if (nv == 0 || nv > kMaxViews) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "view count out of range");
  if (!cams) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null camera");
  std::vector<CameraDev> cd(nv);
  for (uint32_t v = 0; v < nv; ++v) {
    tdgs_status st = check_camera(ctx, cams + v, &cd[v]);
    if (st != TDGS_OK) return st;
  }
  if (n && (!g || !cov)) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null pointer");
  if (!aligned(g, 16) || !aligned(cov, 16)) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "misaligned pointer");
  if (static_cast<uint64_t>(n) * nv > 0xffffffffull)
    return fail(ctx, TDGS_ERR_OVERFLOW, "too many Gaussians in one batch");
  const size_t total = static_cast<size_t>(n) * nv;
  tdgs_status st = ensure(ctx, ctx->f_rec3, total * 16 + 16, s);
  if (st == TDGS_OK) st = ensure(ctx, ctx->f_conic, total * 16 + 16, s);
  if (st == TDGS_OK) st = ensure(ctx, ctx->d_cams, sizeof(CameraDev) * nv, s);
  if (st != TDGS_OK) return st;
  TDGS_CUDA(ctx, cudaMemcpyAsync(ctx->d_cams.p, cd.data(), sizeof(CameraDev) * nv, cudaMemcpyHostToDevice, s));
  // the count kernel projects each view's Gaussians first (preprocessing
  // fused with the count) and stores records and conics view after view
  std::vector<tdgs_view> views(nv);
  const tdgs_gaussian2d* rec = static_cast<const tdgs_gaussian2d*>(ctx->f_rec3.p);
  for (uint32_t v = 0; v < nv; ++v) views[v] = tdgs_view{rec + static_cast<size_t>(v) * n, n,
                                                        tdgs_frame{cams[v].width, cams[v].height}};
  st = stage_views(ctx, views.data(), nv);
  if (st != TDGS_OK) return st;
  ctx->reserved = false;
  ctx->proj = Proj3D{reinterpret_cast<const float4*>(g), reinterpret_cast<const float4*>(cov),
                     static_cast<float4*>(ctx->f_rec3.p), static_cast<float4*>(ctx->f_conic.p),
                     static_cast<const CameraDev*>(ctx->d_cams.p), cd[0]};
  ctx->proj_on = true;
  st = sort_views_exact(ctx, s, m_out);
  ctx->proj_on = false;
  return st;
}

}  // namespace

extern "C" {

tdgs_status tdgs_sort_frame(tdgs_context* ctx, const tdgs_gaussian2d* g, uint32_t n,
                            tdgs_frame f, const uint64_t** sorted_keys,
                            const uint32_t** sorted_values, const tdgs_range** ranges,
                            uint32_t* m_out, void* stream) {
  if (!ctx || !sorted_keys || !sorted_values || !ranges || !m_out)
    return TDGS_ERR_INVALID_ARGUMENT;
  *m_out = 0;
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tdgs_view view{g, n, f};
  tdgs_status st = stage_views(ctx, &view, 1);
  if (st != TDGS_OK) return st;
  ctx->reserved = false;
  uint32_t m = 0;
  st = sort_views_exact(ctx, s, &m);
  if (st != TDGS_OK) return st;
  *sorted_keys = static_cast<const uint64_t*>(ctx->f_keys.p);
  *sorted_values = static_cast<const uint32_t*>(ctx->f_values.p);
  *ranges = static_cast<const tdgs_range*>(ctx->f_ranges.p);
  *m_out = m;
  return TDGS_OK;
}

tdgs_status tdgs_preprocess(tdgs_context* ctx, const tdgs_gaussian3d* g, const tdgs_cov3d* cov,
                            uint32_t n, const tdgs_camera* cam, tdgs_gaussian2d* records,
                            float* conic_opacity, void* stream) {
  if (!ctx) return TDGS_ERR_INVALID_ARGUMENT;
  CameraDev cd;
  tdgs_status st = check_camera(ctx, cam, &cd);
  if (st != TDGS_OK) return st;
  if (n == 0) return TDGS_OK;
  if (!g || !cov || !records) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null pointer");
  if (!aligned(g, 16) || !aligned(cov, 16) || !aligned(records, 16) ||
      (conic_opacity && !aligned(conic_opacity, 16)))
    return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "misaligned pointer");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TDGS_TRACED(ctx, kKPreprocess, n, s,
              launch_preprocess(reinterpret_cast<const float4*>(g), reinterpret_cast<const float4*>(cov), n, cd,
                                reinterpret_cast<float4*>(records), reinterpret_cast<float4*>(conic_opacity), s));
  return TDGS_OK;
}

tdgs_status tdgs_sort_frame_3d(tdgs_context* ctx, const tdgs_gaussian3d* g, const tdgs_cov3d* cov,
                               uint32_t n, const tdgs_camera* cam, const tdgs_gaussian2d** records,
                               const float** conic_opacity, const uint64_t** sorted_keys,
                               const uint32_t** sorted_values, const tdgs_range** ranges,
                               uint32_t* m_out, void* stream) {
  if (!ctx || !sorted_keys || !sorted_values || !ranges || !m_out) return TDGS_ERR_INVALID_ARGUMENT;
  *m_out = 0;
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t m = 0;
  tdgs_status st = sort_views_3d(ctx, g, cov, n, cam, 1, s, &m);
  if (st != TDGS_OK) return st;
  if (records) *records = static_cast<const tdgs_gaussian2d*>(ctx->f_rec3.p);
  if (conic_opacity) *conic_opacity = static_cast<const float*>(ctx->f_conic.p);
  *sorted_keys = static_cast<const uint64_t*>(ctx->f_keys.p);
  *sorted_values = static_cast<const uint32_t*>(ctx->f_values.p);
  *ranges = static_cast<const tdgs_range*>(ctx->f_ranges.p);
  *m_out = m;
  return TDGS_OK;
}

tdgs_status tdgs_sort_views_3d(tdgs_context* ctx, const tdgs_gaussian3d* g, const tdgs_cov3d* cov, uint32_t n,
                               const tdgs_camera* cams, uint32_t num_views, tdgs_view_result* results,
                               void* stream) {
  if (!ctx || !results) return TDGS_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  uint32_t m = 0;
  tdgs_status st = sort_views_3d(ctx, g, cov, n, cams, num_views, s, &m);
  if (st != TDGS_OK) return st;
  return fill_results(ctx, results, num_views, s);
}

}  // extern "C"

namespace tdgs {
// Failure-detection check (diag.cu): two blocks of which only one reaches
// the radix passes' grid barrier on bar (two zeroed words of its own); the
// bounded wait gives up and latches TDGS_ERR_TIMEOUT in err.
cudaError_t launch_diag_barrier_timeout(uint32_t* bar, uint32_t* err, cudaStream_t s);
}  // namespace tdgs

extern "C" {

tdgs_status tdgs_diag_barrier_timeout(tdgs_context* ctx, void* stream) {
  if (!ctx) return TDGS_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tdgs_status st = ensure(ctx, ctx->diag, 16, s);
  if (st != TDGS_OK) return st;
  TDGS_CUDA(ctx, cudaMemsetAsync(ctx->diag.p, 0, 16, s));
  TDGS_CUDA(ctx, launch_diag_barrier_timeout(static_cast<uint32_t*>(ctx->diag.p), err_word(ctx), s));
  return TDGS_OK;
}

tdgs_status tdgs_context_projected(tdgs_context* ctx, const tdgs_gaussian2d** records,
                                   const float** conic_opacity) {
  if (!ctx) return TDGS_ERR_INVALID_ARGUMENT;
  if (records) *records = static_cast<const tdgs_gaussian2d*>(ctx->f_rec3.p);
  if (conic_opacity) *conic_opacity = static_cast<const float*>(ctx->f_conic.p);
  return TDGS_OK;
}

tdgs_status tdgs_sort_frame_normalized(tdgs_context* ctx, const tdgs_gaussian2d* g, uint32_t n, tdgs_frame f,
                                       const uint32_t** sorted_keys, const uint32_t** sorted_values,
                                       const tdgs_range** ranges, uint32_t* m_out, void* stream) {
  if (!ctx || !sorted_keys || !sorted_values || !ranges || !m_out) return TDGS_ERR_INVALID_ARGUMENT;
  *m_out = 0;
  if (f.width == 0 || f.height == 0) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "empty image");
  const uint64_t T = static_cast<uint64_t>((f.width + 15) / 16) * ((f.height + 15) / 16);
  if (T > (1u << 20)) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "the 32-bit key holds at most 2^20 tiles");
  if (n && !g) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null pointer");
  if (!aligned(g, 16)) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "misaligned pointer");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t n4 = static_cast<size_t>(n) * 4 + 16;
  tdgs_status st = ensure(ctx, ctx->n_counts, n4, s);
  if (st == TDGS_OK) st = ensure(ctx, ctx->n_offs, n4, s);
  if (st == TDGS_OK) st = ensure(ctx, ctx->n_norm, 16, s);
  if (st == TDGS_OK) st = ensure(ctx, ctx->n_ranges, T * 8 + 16, s);
  if (st != TDGS_OK) return st;
  uint32_t* counts = static_cast<uint32_t*>(ctx->n_counts.p);
  uint32_t* offs = static_cast<uint32_t*>(ctx->n_offs.p);
  uint32_t* norm = static_cast<uint32_t*>(ctx->n_norm.p);
  uint2* rg = static_cast<uint2*>(ctx->n_ranges.p);
  const float4* g4 = reinterpret_cast<const float4*>(g);
  const FrameGeom geom = make_geom(f);
  TDGS_CUDA(ctx, cudaMemsetAsync(rg, 0, T * 8, s));
  uint32_t m = 0;
  if (n) {
    TDGS_TRACED(ctx, kKCount, n, s, launch_count_tiles(g4, n, geom, counts, err_word(ctx), s));
    TDGS_CUDA(ctx, cudaMemsetAsync(norm, 0xff, 4, s));
    TDGS_CUDA(ctx, cudaMemsetAsync(norm + 1, 0, 4, s));
    TDGS_TRACED(ctx, kKNormRange, n, s, launch_norm_range(g4, counts, n, norm, s));
    st = do_scan(ctx, kKScan, counts, nullptr, nullptr, FrameGeom{}, n, offs, &ctx->d_status->total, nullptr, s);
    if (st != TDGS_OK) return st;
    TDGS_CUDA(ctx, cudaMemcpyAsync(ctx->h_status, ctx->d_status, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    TDGS_CUDA(ctx, cudaStreamSynchronize(s));
    if (ctx->h_status->err) return read_and_clear_error(ctx, s);
    if (ctx->h_status->total > 0xffffffffull) return fail(ctx, TDGS_ERR_OVERFLOW, "pair count above 2^32-1");
    m = static_cast<uint32_t>(ctx->h_status->total);
  }
  const size_t m4 = static_cast<size_t>(m) * 4 + 16;
  for (int i = 0; i < 2 && st == TDGS_OK; ++i) {
    st = ensure(ctx, ctx->n_keys[i], m4, s);
    if (st == TDGS_OK) st = ensure(ctx, ctx->n_vals[i], m4, s);
  }
  if (st != TDGS_OK) return st;
  uint32_t* k[2] = {static_cast<uint32_t*>(ctx->n_keys[0].p), static_cast<uint32_t*>(ctx->n_keys[1].p)};
  uint32_t* v[2] = {static_cast<uint32_t*>(ctx->n_vals[0].p), static_cast<uint32_t*>(ctx->n_vals[1].p)};
  uint32_t res = 0;
  if (m) {
    TDGS_TRACED(ctx, kKNormDup, n, s, launch_duplicate_norm(g4, offs, n, geom, k[0], v[0], m, norm, err_word(ctx), s));
    uint32_t tb = 0;
    while ((1ull << tb) < T) ++tb;
    const DepthPlan dp = plan_key32_sort(m, 10 + tb, ctx->tuning.ctas_per_sm);
    if (dp.grid == 0) return fail(ctx, TDGS_ERR_CUDA, "device query for the sort plan failed");
    st = ensure(ctx, ctx->sort_scratch, dp.scratch_words * 4, s);
    if (st != TDGS_OK) return st;
    for (uint32_t p = 0; p < dp.passes; ++p)
      TDGS_TRACED(ctx, kKNormPass, m, s,
                  launch_depth_pass(dp, p, k[p & 1], v[p & 1], k[(p + 1) & 1], v[(p + 1) & 1], m,
                                    static_cast<uint32_t*>(ctx->sort_scratch.p), ctx->d_tickets + 2,
                                    err_word(ctx), s));
    res = dp.result;
    TDGS_TRACED(ctx, kKNormRanges, m, s,
                launch_tile_ranges_norm(k[res], m, static_cast<uint32_t>(T), rg, err_word(ctx), s));
  }
  *sorted_keys = k[res];
  *sorted_values = v[res];
  *ranges = reinterpret_cast<const tdgs_range*>(rg);
  *m_out = m;
  return TDGS_OK;
}

tdgs_status tdgs_render(tdgs_context* ctx, const tdgs_gaussian2d* records, const float* conic_opacity,
                        const float* rgb, uint32_t n, const uint32_t* sorted_values, const tdgs_range* ranges,
                        tdgs_frame f, const float* background, float* image, void* stream) {
  if (!ctx) return TDGS_ERR_INVALID_ARGUMENT;
  if (f.width == 0 || f.height == 0) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "empty image");
  if (!ranges || !image || !background) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null pointer");
  if (n && (!records || !conic_opacity || !rgb))
    return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "null pointer");
  if (!aligned(records, 16) || !aligned(conic_opacity, 16) || !aligned(rgb, 4) || !aligned(sorted_values, 4) ||
      !aligned(ranges, 8) || !aligned(image, 4))
    return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "misaligned pointer");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t tiles = static_cast<uint64_t>((f.width + 15) / 16) * ((f.height + 15) / 16);
  if (tiles > 0x7fffffffull) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "image too large");
  const float4* rec4 = reinterpret_cast<const float4*>(records);
  const float4* con4 = reinterpret_cast<const float4*>(conic_opacity);
  const uint2* rg = reinterpret_cast<const uint2*>(ranges);
  if (ctx->render_wave == 0) ctx->render_wave = render_wave_blocks(ctx->device);
  if (tiles <= ctx->render_wave) {  // one wave: the order cannot shorten it
    TDGS_TRACED(ctx, kKRender, tiles, s,
                launch_render(rec4, con4, rgb, sorted_values, rg, f.width, f.height, background, n, image,
                              err_word(ctx), s));
    return TDGS_OK;
  }
  tdgs_status st = ensure(ctx, ctx->r_order, tiles * 4, s);
  if (st != TDGS_OK) return st;
  uint32_t* order = static_cast<uint32_t*>(ctx->r_order.p);
  TDGS_TRACED(ctx, kKRenderOrder, tiles, s, launch_render_order(rg, static_cast<uint32_t>(tiles), order, s));
  TDGS_TRACED(ctx, kKRender, tiles, s,
              launch_render_ordered(rec4, con4, rgb, sorted_values, rg, order, f.width, f.height, background, n,
                                    image, err_word(ctx), s));
  return TDGS_OK;
}

tdgs_status tdgs_sort_views(tdgs_context* ctx, const tdgs_view* views, uint32_t num_views,
                            tdgs_view_result* results, void* stream) {
  if (!ctx || !results) return TDGS_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tdgs_status st = stage_views(ctx, views, num_views);
  if (st != TDGS_OK) return st;
  ctx->reserved = false;
  uint32_t m = 0;
  st = sort_views_exact(ctx, s, &m);
  if (st != TDGS_OK) return st;
  return fill_results(ctx, results, num_views, s);
}

tdgs_status tdgs_reserve_views(tdgs_context* ctx, const tdgs_view* views, uint32_t num_views,
                               uint64_t pair_capacity, void* stream) {
  if (!ctx) return TDGS_ERR_INVALID_ARGUMENT;
  if (pair_capacity > 0xffffffffull) return fail(ctx, TDGS_ERR_OVERFLOW, "capacity above 2^32-1");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  tdgs_status st = stage_views(ctx, views, num_views);
  if (st == TDGS_OK) st = ensure_record_buffers(ctx, s);
  if (st == TDGS_OK) st = ensure_pair_buffers(ctx, pair_capacity, s);
  if (st != TDGS_OK) return st;
  TDGS_CUDA(ctx, cudaStreamSynchronize(s));
  ctx->capacity = pair_capacity;
  ctx->reserved = true;
  return TDGS_OK;
}

tdgs_status tdgs_sort_views_async(tdgs_context* ctx, const tdgs_view* views, uint32_t num_views,
                                  void* stream) {
  if (!ctx) return TDGS_ERR_INVALID_ARGUMENT;
  if (!ctx->reserved) return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "call tdgs_reserve_views first");
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint32_t n_prev = ctx->n_all, t_prev = ctx->t_all, nv_prev = ctx->nv;
  tdgs_status st = stage_views(ctx, views, num_views);
  if (st != TDGS_OK) return st;
  if (ctx->n_all != n_prev || ctx->t_all != t_prev || ctx->nv != nv_prev)
    return fail(ctx, TDGS_ERR_INVALID_ARGUMENT, "views differ in shape from the reservation");
  st = run_front(ctx, s);
  if (st != TDGS_OK) return st;
  return run_back(ctx, static_cast<uint32_t>(ctx->capacity), &ctx->d_status->total, s);
}

tdgs_status tdgs_views_results(tdgs_context* ctx, tdgs_view_result* results, uint32_t num_views,
                               void* stream) {
  if (!ctx || !results || num_views != ctx->nv) return TDGS_ERR_INVALID_ARGUMENT;
  DeviceGuard dg(ctx->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return fill_results(ctx, results, num_views, s);
}

}  // extern "C"
