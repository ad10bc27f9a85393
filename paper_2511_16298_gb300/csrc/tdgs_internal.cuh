// Internal declarations shared by the CUDA translation units of libtdgs.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>

#include "tdgs.h"

namespace tdgs {

constexpr int kTile = 16;             // 16x16-pixel screen tiles (Sec. II-A)
constexpr uint32_t kSpinLimit = 1u << 21;  // bounded cross-block waits (~0.1-1 s)

// ---------------------------------------------------------------- geometry
struct FrameGeom {
  int32_t gx, gy;    // tiles per row / column
  float gxf, gyf;    // the same as floats, for clamping
};

inline FrameGeom make_geom(tdgs_frame f) {
  FrameGeom g;
  g.gx = static_cast<int32_t>((f.width + kTile - 1) / kTile);
  g.gy = static_cast<int32_t>((f.height + kTile - 1) / kTile);
  g.gxf = static_cast<float>(g.gx);
  g.gyf = static_cast<float>(g.gy);
  return g;
}

// Outcome of the tile test for one Gaussian.
struct TileRect {
  int32_t x0, y0, x1, y1;  // covered tiles [x0,x1) x [y0,y1)
  uint32_t count;          // (x1-x0)*(y1-y0), 0 when culled/off-screen/invalid
  bool invalid;            // visible but with a bad mean or depth
};

// Tile rectangle of a projected Gaussian (Sec. II-A: the footprint's
// axis-aligned box, intersected with the 16x16 tile grid).  Box edges are
// rounded float32 values taken in a fixed order, with no contraction:
// x0 = floor((x - r) / 16), x1 = floor(((x + r) + 15) / 16), likewise for y,
// each clamped to [0, grid].  Multiplying by 1/16 is exact.
__device__ __forceinline__ TileRect tile_rect(float x, float y, float depth, int32_t r,
                                              const FrameGeom& fg) {
  TileRect q;
  q.x0 = q.y0 = q.x1 = q.y1 = 0;
  q.count = 0;
  q.invalid = false;
  if (r <= 0) return q;
  if (!isfinite(x) || !isfinite(y)) {
    q.invalid = true;
    return q;
  }
  const float rf = __int2float_rn(r);
  const float sx0 = __fsub_rn(x, rf);
  const float sx1 = __fadd_rn(__fadd_rn(x, rf), 15.0f);
  const float sy0 = __fsub_rn(y, rf);
  const float sy1 = __fadd_rn(__fadd_rn(y, rf), 15.0f);
  const float fx0 = fminf(fmaxf(floorf(__fmul_rn(sx0, 0.0625f)), 0.0f), fg.gxf);
  const float fx1 = fminf(fmaxf(floorf(__fmul_rn(sx1, 0.0625f)), 0.0f), fg.gxf);
  const float fy0 = fminf(fmaxf(floorf(__fmul_rn(sy0, 0.0625f)), 0.0f), fg.gyf);
  const float fy1 = fminf(fmaxf(floorf(__fmul_rn(sy1, 0.0625f)), 0.0f), fg.gyf);
  q.x0 = __float2int_rz(fx0);
  q.x1 = __float2int_rz(fx1);
  q.y0 = __float2int_rz(fy0);
  q.y1 = __float2int_rz(fy1);
  if (q.x1 <= q.x0 || q.y1 <= q.y0) {
    q.x0 = q.y0 = q.x1 = q.y1 = 0;
    return q;
  }
  // Keys carry raw depth bits: only finite depths > +0.0 keep their order.
  if (!(isfinite(depth) && depth > 0.0f)) {
    q.invalid = true;
    q.x0 = q.y0 = q.x1 = q.y1 = 0;
    return q;
  }
  q.count = static_cast<uint32_t>(q.x1 - q.x0) * static_cast<uint32_t>(q.y1 - q.y0);
  return q;
}

__device__ __forceinline__ TileRect tile_rect(const float4 rec, const FrameGeom& fg) {
  return tile_rect(rec.x, rec.y, rec.z, __float_as_int(rec.w), fg);
}

// ------------------------------------------------------------ device sync
// The first non-zero code wins; later errors are dropped.  err[1] records
// which site latched it (kSite* below), for the host's error message.
enum ErrorSite : uint32_t {
  kSiteNone = 0, kSiteCount, kSiteScan, kSiteScanTimeout, kSiteDuplicate, kSiteRanges,
  kSiteRadixKeys, kSiteRadixRange, kSiteRadixCapacity, kSiteBarrier, kSiteViewsCount, kSiteViewsDup,
  kSiteRender
};
__device__ __forceinline__ void latch_error(uint32_t* err, uint32_t code, uint32_t site = kSiteNone) {
  if (atomicCAS(err, 0u, code) == 0u) err[1] = site;
}

__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint32_t* p, uint32_t v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ uint64_t ld_acquire(const uint64_t* p) {
  uint64_t v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release(uint64_t* p, uint64_t v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31u; }
__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ------------------------------------------------------------- host side
// Per-call status helpers used by the API layer.
struct Scratch {
  void* ptr = nullptr;
  size_t bytes = 0;
};

// Launchers (each returns a cudaError_t from the launch).
cudaError_t launch_count_tiles(const float4* g, uint32_t n, FrameGeom fg, uint32_t* counts,
                               uint32_t* err, cudaStream_t s);

// Decoupled look-back exclusive scan.  With recs != nullptr the counts are
// computed from the records (count and scan fused); otherwise read from
// counts.  status: one uint64 per kScanTileItems (8192) counts, zeroed by the caller.
constexpr uint32_t kScanTileItems = 8192;
cudaError_t launch_scan(const uint32_t* counts, const float4* recs, const uint32_t* gather,
                        FrameGeom fg, uint32_t n, uint32_t* offsets, uint64_t* status,
                        uint32_t* ticket, uint32_t ticket_base, uint64_t* total64,
                        uint32_t* total32, uint32_t* err, cudaStream_t s);

cudaError_t launch_duplicate(const float4* g, const uint32_t* offsets, uint32_t n,
                             FrameGeom fg, uint64_t* keys, uint32_t* values, uint32_t cap,
                             uint32_t* err, cudaStream_t s);

cudaError_t launch_tile_ranges(const uint64_t* keys, uint32_t m, uint32_t num_tiles,
                               uint2* ranges, uint32_t* err, cudaStream_t s);
// The paper's 32-bit normalised key (Sec. IV-B): depth range of the
// Gaussians with pairs (norm[0..1], float bits, all ones / zero on entry),
// duplication into tile << 10 | 10-bit normalised depth, ranges from them.
cudaError_t launch_norm_range(const float4* g, const uint32_t* counts, uint32_t n, uint32_t* norm, cudaStream_t s);
cudaError_t launch_duplicate_norm(const float4* g, const uint32_t* offsets, uint32_t n, FrameGeom fg,
                                  uint32_t* keys, uint32_t* values, uint32_t cap, const uint32_t* norm,
                                  uint32_t* err, cudaStream_t s);
cudaError_t launch_tile_ranges_norm(const uint32_t* keys, uint32_t m, uint32_t num_tiles, uint2* ranges,
                                    uint32_t* err, cudaStream_t s);

// ---- depth-first frame path over a table of views (one view = one frame)
constexpr uint32_t kMaxViews = 256;
struct ViewTable {             // device arrays
  const float4* const* g;      // [nv] records of each view
  const uint32_t* rec_begin;   // [nv+1] global index of each view's first record
  const uint32_t* tile_begin;  // [nv+1] global id of each view's first tile
  const FrameGeom* geom;       // [nv]
  uint64_t* vtot;              // [nv] pair count per view (accumulated, zeroed beforehand)
  uint32_t* pbeg;              // [nv+1] first pair of each view in the sorted list
  uint32_t nv;
};

// Largest v with begin[v] <= i (begin ascending, begin[0] = 0).
__device__ __forceinline__ uint32_t find_view(const uint32_t* begin, uint32_t nv, uint32_t i) {
  uint32_t lo = 0, hi = nv;  // answer in [lo, hi)
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (begin[mid] <= i) lo = mid; else hi = mid;
  }
  return lo;
}

// Counts, depth keys and indices of all records, per-view pair totals, and
// (last block) the first pair of each view and the pair count in *total.
// ticket: a zero word, left zero.  range: four words, [0..1] all ones and
// zero on entry and exit; [2..3] receive the smallest and largest depth key
// of a Gaussian with pairs.
// Bitonic sort of m (key, value) pairs by (key, value) (tdgs_sort_pairs_bitonic):
// kin/vin -> kout/vout (may alias), scratch ks/vs of bitonic_padded(m) pairs.
uint32_t bitonic_padded(uint32_t m);
uint32_t bitonic_launches(uint32_t m);
cudaError_t launch_bitonic(const uint64_t* kin, const uint32_t* vin, uint32_t m, uint64_t* kout, uint32_t* vout,
                           uint64_t* ks, uint32_t* vs, cudaStream_t s);

// Front-to-back blending of each 16x16 tile's sorted Gaussians into an
// interleaved float RGB image (height x width x 3); bg: 3 host floats; n:
// Gaussians (a sorted value >= n is skipped and latches an error).
cudaError_t launch_render(const float4* rec, const float4* conic, const float* rgb, const uint32_t* values,
                          const uint2* ranges, uint32_t width, uint32_t height, const float* bg, uint32_t n,
                          float* image, uint32_t* err, cudaStream_t s);

// Camera of the preprocessing kernel (the layout of tdgs_camera).
struct CameraDev {
  float rot[9];
  float trans[3];
  float fx, fy, cx, cy, near_z;
  uint32_t width, height;
};
static_assert(sizeof(CameraDev) == 76, "camera block");
// Preprocessing of n 3D Gaussians (g: mean + opacity; cov: two 16-byte
// words per Gaussian) into 16-byte records and (if conic != nullptr)
// conic/opacity words.
cudaError_t launch_preprocess(const float4* g, const float4* cov, uint32_t n, const CameraDev& cam, float4* rec,
                              float4* conic, cudaStream_t s);

// Preprocessing fused into the count kernel: every view is the same n3
// Gaussians seen by its own camera; global record i of view v (local
// index l = i - rec_begin[v]) is projected from g[l] and cov[2l..2l+1] for
// cams[v], stored as rec[i] / conic[i], and counted.
struct Proj3D {
  const float4* g;
  const float4* cov;
  float4* rec;
  float4* conic;
  const CameraDev* cams;  // device, one per view
  CameraDev cam0;         // cams[0], passed by value (kernel parameter space) for one view
};

// host_status (optional): device address of mapped pinned memory that
// also receives {uint64 pair count, uint32 error, uint32 site} from the
// last block (the host reads it after an event on the kernel, no copy).
cudaError_t launch_views_count(const ViewTable& vt, uint32_t n_all, uint32_t* counts,
                               uint32_t* dkey, uint32_t* dval, uint32_t* err, uint32_t* ticket,
                               uint64_t* total, uint32_t* range, void* host_status, cudaStream_t s,
                               const Proj3D* proj = nullptr);
// sdo: receives {depth key, record index} per depth position (read by the
// expanding tile pass with one 8-byte load per pair).
cudaError_t launch_views_dup(const ViewTable& vt, const uint32_t* sorder, const uint32_t* soff,
                             uint32_t n_all, uint32_t rbits, void* out, bool wide, uint32_t cap,
                             uint2* sdo, uint32_t* err, cudaStream_t s);

// Radix passes of the frame path (radix_frame.cu, depth_sort.cu).
// Depth sort of the N Gaussians: (uint32 depth key, uint32 index), over
// keys compressed to their range (key - smallest; culled Gaussians one past
// the largest) with as many 9-bit digits as that range needs (3 for a range
// below 2^27, 4 at most).  When the Gaussians fit one 8192-key chunk per
// resident CTA, the whole sort and the scan of the tile counts in depth
// order run in one cooperative launch (launch_depth_sort).  Larger N (below
// 2^30) take the onesweep passes over 32-bit keys (onesweep.cu): a
// histogram launch and kDepthOnesweepPasses pass launches, each reading the
// pass plan from the key range (passes beyond it end at once), the result
// in buffer pair 1; the scan of the counts in depth order follows.
// Otherwise one launch per pass over all 32 bits: 8-bit (4 passes) or, if
// tuned, 11-bit (3 passes) digits.
struct DepthPlan {
  bool resident;          // one launch; keys compressed to their range, passes chosen on the device
  bool onesweep;          // the onesweep passes over compressed 32-bit keys
  int bits;
  uint32_t passes, grid;  // passes: the most that run; grid 0: the device query failed
  uint32_t result;        // which of the three buffer pairs holds the sorted keys and indices
  size_t scratch_words;
};
DepthPlan plan_depth_sort(uint32_t n, int tuned_bits, int ctas_per_sm);
// Stable sort of m (u32 key, u32 value) pairs on the low key_bits bits with
// the per-pass 11-bit kernel (launch_depth_pass); result in pair passes & 1.
DepthPlan plan_key32_sort(uint32_t m, uint32_t key_bits, int ctas_per_sm);
cudaError_t launch_depth_pass(const DepthPlan& dp, uint32_t pass, const uint32_t* kin, const uint32_t* vin,
                              uint32_t* kout, uint32_t* vout, uint32_t n, uint32_t* scratch, uint32_t* bar,
                              uint32_t* err, cudaStream_t s);
// Single-launch depth sort (depth_sort.cu).  Grid: one CTA per SM (0 if
// the device query failed); it takes n <= depth_sort_count_capacity(grid)
// keys (one tile of 8192 per CTA), with or without the count step.
// Results: v1 = record indices in depth order, offsets = the exclusive scan
// of the tile counts in that order (the pair offsets in depth order); k1
// receives the counts in depth order, (k2, v2) are intermediate.  range:
// [0..1] running smallest / largest key of a Gaussian with pairs (all ones
// / zero between frames), [2..3] that range for the sort, [4] receives the
// number of passes run.  scratch: depth_sort_scratch_words(grid) words of
// state kept between launches, zero before the first launch and after an
// error latched in err.
//  * With count (launch_count_depth_sort) the tile count step runs in the
//    same launch: the records of the view table in; each view's pair total
//    and first pair (vt), M (total) and range[2..3] out, and one 8-byte
//    word to host_status (mapped host memory, or null): host_seq (16 bits)
//    << 48 | min(latched error, 255) << 40 | min(M, 2^40 - 1); counts
//    receives only counts of 1023 or more.
//  * Without (launch_depth_sort): key0 = the count kernel's depth keys,
//    counts its tile counts, range[2..3] its range.
struct DepthSortArgs {
  const uint32_t* key0;
  ViewTable vt;
  uint64_t* total;
  uint32_t* host_status;
  uint32_t host_seq;
  uint32_t *k1, *v1, *k2, *v2;
  uint32_t* counts;
  uint32_t* offsets;
  uint32_t* range;
  uint32_t n;
  uint32_t* scratch;
  uint32_t* err;
};
uint32_t depth_sort_grid();
uint32_t depth_sort_count_capacity(uint32_t grid);
size_t depth_sort_scratch_words(uint32_t grid);
cudaError_t launch_depth_sort(uint32_t grid, const DepthSortArgs& a, cudaStream_t s);
cudaError_t launch_count_depth_sort(uint32_t grid, const DepthSortArgs& a, cudaStream_t s);
// Stable pass over the packed stream on tile bits [shift, shift + width).
// expand: write the final (local tile << 32 | depth bits) keys and local
// indices; with rmin/rmax, record each global tile's first/last sorted
// position; with ranges (a single pass over the whole tile id), write the
// view-local tile ranges from the digit totals.
// m_dev (optional): device copy of the element count, capped at m.
struct StreamPass {
  bool wide, expand;
  uint32_t bits;           // compiled digit width (stream_kernel_bits)
  uint32_t grid;
  const void* kin;
  void* kout;
  uint32_t* vout;
  uint32_t m;
  const uint64_t* m_dev;
  uint32_t shift, width, rbits;
  const uint2* sdo;  // by depth position: {depth bits, record index}
  const ViewTable* views;  // expand only
  uint32_t* rmin;
  uint32_t* rmax;
  uint2* ranges;
  uint32_t t_all;
};
// Compiled digit width (6, 8 or 12) that holds a `width`-bit digit.
uint32_t stream_kernel_bits(uint32_t width);
uint32_t stream_grid(bool wide, bool expand, uint32_t bits, uint32_t m, int ctas_per_sm);
size_t stream_scratch_words(bool wide, bool expand, uint32_t bits, uint32_t grid);
cudaError_t launch_stream_pass(const StreamPass& sp, uint32_t* scratch, uint32_t* bar,
                               uint32_t* err, cudaStream_t s);

// ---------------------------------------------------------------- tuning
// Knobs picked by the autotuner (0 / -1 = built-in choice).
struct Tuning {
  int sort_variant = -1;     // tdgs_sort_pairs pass kernel
  int tile_digit_bits = 0;   // frame tile passes: widest digit, 4..12 (0 = 8)
  int ctas_per_sm = 0;       // persistent radix grids: CTAs per SM (0 = kernel default)
  int depth_digit_bits = 0;  // depth sort: 11 (3 passes) or 8 (4 passes); 0 = 8
};

// ----------------------------------------------------------- radix sort
constexpr int kMaxPasses = 8;

struct SortPlan {
  uint32_t key_bits;   // sorted bits of the transformed key
  uint32_t passes;     // number of digit passes
  uint32_t digit_bits; // digit width of every pass but possibly the last
  uint32_t shift[kMaxPasses];
  uint32_t mask[kMaxPasses];
  bool drop31;         // transformed key skips bit 31
  uint64_t bad_mask;   // key bits that must be zero
  uint32_t variant;    // which compiled pass kernel
  uint32_t bins;       // digit bins of that kernel
  uint32_t tile_keys;  // keys per shared-memory tile of a chunk
  uint32_t grid;       // resident CTAs = chunks (0 if the device query failed)
};

// Tunable pass-kernel configurations (digit bits, threads, items/thread,
// CTAs per SM its register budget is sized for).
struct PassVariant {
  int bits, threads, items, blocks_per_sm;
};
int num_pass_variants();
PassVariant pass_variant(int i);
int default_pass_variant(uint32_t digit_bits);

// Plans a sort of m keys on the current device.
SortPlan make_sort_plan(uint32_t m, uint32_t tile_bits, uint32_t flags, const Tuning& tu);
// uint32 words of scratch one pass needs (chunk histograms, prefixes, totals).
size_t radix_scratch_words(const SortPlan& plan);
// One digit pass (cooperative launch).  bar: two zero-initialised words.
cudaError_t launch_radix_pass(const SortPlan& plan, uint32_t pass, const uint64_t* kin,
                              const uint32_t* vin, uint64_t* kout, uint32_t* vout, uint32_t m,
                              uint32_t* scratch, uint32_t* bar, uint32_t* err, cudaStream_t s);

// Onesweep form of tdgs_sort_pairs (onesweep.cu): one histogram launch
// that reads the keys once, then one launch per digit pass with a
// decoupled look-back.  Eligible for 0 < m < 2^30 pairs with all four
// buffers 16-byte aligned (the tiles arrive by bulk copies).  Scratch:
// onesweep_scratch_words(m) uint32 words whose first
// onesweep_header_words() are zero when first used (the kernels leave
// them zero).  Passes ping-pong between (keys, values) and the alternates.
bool onesweep_eligible(uint32_t m, const void* keys, const void* values, const void* keys_alt,
                       const void* values_alt);
size_t onesweep_scratch_words(uint32_t m);
size_t onesweep_header_words();
uint32_t onesweep_tile_keys();
cudaError_t launch_onesweep_hist(const SortPlan& plan, const uint64_t* keys, uint32_t m, uint32_t* scratch,
                                 uint32_t* err, cudaStream_t s);
cudaError_t launch_onesweep_pass(const SortPlan& plan, uint32_t pass, const uint64_t* kin, const uint32_t* vin,
                                 uint64_t* kout, uint32_t* vout, uint32_t m, uint32_t* scratch, uint32_t* err,
                                 cudaStream_t s);
// The same passes over the depth sort's 32-bit keys (dk[0], dv[0]: keys and
// indices from the count kernel; range: the key range it published in
// range[2..3]; the histogram writes the pass count to range[4]).  The pass
// plan is read on the device: launch the histogram,
// then passes 0 .. kDepthOnesweepPasses - 1 in order; passes the range does
// not need end at once, and the last pass that runs writes dk[1], dv[1]
// (dk[2], dv[2] hold intermediate passes).  Scratch as above for m = n,
// separate from any other sort's while both may be in use.
constexpr uint32_t kDepthOnesweepPasses = 4;  // 32 bits in 9-bit digits
cudaError_t launch_depth_onesweep_hist(const uint32_t* keys, uint32_t n, uint32_t* range, uint32_t* scratch,
                                       uint32_t* err, cudaStream_t s);
cudaError_t launch_depth_onesweep_pass(uint32_t pass, uint32_t* const dk[3], uint32_t* const dv[3], uint32_t n,
                                       const uint32_t* range, uint32_t* scratch, uint32_t* err, cudaStream_t s);

}  // namespace tdgs
