/*
 * tdgs.h -- C ABI of the GB300 (sm_103a) 3D Gaussian Splatting tile depth sort.
 *
 * The library computes the steps that sit between Preprocessing and
 * Rendering in the 3DGS pipeline (arXiv 2511.16298, Sec. II-A
 * "Duplication with Tiles" and "Sorting"; Table III shows PrefixSum feeding
 * DuplicateWithTile; Table VI times Scan, Duplicate with tiles, Sorting and
 * Identify Range as separate stages):
 *
 *   1. tdgs_count_tiles    tiles touched by each projected Gaussian
 *   2. tdgs_scan           exclusive prefix sum of those counts
 *   3. tdgs_duplicate_keys one (tile << 32 | depth bits, index) pair per
 *                          Gaussian-tile instance
 *   4. tdgs_sort_pairs     stable sort of the pairs by key (tile, then depth)
 *   5. tdgs_tile_ranges    [start, end) of every tile in the sorted list
 *   +  tdgs_sort_frame     all five steps on context-owned buffers
 *   +  tdgs_sort_views     many views of one scene in one batched call
 *   0. tdgs_preprocess     the Preprocessing stage before step 1: 3D
 *                          Gaussians -> projected records for one camera
 *   +  tdgs_sort_frame_3d  preprocessing and steps 1-5 in one call
 *   +  tdgs_sort_frame_normalized  steps 1-5 with the paper's 32-bit
 *                          normalised key (lossy; for comparison)
 *   6. tdgs_render         the Rendering stage after step 5: front-to-back
 *                          alpha blending of every tile into an image
 *
 * Conventions shared by every call
 *   - Data pointers are DEVICE pointers unless a parameter says "host".
 *   - Calls are asynchronous on `stream` (a cudaStream_t; NULL = legacy
 *     default stream).  The caller owns inputs and outputs of the per-step
 *     calls and keeps them alive until the stream has finished the work.
 *   - A call returns TDGS_OK or the first error it detects on the host
 *     (NULL pointer with a non-zero size, misaligned pointer, zero image
 *     size, out-of-range parameter, CUDA launch failure).  No call throws,
 *     aborts or prints.
 *   - Errors that only the GPU can see (an invalid depth or mean on a
 *     visible Gaussian, a pair count above 2^32-1, a key wider than the
 *     declared bits, a pair written beyond the given capacity, a
 *     cross-block wait that exceeded its iteration bound) are latched in
 *     the context and returned by the next tdgs_context_sync() or
 *     tdgs_sort_frame() on that context, which also clears them.
 *   - n = 0 and m = 0 are valid everywhere.
 *   - A context may be used from one host thread and one stream at a time;
 *     use one context per concurrent stream.
 */
#ifndef TDGS_H_
#define TDGS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TDGS_OK = 0,
  TDGS_ERR_INVALID_ARGUMENT = 1, /* bad pointer/size/flag, or invalid Gaussian */
  TDGS_ERR_OUT_OF_MEMORY = 2,    /* device allocation failed                  */
  TDGS_ERR_OVERFLOW = 3,         /* pair count above 2^32 - 1                 */
  TDGS_ERR_CUDA = 4,             /* a CUDA runtime call failed                */
  TDGS_ERR_TIMEOUT = 5,          /* a bounded cross-block wait gave up        */
  TDGS_ERR_CAPACITY = 6          /* output capacity smaller than required     */
} tdgs_status;

/* One projected Gaussian, 16 bytes, 16-byte aligned in arrays: the packing
 * of Table IV, Group 1 (2D mean in pixels, view depth, pixel radius).
 * radius <= 0 marks a culled Gaussian. */
typedef struct {
  float x, y;
  float depth;
  int32_t radius;
} tdgs_gaussian2d;

/* Image size in pixels; tiles are 16x16, partial edge tiles count. */
typedef struct {
  uint32_t width, height;
} tdgs_frame;

/* Tile range in the sorted list; an empty tile is {0, 0}. */
typedef struct {
  uint32_t start, end;
} tdgs_range;

typedef struct tdgs_context tdgs_context; /* opaque */

/* tdgs_sort_pairs flag: every key has bit 31 clear (true for keys made by
 * tdgs_duplicate_keys, whose depths are positive), so the sort skips that
 * bit.  A key with bit 31 set latches TDGS_ERR_INVALID_ARGUMENT. */
#define TDGS_SORT_DEPTH_POSITIVE 1u

/* ------------------------------------------------------------ context --- */

/* Create a context on CUDA device `device`.  The context owns the scratch
 * memory of the calls below (look-back status words, histograms, offsets)
 * and the output buffers of tdgs_sort_frame, growing them on demand.
 * *out is set to NULL on failure. */
tdgs_status tdgs_context_create(tdgs_context** out, int device);

/* Free every buffer the context owns.  NULL is a no-op.  The caller must
 * ensure no work on the context is still running. */
void tdgs_context_destroy(tdgs_context* ctx);

/* Wait for `stream`, then return and clear the first device-latched error
 * (TDGS_OK if none). */
tdgs_status tdgs_context_sync(tdgs_context* ctx, void* stream);

/* Static description of a status code; never NULL. */
const char* tdgs_status_string(tdgs_status s);

/* Human-readable detail of the last failure on this context ("" if none).
 * Valid until the next call on the context. */
const char* tdgs_last_error(const tdgs_context* ctx);

/* Grid helpers: gx = ceil(width/16), gy = ceil(height/16), T = gx*gy and
 * tile bits = ceil(log2 T) (0 when T = 1). */
uint32_t tdgs_num_tiles(tdgs_frame f);
uint32_t tdgs_tile_bits(tdgs_frame f);

/* Tuning of the sort's digit passes (used by the autotuner; the paper has
 * no counterpart).  Variant i is a compiled pass kernel with
 * 2^bits digit bins, `threads` threads per block, `items` keys per thread
 * and registers budgeted for `blocks_per_sm` resident blocks per SM.
 * tdgs_context_set_sort_variant(ctx, -1) restores the built-in choice; an
 * index out of range returns TDGS_ERR_INVALID_ARGUMENT.  Any output
 * pointer may be NULL. */
int tdgs_sort_variant_count(void);
tdgs_status tdgs_sort_variant_info(int i, int* bits, int* threads, int* items, int* blocks_per_sm);
tdgs_status tdgs_context_set_sort_variant(tdgs_context* ctx, int variant);

/* Further tuning knobs of a context (value 0, or -1 for the sort variant,
 * restores the built-in choice); out-of-range keys or values return
 * TDGS_ERR_INVALID_ARGUMENT.
 *   TDGS_TUNE_SORT_VARIANT     pass kernel of tdgs_sort_pairs (as above)
 *   TDGS_TUNE_TILE_DIGIT_BITS  widest digit (4..12) of the frame's passes
 *                              over the tile bits (built-in: 8)
 *   TDGS_TUNE_CTAS_PER_SM      CTAs per SM of the persistent radix grids
 *                              (capped by occupancy)
 *   TDGS_TUNE_DEPTH_DIGIT_BITS digit width of the frame's depth sort when
 *                              it runs as one launch per pass over all 32
 *                              key bits (frames or batches of 2^30
 *                              Gaussians or more): 8 (4 passes, the
 *                              built-in choice) or 11 (3 passes).  Below
 *                              that the depth sort takes 9-bit digits over
 *                              the keys less the smallest and only the
 *                              passes their range needs: one launch up to
 *                              one 8192-key tile per resident CTA (about
 *                              1.25M Gaussians on 152 SMs), the onesweep
 *                              passes above. */
enum {
  TDGS_TUNE_SORT_VARIANT = 0,
  TDGS_TUNE_TILE_DIGIT_BITS = 1,
  TDGS_TUNE_CTAS_PER_SM = 3,
  TDGS_TUNE_DEPTH_DIGIT_BITS = 4
};
tdgs_status tdgs_context_set_tuning(tdgs_context* ctx, int key, int value);
tdgs_status tdgs_context_get_tuning(const tdgs_context* ctx, int key, int* value);

/* Tracing (the paper has no counterpart; its Table VI times each stage
 * separately, which this reproduces on the GPU).  Every kernel launch made
 * through a context increments a counter.  With timing enabled, the
 * library brackets each launch with CUDA events on the launching stream;
 * tdgs_context_kernel_times waits for those events and returns, per
 * kernel name, the launches, the items processed (Gaussians or pairs) and
 * the summed device time in ms, then clears the record.  It writes at most
 * `max` entries and returns how many kernels have data (or -1 on error).
 * Enabling or disabling timing clears the record. */
typedef struct {
  const char* name; /* static string */
  uint64_t launches;
  uint64_t items;
  double total_ms;
} tdgs_kernel_time;

uint64_t tdgs_context_launch_count(const tdgs_context* ctx);
tdgs_status tdgs_context_enable_timing(tdgs_context* ctx, int enable);
int tdgs_context_kernel_times(tdgs_context* ctx, tdgs_kernel_time* out, int max);

/* Digit passes the last depth sort of the fused frame ran on this context
 * over keys compressed to their range (the single launch or the onesweep
 * passes; the count follows the frame's depth range: 1 to 4), or 0 if
 * none has run.  Waits for the work on `stream`. */
tdgs_status tdgs_context_depth_passes(tdgs_context* ctx, int* passes, void* stream);

/* ------------------------------------------------------- the five steps --- */

/* Step 1 (Sec. II-A: each projected Gaussian is represented by the
 * axis-aligned box of its footprint and touches every 16x16 tile the box
 * intersects).  For i < n: tiles_touched[i] = (x1-x0)*(y1-y0) where, in
 * float32 and in this order, x0 = floor((x - r) / 16),
 * x1 = floor(((x + r) + 15) / 16), likewise for y, each clamped to
 * [0, gx] (resp. [0, gy]); 0 when radius <= 0 or the box misses the image.
 * g: n records (16-byte aligned); tiles_touched: n uint32.
 * A visible Gaussian (radius > 0) with a non-finite mean, or with a
 * non-empty box and a depth that is not finite and > 0, latches
 * TDGS_ERR_INVALID_ARGUMENT (its count is written as 0). */
tdgs_status tdgs_count_tiles(tdgs_context* ctx, const tdgs_gaussian2d* g, uint32_t n,
                             tdgs_frame f, uint32_t* tiles_touched, void* stream);

/* Step 2 (Table III, PrefixSum over Tiles_touched): offsets[i] = sum of
 * counts[j] for j < i; *total_dev (device, one uint32) = sum of all counts.
 * A sum above 2^32-1 latches TDGS_ERR_OVERFLOW (total_dev then holds
 * 0xFFFFFFFF).  counts and offsets may not overlap.  total_dev may be NULL. */
tdgs_status tdgs_scan(tdgs_context* ctx, const uint32_t* counts, uint32_t n,
                      uint32_t* offsets, uint32_t* total_dev, void* stream);

/* Step 3 (Sec. II-A: Gaussians are duplicated across the tiles their box
 * intersects, forming key-value pairs keyed by tile and depth).  Gaussian i
 * writes its pairs at offsets[i], offsets[i]+1, ... with rows (ty) outer and
 * columns (tx) inner:
 *   keys[k]   = ((uint64_t)(ty*gx + tx) << 32) | float32 bit pattern of depth
 *   values[k] = i
 * offsets must be the exclusive scan of the step-1 counts of the same g and
 * f.  m_capacity = length of keys and values; a pair that would land at or
 * beyond it is dropped and latches TDGS_ERR_CAPACITY.
 * keys 8-byte aligned, values 4-byte aligned. */
tdgs_status tdgs_duplicate_keys(tdgs_context* ctx, const tdgs_gaussian2d* g,
                                const uint32_t* offsets, uint32_t n, tdgs_frame f,
                                uint64_t* keys, uint32_t* values, uint32_t m_capacity,
                                void* stream);

/* Step 4 (Sec. II-A Sorting: by tile index, then by depth within a tile).
 * Stable ascending sort of the m pairs by key.  Only key bits [0, 32 +
 * tile_bits) take part (bit 31 is skipped with TDGS_SORT_DEPTH_POSITIVE);
 * a key with a higher bit set latches TDGS_ERR_INVALID_ARGUMENT.
 * keys/values are the input; keys_alt/values_alt are caller-provided
 * buffers of the same length.  The sort ping-pongs between the two, and
 * *result_in_alt (host int) tells where the sorted pairs are: 0 = keys/
 * values, 1 = keys_alt/values_alt.  The other pair of buffers is clobbered.
 * tile_bits <= 32.  Keys changed by someone else while the sort runs can
 * send a pair outside [0, m); it is dropped and TDGS_ERR_CAPACITY latched.
 * Form: with all four buffers 16-byte aligned and m < 2^30 (and no sort
 * variant chosen by tdgs_context_set_sort_variant), a onesweep LSD radix sort:
 * one launch reads the keys once for the first digit's counts, then one
 * launch per 9-bit digit reads and writes every pair once (its tiles go
 * through shared memory by bulk copy; scan blocks of the same cooperative
 * launch turn the tiles' digit counts into prefixes); every other case
 * takes the chunked per-digit passes.  Both give the same bytes. */
tdgs_status tdgs_sort_pairs(tdgs_context* ctx, uint64_t* keys, uint32_t* values,
                            uint64_t* keys_alt, uint32_t* values_alt, uint32_t m,
                            uint32_t tile_bits, uint32_t flags, int* result_in_alt,
                            void* stream);

/* Step 4 as the paper builds it (Sec. III, Algorithms 1-2): a bitonic
 * sorting network over the pairs padded to a power of two (at least 4096),
 * ascending by key and then by value.  When pairs with equal keys appear
 * with ascending values -- as tdgs_duplicate_keys emits them -- the result
 * is identical to tdgs_sort_pairs; otherwise equal keys end up ordered by
 * value.  keys_in/values_in (m pairs) are read; keys_out/values_out receive
 * the sorted pairs and may be the same arrays.  The context holds a scratch
 * copy of the padded pairs (12 bytes per padded pair).  m <= 2^31.  It is
 * slower than tdgs_sort_pairs on this GPU (O(m log^2 m) work against a few
 * radix passes) and is kept as the paper's method for comparison. */
tdgs_status tdgs_sort_pairs_bitonic(tdgs_context* ctx, const uint64_t* keys_in, const uint32_t* values_in,
                                    uint64_t* keys_out, uint32_t* values_out, uint32_t m, void* stream);

/* Step 5 (Identify Range, Sec. IV-B and Table VI): ranges[t] = first and
 * one-past-last position of tile t (= key >> 32) in sorted_keys, {0, 0} for
 * a tile with no pairs.  sorted_keys must be ordered by tile.  A tile id
 * >= num_tiles latches TDGS_ERR_INVALID_ARGUMENT.  ranges: num_tiles
 * entries, 8-byte aligned. */
tdgs_status tdgs_tile_ranges(tdgs_context* ctx, const uint64_t* sorted_keys, uint32_t m,
                             uint32_t num_tiles, tdgs_range* ranges, void* stream);

/* Steps 1-5 fused.  Writes host *m_out (pair count), and *sorted_keys,
 * *sorted_values (m entries) and *ranges (tdgs_num_tiles(f) entries) as
 * device pointers into buffers owned by the context, valid until the next
 * call on the context or its destruction.  The call waits once for the
 * pair count (a 4-byte device-to-host read), so it returns the errors of
 * steps 1-2 directly; errors of later steps are returned by the next
 * tdgs_context_sync or tdgs_sort_frame. */
tdgs_status tdgs_sort_frame(tdgs_context* ctx, const tdgs_gaussian2d* g, uint32_t n,
                            tdgs_frame f, const uint64_t** sorted_keys,
                            const uint32_t** sorted_values, const tdgs_range** ranges,
                            uint32_t* m_out, void* stream);

/* ------------------------------------------------------ preprocessing --- */

/* One 3D Gaussian as the preprocessing stage reads it (Table I, Group 1:
 * mean in world units and opacity), 16 bytes, 16-byte aligned in arrays. */
typedef struct {
  float x, y, z, opacity;
} tdgs_gaussian3d;

/* Its 3D covariance (Table I, Group 2: the six entries of the symmetric
 * matrix in two 16-byte texels; pad0 and pad1 are ignored), 32 bytes,
 * 16-byte aligned in arrays. */
typedef struct {
  float xx, xy, xz, yy, yz, zz, pad0, pad1;
} tdgs_cov3d;

/* Pinhole camera: camera-space point = rot * p + trans (rot row-major;
 * camera x to the right and y down in the image, z along the view
 * direction), focal lengths and principal point in pixels, near plane and
 * image size in pixels.  76 bytes, passed by HOST pointer. */
typedef struct {
  float rot[9];
  float trans[3];
  float fx, fy, cx, cy;
  float near_z;
  uint32_t width, height;
} tdgs_camera;

/* Preprocessing (Sec. II-A "Preprocessing": frustum culling and projection
 * of each Gaussian to its elliptical footprint; inputs Table I, outputs
 * Table IV Groups 1-2).  The paper prints no formulas; the library applies
 * the EWA projection of 3D Gaussian splatting, in float32 with every
 * operation rounded in this order:
 *   t = rot p + trans; culled unless t.z > near_z
 *   u = t.x / t.z, v = t.y / t.z; record x = fx u + cx, y = fy v + cy,
 *   depth = t.z
 *   uc, vc = u, v clamped to +-(0.65 width / fx), +-(0.65 height / fy)
 *   J = [[fx / t.z, 0, -fx uc / t.z], [0, fy / t.z, -fy vc / t.z]]
 *   S2 = (J rot) S3 (J rot)^T + 0.3 I; culled unless det(S2) > 0
 *   conic = (S2yy, -S2xy, S2xx) / det
 *   radius = ceil(3 sqrt(mid + sqrt(max(0.1, mid^2 - det)))),
 *   mid = (S2xx + S2yy) / 2; culled unless x, y, depth and radius are finite;
 *   radius capped at 2^30.
 * A culled Gaussian gets the record {0, 0, 0, 0} (radius 0: no tiles) and
 * the conic {0, 0, 0, 0}.
 * g, cov: n device entries; records: n device entries (16-byte aligned);
 * conic_opacity: NULL or n x 4 device floats (conic a, b, c, opacity),
 * 16-byte aligned.  cam: host.  Returns TDGS_ERR_INVALID_ARGUMENT for fx or
 * fy not > 0 or not finite, a zero image size, or NULL / misaligned
 * pointers with n > 0. */
tdgs_status tdgs_preprocess(tdgs_context* ctx, const tdgs_gaussian3d* g, const tdgs_cov3d* cov,
                            uint32_t n, const tdgs_camera* cam, tdgs_gaussian2d* records,
                            float* conic_opacity, void* stream);

/* Preprocessing and steps 1-5 for the camera's image, with the projection
 * fused into the count kernel of the fused frame (each Gaussian is
 * projected, stored and counted in one pass; results identical to
 * tdgs_preprocess followed by tdgs_sort_frame).  *records and
 * *conic_opacity (each may
 * be NULL to skip) receive device pointers to the n projected records and
 * n x 4 conic/opacity floats, valid like the sorted buffers (until the next
 * call on the context). */
tdgs_status tdgs_sort_frame_3d(tdgs_context* ctx, const tdgs_gaussian3d* g, const tdgs_cov3d* cov,
                               uint32_t n, const tdgs_camera* cam, const tdgs_gaussian2d** records,
                               const float** conic_opacity, const uint64_t** sorted_keys,
                               const uint32_t** sorted_values, const tdgs_range** ranges,
                               uint32_t* m_out, void* stream);

/* Device pointers to the projected records (16 bytes each) and conic /
 * opacity words (4 floats each) of the last tdgs_sort_frame_3d or
 * tdgs_sort_views_3d call on ctx (view after view), valid until the next
 * call on the context. */
tdgs_status tdgs_context_projected(tdgs_context* ctx, const tdgs_gaussian2d** records,
                                   const float** conic_opacity);

/* Steps 1-5 with the paper's 32-bit key (Sec. IV-B "key normalization":
 * 20 bits of tile number and the depth normalised to the range 2^10).  The
 * figure fixing the layout is not in the text; the library's reading:
 *   visible = Gaussians with pairs; dmin, dmax = their smallest and largest
 *   depth; scale = 1024 / (dmax - dmin) (0 if equal);
 *   q = min(1023, floor((depth - dmin) * scale)) in float32 in this order;
 *   key = tile << 10 | q (bits 30-31 clear: a positive float's bit pattern)
 * The pairs are emitted like tdgs_duplicate_keys and sorted stably by the
 * 32-bit key; ranges come from key >> 10.  Depths closer than 1/1024 of the
 * range get one q and keep index order, so the order differs from
 * tdgs_sort_frame wherever that happens (it is lossy by design).  At most
 * 2^20 tiles (else TDGS_ERR_INVALID_ARGUMENT).  Outputs: device pointers into
 * context-owned buffers (m keys, m values, tdgs_num_tiles(f) ranges), valid
 * until the next call on the context; host *m_out.  Waits once (pair count). */
tdgs_status tdgs_sort_frame_normalized(tdgs_context* ctx, const tdgs_gaussian2d* g, uint32_t n, tdgs_frame f,
                                       const uint32_t** sorted_keys, const uint32_t** sorted_values,
                                       const tdgs_range** ranges, uint32_t* m_out, void* stream);

/* Rendering (Sec. II-A "Rendering"; Sec. IV-C: one 16x16 tile per thread
 * block; one pixel per thread here, exponent coefficients staged in shared
 * memory, and each warp skips the staged Gaussians whose cut-off ellipse
 * cannot reach its rows, which leaves every pixel unchanged).  Each pixel blends its tile's Gaussians
 * sorted_values[ranges[t].start .. ranges[t].end) front to back; the
 * paper prints no formulas, the library applies the compositing of 3D
 * Gaussian splatting in float32 (multiply-adds may be fused, exp is CUDA's
 * fast __expf; sample point = the pixel's integer coordinate; T = 1, C = 0):
 *   d = (x - px, y - py); power = -0.5 (a dx^2 + c dy^2) - b dx dy
 *   skip if power > 0; alpha = min(0.99, opacity exp(power));
 *   skip if alpha < 1/255; T' = T (1 - alpha); stop if T' < 1e-4;
 *   C += rgb alpha T; T = T'
 * and the pixel is C + T background.
 * records (n, 16-byte aligned), conic_opacity (n x 4 floats: a, b, c,
 * opacity; 16-byte aligned), rgb (n x 3 floats), sorted_values and ranges
 * (as tdgs_sort_frame returns them; sorted_values may be NULL when every
 * range is empty): device.  background: 3 HOST floats.
 * image: device, height x width x 3 floats (interleaved RGB, row-major).
 * A sorted value >= n is skipped and latches TDGS_ERR_INVALID_ARGUMENT; a
 * range whose start is not below its end is an empty tile.
 * Scheduling: when the image has more tiles than one wave of resident
 * rendering blocks, a one-block kernel first orders the tiles by Gaussian
 * count (heaviest first, 64 buckets) into a context-owned buffer of 4 B
 * per tile, which the first such call allocates (draining the stream), and
 * block b renders the b-th tile of that order; otherwise the tiles render
 * in raster order with one launch.  No pixel depends on the order. */
tdgs_status tdgs_render(tdgs_context* ctx, const tdgs_gaussian2d* records, const float* conic_opacity,
                        const float* rgb, uint32_t n, const uint32_t* sorted_values, const tdgs_range* ranges,
                        tdgs_frame f, const float* background, float* image, void* stream);

/* ------------------------------------------------ failure detection --- */

/* Failure-detection check of the cross-block waits: launches two blocks of
 * which only one reaches the library's grid barrier (the same code the
 * radix passes use, on barrier words of its own).  The waiting block gives
 * up after the barrier's bounded wait (2^21 polls, about 0.1-2 s) and
 * latches TDGS_ERR_TIMEOUT, which the next tdgs_context_sync (or
 * tdgs_sort_frame) returns and clears; the context stays usable.  No GPU
 * fault or hang is involved. */
tdgs_status tdgs_diag_barrier_timeout(tdgs_context* ctx, void* stream);

/* ------------------------------------------------- scan without allocation */

/* The exclusive scan of tdgs_scan (offsets, total, 64-bit overflow check)
 * for callers that cannot allocate device memory: real-time loops that
 * must never reach the device allocator (an allocation can block or
 * synchronise the device), or plugins whose device memory belongs to a
 * host application that does not let them allocate.  The paper has no
 * counterpart; it is a deployment convenience.
 *
 * It needs no context and allocates nothing (no cudaMalloc, cudaFree or
 * allocating library call).  Its scratch -- look-back status words, the
 * tile ticket and an error word -- is one fixed array of about 16 KB in
 * the library's device memory, present on every GPU that loads the library
 * until the process exits.  Limits and behaviour:
 *   - n <= 16,777,216 counts; a larger n returns TDGS_ERR_INVALID_ARGUMENT.
 *   - The first call in each CUDA context (normally once per device: the
 *     device's primary context) looks up the array's address in that
 *     context; make that first call before any stream capture.
 *   - Every call shares the array, which keeps the last call's contents;
 *     each call clears the words it uses on `stream` before its kernel.
 *     Calls whose GPU work overlaps (different streams, or threads without
 *     ordering) race and give wrong results.  Order them on one stream.
 *   - total_dev (may be NULL) receives the sum, 0xFFFFFFFF on overflow;
 *     error_dev (may be NULL) receives 0 or the error the GPU detected
 *     (TDGS_ERR_OVERFLOW, or TDGS_ERR_TIMEOUT from a bounded wait).
 *   - n == 0 writes total 0 and error 0 and launches no scan kernel.
 * counts, offsets, total_dev, error_dev: device pointers, 4-byte aligned. */
tdgs_status tdgs_scan_noalloc(const uint32_t* counts, uint32_t n, uint32_t* offsets,
                              uint32_t* total_dev, uint32_t* error_dev, void* stream);

/* ------------------------------------------------------ several views --- */

/* One view of a batch: its projected Gaussians (device, 16-byte aligned)
 * and its image size. */
typedef struct {
  const tdgs_gaussian2d* g;
  uint32_t n;
  tdgs_frame f;
} tdgs_view;

/* Sorted result of one view: pointers into context-owned device buffers
 * (valid until the next call on the context), its pair count and tiles.
 * Keys carry the view's LOCAL tile id; values are indices into the view's
 * own Gaussian array; ranges index the view's own list. */
typedef struct {
  const uint64_t* keys;
  const uint32_t* values;
  const tdgs_range* ranges;
  uint32_t m;
  uint32_t num_tiles;
} tdgs_view_result;

/* Steps 1-5 for up to 256 views with one set of passes (the batched form of
 * the Sorting step, Sec. II-A, over several cameras): each view's result is
 * byte-identical to tdgs_sort_frame on that view alone.  Waits once for the
 * pair count; results[num_views] (host) is filled. */
tdgs_status tdgs_sort_views(tdgs_context* ctx, const tdgs_view* views, uint32_t num_views,
                            tdgs_view_result* results, void* stream);

/* Allocate everything a batch of this shape needs (same view count, total
 * Gaussians and total tiles) for up to pair_capacity pairs.  Waits. */
tdgs_status tdgs_reserve_views(tdgs_context* ctx, const tdgs_view* views, uint32_t num_views,
                               uint64_t pair_capacity, void* stream);

/* The same work as tdgs_sort_views without any host wait or allocation, so
 * it can be captured in a CUDA graph and replayed: kernels read the pair
 * count from device memory.  Requires tdgs_reserve_views with the same
 * shape.  A batch with more pairs than the reserved capacity latches
 * TDGS_ERR_CAPACITY (reserve more and run again).  The view table is read
 * from a host staging buffer the context owns, refreshed by each call. */
tdgs_status tdgs_sort_views_async(tdgs_context* ctx, const tdgs_view* views, uint32_t num_views,
                                  void* stream);

/* After tdgs_sort_views_async: wait for `stream`, return the first latched
 * error, else fill results[num_views]. */
tdgs_status tdgs_views_results(tdgs_context* ctx, tdgs_view_result* results, uint32_t num_views,
                               void* stream);

/* Preprocessing and steps 1-5 for num_views (<= 256) cameras of the same
 * n 3D Gaussians in one batch (the multi-view form of tdgs_sort_frame_3d;
 * the sort is that of tdgs_sort_views): view v is camera cams[v] (host
 * array) with its own image size; results[num_views] (host) as
 * tdgs_sort_views fills them, each byte-identical to tdgs_sort_frame_3d
 * with that camera alone.  The projected records and conics of view v are
 * n entries at offset v * n of the buffers tdgs_context_projected returns.
 * n * num_views < 2^32. */
tdgs_status tdgs_sort_views_3d(tdgs_context* ctx, const tdgs_gaussian3d* g, const tdgs_cov3d* cov, uint32_t n,
                               const tdgs_camera* cams, uint32_t num_views, tdgs_view_result* results,
                               void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TDGS_H_ */
