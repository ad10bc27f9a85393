// Rendering (Sec. II-A "Rendering"; Sec. IV-C "Efficient Tile-Based
// Rendering"): one thread block per 16x16 tile blends the tile's sorted
// Gaussians front to back into every pixel.  Each thread owns kPix pixels
// of one column (rows t / 16 + kRowStep * k) and the three colour channels
// are unrolled.  The paper gives each thread four pixels so one Gaussian
// fetch serves four SIMD lanes; on this GPU one pixel per thread (256
// threads per tile) measured fastest -- 0.44 / 0.36 / 0.34 ms for 4 / 2 / 1
// pixels per thread on the 1280x720 frame of the 500k scene -- because
// tiles with many Gaussians set the kernel's end and more threads per tile
// finish them sooner; kPix stays a compile-time choice.
//
// Further measures on that frame (0.32 -> 0.21 ms together):
//  * tiles run heaviest first when they take more than one wave of
//    resident blocks.  A one-block kernel buckets the tiles by their
//    Gaussian count (64 buckets, descending) and block b renders the b-th
//    tile of that order, so the long tiles start in the first wave instead
//    of setting the end of the last one (longest-processing-time list
//    scheduling).  The order inside a bucket comes from shared-memory
//    atomics and may differ between calls; no pixel depends on it.  Images
//    whose tiles all fit in one wave render in raster order without it.
//  * the staged conic is stored as (-a/2, -b, -c/2), so the exponent is
//    dx (A dx + B dy) + C dy^2 in five operations; each staged Gaussian is
//    two 16-byte shared-memory words, read with two loads per step; the
//    blend loop is unrolled eight times (242 -> 231 us against four; two
//    pixels per thread measured 243-265 us).  A finished pixel keeps
//    testing its flag each step: letting it run on with T = 0 instead made
//    whole finished warps do every step's arithmetic (361 against 241 us).
//  * row culling per warp: a Gaussian reaches a pixel only inside the
//    ellipse where power >= cut, so when it is staged, its thread marks
//    the warps (row pairs of the tile) the ellipse can reach, with a
//    margin; each warp then blends only the list of staged Gaussians that
//    reach it, kept in front-to-back order by one ballot per 32.  What a
//    warp skips is what its pixels' own cut test would have skipped, so
//    the image is unchanged (a probe: 220 -> 198 us; here the kernel
//    takes 39 registers, 6 blocks per SM, and a render call 0.234 ->
//    0.217 ms, 0.208 ms with the quarter-pixel margin of warp_mask
//    instead of one pixel).  Asking for 8 blocks per SM (32 registers)
//    spills and loses most of the gain.
//
// Per pixel (sample point = the pixel's integer coordinate), in float32
// with CUDA's fast exponential and multiply-adds (the result is compared
// with the oracle's blend within a tolerance):
//   d = mean - pixel; power = -0.5 (a dx^2 + c dy^2) - b dx dy
//   skip if power > 0; alpha = min(0.99, opacity exp(power));
//   skip if alpha < 1/255; T' = T (1 - alpha); stop if T' < 1e-4;
//   C += rgb alpha T; T = T'
// and the pixel is C + T background.  The block stops fetching when all
// its pixels have stopped.
#include "render.cuh"
#include "tdgs_internal.cuh"

namespace tdgs {

namespace {

constexpr int kPix = 1;                        // pixels per thread
constexpr int kRenderThreads = 256 / kPix;      // one 16x16 tile per block
constexpr int kRowStep = kRenderThreads / 16;   // rows between a thread's pixels
constexpr int kOrderThreads = 1024;             // the tile-order kernel's one block
constexpr uint32_t kOrderBuckets = 64;          // Gaussian-count buckets, heaviest first
static_assert(kOrderBuckets == 64, "the bucket scan takes two counts per lane of one warp");

constexpr int kRenderWarps = kRenderThreads / 32;
static_assert(kRenderWarps <= 8, "one bit per warp in an 8-bit mask");

__device__ __forceinline__ uint32_t tile_len(uint2 r) { return r.y > r.x ? r.y - r.x : 0u; }

// Warps of the tile a staged Gaussian can reach (bit w: warp w, whose
// pixels sit on rows 2w, 2w+1 (+ kRowStep k) of the tile).  A pixel passes
// the cut test only inside the ellipse d^T Q d <= K, K = -2 cut, where
// Q = [[a, b], [b, c]] is the conic; its squared half-extents are
// K a / det in y and K c / det in x (det = ac - b^2).  A warp is left out
// when all its rows lie farther from the mean than 1.01 half-extents plus
// a quarter pixel (tested on squares), and every warp when the columns of
// the tile do.  det comes from one fused multiply-add (relative error
// below 6e-5 when det > 1e-3 ac, inside the 1 %); with |cut| <= ln 255 and
// the terms of the exponent below sqrt(ac / det) K, float rounding moves
// the cut boundary by about 1e-3 pixel at most, inside the quarter pixel.
// Flatter conics, Q not positive definite, or anything not finite reach
// every warp.  K < 0: no pixel passes the cut test (no warp).
__device__ __forceinline__ uint32_t warp_mask(float mx, float my, float4 c, float cut, float tx0, float ty0) {
  const float K = -2.0f * cut;
  if (K < 0.0f) return 0u;
  const uint32_t all = (1u << kRenderWarps) - 1u;
  const float ac = c.x * c.z;
  const float det = fmaf(-c.y, c.y, ac);
  if (!(c.x > 0.0f && c.z > 0.0f && det > 1e-3f * ac && K < 1e30f)) return all;
  const float hy2 = __fdividef(K * c.x, det) * 1.0201f;
  const float hx2 = __fdividef(K * c.z, det) * 1.0201f;
  if (!(hy2 < 1e30f && hx2 < 1e30f)) return all;
  const float ex = fmaxf(fmaxf(tx0 - mx, mx - (tx0 + 15.0f)) - 0.25f, 0.0f);
  if (ex * ex > hx2) return 0u;
  const float yr = my - ty0;  // the mean's row inside the tile
  uint32_t m = 0;
#pragma unroll
  for (int w = 0; w < kRenderWarps; ++w)
#pragma unroll
    for (int k = 0; k < kPix; ++k) {
      const float r0 = static_cast<float>(2 * w + kRowStep * k);
      const float ey = fmaxf(fmaxf(r0 - yr, yr - (r0 + 1.0f)) - 0.25f, 0.0f);
      if (ey * ey <= hy2) m |= 1u << w;
    }
  return m;
}

// order[0 .. tiles) = every tile once, by descending bucket of its
// Gaussian count: bucket = (max - len) * 63 / max (0 when every tile is
// empty).  Positions come from the exclusive bucket scan, so they are a
// permutation of 0 .. tiles-1.
__global__ void __launch_bounds__(kOrderThreads)
    k_render_order(const uint2* __restrict__ ranges, uint32_t tiles, uint32_t* __restrict__ order) {
  __shared__ uint32_t s_max[kOrderThreads / 32];
  __shared__ uint32_t s_cnt[kOrderBuckets];
  const uint32_t t = threadIdx.x;
  uint32_t mx = 0;
  for (uint32_t i = t; i < tiles; i += kOrderThreads) mx = max(mx, tile_len(ranges[i]));
  mx = __reduce_max_sync(0xffffffffu, mx);
  if ((t & 31) == 0) s_max[t >> 5] = mx;
  if (t < kOrderBuckets) s_cnt[t] = 0;
  __syncthreads();
  mx = 0;
#pragma unroll
  for (int w = 0; w < kOrderThreads / 32; ++w) mx = max(mx, s_max[w]);
  auto bucket = [mx](uint32_t len) -> uint32_t {
    return mx ? static_cast<uint32_t>(static_cast<uint64_t>(mx - len) * (kOrderBuckets - 1) / mx) : 0u;
  };
  for (uint32_t i = t; i < tiles; i += kOrderThreads) atomicAdd(&s_cnt[bucket(tile_len(ranges[i]))], 1u);
  __syncthreads();
  if (t < 32) {  // exclusive scan of the 64 bucket counts: two per lane
    const uint32_t c0 = s_cnt[2 * t], c1 = s_cnt[2 * t + 1];
    uint32_t incl = c0 + c1;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
      const uint32_t o = __shfl_up_sync(0xffffffffu, incl, d);
      if (static_cast<int>(t) >= d) incl += o;
    }
    const uint32_t excl = incl - c0 - c1;
    s_cnt[2 * t] = excl;
    s_cnt[2 * t + 1] = excl + c0;
  }
  __syncthreads();
  for (uint32_t i = t; i < tiles; i += kOrderThreads)
    order[atomicAdd(&s_cnt[bucket(tile_len(ranges[i]))], 1u)] = i;
}


__global__ void __launch_bounds__(kRenderThreads)
    k_render(const float4* __restrict__ rec, const float4* __restrict__ conic, const float* __restrict__ rgb,
             const uint32_t* __restrict__ values, const uint2* __restrict__ ranges,
             const uint32_t* __restrict__ order, uint32_t gx, uint32_t width,
             uint32_t height, float3 bg, uint32_t n, float* __restrict__ image, uint32_t* err) {
  // staged Gaussians, two 16-byte loads per step: (x, y, cut, -c/2) and
  // (-a/2, -b, opacity, -); cut = the exponent below which alpha < 1/255
  __shared__ float4 s_g0[kRenderThreads];
  __shared__ float4 s_g1[kRenderThreads];
  __shared__ float s_rgb[kRenderThreads][3];
  __shared__ uint8_t s_mask[kRenderThreads];                 // warps each staged Gaussian reaches
  __shared__ uint8_t s_list[kRenderWarps][kRenderThreads];  // per warp: staged Gaussians to blend
  const uint32_t tile = order ? order[blockIdx.x] : blockIdx.x, t = threadIdx.x;
  const uint32_t px = (tile % gx) * 16 + (t & 15);
  const uint32_t py0 = (tile / gx) * 16 + (t >> 4);
  const float fx = __uint2float_rn(px);
  const uint32_t warp = t >> 5, lane = t & 31;
  float fy[kPix], T[kPix], C[kPix][3];
  bool done[kPix];
#pragma unroll
  for (int k = 0; k < kPix; ++k) {
    const uint32_t py = py0 + kRowStep * k;
    fy[k] = __uint2float_rn(py);
    T[k] = 1.0f;
    C[k][0] = C[k][1] = C[k][2] = 0.0f;
    done[k] = !(px < width && py < height);
  }
  const uint2 r = ranges[tile];
  bool bad = false;
  for (uint32_t b = r.x; b < r.y; b += kRenderThreads) {
    bool mine_done = true;
#pragma unroll
    for (int k = 0; k < kPix; ++k) mine_done = mine_done && done[k];
    if (__syncthreads_count(mine_done) == kRenderThreads) break;
    const uint32_t idx = b + t;
    if (idx < r.y) {
      uint32_t g = values[idx];
      if (g >= n) {  // not an index of this frame: skipped and reported
        bad = true;
        s_g0[t] = make_float4(0.f, 0.f, __int_as_float(0x7f800000), 0.f);
        s_g1[t] = make_float4(0.f, 0.f, 0.f, 0.f);
        s_mask[t] = 0;
        s_rgb[t][0] = s_rgb[t][1] = s_rgb[t][2] = 0.f;
      } else {
        const float4 q = __ldg(rec + g);
        const float4 c = __ldg(conic + g);
        // opacity * exp(power) < 1/255 exactly when power < -ln(255 opacity):
        // far pixels skip the exponential (the 1/255 test below stays)
        const float cut = c.w > 0.0f ? -__logf(255.0f * c.w) : __int_as_float(0x7f800000);
        s_g0[t] = make_float4(q.x, q.y, cut, -0.5f * c.z);
        s_g1[t] = make_float4(-0.5f * c.x, -c.y, c.w, 0.f);
        s_mask[t] = static_cast<uint8_t>(
            warp_mask(q.x, q.y, c, cut, __uint2float_rn((tile % gx) * 16), __uint2float_rn((tile / gx) * 16)));
        s_rgb[t][0] = __ldg(rgb + 3 * static_cast<size_t>(g));
        s_rgb[t][1] = __ldg(rgb + 3 * static_cast<size_t>(g) + 1);
        s_rgb[t][2] = __ldg(rgb + 3 * static_cast<size_t>(g) + 2);
      }
    }
    __syncthreads();
    const uint32_t cnt = min(static_cast<uint32_t>(kRenderThreads), r.y - b);
    // this warp's list of the staged Gaussians that can reach its rows
    uint32_t nw = 0;
#pragma unroll
    for (uint32_t k = 0; k < kRenderThreads / 32; ++k) {
      const uint32_t e = k * 32 + lane;
      const bool hit = e < cnt && ((s_mask[e] >> warp) & 1u);
      const uint32_t bal = __ballot_sync(0xffffffffu, hit);
      if (hit) s_list[warp][nw + __popc(bal & ((1u << lane) - 1u))] = static_cast<uint8_t>(e);
      nw += __popc(bal);
    }
    __syncwarp();
#pragma unroll 8
    for (uint32_t jj = 0; jj < nw; ++jj) {
      const uint32_t j = s_list[warp][jj];
      const float4 g0 = s_g0[j];
      const float4 g1 = s_g1[j];
      const float dx = g0.x - fx;
#pragma unroll
      for (int k = 0; k < kPix; ++k) {
        if (done[k]) continue;
        const float dy = g0.y - fy[k];
        const float power = fmaf(dx, fmaf(g1.x, dx, g1.y * dy), g0.w * dy * dy);
        if (power > 0.0f || power < g0.z) continue;
        const float alpha = fminf(0.99f, g1.z * __expf(power));
        if (alpha < 1.0f / 255.0f) continue;
        const float test_t = T[k] * (1.0f - alpha);
        if (test_t < 0.0001f) {
          done[k] = true;
          continue;
        }
        const float w = alpha * T[k];
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) C[k][ch] += s_rgb[j][ch] * w;
        T[k] = test_t;
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && (t & 31) == 0) latch_error(err, TDGS_ERR_INVALID_ARGUMENT, kSiteRender);
#pragma unroll
  for (int k = 0; k < kPix; ++k) {
    const uint32_t py = py0 + kRowStep * k;
    if (px < width && py < height) {
      float* o = image + 3 * (static_cast<size_t>(py) * width + px);
      o[0] = C[k][0] + T[k] * bg.x;
      o[1] = C[k][1] + T[k] * bg.y;
      o[2] = C[k][2] + T[k] * bg.z;
    }
  }
}

}  // namespace

cudaError_t launch_render_order(const uint2* ranges, uint32_t tiles, uint32_t* order, cudaStream_t s) {
  if (tiles == 0) return cudaSuccess;
  k_render_order<<<1, kOrderThreads, 0, s>>>(ranges, tiles, order);
  return cudaGetLastError();
}

cudaError_t launch_render_ordered(const float4* rec, const float4* conic, const float* rgb, const uint32_t* values,
                                  const uint2* ranges, const uint32_t* order, uint32_t width, uint32_t height,
                                  const float* bg, uint32_t n, float* image, uint32_t* err, cudaStream_t s) {
  const uint32_t gx = (width + 15) / 16, gy = (height + 15) / 16;
  const uint32_t tiles = gx * gy;
  if (tiles == 0) return cudaSuccess;
  k_render<<<tiles, kRenderThreads, 0, s>>>(rec, conic, rgb, values, ranges, order, gx, width, height,
                                            make_float3(bg[0], bg[1], bg[2]), n, image, err);
  return cudaGetLastError();
}

cudaError_t launch_render(const float4* rec, const float4* conic, const float* rgb, const uint32_t* values,
                          const uint2* ranges, uint32_t width, uint32_t height, const float* bg, uint32_t n,
                          float* image, uint32_t* err, cudaStream_t s) {
  return launch_render_ordered(rec, conic, rgb, values, ranges, nullptr, width, height, bg, n, image, err, s);
}

uint32_t render_wave_blocks(int device) {
  int sms = 0, per_sm = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_render, kRenderThreads, 0) != cudaSuccess) return 0;
  return static_cast<uint32_t>(sms) * static_cast<uint32_t>(per_sm);
}

}  // namespace tdgs
