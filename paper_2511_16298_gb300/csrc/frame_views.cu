// Depth-first fused frame over a table of views (Sec. II-A: Duplication
// with Tiles, Sorting, and the Identify Range step of Sec. IV-B).  One view
// is one frame; several views of one scene are sorted together with one
// set of passes, each view keeping its local tile ids and its own list.
//
// The Gaussians of all views are sorted by depth first; every Gaussian's
// pairs are then emitted in that depth order as packed elements
// (global tile << rbits | depth position), and a stable sort on the tile
// bits alone yields the order by (tile, depth, index) that a stable sort of
// the 64-bit keys defines: ties of the 64-bit key are pairs of distinct
// Gaussians of one view in the same tile with equal depth, and both orders
// put them in index order.
#include "tdgs_internal.cuh"

namespace tdgs {

// Per record (global index i over all views): tile count, depth sort key
// (raw depth bits of a visible Gaussian, all ones otherwise so culled ones
// sort last), the record index, and the per-view pair totals.
__global__ void __launch_bounds__(256)
    k_views_count(ViewTable vt, uint32_t n_all, uint32_t* __restrict__ counts,
                  uint32_t* __restrict__ dkey, uint32_t* __restrict__ dval, uint32_t* err) {
  __shared__ uint32_t s_begin[kMaxViews + 1];
  __shared__ unsigned long long s_tot[kMaxViews];
  for (uint32_t v = threadIdx.x; v <= vt.nv; v += blockDim.x) s_begin[v] = vt.rec_begin[v];
  for (uint32_t v = threadIdx.x; v < vt.nv; v += blockDim.x) s_tot[v] = 0;
  __syncthreads();
  bool bad = false;
  const uint32_t stride = gridDim.x * blockDim.x;
  // warp-uniform loop so the per-view totals can be reduced across the warp
  for (uint32_t i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n_all; i0 += stride) {
    const uint32_t i = i0 + lane_id();
    uint32_t v = 0, cnt = 0;
    if (i < n_all) {
      v = vt.nv == 1 ? 0u : find_view(s_begin, vt.nv, i);
      const float4 rec = __ldg(vt.g[v] + (i - s_begin[v]));
      const TileRect q = tile_rect(rec, vt.geom[v]);
      bad |= q.invalid;
      cnt = q.count;
      counts[i] = q.count;
      dkey[i] = q.count ? __float_as_uint(rec.z) : 0xffffffffu;
      dval[i] = i;
    }
    const uint32_t v0 = __shfl_sync(0xffffffffu, v, 0);
    if (__all_sync(0xffffffffu, v == v0 || i >= n_all)) {
      unsigned long long sum = cnt;
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
      if (lane_id() == 0 && sum) atomicAdd(&s_tot[v0], sum);
    } else if (cnt) {
      atomicAdd(&s_tot[v], static_cast<unsigned long long>(cnt));
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane_id() == 0) latch_error(err, TDGS_ERR_INVALID_ARGUMENT, kSiteViewsCount);
  __syncthreads();
  for (uint32_t v = threadIdx.x; v < vt.nv; v += blockDim.x)
    if (s_tot[v]) atomicAdd(reinterpret_cast<unsigned long long*>(vt.vtot + v), s_tot[v]);
}

cudaError_t launch_views_count(const ViewTable& vt, uint32_t n_all, uint32_t* counts,
                               uint32_t* dkey, uint32_t* dval, uint32_t* err, cudaStream_t s) {
  if (n_all == 0) return cudaSuccess;
  const uint32_t blocks = (n_all + 255) / 256;
  const uint32_t grid = blocks < 152u * 8u ? blocks : 152u * 8u;
  k_views_count<<<grid, 256, 0, s>>>(vt, n_all, counts, dkey, dval, err);
  return cudaGetLastError();
}

// pbeg[v] = pairs of views < v (views are contiguous in the sorted list
// because global tile ids are view-major).
__global__ void __launch_bounds__(32) k_views_pair_begin(ViewTable vt) {
  if (threadIdx.x == 0) {
    uint64_t run = 0;
    for (uint32_t v = 0; v < vt.nv; ++v) {
      vt.pbeg[v] = static_cast<uint32_t>(run);
      run += vt.vtot[v];
    }
    vt.pbeg[vt.nv] = static_cast<uint32_t>(run);
  }
}

cudaError_t launch_views_pair_begin(const ViewTable& vt, cudaStream_t s) {
  k_views_pair_begin<<<1, 32, 0, s>>>(vt);
  return cudaGetLastError();
}

// Duplicate in depth order: depth position j is record sorder[j]; its
// pairs start at soff[j]; each is (global tile << rbits) | j.  Warp-level
// load-balanced expansion: lane l takes pair chunk + l, finds its owner by
// a 5-step binary search over the lanes' start offsets, and derives the
// tile from the local index (rows outer, columns inner).
template <typename K>
__global__ void __launch_bounds__(256)
    k_views_dup(ViewTable vt, const uint32_t* __restrict__ sorder,
                const uint32_t* __restrict__ soff, uint32_t n_all, uint32_t rbits,
                K* __restrict__ out, uint32_t cap, uint32_t* err) {
  __shared__ uint32_t s_begin[kMaxViews + 1];
  for (uint32_t v = threadIdx.x; v <= vt.nv; v += blockDim.x) s_begin[v] = vt.rec_begin[v];
  __syncthreads();
  const uint32_t lane = lane_id();
  const uint32_t warps_total = (gridDim.x * blockDim.x) >> 5;
  bool over = false;
  for (uint32_t wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
       static_cast<uint64_t>(wg) * 32u < n_all; wg += warps_total) {
    const uint32_t j = wg * 32u + lane;
    TileRect q;
    q.x0 = q.y0 = q.x1 = q.y1 = 0;
    q.count = 0;
    uint64_t start = 0;
    int32_t gx = 1;
    uint32_t tb = 0;
    const uint32_t gi = j < n_all ? __ldg(sorder + j) : 0xffffffffu;
    if (gi < n_all) {  // a depth order that is not a permutation is never followed out of bounds
      const uint32_t v = vt.nv == 1 ? 0u : find_view(s_begin, vt.nv, gi);
      const FrameGeom fg = vt.geom[v];
      q = tile_rect(__ldg(vt.g[v] + (gi - s_begin[v])), fg);
      start = __ldg(soff + j);
      gx = fg.gx;
      tb = vt.tile_begin[v];
    }
    const uint64_t end = start + q.count;
    uint64_t end_max = end;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      const uint64_t o = __shfl_xor_sync(0xffffffffu, end_max, d);
      end_max = o > end_max ? o : end_max;
    }
    if (gi >= n_all) start = end_max;
    const uint64_t begin = __shfl_sync(0xffffffffu, start, 0);
    const int32_t w = q.x1 - q.x0;
    for (uint64_t c = begin; c < end_max; c += 32) {
      const uint64_t p = c + lane;
      uint32_t lo = 0;
#pragma unroll
      for (uint32_t step = 16; step > 0; step >>= 1) {
        const uint64_t sc = __shfl_sync(0xffffffffu, start, lo + step);
        if (sc <= p) lo += step;
      }
      const uint64_t s0 = __shfl_sync(0xffffffffu, start, lo);
      const int32_t ow = __shfl_sync(0xffffffffu, w, lo);
      const int32_t ox0 = __shfl_sync(0xffffffffu, q.x0, lo);
      const int32_t oy0 = __shfl_sync(0xffffffffu, q.y0, lo);
      const int32_t ogx = __shfl_sync(0xffffffffu, gx, lo);
      const uint32_t otb = __shfl_sync(0xffffffffu, tb, lo);
      if (p < end_max && ow > 0) {
        const uint32_t jj = static_cast<uint32_t>(p - s0);
        const uint32_t ry = jj / static_cast<uint32_t>(ow);
        const uint32_t rx = jj - ry * static_cast<uint32_t>(ow);
        const uint64_t tile = otb + static_cast<uint64_t>(oy0 + ry) * static_cast<uint64_t>(ogx) +
                              static_cast<uint64_t>(ox0 + rx);
        if (p < cap) out[p] = static_cast<K>((tile << rbits) | (wg * 32u + lo));
        else over = true;
      }
    }
  }
  if (__any_sync(0xffffffffu, over) && lane == 0) latch_error(err, TDGS_ERR_CAPACITY, kSiteViewsDup);
}

cudaError_t launch_views_dup(const ViewTable& vt, const uint32_t* sorder, const uint32_t* soff,
                             uint32_t n_all, uint32_t rbits, void* out, bool wide, uint32_t cap,
                             uint32_t* err, cudaStream_t s) {
  if (n_all == 0) return cudaSuccess;
  const uint32_t warps = (n_all + 31) / 32;
  const uint32_t blocks = (warps + 7) / 8;
  const uint32_t grid = blocks < 152u * 32u ? blocks : 152u * 32u;
  if (wide)
    k_views_dup<uint64_t><<<grid, 256, 0, s>>>(vt, sorder, soff, n_all, rbits,
                                               static_cast<uint64_t*>(out), cap, err);
  else
    k_views_dup<uint32_t><<<grid, 256, 0, s>>>(vt, sorder, soff, n_all, rbits,
                                               static_cast<uint32_t*>(out), cap, err);
  return cudaGetLastError();
}

// Identify Range: local [start, end) per tile from the first/last sorted
// positions recorded by the last tile pass; {0, 0} for an empty tile.
__global__ void __launch_bounds__(256)
    k_views_ranges(ViewTable vt, const uint32_t* __restrict__ rmin, const uint32_t* __restrict__ rmax,
                   uint32_t t_all, uint2* __restrict__ ranges) {
  __shared__ uint32_t s_tb[kMaxViews + 1];
  __shared__ uint32_t s_pb[kMaxViews + 1];
  for (uint32_t v = threadIdx.x; v <= vt.nv; v += blockDim.x) {
    s_tb[v] = vt.tile_begin[v];
    s_pb[v] = vt.pbeg[v];
  }
  __syncthreads();
  for (uint32_t t = blockIdx.x * blockDim.x + threadIdx.x; t < t_all; t += gridDim.x * blockDim.x) {
    const uint32_t lo = rmin[t];
    if (lo == 0xffffffffu) {
      ranges[t] = make_uint2(0u, 0u);
    } else {
      const uint32_t pb = s_pb[vt.nv == 1 ? 0u : find_view(s_tb, vt.nv, t)];
      ranges[t] = make_uint2(lo - pb, rmax[t] - pb);
    }
  }
}

cudaError_t launch_views_ranges(const ViewTable& vt, const uint32_t* rmin, const uint32_t* rmax,
                                uint32_t t_all, uint2* ranges, cudaStream_t s) {
  if (t_all == 0) return cudaSuccess;
  const uint32_t blocks = (t_all + 255) / 256;
  const uint32_t grid = blocks < 152u * 8u ? blocks : 152u * 8u;
  k_views_ranges<<<grid, 256, 0, s>>>(vt, rmin, rmax, t_all, ranges);
  return cudaGetLastError();
}

}  // namespace tdgs
