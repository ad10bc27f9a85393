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
#include "project.cuh"

namespace tdgs {

// Per record (global index i over all views): tile count, depth sort key
// (raw depth bits of a visible Gaussian, all ones otherwise so culled ones
// sort last), the record index, and the per-view pair totals.  The last
// block to finish turns the totals into pbeg (first pair of each view in
// the sorted list; views are contiguous there because global tile ids are
// view-major), writes the pair count M to *total and resets the ticket.
// range[0..1] accumulate the smallest and largest depth key of a Gaussian
// with pairs (reset to all ones / zero by the last block, which publishes
// them in range[2..3] for the depth sort).
// kProject: every view's records are first computed from the same 3D
// Gaussians with the view's camera (the preprocessing stage fused into the
// count, proj::project) and stored for the later kernels.
constexpr int kCountUnroll = 4;
template <bool kProject>
__global__ void __launch_bounds__(256)
    k_views_count(ViewTable vt, uint32_t n_all, uint32_t* __restrict__ counts,
                  uint32_t* __restrict__ dkey, uint32_t* __restrict__ dval, uint32_t* err,
                  uint32_t* ticket, uint64_t* total, uint32_t* range, uint32_t* host_status, Proj3D pj) {
  __shared__ uint32_t s_begin[kMaxViews + 1];
  __shared__ unsigned long long s_tot[kMaxViews];
  __shared__ const float4* s_g[kMaxViews];
  __shared__ FrameGeom s_geom[kMaxViews];
  __shared__ bool s_last;
  __shared__ uint32_t s_lo, s_hi;
  __shared__ CameraDev s_cam[kProject ? kMaxViews : 1];
  __shared__ float2 s_lim[kProject ? kMaxViews : 1];
  for (uint32_t v = threadIdx.x; v <= vt.nv; v += blockDim.x) s_begin[v] = vt.rec_begin[v];
  for (uint32_t v = threadIdx.x; v < vt.nv; v += blockDim.x) {
    s_tot[v] = 0;
    s_g[v] = vt.g[v];
    s_geom[v] = vt.geom[v];
    if constexpr (kProject) {
      s_cam[v] = pj.cams[v];
      s_lim[v] = proj::slope_limits(pj.cams[v]);
    }
  }
  if (threadIdx.x == 0) {
    s_lo = 0xffffffffu;
    s_hi = 0u;
  }
  __syncthreads();
  bool bad = false;
  uint32_t lo = 0xffffffffu, hi = 0u;  // depth keys of Gaussians with pairs
  // one view reads its camera from the kernel parameters, many views
  // from shared memory
  const float2 lim0 = kProject ? proj::slope_limits(pj.cam0) : make_float2(0.f, 0.f);
  const uint32_t lane = lane_id();
  const uint32_t stride = gridDim.x * blockDim.x;
  // warp-uniform loop so the per-view totals can be reduced across the
  // warp; kUnroll records per thread are in flight at once (two when each
  // needs three 16-byte loads and the projection)
  constexpr int kUnroll = kProject ? 2 : kCountUnroll;
  for (uint32_t i0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); i0 < n_all; i0 += stride * kUnroll) {
    float4 rec[kUnroll];
    uint32_t vv[kUnroll];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t i = i0 + u * stride + lane;
      vv[u] = 0;
      rec[u] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (i < n_all) {
        if constexpr (kProject) {
          float4 co;
          if (vt.nv == 1) {
            proj::project(__ldg(pj.g + i), __ldg(pj.cov + 2 * static_cast<size_t>(i)),
                          __ldg(pj.cov + 2 * static_cast<size_t>(i) + 1), pj.cam0, lim0, rec[u], co);
          } else {
            vv[u] = find_view(s_begin, vt.nv, i);
            const uint32_t l = i - s_begin[vv[u]];
            proj::project(__ldg(pj.g + l), __ldg(pj.cov + 2 * static_cast<size_t>(l)),
                          __ldg(pj.cov + 2 * static_cast<size_t>(l) + 1), s_cam[vv[u]], s_lim[vv[u]], rec[u], co);
          }
          pj.rec[i] = rec[u];
          pj.conic[i] = co;
        } else {
          vv[u] = vt.nv == 1 ? 0u : find_view(s_begin, vt.nv, i);
          rec[u] = __ldg(s_g[vv[u]] + (i - s_begin[vv[u]]));
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const uint32_t i = i0 + u * stride + lane;
      uint32_t cnt = 0;
      const uint32_t v = vv[u];
      if (i < n_all) {
        const TileRect q = tile_rect(rec[u], s_geom[v]);
        bad |= q.invalid;
        cnt = q.count;
        counts[i] = q.count;
        const uint32_t key = q.count ? __float_as_uint(rec[u].z) : 0xffffffffu;
        dkey[i] = key;
        dval[i] = i;
        if (q.count) {
          lo = min(lo, key);
          hi = max(hi, key);
        }
      }
      const uint32_t v0 = __shfl_sync(0xffffffffu, v, 0);
      if (__all_sync(0xffffffffu, v == v0 || i >= n_all)) {
        unsigned long long sum = cnt;
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, d);
        if (lane == 0 && sum) atomicAdd(&s_tot[v0], sum);
      } else if (cnt) {
        atomicAdd(&s_tot[v], static_cast<unsigned long long>(cnt));
      }
    }
  }
  if (__any_sync(0xffffffffu, bad) && lane == 0) latch_error(err, TDGS_ERR_INVALID_ARGUMENT, kSiteViewsCount);
  lo = __reduce_min_sync(0xffffffffu, lo);
  hi = __reduce_max_sync(0xffffffffu, hi);
  if (lane == 0) {
    atomicMin(&s_lo, lo);
    atomicMax(&s_hi, hi);
  }
  __syncthreads();
  for (uint32_t v = threadIdx.x; v < vt.nv; v += blockDim.x)
    if (s_tot[v]) atomicAdd(reinterpret_cast<unsigned long long*>(vt.vtot + v), s_tot[v]);
  if (threadIdx.x == 0) {
    if (s_lo != 0xffffffffu) atomicMin(range, s_lo);
    if (s_hi != 0u) atomicMax(range + 1, s_hi);
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (s_last) {
    __threadfence();
    for (uint32_t v = threadIdx.x; v < vt.nv; v += blockDim.x) s_tot[v] = __ldcg(reinterpret_cast<unsigned long long*>(vt.vtot + v));
    __syncthreads();
    if (threadIdx.x == 0) {
      uint64_t run = 0;
      for (uint32_t v = 0; v < vt.nv; ++v) {
        vt.pbeg[v] = static_cast<uint32_t>(run);
        run += s_tot[v];
      }
      vt.pbeg[vt.nv] = static_cast<uint32_t>(run);
      *total = run;
      if (host_status) {
        // the same for the host, in mapped pinned memory: {total, error,
        // site} (errors latched by every other block are visible here)
        reinterpret_cast<volatile unsigned long long*>(host_status)[0] = run;
        reinterpret_cast<volatile uint32_t*>(host_status)[2] = __ldcg(err);
        reinterpret_cast<volatile uint32_t*>(host_status)[3] = __ldcg(err + 1);
        __threadfence_system();
      }
      range[2] = __ldcg(range);
      range[3] = __ldcg(range + 1);
      range[0] = 0xffffffffu;
      range[1] = 0u;
      *ticket = 0;
    }
  }
}

cudaError_t launch_views_count(const ViewTable& vt, uint32_t n_all, uint32_t* counts,
                               uint32_t* dkey, uint32_t* dval, uint32_t* err, uint32_t* ticket,
                               uint64_t* total, uint32_t* range, void* host_status, cudaStream_t s,
                               const Proj3D* proj) {
  const uint32_t per_block = 256u * (proj ? 2u : static_cast<uint32_t>(kCountUnroll));
  const uint32_t blocks = (n_all + per_block - 1) / per_block;
  const uint32_t grid = blocks < 1u ? 1u : (blocks < 152u * 8u ? blocks : 152u * 8u);
  if (proj)
    k_views_count<true><<<grid, 256, 0, s>>>(vt, n_all, counts, dkey, dval, err, ticket, total, range,
                                             static_cast<uint32_t*>(host_status), *proj);
  else
    k_views_count<false><<<grid, 256, 0, s>>>(vt, n_all, counts, dkey, dval, err, ticket, total, range,
                                              static_cast<uint32_t*>(host_status), Proj3D{});
  return cudaGetLastError();
}

// Duplicate in depth order: depth position j is record sorder[j]; its
// pairs start at soff[j]; each is (global tile << rbits) | j.  A warp owns
// 32 consecutive depth positions; their pairs are consecutive in the
// output.  Lane l of a window writes the 4 pairs of quad l (quads are
// aligned to 4 output elements, so whole quads are one 16-byte store): it
// finds the owner of its first pair by a binary search over the warp's
// 32 starts in shared memory, splits that pair's index inside the
// rectangle into row and column once (float reciprocal with one exact
// correction step, or an integer division past 2^22), then steps column
// by column, wrapping rows and moving to the next Gaussian when its pairs
// are done.  Rows are outer, columns inner.
template <typename K>
__device__ __forceinline__ void store_quad(K* dst, const K (&e)[4], uint32_t valid_mask) {
  if (valid_mask == 0xfu) {
    if constexpr (sizeof(K) == 4) {
      *reinterpret_cast<uint4*>(dst) = make_uint4(e[0], e[1], e[2], e[3]);
    } else {
      reinterpret_cast<ulonglong2*>(dst)[0] = make_ulonglong2(e[0], e[1]);
      reinterpret_cast<ulonglong2*>(dst)[1] = make_ulonglong2(e[2], e[3]);
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (valid_mask & (1u << i)) dst[i] = e[i];
  }
}

template <typename K>
__global__ void __launch_bounds__(256)
    k_views_dup(ViewTable vt, const uint32_t* __restrict__ sorder,
                const uint32_t* __restrict__ soff, uint32_t n_all, uint32_t rbits,
                K* __restrict__ out, uint32_t cap, uint2* __restrict__ sdo, uint32_t* err) {
  __shared__ uint32_t s_begin[kMaxViews + 1];
  __shared__ const float4* s_g[kMaxViews];
  __shared__ FrameGeom s_geom[kMaxViews];
  __shared__ uint32_t s_tb[kMaxViews];
  // per warp and lane: first pair relative to the warp's first pair
  // (non-decreasing; [32] = end of the warp's range), global id of the
  // rectangle's first tile, width, 1 / width, tiles per row of the view
  __shared__ uint32_t s_st[8][33];
  __shared__ uint32_t s_first[8][32];
  __shared__ uint32_t s_w[8][32];
  __shared__ float s_rw[8][32];
  __shared__ uint32_t s_gx[8][32];
  for (uint32_t v = threadIdx.x; v <= vt.nv; v += blockDim.x) s_begin[v] = vt.rec_begin[v];
  for (uint32_t v = threadIdx.x; v < vt.nv; v += blockDim.x) {
    s_g[v] = vt.g[v];
    s_geom[v] = vt.geom[v];
    s_tb[v] = vt.tile_begin[v];
  }
  __syncthreads();
  const uint32_t lane = lane_id(), w8 = threadIdx.x >> 5;
  const uint32_t warps_total = (gridDim.x * blockDim.x) >> 5;
  bool over = false;
  for (uint32_t wg = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
       static_cast<uint64_t>(wg) * 32u < n_all; wg += warps_total) {
    const uint32_t j = wg * 32u + lane;
    TileRect q;
    q.x0 = q.y0 = q.x1 = q.y1 = 0;
    q.count = 0;
    uint64_t start = 0;
    uint32_t first = 0, gx = 1;
    const uint32_t gi = j < n_all ? __ldg(sorder + j) : 0xffffffffu;
    if (gi < n_all) {  // a depth order that is not a permutation is never followed out of bounds
      const uint32_t v = vt.nv == 1 ? 0u : find_view(s_begin, vt.nv, gi);
      const FrameGeom fg = s_geom[v];
      const float4 rec = __ldg(s_g[v] + (gi - s_begin[v]));
      q = tile_rect(rec, fg);
      start = __ldg(soff + j);
      gx = static_cast<uint32_t>(fg.gx);
      first = s_tb[v] + static_cast<uint32_t>(q.y0) * gx + static_cast<uint32_t>(q.x0);
      // the depth key of the count kernel, beside the record index
      sdo[j] = make_uint2(q.count ? __float_as_uint(rec.z) : 0xffffffffu, gi);
    }
    // pairs of consecutive depth positions are consecutive, so the warp's
    // last valid lane ends its range
    const uint32_t last = min(31u, n_all - 1u - wg * 32u);
    const uint64_t end_max = __shfl_sync(0xffffffffu, start + q.count, last);
    if (end_max > cap) over = true;
    // Positions relative to the warp's first pair, in 32 bits; pairs at or
    // beyond cap are not written.
    const uint64_t begin = __shfl_sync(0xffffffffu, start, 0);
    const uint64_t stop = end_max < cap ? end_max : cap;
    const uint64_t span = stop > begin ? stop - begin : 0;
    const uint32_t nrel = span < 0xfffffff0ull ? static_cast<uint32_t>(span) : 0xfffffff0u;
    const uint64_t srel64 = start - begin;
    const uint32_t wd = static_cast<uint32_t>(q.x1 - q.x0);
    s_st[w8][lane] = (j < n_all && srel64 < nrel) ? static_cast<uint32_t>(srel64) : nrel;
    if (lane == 0) s_st[w8][32] = nrel;
    s_first[w8][lane] = first;
    s_w[w8][lane] = wd;
    s_rw[w8][lane] = wd ? __frcp_rn(static_cast<float>(wd)) : 0.0f;
    s_gx[w8][lane] = gx;
    __syncwarp();
    const uint32_t lead = static_cast<uint32_t>(begin & 3u);  // quads are aligned to 4 output elements
    const uint32_t nquad = (nrel + lead + 3u) / 4u;
    K* qout = out + (begin - lead);
    const uint32_t rank0 = wg * 32u;
    for (uint32_t q0 = 0; q0 < nquad; q0 += 32) {
      const uint32_t qi = q0 + lane;
      if (qi < nquad) {
        // relative position of the quad's first element, modulo 2^32: the
        // first quad's lead elements wrap to 2^32 - lead .. 2^32 - 1, at or
        // above nrel (<= 0xfffffff0), so one unsigned test skips them
        const uint32_t r0 = qi * 4u - lead;
        const uint32_t x = qi ? r0 : 0u;
        uint32_t owner = 0;
#pragma unroll
        for (uint32_t step = 16; step > 0; step >>= 1)
          if (s_st[w8][owner + step] <= x) owner += step;
        // row and column of pair x inside the owner's rectangle
        uint32_t ow = s_w[w8][owner];
        const uint32_t jj = x - s_st[w8][owner];
        uint32_t ry, rx;
        if (jj < (1u << 22)) {
          ry = __float2uint_rz(__fmul_rn(__uint2float_rn(jj), s_rw[w8][owner]));
          rx = jj - ry * ow;
          if (static_cast<int32_t>(rx) < 0) {
            --ry;
            rx += ow;
          } else if (rx >= ow) {
            ++ry;
            rx -= ow;
          }
        } else {
          ry = jj / ow;
          rx = jj - ry * ow;
        }
        uint32_t ogx = s_gx[w8][owner];
        uint32_t row = s_first[w8][owner] + ry * ogx;
        uint32_t next = s_st[w8][owner + 1];
        K e[4];
        uint32_t valid = 0;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const uint32_t ru = r0 + static_cast<uint32_t>(i);
          e[i] = K(0);
          if (ru < nrel) {
            while (next <= ru) {  // the owner's pairs are done: the next Gaussian with pairs
              ++owner;
              next = s_st[w8][owner + 1];
              if (next > ru) {
                ow = s_w[w8][owner];
                ogx = s_gx[w8][owner];
                row = s_first[w8][owner];
                rx = 0;
              }
            }
            e[i] = (static_cast<K>(row + rx) << rbits) | static_cast<K>(rank0 + owner);
            valid |= 1u << i;
            if (++rx == ow) {
              rx = 0;
              row += ogx;
            }
          }
        }
        store_quad<K>(qout + static_cast<size_t>(qi) * 4, e, valid);
      }
    }
    __syncwarp();
  }
  if (__any_sync(0xffffffffu, over) && lane == 0) latch_error(err, TDGS_ERR_CAPACITY, kSiteViewsDup);
}

cudaError_t launch_views_dup(const ViewTable& vt, const uint32_t* sorder, const uint32_t* soff,
                             uint32_t n_all, uint32_t rbits, void* out, bool wide, uint32_t cap,
                             uint2* sdo, uint32_t* err, cudaStream_t s) {
  if (n_all == 0) return cudaSuccess;
  const uint32_t warps = (n_all + 31) / 32;
  const uint32_t blocks = (warps + 7) / 8;
  const uint32_t grid = blocks < 152u * 32u ? blocks : 152u * 32u;
  if (wide)
    k_views_dup<uint64_t><<<grid, 256, 0, s>>>(vt, sorder, soff, n_all, rbits,
                                               static_cast<uint64_t*>(out), cap, sdo, err);
  else
    k_views_dup<uint32_t><<<grid, 256, 0, s>>>(vt, sorder, soff, n_all, rbits,
                                               static_cast<uint32_t*>(out), cap, sdo, err);
  return cudaGetLastError();
}

}  // namespace tdgs
