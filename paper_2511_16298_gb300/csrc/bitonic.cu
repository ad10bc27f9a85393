// The paper's sorting network (Sec. III "Optimizing Texture Memory Based
// Sorting", Algorithms 1-2): a bitonic sort of the (key, value) pairs,
// padded to a power of two, ascending by key then value.  When equal keys
// enter with ascending values -- as tdgs_duplicate_keys emits them -- this
// is the order of the stable sort, so the result is identical to
// tdgs_sort_pairs.
//
// The paper keeps each compare partner adjacent in a 2D texture (layout
// transformation) and fuses the last two steps of a stage into one kernel
// over a 4-element texel (stage fusion).  On this GPU the fastest memories
// next to a thread are its registers and its CTA's shared memory, so the
// same two ideas become:
//   * every step whose partner distance is below the tile (4096 pairs) runs
//     in shared memory: the first 12 stages entirely in one kernel, and the
//     last 12 steps of every later stage fused into one pass over the tile;
//   * steps with a larger partner distance are fused up to four at a time:
//     each thread loads the 16 pairs those steps connect into registers
//     (partners adjacent), runs the four compare-exchange levels there and
//     writes them back.
// Direction of a compare-exchange in stage k (sub-sequences of 2^k pairs):
// ascending when bit k of the global index is 0 (always, in the last stage).
#include "tdgs_internal.cuh"

namespace tdgs {

namespace {

constexpr int kBitonicTileLog = 12;
constexpr uint32_t kBitonicTile = 1u << kBitonicTileLog;  // pairs per CTA tile
constexpr int kBitonicThreads = 512;
constexpr int kFuse = 4;  // global steps per pass

struct Pair {
  uint64_t k;
  uint32_t v;
};

// a > b in (key, value) order
__device__ __forceinline__ bool greater(uint64_t ka, uint32_t va, uint64_t kb, uint32_t vb) {
  return ka > kb || (ka == kb && va > vb);
}

__device__ __forceinline__ void cmp_swap(uint64_t& ka, uint32_t& va, uint64_t& kb, uint32_t& vb, bool asc) {
  if (greater(ka, va, kb, vb) == asc) {
    const uint64_t tk = ka;
    ka = kb;
    kb = tk;
    const uint32_t tv = va;
    va = vb;
    vb = tv;
  }
}

// Steps j = j_hi .. 0 of stage k on the tile in shared memory; base = the
// tile's first global index.
__device__ __forceinline__ void tile_steps(uint64_t* sk, uint32_t* sv, uint32_t base, int k, int j_hi) {
  for (int j = j_hi; j >= 0; --j) {
    for (uint32_t q = threadIdx.x; q < kBitonicTile / 2; q += kBitonicThreads) {
      const uint32_t i = ((q >> j) << (j + 1)) | (q & ((1u << j) - 1u));
      const uint32_t p = i | (1u << j);
      const bool asc = (((base + i) >> k) & 1u) == 0u;
      uint64_t ka = sk[i], kb = sk[p];
      uint32_t va = sv[i], vb = sv[p];
      cmp_swap(ka, va, kb, vb, asc);
      sk[i] = ka;
      sk[p] = kb;
      sv[i] = va;
      sv[p] = vb;
    }
    __syncthreads();
  }
}

// Stages 1..min(log2 n2, 12) on each tile: loads from the input (pairs at
// or beyond m are the padding (all ones, all ones)), writes the tile to out
// (the first m pairs only when out is the caller's array: last == true).
__global__ void __launch_bounds__(kBitonicThreads)
    k_bitonic_tiles(const uint64_t* __restrict__ kin, const uint32_t* __restrict__ vin, uint32_t m,
                    int stages, uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, bool last) {
  __shared__ uint64_t sk[kBitonicTile];
  __shared__ uint32_t sv[kBitonicTile];
  const uint32_t base = blockIdx.x * kBitonicTile;
  for (uint32_t i = threadIdx.x; i < kBitonicTile; i += kBitonicThreads) {
    const uint32_t g = base + i;
    sk[i] = g < m ? kin[g] : ~0ull;
    sv[i] = g < m ? vin[g] : ~0u;
  }
  __syncthreads();
  for (int k = 1; k <= stages; ++k) tile_steps(sk, sv, base, k, k - 1);
  for (uint32_t i = threadIdx.x; i < kBitonicTile; i += kBitonicThreads) {
    const uint32_t g = base + i;
    if (!last || g < m) {
      kout[g] = sk[i];
      vout[g] = sv[i];
    }
  }
}

// The last 12 steps of stage k on each tile (stage fusion).
__global__ void __launch_bounds__(kBitonicThreads)
    k_bitonic_merge_tiles(uint64_t* __restrict__ k_io, uint32_t* __restrict__ v_io, int k, uint32_t m,
                          uint64_t* __restrict__ kout, uint32_t* __restrict__ vout, bool last) {
  __shared__ uint64_t sk[kBitonicTile];
  __shared__ uint32_t sv[kBitonicTile];
  const uint32_t base = blockIdx.x * kBitonicTile;
  for (uint32_t i = threadIdx.x; i < kBitonicTile; i += kBitonicThreads) {
    sk[i] = k_io[base + i];
    sv[i] = v_io[base + i];
  }
  __syncthreads();
  tile_steps(sk, sv, base, k, kBitonicTileLog - 1);
  for (uint32_t i = threadIdx.x; i < kBitonicTile; i += kBitonicThreads) {
    const uint32_t g = base + i;
    if (!last || g < m) {
      kout[g] = sk[i];
      vout[g] = sv[i];
    }
  }
}

// Steps j_hi .. j_lo (r = j_hi - j_lo + 1 <= kFuse, j_lo >= 12) of stage k
// in one pass: each thread owns the 2^r pairs these steps connect.
template <int r>
__global__ void __launch_bounds__(256)
    k_bitonic_global(uint64_t* __restrict__ keys, uint32_t* __restrict__ vals, uint32_t n2, int k, int j_lo) {
  constexpr int kN = 1 << r;
  const uint32_t groups = n2 >> r;
  for (uint32_t q = blockIdx.x * blockDim.x + threadIdx.x; q < groups; q += gridDim.x * blockDim.x) {
    const uint32_t low = q & ((1u << j_lo) - 1u);
    const uint32_t base = ((q >> j_lo) << (j_lo + r)) | low;
    const bool asc = ((base >> k) & 1u) == 0u;
    uint64_t ek[kN];
    uint32_t ev[kN];
#pragma unroll
    for (int s = 0; s < kN; ++s) {
      const uint32_t idx = base + (static_cast<uint32_t>(s) << j_lo);
      ek[s] = keys[idx];
      ev[s] = vals[idx];
    }
#pragma unroll
    for (int b = r - 1; b >= 0; --b) {
#pragma unroll
      for (int s = 0; s < kN; ++s)
        if (!(s & (1 << b))) cmp_swap(ek[s], ev[s], ek[s | (1 << b)], ev[s | (1 << b)], asc);
    }
#pragma unroll
    for (int s = 0; s < kN; ++s) {
      const uint32_t idx = base + (static_cast<uint32_t>(s) << j_lo);
      keys[idx] = ek[s];
      vals[idx] = ev[s];
    }
  }
}

uint32_t grid_of(uint32_t items, uint32_t per_block) {
  const uint32_t b = (items + per_block - 1) / per_block;
  const uint32_t cap = 152u * 16u;
  return b < 1u ? 1u : (b < cap ? b : cap);
}

cudaError_t launch_global(uint64_t* keys, uint32_t* vals, uint32_t n2, int k, int j_lo, int r, cudaStream_t s) {
  const uint32_t grid = grid_of(n2 >> r, 256);
  switch (r) {
    case 1: k_bitonic_global<1><<<grid, 256, 0, s>>>(keys, vals, n2, k, j_lo); break;
    case 2: k_bitonic_global<2><<<grid, 256, 0, s>>>(keys, vals, n2, k, j_lo); break;
    case 3: k_bitonic_global<3><<<grid, 256, 0, s>>>(keys, vals, n2, k, j_lo); break;
    default: k_bitonic_global<4><<<grid, 256, 0, s>>>(keys, vals, n2, k, j_lo); break;
  }
  return cudaGetLastError();
}

}  // namespace

uint32_t bitonic_padded(uint32_t m) {
  uint32_t n2 = kBitonicTile;
  while (n2 < m) n2 <<= 1;
  return n2;
}

uint32_t bitonic_launches(uint32_t m) {
  const uint32_t n2 = bitonic_padded(m);
  int x = 0;
  while ((1u << x) < n2) ++x;
  uint32_t launches = 1;
  for (int k = kBitonicTileLog + 1; k <= x; ++k) launches += (k - kBitonicTileLog + kFuse - 1) / kFuse + 1;
  return launches;
}

cudaError_t launch_bitonic(const uint64_t* kin, const uint32_t* vin, uint32_t m, uint64_t* kout, uint32_t* vout,
                           uint64_t* ks, uint32_t* vs, cudaStream_t s) {
  if (m == 0) return cudaSuccess;
  const uint32_t n2 = bitonic_padded(m);
  int x = 0;
  while ((1u << x) < n2) ++x;
  const uint32_t tiles = n2 / kBitonicTile;
  const bool one = x <= kBitonicTileLog;
  k_bitonic_tiles<<<tiles, kBitonicThreads, 0, s>>>(kin, vin, m, x < kBitonicTileLog ? x : kBitonicTileLog,
                                                     one ? kout : ks, one ? vout : vs, one);
  cudaError_t e = cudaGetLastError();
  for (int k = kBitonicTileLog + 1; e == cudaSuccess && k <= x; ++k) {
    for (int j_hi = k - 1; e == cudaSuccess && j_hi >= kBitonicTileLog;) {
      const int r = j_hi - kBitonicTileLog + 1 < kFuse ? j_hi - kBitonicTileLog + 1 : kFuse;
      e = launch_global(ks, vs, n2, k, j_hi - r + 1, r, s);
      j_hi -= r;
    }
    if (e != cudaSuccess) break;
    const bool last = k == x;
    k_bitonic_merge_tiles<<<tiles, kBitonicThreads, 0, s>>>(ks, vs, k, m, last ? kout : ks, last ? vout : vs, last);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace tdgs
