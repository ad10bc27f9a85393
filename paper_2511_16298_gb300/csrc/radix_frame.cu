// Radix passes of the depth-first frame path: the depth sort of the N
// Gaussians and the stable passes over the packed (tile, depth rank)
// stream, the last of which expands to the final keys and indices.
#include "radix.cuh"

namespace tdgs {

namespace {
using radix::make_kernel;
const radix::Kernel& depth_kernel(int digit_bits) {
  static const radix::Kernel k11 = make_kernel<uint32_t, true, false, 11, 256, 16>();
  static const radix::Kernel k8 = make_kernel<uint32_t, true, false, 8, 256, 16>();
  return digit_bits == 11 ? k11 : k8;
}
// Tile passes: digit kernels of 6, 8 and 12 bits, narrow (32-bit) or wide
// (64-bit) packed elements, plain or expanding.
const radix::Kernel& stream_kernel(bool wide, bool expand, uint32_t bits) {
  static const radix::Kernel k[12] = {
      make_kernel<uint32_t, false, false, 6, 256, 16>(),  make_kernel<uint32_t, false, true, 6, 256, 16>(),
      make_kernel<uint64_t, false, false, 6, 256, 16>(),  make_kernel<uint64_t, false, true, 6, 256, 16>(),
      make_kernel<uint32_t, false, false, 8, 256, 16>(),  make_kernel<uint32_t, false, true, 8, 256, 16>(),
      make_kernel<uint64_t, false, false, 8, 256, 16>(),  make_kernel<uint64_t, false, true, 8, 256, 16>(),
      make_kernel<uint32_t, false, false, 12, 256, 16>(), make_kernel<uint32_t, false, true, 12, 256, 16>(),
      make_kernel<uint64_t, false, false, 12, 256, 16>(), make_kernel<uint64_t, false, true, 12, 256, 16>(),
  };
  const int w = bits <= 6 ? 0 : (bits <= 8 ? 1 : 2);
  return k[w * 4 + (wide ? 2 : 0) + (expand ? 1 : 0)];
}
}  // namespace

uint32_t stream_kernel_bits(uint32_t width) { return width <= 6 ? 6u : (width <= 8 ? 8u : 12u); }

DepthPlan plan_depth_sort(uint32_t n, int tuned_bits, int ctas_per_sm) {
  DepthPlan p{};
  const uint32_t nn = n ? n : 1;
  const uint32_t g = depth_sort_grid();
  if (g && nn <= depth_sort_count_capacity(g)) {
    p.resident = true;
    p.bits = 9;
    p.passes = 4;  // at most; the kernel runs as many as the key range needs
    p.grid = g;
    p.result = 1;
    p.scratch_words = 0;  // its state lives in a buffer of its own (depth_sort_scratch_words)
    return p;
  }
  p.resident = false;
  if (g && nn < (1u << 30)) {
    p.onesweep = true;
    p.bits = 9;
    p.passes = kDepthOnesweepPasses;  // launches; the device runs as many as the key range needs
    p.grid = g;
    p.result = 1;
    p.scratch_words = 0;  // its scratch is a buffer of its own (onesweep_scratch_words)
    return p;
  }
  p.bits = tuned_bits == 11 ? 11 : 8;
  p.passes = p.bits == 11 ? 3u : 4u;
  p.grid = radix::grid_for(depth_kernel(p.bits), nn, ctas_per_sm);
  p.result = p.passes & 1u;
  p.scratch_words = radix::scratch_words(depth_kernel(p.bits), p.grid);
  return p;
}

DepthPlan plan_key32_sort(uint32_t m, uint32_t key_bits, int ctas_per_sm) {
  DepthPlan p{};
  p.resident = false;
  p.bits = 11;
  p.passes = key_bits ? (key_bits + 10) / 11 : 1;
  p.grid = radix::grid_for(depth_kernel(11), m ? m : 1, ctas_per_sm);
  p.result = p.passes & 1u;
  p.scratch_words = radix::scratch_words(depth_kernel(11), p.grid);
  return p;
}

namespace {
void depth_digit(uint32_t bits, uint32_t pass, uint32_t* shift, uint32_t* mask) {
  *shift = pass * bits;
  *mask = *shift + bits <= 32 ? (1u << bits) - 1 : (1u << (32 - *shift)) - 1;
}
}  // namespace

cudaError_t launch_depth_pass(const DepthPlan& dp, uint32_t pass, const uint32_t* kin, const uint32_t* vin,
                              uint32_t* kout, uint32_t* vout, uint32_t n, uint32_t* scratch, uint32_t* bar,
                              uint32_t* err, cudaStream_t s) {
  radix::PassArgs a{};
  a.m = n;
  depth_digit(static_cast<uint32_t>(dp.bits), pass, &a.shift, &a.mask);
  a.bar = bar;
  a.err = err;
  return radix::launch(depth_kernel(dp.bits), dp.grid, kin, vin, kout, vout, a, scratch, s);
}

uint32_t stream_grid(bool wide, bool expand, uint32_t bits, uint32_t m, int ctas_per_sm) {
  return radix::grid_for(stream_kernel(wide, expand, bits), m, ctas_per_sm);
}
size_t stream_scratch_words(bool wide, bool expand, uint32_t bits, uint32_t grid) {
  return radix::scratch_words(stream_kernel(wide, expand, bits), grid);
}

cudaError_t launch_stream_pass(const StreamPass& sp, uint32_t* scratch, uint32_t* bar,
                               uint32_t* err, cudaStream_t s) {
  radix::PassArgs a{};
  a.m = sp.m;
  a.m_dev = sp.m_dev;
  a.shift = sp.shift;
  a.mask = sp.width >= 32 ? 0xffffffffu : (1u << sp.width) - 1;
  a.rbits = sp.rbits;
  a.sdo = sp.sdo;
  if (sp.expand && sp.views) {
    a.vrec_begin = sp.views->rec_begin;
    a.vtile_begin = sp.views->tile_begin;
    a.nv = sp.views->nv;
    a.pbeg = sp.views->pbeg;
  }
  a.rmin = sp.rmin;
  a.rmax = sp.rmax;
  a.ranges = sp.ranges;
  a.t_all = sp.t_all;
  a.bar = bar;
  a.err = err;
  return radix::launch(stream_kernel(sp.wide, sp.expand, sp.bits), sp.grid, sp.kin, nullptr, sp.kout, sp.vout,
                       a, scratch, s);
}

}  // namespace tdgs
