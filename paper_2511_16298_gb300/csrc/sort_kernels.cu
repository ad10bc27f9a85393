// tdgs_sort_pairs: stable sort of (uint64 key, uint32 value) pairs by the
// significant key bits (Sec. II-A Sorting), built from the radix pass of
// radix.cuh.  This file holds the compiled pass variants (digit width,
// threads, keys per thread) and the plan that picks passes and digits.
#include "radix.cuh"

namespace tdgs {

namespace {
using radix::make_kernel;
const radix::Kernel& variant_kernel(int i) {
  static const radix::Kernel kV[] = {
      make_kernel<uint64_t, true, false, 8, 256, 16>(),
      make_kernel<uint64_t, true, false, 9, 256, 16>(),
      make_kernel<uint64_t, true, false, 10, 256, 16>(),
      make_kernel<uint64_t, true, false, 11, 256, 16>(),
      make_kernel<uint64_t, true, false, 9, 256, 16, 3>(),
      make_kernel<uint64_t, true, false, 9, 256, 12, 3>(),
      make_kernel<uint64_t, true, false, 8, 256, 12, 3>(),
      make_kernel<uint64_t, true, false, 9, 256, 8, 4>(),
      make_kernel<uint64_t, true, false, 9, 512, 16>(),
  };
  return kV[i];
}
constexpr int kNumVariants = 9;
}  // namespace

int num_pass_variants() { return kNumVariants; }
PassVariant pass_variant(int i) {
  const radix::Kernel& k = variant_kernel(i);
  return PassVariant{k.bits, k.threads, k.items, k.min_blocks};
}

int default_pass_variant(uint32_t digit_bits) {
  if (digit_bits <= 8) return 0;
  if (digit_bits <= 9) return 1;
  if (digit_bits <= 10) return 2;
  return 3;
}

SortPlan make_sort_plan(uint32_t m, uint32_t tile_bits, uint32_t flags, const Tuning& tu) {
  const int variant_override = tu.sort_variant;
  SortPlan p{};
  p.drop31 = (flags & TDGS_SORT_DEPTH_POSITIVE) != 0;
  p.key_bits = 32 + tile_bits - (p.drop31 ? 1 : 0);
  p.bad_mask = tile_bits >= 32 ? 0ull : ~((1ull << (32 + tile_bits)) - 1);
  if (p.drop31) p.bad_mask |= 1ull << 31;
  // 9-bit digits by default: wider digits save a pass but scatter shorter
  // runs per digit (a 4096-key tile writes ~8 keys per digit at 9 bits, ~2
  // at 11), and the partial-sector writes cost more than the pass
  uint32_t max_bits = 9;
  const bool forced = variant_override >= 0 && variant_override < kNumVariants;
  if (forced) {
    max_bits = static_cast<uint32_t>(variant_kernel(variant_override).bits);
    p.variant = static_cast<uint32_t>(variant_override);
  }
  p.passes = (p.key_bits + max_bits - 1) / max_bits;
  p.digit_bits = (p.key_bits + p.passes - 1) / p.passes;
  if (!forced) p.variant = static_cast<uint32_t>(default_pass_variant(p.digit_bits));
  for (uint32_t i = 0; i < p.passes; ++i) {
    p.shift[i] = i * p.digit_bits;
    const uint32_t w = p.key_bits - p.shift[i] < p.digit_bits ? p.key_bits - p.shift[i] : p.digit_bits;
    p.mask[i] = (1u << w) - 1;
  }
  const radix::Kernel& k = variant_kernel(static_cast<int>(p.variant));
  p.tile_keys = static_cast<uint32_t>(k.threads * k.items);
  p.bins = 1u << k.bits;
  p.grid = radix::grid_for(k, m, tu.ctas_per_sm);
  return p;
}

size_t radix_scratch_words(const SortPlan& plan) {
  return radix::scratch_words(variant_kernel(static_cast<int>(plan.variant)), plan.grid);
}

cudaError_t launch_radix_pass(const SortPlan& plan, uint32_t pass, const uint64_t* kin,
                              const uint32_t* vin, uint64_t* kout, uint32_t* vout, uint32_t m,
                              uint32_t* scratch, uint32_t* bar, uint32_t* err, cudaStream_t s) {
  radix::PassArgs a{};
  a.m = m;
  a.shift = plan.shift[pass];
  a.mask = plan.mask[pass];
  a.drop31 = plan.drop31 ? 1 : 0;
  a.bad_mask = pass == 0 ? plan.bad_mask : 0ull;
  a.bar = bar;
  a.err = err;
  return radix::launch(variant_kernel(static_cast<int>(plan.variant)), plan.grid, kin, vin, kout,
                       vout, a, scratch, s);
}

}  // namespace tdgs
