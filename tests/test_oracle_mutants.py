"""The pins have teeth: plausible mistakes planted in a copy of the oracle
(compiled on the CPU into a temporary library) each fail at least one pin.
The real oracle source is never modified.  Each mutant runs in its own
process; a mutant that crashes counts as caught."""
import json
import os
import subprocess
import sys

import pytest

from oracle import oracle as O

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                   "tdgs_oracle.cpp")

MUTANTS = {
    "round_up_16": ("sx1 = sx1 + 15.0f;", "sx1 = sx1 + 16.0f;"),
    "round_up_missing_y": ("sy1 = sy1 + 15.0f;", ""),
    "y_uses_x": ("volatile float sy0 = g.y - r;", "volatile float sy0 = g.x - r;"),
    "clamp_grid_minus_one": ("q.x1 = static_cast<int32_t>(clampf(fx1, static_cast<float>(gx)));",
                             "q.x1 = static_cast<int32_t>(clampf(fx1, static_cast<float>(gx - 1)));"),
    "tile_transposed": ("static_cast<uint64_t>(ty) * static_cast<uint64_t>(gx) +\n"
                        "                              static_cast<uint64_t>(tx);",
                        "static_cast<uint64_t>(tx) * static_cast<uint64_t>(gy) +\n"
                        "                              static_cast<uint64_t>(ty);"),
    "depth_converted_not_bits": ("const uint64_t dbits = bits_of(g[i].depth);",
                                 "const uint64_t dbits = static_cast<uint32_t>(g[i].depth * 1000.0f);"),
    "accepts_zero_depth": ("return std::isfinite(d) && d > 0.0f;", "return std::isfinite(d) && d >= 0.0f;"),
    "inclusive_scan": ("    offsets[i] = static_cast<uint32_t>(run);\n    run += counts[i];",
                       "    run += counts[i];\n    offsets[i] = static_cast<uint32_t>(run);"),
    "no_overflow_check": ("return run > 0xFFFFFFFFull ? kOverflow : kOk;", "return kOk;"),
    "sort_by_tile_only": ("return keys[a] < keys[b]; });", "return (keys[a] >> 32) < (keys[b] >> 32); });"),
    "ties_reversed": ("return keys[a] < keys[b]; });",
                      "return keys[a] < keys[b] || (keys[a] == keys[b] && a > b); });"),
    "range_end_short": ("ranges[2 * prev + 1] = m;", "ranges[2 * prev + 1] = m - 1;"),
    "range_start_skipped": ("      ranges[2 * t] = k;\n", "      ranges[2 * t] = k ? k - 1 : 0;\n"),
    "no_lowpass": ("M[0][2] * T[0][2]) + 0.3f;", "M[0][2] * T[0][2]);"),
    "smaller_eigenvalue": ("const float lambda = mid + std::sqrt", "const float lambda = mid - std::sqrt"),
    "no_discriminant_floor": ("std::fmax(0.1f, disc)", "std::fmax(0.0f, disc)"),
    "jacobian_sign": ("j02 = -((cam->fx * uc) / tz);", "j02 = ((cam->fx * uc) / tz);"),
    "no_slope_clamp": ("const float uc = std::fmin(lim_x, std::fmax(-lim_x, u));", "const float uc = u;"),
    "cull_at_near_plane": ("bool keep = tz > cam->near_z;", "bool keep = tz >= cam->near_z;"),
    "two_sigma": ("std::ceil(3.0f * std::sqrt(lambda))", "std::ceil(2.0f * std::sqrt(lambda))"),
    "conic_swapped": ("co[0] = d / det;", "co[0] = a / det;"),
    "render_no_early_stop": ("if (test_t < 0.0001f) break;", ""),
    "render_back_to_front": ("        const uint32_t i = sorted_values[k];",
                             "        const uint32_t i = sorted_values[ranges[2 * t] + ranges[2 * t + 1] - 1 - k];"),
    "render_no_alpha_cap": ("std::fmin(0.99f, co[3] * std::exp(power))", "co[3] * std::exp(power)"),
    "render_cut_1_64": ("if (alpha < 1.0f / 255.0f) continue;", "if (alpha < 1.0f / 64.0f) continue;"),
    "render_t_before_colour": ("for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * static_cast<size_t>(i) + ch] * alpha * T;\n        T = test_t;",
                               "T = test_t;\n        for (int ch = 0; ch < 3; ++ch) C[ch] += rgb[3 * static_cast<size_t>(i) + ch] * alpha * T;"),
    "render_no_background": ("o[ch] = C[ch] + T * background[ch];", "o[ch] = C[ch];"),
    "render_tile_transposed": ("const uint32_t t = (py / 16u) * gx + px / 16u;",
                               "const uint32_t t = (px / 16u) * gx + py / 16u;"),
    "render_cross_sign": ("- co[1] * dx * dy;", "+ co[1] * dx * dy;"),
    "render_pixel_centre": ("const float fx = static_cast<float>(px), fy = static_cast<float>(py);",
                            "const float fx = static_cast<float>(px) + 0.5f, fy = static_cast<float>(py) + 0.5f;"),
    "norm_scale_1023": ("1024.0f / (dmax - dmin)", "1023.0f / (dmax - dmin)"),
    "norm_no_clamp": ("f >= 1023.0f ? 1023u : static_cast<uint32_t>(f)", "static_cast<uint32_t>(f)"),
    "norm_range_includes_culled": ("    if (!counts[i]) continue;\n    m += counts[i];",
                                   "    if (g[i].depth < dmin || !any) { dmin = g[i].depth; any = true; }\n"
                                   "    if (!counts[i]) continue;\n    m += counts[i];"),
    "norm_ties_reversed": ("[&k0](uint32_t a, uint32_t b) { return k0[a] < k0[b]; }",
                           "[&k0](uint32_t a, uint32_t b) { return k0[a] < k0[b] || (k0[a] == k0[b] && a > b); }"),
    "norm_shift_12": ("k0.push_back((tile << 10) | qd);", "k0.push_back((tile << 12) | qd);"),
    "rotation_transposed": ("T[0][k] = j00 * R[k] + j02 * R[6 + k];", "T[0][k] = j00 * R[3 * k] + j02 * R[6 + k];"),
}


def test_unmutated_oracle_passes_every_pin(oracle):
    """A mutant counts as caught only if the real oracle passes the same pins."""
    from tests import oracle_pins as P
    assert P.run_all(oracle) == []


@pytest.fixture(scope="module")
def src_text():
    return open(SRC).read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, src_text, tmp_path):
    old, new = MUTANTS[name]
    assert src_text.count(old) >= 1, f"mutation site for {name} not found"
    mutated = src_text.replace(old, new, 1)
    src = tmp_path / "mutant.cpp"
    src.write_text(mutated)
    lib = O.compile_oracle(str(src), str(tmp_path / "libmutant.so"))
    root = os.path.dirname(os.path.dirname(SRC))
    proc = subprocess.run([sys.executable, "-m", "tests.oracle_pins", lib], cwd=root,
                          capture_output=True, text=True, timeout=300)
    if proc.returncode == 0:
        failed = json.loads(proc.stdout.strip().splitlines()[-1])
        assert failed, f"mutant {name} passed every pin"
