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
}


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
