"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Everything on the path is integer or a float32 computation with a pinned
operation order, so the bar is bit-exact: counts, offsets, keys, values and
ranges must be identical, and error statuses must agree.
"""
import functools

import numpy as np
import pytest
import torch

from paper_2511_16298_gb300 import synth
from paper_2511_16298_gb300 import tdgs as T
from tests import oracle_pins as P

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    from paper_2511_16298_gb300 import build
    build.build()
    c = T.Context(0)
    yield c
    c.close()


def u64(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def u32(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


@functools.lru_cache(maxsize=1)
def frames_small():
    out = [synth.frame_small(0), synth.frame_small(3, n=777, width=100, height=37)]
    for s in range(6):
        out.append(synth.frame_random(s, int(np.random.default_rng(s).integers(1, 9000)),
                                      int(np.random.default_rng(s + 50).integers(1, 700)),
                                      int(np.random.default_rng(s + 90).integers(1, 500)),
                                      depth_ties=0.2 * (s % 2)))
    for s in range(30):
        g, W, H = P.tiny_frame(s)
        out.append(synth.Frame(W, H, g, f"tiny{s}"))
    out.append(synth.frame_random(9, 3000, 16, 16))         # one tile, 0 tile bits
    out.append(synth.frame_random(10, 5000, 17, 1))         # 2 x 1 tiles
    out.append(synth.frame_large(1, n=50_000, width=640, height=360))
    return out


# ------------------------------------------------------------------ steps
@pytest.mark.parametrize("fi", range(41))
def test_count_scan_duplicate(ctx, oracle, fi):
    fr = frames_small()[fi]
    g = T.records_to_tensor(fr.gaussians, DEV)
    ref = oracle.sort_frame(fr.gaussians, fr.width, fr.height)
    assert ref["status"] == 0
    counts = ctx.count_tiles(g, fr.width, fr.height)
    ctx.sync()
    assert np.array_equal(u32(counts), ref["counts"])
    offsets, total = ctx.scan(counts)
    ctx.sync()
    assert np.array_equal(u32(offsets), ref["offsets"])
    assert int(u32(total)[0]) == ref["m"]
    keys, values = ctx.duplicate_keys(g, offsets, fr.width, fr.height, ref["m"])
    ctx.sync()
    assert np.array_equal(u64(keys), ref["unsorted_keys"])
    assert np.array_equal(u32(values), ref["unsorted_values"])
    sk, sv = ctx.sort_pairs(keys, values, fr.tile_bits, T.SORT_DEPTH_POSITIVE)
    ctx.sync()
    assert np.array_equal(u64(sk), ref["keys"])
    assert np.array_equal(u32(sv), ref["values"])
    r = ctx.tile_ranges(sk, fr.num_tiles)
    ctx.sync()
    assert np.array_equal(u32(r), ref["ranges"])


@pytest.mark.parametrize("n", [1, 2, 2047, 2048, 2049, 65536 + 7, 3_000_001])
def test_scan_sizes(ctx, oracle, n):
    rng = np.random.default_rng(n)
    c = rng.integers(0, 1500, size=n).astype(np.uint32)
    st, off, total = oracle.scan(c)
    o, t = ctx.scan(torch.from_numpy(c.view(np.int32)).to(DEV))
    ctx.sync()
    assert np.array_equal(u32(o), off) and int(u32(t)[0]) == total


def test_scan_overflow(ctx, oracle):
    c = np.full(5000, 2**20, dtype=np.uint32)  # total 5000 * 2^20 > 2^32
    st, _, total = oracle.scan(c)
    assert st == P_OVERFLOW
    o, t = ctx.scan(torch.from_numpy(c.view(np.int32)).to(DEV))
    with pytest.raises(T.TdgsError) as e:
        ctx.sync()
    assert e.value.status == T.OVERFLOW
    assert int(u32(t)[0]) == 0xFFFFFFFF


P_OVERFLOW = 3


@pytest.mark.parametrize("case", ["nan_depth", "zero_depth", "neg_zero_depth", "inf_x", "neg_depth"])
def test_invalid_gaussian(ctx, oracle, case):
    vals = {"nan_depth": (10.0, 10.0, float("nan")), "zero_depth": (10.0, 10.0, 0.0),
            "neg_zero_depth": (10.0, 10.0, -0.0), "inf_x": (float("inf"), 10.0, 1.0),
            "neg_depth": (10.0, 10.0, -2.0)}[case]
    g = synth.records([5.0, vals[0], 30.0], [5.0, vals[1], 30.0], [1.0, vals[2], 2.0], [2, 3, 4])
    st, _ = oracle.count_tiles(g, 64, 64)
    assert st == 1
    gt = T.records_to_tensor(g, DEV)
    ctx.count_tiles(gt, 64, 64)
    with pytest.raises(T.TdgsError) as e:
        ctx.sync()
    assert e.value.status == T.INVALID_ARGUMENT
    with pytest.raises(T.TdgsError) as e:
        ctx.sort_frame(gt, 64, 64)
    assert e.value.status == T.INVALID_ARGUMENT
    ctx.sync()  # error was cleared


def _random_pairs(m, seed, key_bits, ties):
    rng = np.random.default_rng(seed)
    if ties:
        pool = rng.integers(0, 1 << key_bits, size=max(1, m // 20), dtype=np.uint64)
        k = pool[rng.integers(0, len(pool), size=m)]
    else:
        k = rng.integers(0, 1 << key_bits, size=m, dtype=np.uint64)
    v = rng.permutation(m).astype(np.uint32)
    return k, v


@pytest.mark.parametrize("variant", range(9))
@pytest.mark.parametrize("m,tile_bits,ties", [(1, 0, False), (4095, 8, True), (4096, 8, False),
                                               (8193, 12, True), (100_003, 13, True),
                                               (250_000, 32, False)])
def test_sort_pairs_variants(ctx, oracle, variant, m, tile_bits, ties):
    if variant >= len(T.sort_variants()):
        pytest.skip("variant not compiled")
    k, v = _random_pairs(m, m + variant, 32 + tile_bits if tile_bits < 32 else 63, ties)
    if tile_bits == 32:
        k |= np.uint64(1) << np.uint64(63)
    _, rk, rv = oracle.sort_pairs(k, v)
    ctx.set_sort_variant(variant)
    try:
        kt = torch.from_numpy(k.view(np.int64)).to(DEV)
        vt = torch.from_numpy(v.view(np.int32)).to(DEV)
        sk, sv = ctx.sort_pairs(kt, vt, tile_bits, 0)
        ctx.sync()
    finally:
        ctx.set_sort_variant(-1)
    assert np.array_equal(u64(sk), rk)
    assert np.array_equal(u32(sv), rv)


@pytest.mark.parametrize("m,tile_bits,ties", [(1, 0, False), (2, 4, True), (3, 12, False), (4, 12, True),
                                               (4095, 8, True), (4096, 12, False), (4097, 12, True),
                                               (4099, 13, False), (8195, 13, True), (1_000_003, 12, True),
                                               (3_000_001, 13, False), (1_500_007, 32, False)])
def test_sort_pairs_onesweep(ctx, oracle, m, tile_bits, ties):
    """The default tdgs_sort_pairs (onesweep: one histogram launch, then one
    look-back pass per digit) at ragged sizes: fewer than four pairs (no
    bulk copy), a ragged last tile with 1-3 pairs read by plain loads, and
    more tiles than resident CTAs (several tiles per CTA)."""
    k, v = _random_pairs(m, 7 * m + tile_bits, 32 + tile_bits if tile_bits < 32 else 63, ties)
    if tile_bits == 32:
        k |= np.uint64(1) << np.uint64(63)
    _, rk, rv = oracle.sort_pairs(k, v)
    kt = torch.from_numpy(k.view(np.int64)).to(DEV)
    vt = torch.from_numpy(v.view(np.int32)).to(DEV)
    sk, sv = ctx.sort_pairs(kt, vt, tile_bits, 0)
    ctx.sync()
    assert np.array_equal(u64(sk), rk)
    assert np.array_equal(u32(sv), rv)


@pytest.mark.parametrize("m,tile_bits,positive", [(70_001, 2, False), (65_537, 3, True), (300_007, 12, True),
                                                    (123_457, 4, False)])
def test_sort_pairs_onesweep_spanning_digits(ctx, oracle, m, tile_bits, positive):
    """Digits that straddle the two key words (7 to 9 bits wide, with and
    without bit 31 dropped), on keys whose top depth bits take two values
    as real depths do: the passes whose per-digit tables sit in swizzled
    slots, and the passes before them, which count their digits."""
    rng = np.random.default_rng(m + tile_bits)
    k = rng.integers(0, 1 << (32 + tile_bits), size=m, dtype=np.uint64)
    top = rng.choice(np.array([7, 8], dtype=np.uint64), size=m)  # bits 27..30
    k = (k & ~np.uint64(0xF << 27)) | (top << np.uint64(27))
    if positive:
        k &= ~np.uint64(1 << 31)
    v = rng.permutation(m).astype(np.uint32)
    _, rk, rv = oracle.sort_pairs(k, v)
    sk, sv = ctx.sort_pairs(torch.from_numpy(k.view(np.int64)).to(DEV), torch.from_numpy(v.view(np.int32)).to(DEV),
                            tile_bits, T.SORT_DEPTH_POSITIVE if positive else 0)
    ctx.sync()
    assert np.array_equal(u64(sk), rk)
    assert np.array_equal(u32(sv), rv)


def test_sort_pairs_onesweep_skewed_and_repeated(ctx, oracle):
    """All keys equal (one digit takes every pair of every tile), one hot tile
    with random depths, then sizes that shrink and grow between calls on the
    same context (the histogram and ticket state must reset itself)."""
    cases = []
    m = 300_001
    cases.append((np.full(m, (5 << 32) | 0x3f800000, dtype=np.uint64), 12))
    rng = np.random.default_rng(11)
    hot = (np.uint64(17) << np.uint64(32)) | rng.integers(0x3f000000, 0x42000000, size=m, dtype=np.uint64)
    cases.append((hot, 12))
    for mm in (2_000_003, 9_999, 777_777, 5):
        cases.append((rng.integers(0, 1 << 44, size=mm, dtype=np.uint64), 12))
    for k, tb in cases:
        v = rng.permutation(len(k)).astype(np.uint32)
        _, rk, rv = oracle.sort_pairs(k, v)
        sk, sv = ctx.sort_pairs(torch.from_numpy(k.view(np.int64)).to(DEV),
                                torch.from_numpy(v.view(np.int32)).to(DEV), tb, 0)
        ctx.sync()
        assert np.array_equal(u64(sk), rk)
        assert np.array_equal(u32(sv), rv)


@pytest.mark.parametrize("m", [5, 70_001])
def test_sort_pairs_keys_8_byte_aligned(ctx, oracle, m):
    """Keys that start 8 bytes past a 16-byte boundary (allowed by the ABI)
    cannot arrive by bulk copies: the sort takes the chunked pass kernels
    (and the scalar histogram path of their first pass)."""
    k, v = _random_pairs(m, 99 + m, 44, True)
    _, rk, rv = oracle.sort_pairs(k, v)
    kt = torch.zeros(m + 1, dtype=torch.int64, device=DEV)
    vt = torch.zeros(m + 1, dtype=torch.int32, device=DEV)
    kt[1:] = torch.from_numpy(k.view(np.int64)).to(DEV)
    vt[1:] = torch.from_numpy(v.view(np.int32)).to(DEV)
    assert kt[1:].data_ptr() % 16 == 8
    sk, sv = ctx.sort_pairs(kt[1:], vt[1:], 12, 0)
    ctx.sync()
    assert np.array_equal(u64(sk), rk)
    assert np.array_equal(u32(sv), rv)


def test_sort_pairs_depth_flag_violation(ctx):
    k = np.array([1, 2, 0x80000000], dtype=np.uint64)
    v = np.arange(3, dtype=np.uint32)
    ctx.sort_pairs(torch.from_numpy(k.view(np.int64)).to(DEV),
                   torch.from_numpy(v.view(np.int32)).to(DEV), 4, T.SORT_DEPTH_POSITIVE)
    with pytest.raises(T.TdgsError) as e:
        ctx.sync()
    assert e.value.status == T.INVALID_ARGUMENT


def test_sort_pairs_key_too_wide(ctx):
    k = np.array([1, 1 << 45], dtype=np.uint64)
    v = np.arange(2, dtype=np.uint32)
    ctx.sort_pairs(torch.from_numpy(k.view(np.int64)).to(DEV),
                   torch.from_numpy(v.view(np.int32)).to(DEV), 8, 0)
    with pytest.raises(T.TdgsError):
        ctx.sync()


def test_tile_ranges_bad_tile(ctx):
    k = np.array([0, 1 << 32, 9 << 32], dtype=np.uint64)
    ctx.tile_ranges(torch.from_numpy(k.view(np.int64)).to(DEV), 4)
    with pytest.raises(T.TdgsError):
        ctx.sync()


# ------------------------------------------------------------ fused frame
def _check_frame(ctx, oracle, fr):
    ref = oracle.sort_frame(fr.gaussians, fr.width, fr.height)
    assert ref["status"] == 0
    g = T.records_to_tensor(fr.gaussians, DEV)
    k, v, r, m = ctx.sort_frame(g, fr.width, fr.height)
    ctx.sync()
    assert m == ref["m"]
    assert np.array_equal(u64(k), ref["keys"])
    assert np.array_equal(u32(v), ref["values"])
    assert np.array_equal(u32(r), ref["ranges"])
    return m


@pytest.mark.parametrize("fi", range(41))
def test_sort_frame_small(ctx, oracle, fi):
    _check_frame(ctx, oracle, frames_small()[fi])


def test_sort_frame_edge_cases(ctx, oracle):
    W, H = 300, 200
    cases = {
        "empty": synth.records([], [], [], []),
        "all_culled": synth.records([10.0] * 50, [10.0] * 50, [1.0] * 50, [0] * 50),
        "offscreen": synth.records([-500.0, 5000.0], [10.0, 10.0], [1.0, 1.0], [5, 5]),
        "whole_screen": synth.records([150.0, 150.0], [100.0, 100.0], [3.0, 2.0], [1000, 400]),
        "equal_depths": synth.records(np.linspace(0, 300, 500), np.linspace(0, 200, 500),
                                      [2.5] * 500, [20] * 500),
        "subnormal_depth": synth.records([10.0, 20.0], [10.0, 20.0], [1e-45, 1e-40], [3, 3]),
    }
    for name, g in cases.items():
        _check_frame(ctx, oracle, synth.Frame(W, H, g, name))


def test_sort_frame_huge_image(ctx, oracle):
    """A 4096x3200 image has more tile-grid cells than the shared-memory
    difference grid holds, so the ranges come from the sorted keys."""
    _check_frame(ctx, oracle, synth.frame_random(21, 30_000, 4096, 3200, max_sigma=200.0))


def test_sort_frame_single_gaussian(ctx, oracle):
    _check_frame(ctx, oracle, synth.Frame(100, 100, synth.records([50.0], [50.0], [3.0], [40]), "one"))


def test_sort_frame_wide_elements(ctx, oracle):
    """Tile bits + depth-rank bits above 32 use 64-bit stream elements."""
    fr = synth.frame_random(22, 300_000, 4000, 4000, max_sigma=30.0)  # 250x250 tiles, 16+19 bits
    _check_frame(ctx, oracle, fr)


@pytest.mark.parametrize("n,width,height", [(400_000, 1920, 1080), (1_300_000, 3840, 2160)])
def test_sort_frame_pass_widths(ctx, oracle, n, width, height):
    """Tile ids of 13 and 15 bits split into passes of 7 + 6 and 8 + 7 bits,
    each pass on the kernel compiled for its own digit width (8-bit, then
    6-bit at 1080p).  400k Gaussians at 1080p pack into 32-bit elements;
    1.3M at 4K (above one depth-sort chunk per CTA: the onesweep depth form)
    into 64-bit ones."""
    _check_frame(ctx, oracle, synth.frame_random(31 + width, n, width, height, max_sigma=12.0))


def test_sort_frame_repeated_calls(ctx, oracle):
    """Many sorts on one context (the look-back epoch tag wraps every 7
    passes) stay exact."""
    for s in range(6):
        _check_frame(ctx, oracle, synth.frame_random(100 + s, 20_000, 500, 300, depth_ties=0.3))


def test_sort_frame_changing_counts(ctx, oracle):
    """Consecutive frames of one shape whose pair counts grow, shrink to
    zero and grow again stay exact (buffers sized from each frame's own
    count)."""
    base = synth.frame_random(300, 20_000, 640, 360, max_sigma=8.0)
    m_base = _check_frame(ctx, oracle, base)
    _check_frame(ctx, oracle, synth.frame_random(301, 20_000, 640, 360, max_sigma=8.0))   # fits
    g3 = base.gaussians.copy()
    g3["radius"] *= 3  # same shape, several times the pairs
    m_big = _check_frame(ctx, oracle, synth.Frame(640, 360, g3, "big"))
    assert m_big > 2 * m_base
    culled = base.gaussians.copy()
    culled["radius"] = 0  # same shape, no pairs
    g = T.records_to_tensor(culled, DEV)
    for _ in range(2):
        k, v, r, m = ctx.sort_frame(g, 640, 360)
        ctx.sync()
        assert m == 0 and not u32(r).any()
    _check_frame(ctx, oracle, base)  # from a zero count back to a full frame


@pytest.mark.parametrize("depths,passes", [
    ((2.5, 2.5), 1),            # one depth: one pass
    ((1.0, 1.01), 2),           # a narrow range: 17 bits of keys
    ((0.5, 80.0), 3),           # a scene-like range: < 2^27 keys
    ((1e-30, 1e30), 4),         # the full range of positive floats
])
def test_depth_sort_pass_count(ctx, oracle, depths, passes):
    """The single-launch depth sort compresses keys to their range and runs
    as many 9-bit passes as the range needs; results stay exact, with
    culled Gaussians and equal depths in the mix."""
    rng = np.random.default_rng(passes)
    n = 30_000
    lo, hi = depths
    d = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))
    d[rng.integers(0, n, size=n // 10)] = lo  # ties at the smallest key
    r = rng.integers(1, 12, size=n)
    r[rng.integers(0, n, size=n // 20)] = 0  # culled
    g = synth.records(rng.uniform(0, 640, n), rng.uniform(0, 360, n), d, r)
    _check_frame(ctx, oracle, synth.Frame(640, 360, g, f"depths-{lo}-{hi}"))
    assert ctx.depth_passes() == passes


def _depth_range_frame(seed, lo, hi, n=20_000):
    rng = np.random.default_rng(seed)
    d = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))
    d[rng.integers(0, n, size=n // 10)] = hi  # ties at the largest key
    r = rng.integers(1, 10, size=n)
    r[rng.integers(0, n, size=n // 20)] = 0  # culled
    g = synth.records(rng.uniform(0, 640, n), rng.uniform(0, 360, n), d, r)
    return synth.Frame(640, 360, g, f"depths-{seed}")


def test_depth_sort_alternating_pass_counts(ctx, oracle):
    """Consecutive frames on one context whose depth ranges need 4, 1, 3,
    2, 4, 2, 3 and 1 passes: the single-launch sort's counters, totals and
    count rows are reset for every pass count (each frame exact)."""
    ranges = [(1e-30, 1e30), (3.0, 3.0), (0.5, 80.0), (1.0, 1.01), (1e-20, 1e20), (2.0, 2.02),
              (0.2, 50.0), (7.0, 7.0)]
    want = [4, 1, 3, 2, 4, 2, 3, 1]
    for i, ((lo, hi), passes) in enumerate(zip(ranges, want)):
        _check_frame(ctx, oracle, _depth_range_frame(40 + i, lo, hi))
        assert ctx.depth_passes() == passes


def test_depth_sort_at_capacity(ctx, oracle):
    """N = SMs x 8192 Gaussians, the most the single-launch depth sort takes
    (every CTA a full chunk), and one more (the onesweep passes)."""
    cap = torch.cuda.get_device_properties(0).multi_processor_count * 8192
    for n in (cap, cap + 1):
        fr = synth.frame_random(77, n, 1280, 720, max_sigma=6.0)
        _check_frame(ctx, oracle, fr)
        assert ctx.depth_passes() >= 1


@pytest.mark.parametrize("mult", [2, 3, 4])
def test_depth_sort_onesweep_sizes(ctx, oracle, mult):
    """Above SMs x 8192 Gaussians the depth sort takes the onesweep passes
    over the compressed 32-bit keys: 2 to 4 times that N (up to 2^22), each
    with a ragged last 4096-key tile."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    n = min(mult * sms * 8192 - 5 * mult, 1 << 22)
    fr = synth.frame_random(90 + mult, n, 1920, 1080, max_sigma=4.0)
    _check_frame(ctx, oracle, fr)
    assert 1 <= ctx.depth_passes() <= 4


def test_depth_sort_onesweep_alternating_pass_counts(ctx, oracle):
    """The onesweep depth form under 4, 1, 3 and 2 passes in a row: the
    passes the key range does not need end at once, the result always lands
    in the same buffers, and the scratch state left by each run serves the
    next."""
    n = torch.cuda.get_device_properties(0).multi_processor_count * 8192 + 4099
    for i, ((lo, hi), passes) in enumerate([((1e-30, 1e30), 4), ((3.0, 3.0), 1), ((0.5, 80.0), 3),
                                             ((1.0, 1.01), 2)]):
        _check_frame(ctx, oracle, _depth_range_frame(60 + i, lo, hi, n=n))
        assert ctx.depth_passes() == passes


def test_depth_sort_onesweep_all_culled_then_visible(ctx, oracle):
    """The onesweep depth form when no Gaussian has pairs (an empty key
    range: one pass over a zero-width digit, M = 0, every range {0, 0}),
    then an ordinary frame of the same size on the same context."""
    n = torch.cuda.get_device_properties(0).multi_processor_count * 8192 + 777
    rng = np.random.default_rng(5)
    culled = synth.records(rng.uniform(0, 640, n), rng.uniform(0, 360, n), rng.uniform(1.0, 9.0, n),
                           np.zeros(n, dtype=np.int64))
    assert _check_frame(ctx, oracle, synth.Frame(640, 360, culled, "all-culled-onesweep")) == 0
    assert ctx.depth_passes() == 1
    _check_frame(ctx, oracle, _depth_range_frame(71, 0.5, 80.0, n=n))
    assert ctx.depth_passes() == 3


def test_sort_frame_scene_1m(ctx, oracle):
    m = _check_frame(ctx, oracle, synth.frame_scene(0))
    assert m > 5_000_000


def test_sort_frame_large_3m(ctx, oracle):
    m = _check_frame(ctx, oracle, synth.frame_large(0))
    assert m > 20_000_000


def test_sort_pairs_over_2p26(ctx):
    """More than 2^26 pairs (digit counts beyond 26 bits): checked by properties
    that determine the stable sort uniquely -- values are the input
    positions, so they must form a permutation, sorted_keys must equal
    keys[values], keys must be non-decreasing and ties must keep input
    order."""
    m = (1 << 26) + 12_345
    rng = np.random.default_rng(5)
    k = rng.integers(0, 1 << 20, size=m, dtype=np.uint64) << np.uint64(12)  # many ties
    kt = torch.from_numpy(k.view(np.int64)).to(DEV)
    vt = torch.arange(m, dtype=torch.int32, device=DEV)
    sk, sv = ctx.sort_pairs(kt, vt, 0, 0)
    ctx.sync()
    del kt
    skn, svn = u64(sk), u32(sv).astype(np.int64)
    assert np.all(skn[1:] >= skn[:-1])
    assert np.array_equal(skn, k[svn])
    assert np.array_equal(np.bincount(svn, minlength=m), np.ones(m, dtype=np.int64))
    tie = skn[1:] == skn[:-1]
    assert np.all(svn[1:][tie] > svn[:-1][tie])
