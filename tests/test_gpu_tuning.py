"""Every tuning setting gives bit-identical results; the autotuner picks a
setting and its table round-trips."""
import numpy as np
import pytest
import torch

from paper_2511_16298_gb300 import autotune, synth
from paper_2511_16298_gb300 import tdgs as T

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx():
    from paper_2511_16298_gb300 import build
    build.build()
    c = T.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("knobs", [
    {"tile_digit_bits": 6},
    {"tile_digit_bits": 4, "ctas_per_sm": 1},
    {"tile_digit_bits": 5, "ctas_per_sm": 3},
    {"tile_digit_bits": 8, "ctas_per_sm": 1, "depth_digit_bits": 8},
    {"tile_digit_bits": 11, "ctas_per_sm": 2, "depth_digit_bits": 11},
])
def test_frame_knobs_exact(ctx, oracle, knobs):
    frames = [synth.frame_small(0), synth.frame_large(2, n=60_000, width=1920, height=1080),
              synth.frame_random(7, 20_000, 4000, 4000, max_sigma=30.0)]  # last one uses wide elements
    ctx.apply_tuning(knobs)
    try:
        for fr in frames:
            ref = oracle.sort_frame(fr.gaussians, fr.width, fr.height)
            k, v, r, m = ctx.sort_frame(T.records_to_tensor(fr.gaussians, DEV), fr.width, fr.height)
            ctx.sync()
            assert m == ref["m"]
            assert np.array_equal(k.cpu().numpy().view(np.uint64), ref["keys"])
            assert np.array_equal(v.cpu().numpy().view(np.uint32), ref["values"])
            assert np.array_equal(r.cpu().numpy().view(np.uint32), ref["ranges"])
        mv = synth.multiview(seed=5, n=30_000, views=4, width=640, height=360)
        out = ctx.sort_views([(T.records_to_tensor(f.gaussians, DEV), f.width, f.height) for f in mv.views])
        for f, (k, v, r, m) in zip(mv.views, out):
            ref = oracle.sort_frame(f.gaussians, f.width, f.height)
            assert np.array_equal(k.cpu().numpy().view(np.uint64), ref["keys"])
    finally:
        ctx.apply_tuning({"tile_digit_bits": 0, "ctas_per_sm": 0, "depth_digit_bits": 0})


def test_tuning_rejects_bad_values(ctx):
    with pytest.raises(T.TdgsError):
        ctx.set_tuning(T.TUNE_TILE_DIGIT_BITS, 13)
    with pytest.raises(T.TdgsError):
        ctx.set_tuning(2, 1)  # no such knob
    with pytest.raises(T.TdgsError):
        ctx.set_tuning(99, 1)
    assert ctx.get_tuning(T.TUNE_TILE_DIGIT_BITS) == 0


def test_autotuner_table(ctx, tmp_path):
    fr = synth.frame_small(1)
    g = T.records_to_tensor(fr.gaussians, DEV)
    res = autotune.tune_views(ctx, [(g, fr.width, fr.height)], reps=1)
    # 3 tile digit widths x 4 CTA counts; the depth digit width stays the
    # built-in choice below the per-pass depth sort's 2^30 Gaussians
    assert res["ms"] > 0 and len(res["trials"]) == 12
    assert all(k["depth_digit_bits"] == 0 for k, _ in res["trials"])
    counts = ctx.count_tiles(g, fr.width, fr.height)
    offs, tot = ctx.scan(counts)
    k, v = ctx.duplicate_keys(g, offs, fr.width, fr.height, int(tot.item()))
    res2 = autotune.tune_sort_pairs(ctx, k, v, fr.tile_bits, reps=1)
    table = autotune.Table(str(tmp_path / "tune.json"))
    table.record(res)
    table.record(res2)
    table.save()
    t2 = autotune.Table(str(tmp_path / "tune.json"))
    assert t2.knobs_for_views([(g, fr.width, fr.height)]) == res["best"]
    assert t2.knobs_for_pairs(k.shape[0], fr.tile_bits, T.SORT_DEPTH_POSITIVE) == res2["best"]
