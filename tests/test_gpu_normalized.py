"""The paper's 32-bit normalised key (tdgs_sort_frame_normalized) against
its own CPU oracle: bit-exact keys, values and ranges (the normalisation is
float32 in a pinned order on both sides, everything else integer)."""
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


def frames():
    out = [synth.frame_small(0), synth.frame_large(1, n=60_000, width=640, height=360)]
    for s in range(4):
        out.append(synth.frame_random(20 + s, 500 + 2500 * s, 100 + 90 * s, 60 + 70 * s, depth_ties=0.3))
    for s in range(6):
        g, W, H = P.tiny_frame(s)
        out.append(synth.Frame(W, H, g, f"tiny{s}"))
    return out


@pytest.mark.parametrize("fi", range(12))
def test_normalized_matches_oracle(ctx, oracle, fi):
    fr = frames()[fi]
    st, ek, ev, er = oracle.sort_frame_normalized(fr.gaussians, fr.width, fr.height)
    g = T.records_to_tensor(fr.gaussians, DEV)
    if st != 0:  # invalid Gaussians: the library reports the same
        with pytest.raises(T.TdgsError):
            ctx.sort_frame_normalized(g, fr.width, fr.height)
        ctx.sync()
        return
    k, v, r, m = ctx.sort_frame_normalized(g, fr.width, fr.height, copy=True)
    assert m == len(ek)
    assert np.array_equal(k.cpu().numpy().view(np.uint32), ek)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ev)
    assert np.array_equal(r.cpu().numpy().view(np.uint32), er)


def test_normalized_scene_full_size(ctx, oracle):
    fr = synth.frame_scene(0)
    k, v, r, m = ctx.sort_frame_normalized(T.records_to_tensor(fr.gaussians, DEV), fr.width, fr.height, copy=True)
    st, ek, ev, er = oracle.sort_frame_normalized(fr.gaussians, fr.width, fr.height)
    assert st == 0 and m == len(ek)
    assert np.array_equal(k.cpu().numpy().view(np.uint32), ek)
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ev)
    assert np.array_equal(r.cpu().numpy().view(np.uint32), er)


def test_normalized_empty_and_limits(ctx):
    e = torch.empty((0, 4), dtype=torch.int32, device=DEV)
    k, v, r, m = ctx.sort_frame_normalized(e, 64, 48)
    assert m == 0 and r.shape == (12, 2) and not r.any()
    with pytest.raises(T.TdgsError) as ex:
        ctx.sort_frame_normalized(e, 16400, 16400)  # more than 2^20 tiles
    assert ex.value.status == T.INVALID_ARGUMENT
