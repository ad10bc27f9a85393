"""The paper's bitonic sorting network (tdgs_sort_pairs_bitonic) against the
CPU oracle.  Pairs from the duplication step (equal keys in ascending value
order) must come out exactly as the stable sort orders them; pairs with
arbitrary values must come out in (key, value) order."""
import numpy as np
import pytest
import torch

from paper_2511_16298_gb300 import synth
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


def to_dev(keys, values):
    return (torch.from_numpy(keys.view(np.int64).copy()).to(DEV),
            torch.from_numpy(values.view(np.int32).copy()).to(DEV))


def check(ctx, oracle, keys, values, inplace=False):
    k, v = to_dev(keys, values)
    if inplace:
        ko, vo = ctx.sort_pairs_bitonic(k, v, k, v)
    else:
        ko, vo = ctx.sort_pairs_bitonic(k, v)
    order = np.argsort(values, kind="stable")  # equal keys enter the stable sort in value order
    st, ek, ev = oracle.sort_pairs(keys[order], values[order])
    assert st == 0
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), ek)
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), ev)


@pytest.mark.parametrize("m", [1, 2, 3, 4095, 4096, 4097, 8192, 12289, 100_000, (1 << 20) + 3])
def test_random_pairs_with_ties(ctx, oracle, m):
    rng = np.random.default_rng(m)
    keys = (rng.integers(0, 64, m, dtype=np.uint64) << np.uint64(32)) | rng.integers(0, 50, m, dtype=np.uint64)
    values = rng.permutation(m).astype(np.uint32)
    check(ctx, oracle, keys, values)


def test_full_width_keys_and_inplace(ctx, oracle):
    rng = np.random.default_rng(7)
    m = 300_001
    keys = rng.integers(0, np.iinfo(np.uint64).max, m, dtype=np.uint64, endpoint=True)
    keys[::7] = np.uint64(0xFFFFFFFFFFFFFFFF)  # the padding value itself
    values = rng.integers(0, 1 << 32, m, dtype=np.uint64).astype(np.uint32)
    values[::7] = np.uint32(0xFFFFFFFF)
    check(ctx, oracle, keys, values, inplace=True)


def test_frame_pairs_equal_stable_sort(ctx, oracle):
    """Duplication output of a frame: identical to the stable radix sort and
    to the oracle's stable sort, with no reordering of the input needed."""
    fr = synth.frame_large(2, n=40_000, width=640, height=360)
    st, counts = oracle.count_tiles(fr.gaussians, fr.width, fr.height)
    st, offs, m = oracle.scan(counts)
    st, keys, values = oracle.duplicate(fr.gaussians, offs, m, fr.width, fr.height)
    k, v = to_dev(keys, values)
    ko, vo = ctx.sort_pairs_bitonic(k, v)
    st, ek, ev = oracle.sort_pairs(keys, values)
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), ek)
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), ev)


def test_scene_frame_full_size(ctx, oracle):
    """The 1M-Gaussian scene's pairs (11.8M, padded to 2^24): identical to
    the oracle."""
    fr = synth.frame_scene(0)
    g = T.records_to_tensor(fr.gaussians, DEV)
    counts = ctx.count_tiles(g, fr.width, fr.height)
    offs, tot = ctx.scan(counts)
    m = int(tot.item())
    k0, v0 = ctx.duplicate_keys(g, offs, fr.width, fr.height, m)
    ko, vo = ctx.sort_pairs_bitonic(k0, v0)
    st, ek, ev = oracle.sort_pairs(k0.cpu().numpy().view(np.uint64), v0.cpu().numpy().view(np.uint32))
    assert np.array_equal(ko.cpu().numpy().view(np.uint64), ek)
    assert np.array_equal(vo.cpu().numpy().view(np.uint32), ev)


def test_empty(ctx):
    e64 = torch.empty(0, dtype=torch.int64, device=DEV)
    e32 = torch.empty(0, dtype=torch.int32, device=DEV)
    ko, vo = ctx.sort_pairs_bitonic(e64, e32)
    assert ko.numel() == 0 and vo.numel() == 0
