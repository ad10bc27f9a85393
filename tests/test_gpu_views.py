"""Batched multi-view sort: every view's result equals the CPU oracle on
that view alone (bit-exact), through the exact call, the asynchronous call
and a replayed CUDA graph."""
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


def check_view(oracle, fr, res):
    k, v, r, m = res
    ref = oracle.sort_frame(fr.gaussians, fr.width, fr.height)
    assert ref["status"] == 0
    assert m == ref["m"]
    assert np.array_equal(k.cpu().numpy().view(np.uint64), ref["keys"])
    assert np.array_equal(v.cpu().numpy().view(np.uint32), ref["values"])
    assert np.array_equal(r.cpu().numpy().view(np.uint32), ref["ranges"])


def small_multiview():
    mv = synth.multiview(seed=3, n=40_000, views=6, width=640, height=360, scale0=0.03)
    # mixed shapes: add frames of other sizes and an empty one
    extra = [synth.frame_small(1, n=5000, width=200, height=90),
             synth.Frame(64, 64, synth.records([], [], [], []), "empty"),
             synth.frame_random(4, 3000, 16, 16)]
    return mv.views + extra


def test_views_exact(ctx, oracle):
    frames = small_multiview()
    gs = [T.records_to_tensor(f.gaussians, DEV) for f in frames]
    out = ctx.sort_views([(g, f.width, f.height) for g, f in zip(gs, frames)])
    for f, res in zip(frames, out):
        check_view(oracle, f, res)


def test_views_async_and_graph(ctx, oracle):
    frames = small_multiview()
    gs = [T.records_to_tensor(f.gaussians, DEV) for f in frames]
    views = [(g, f.width, f.height) for g, f in zip(gs, frames)]
    frames2 = [synth.frame_random(50 + i, f.n, f.width, f.height) for i, f in enumerate(frames)]
    gs2 = [T.records_to_tensor(f.gaussians, DEV) for f in frames2]
    m2 = sum(r[3] for r in ctx.sort_views([(g, f.width, f.height) for g, f in zip(gs2, frames2)]))
    exact = ctx.sort_views(views, copy=True)
    # the graph is replayed on both data sets: reserve for the larger one
    cap = max(sum(r[3] for r in exact), m2) + 1000
    ctx.reserve_views(views, cap)
    ctx.sort_views_async(views)
    for e, res in zip(exact, ctx.views_results(len(views))):
        for a, b in zip(e[:3], res[:3]):
            assert torch.equal(a, b)
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            ctx.sort_views_async(views)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        graph.replay()
        for e, res in zip(exact, ctx.views_results(len(views))):
            for a, b in zip(e[:3], res[:3]):
                assert torch.equal(a, b)
    # new data of the same shape replays through the same graph
    for g, g2 in zip(gs, gs2):
        g.copy_(g2)
    graph.replay()
    for f, res in zip(frames2, ctx.views_results(len(views))):
        check_view(oracle, f, res)


def test_views_graph_onesweep_depth(ctx, oracle):
    """A batch above one depth-sort chunk per CTA (3 x 500k Gaussians: the
    onesweep depth form, whose pass plan is read on the device) captured
    in a CUDA graph: replays equal the exact call, and new depths through
    the same graph match the oracle."""
    mv = synth.multiview(seed=5, n=500_000, views=3, width=1280, height=720, scale0=0.05)
    frames = mv.views
    gs = [T.records_to_tensor(f.gaussians, DEV) for f in frames]
    views = [(g, f.width, f.height) for g, f in zip(gs, frames)]
    rng = np.random.default_rng(8)
    frames2 = []
    for f in frames:  # same positions and radii, other depths (another depth range)
        g2 = f.gaussians.copy()
        g2["depth"] = (g2["depth"] * rng.uniform(0.5, 4.0, size=f.n)).astype(np.float32)
        frames2.append(synth.Frame(f.width, f.height, g2, f.name + "-redepth"))
    exact = ctx.sort_views(views, copy=True)
    cap = sum(r[3] for r in exact) + 1000  # same rectangles: the same pair count
    ctx.reserve_views(views, cap)
    ctx.sort_views_async(views)  # the first call on this shape, outside the capture
    for e, res in zip(exact, ctx.views_results(len(views))):
        for a, b in zip(e[:3], res[:3]):
            assert torch.equal(a, b)
    graph = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        with torch.cuda.graph(graph, stream=side):
            ctx.sort_views_async(views)
    torch.cuda.current_stream().wait_stream(side)
    for _ in range(2):
        graph.replay()
        for e, res in zip(exact, ctx.views_results(len(views))):
            for a, b in zip(e[:3], res[:3]):
                assert torch.equal(a, b)
    for g, f2 in zip(gs, frames2):
        g.copy_(T.records_to_tensor(f2.gaussians, DEV))
    graph.replay()
    res = ctx.views_results(len(views))
    check_view(oracle, frames2[1], res[1])


def test_views_capacity_exceeded(ctx):
    frames = [synth.frame_small(0)]
    g = T.records_to_tensor(frames[0].gaussians, DEV)
    views = [(g, 256, 256)]
    ctx.reserve_views(views, 1000)  # far fewer than the 57k pairs
    ctx.sort_views_async(views)
    with pytest.raises(T.TdgsError) as e:
        ctx.views_results(1)
    assert e.value.status == T.CAPACITY


def test_views_full_config_sampled(ctx, oracle):
    """The 64-camera, 500k-Gaussian batch at full size; five views checked
    against the oracle one by one."""
    mv = synth.multiview(seed=0)
    gs = [T.records_to_tensor(f.gaussians, DEV) for f in mv.views]
    out = ctx.sort_views([(g, f.width, f.height) for g, f in zip(gs, mv.views)])
    ms = [r[3] for r in out]
    assert min(ms) > 0
    for i in (0, 17, 31, 50, 63):
        check_view(oracle, mv.views[i], out[i])


def test_views_maximum_count(ctx, oracle):
    """256 views (the maximum) of ragged sizes, some empty, in one batch;
    257 views are rejected."""
    rng = np.random.default_rng(17)
    frames = []
    for i in range(256):
        n = 0 if i % 37 == 0 else int(rng.integers(1, 400))
        w, h = int(rng.integers(1, 300)), int(rng.integers(1, 200))
        frames.append(synth.frame_random(100 + i, n, w, h) if n else synth.Frame(w, h, synth.records([], [], [], []), "e"))
    gs = [T.records_to_tensor(f.gaussians, DEV) for f in frames]
    res = ctx.sort_views([(g, f.width, f.height) for g, f in zip(gs, frames)], copy=True)
    for f, r in zip(frames, res):
        check_view(oracle, f, r)
    with pytest.raises(T.TdgsError) as e:
        ctx.sort_views([(gs[1], frames[1].width, frames[1].height)] * 257)
    assert e.value.status == T.INVALID_ARGUMENT
