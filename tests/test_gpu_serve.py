"""Served results are byte-identical to each frame sorted alone, with and
without continuous batching, and match the CPU oracle."""
import numpy as np
import pytest
import torch

from paper_2511_16298_gb300 import serve, synth
from paper_2511_16298_gb300 import tdgs as T

pytestmark = pytest.mark.gpu


def make_requests(count=14, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        w, h = synth.RESOLUTIONS[int(rng.integers(0, 3))]
        n = int(np.exp(rng.uniform(np.log(2_000), np.log(120_000))))
        out.append(synth.frame_scene(1000 + i, n, w, h))
    return out


@pytest.mark.parametrize("batching", [True, False])
def test_served_equals_alone(oracle, batching):
    from paper_2511_16298_gb300 import build
    build.build()
    frames = make_requests()
    ex = serve.GpuExecutor(0, slots=2, keep_results=True)
    host = [torch.from_numpy(np.ascontiguousarray(f.gaussians).view(np.int32).reshape(-1, 4)).pin_memory()
            for f in frames]
    with serve.Server(ex, slots=2, hbm_budget=40 << 30, max_batch=8, batching=batching) as s:
        futs = [s.submit(i, h, f.n, f.width, f.height) for i, (h, f) in enumerate(zip(host, frames))]
        res = [f.result(timeout=120) for f in futs]
    if batching:
        assert max(s.batches) >= 1
    with T.Context(0) as ctx:
        for f, r in zip(frames, res):
            k, v, rg, m = ctx.sort_frame(T.records_to_tensor(f.gaussians, "cuda:0"), f.width, f.height,
                                         copy=True)
            ctx.sync()
            assert r.m == m
            assert torch.equal(r.keys, k) and torch.equal(r.values, v) and torch.equal(r.ranges, rg)
    for i in (0, 5):
        ref = oracle.sort_frame(frames[i].gaussians, frames[i].width, frames[i].height)
        assert np.array_equal(res[i].keys.cpu().numpy().view(np.uint64), ref["keys"])
        assert np.array_equal(res[i].values.cpu().numpy().view(np.uint32), ref["values"])
    ex.close()


def test_invalid_request_fails_alone():
    from paper_2511_16298_gb300 import build
    build.build()
    frames = make_requests(6, seed=2)
    bad = synth.frame_small(9, n=1000)
    bad.gaussians["depth"][10] = np.float32(np.nan)
    frames.insert(3, bad)
    ex = serve.GpuExecutor(0, slots=1, keep_results=False)
    host = [torch.from_numpy(np.ascontiguousarray(f.gaussians).view(np.int32).reshape(-1, 4)).pin_memory()
            for f in frames]
    with serve.Server(ex, slots=1, max_batch=16) as s:
        futs = [s.submit(i, h, f.n, f.width, f.height) for i, (h, f) in enumerate(zip(host, frames))]
        outs = []
        for f in futs:
            try:
                outs.append(f.result(timeout=120).m)
            except T.TdgsError as e:
                outs.append(e.status)
    assert outs[3] == T.INVALID_ARGUMENT
    assert all(isinstance(o, int) and o > 0 for i, o in enumerate(outs) if i != 3)
    ex.close()
