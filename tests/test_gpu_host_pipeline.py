"""HostPipeline (frames from pinned host memory to sorted results in pinned
host memory, two frames in flight) returns exactly what the oracle returns
for each frame, in submission order, across frames of different sizes."""
import numpy as np
import pytest
import torch

from paper_2511_16298_gb300 import synth
from paper_2511_16298_gb300.host_pipeline import HostPipeline

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_pipeline_matches_oracle(oracle, depth):
    from paper_2511_16298_gb300 import build
    build.build()
    frames = [synth.frame_random(s, 2000 + 3000 * s, 320 + 64 * s, 200 + 16 * s) for s in range(5)]
    frames.append(synth.frame_small(0))
    with HostPipeline(0, depth=depth) as pipe:
        hs = [torch.from_numpy(np.ascontiguousarray(f.gaussians).view(np.int32).reshape(-1, 4)).pin_memory()
              for f in frames]
        # streaming use: the oldest result is read (and detached) before a
        # new frame reuses its slot
        tickets, got = [], []
        for h, f in zip(hs, frames):
            if len(tickets) == depth:
                got.append(pipe.result(tickets.pop(0)).copy())
            tickets.append(pipe.submit(h, f.width, f.height))
        while tickets:
            got.append(pipe.result(tickets.pop(0)).copy())
    for f, r in zip(frames, got):
        ref = oracle.sort_frame(f.gaussians, f.width, f.height)
        assert r.m == ref["m"]
        assert np.array_equal(r.keys.numpy().view(np.uint64), ref["keys"])
        assert np.array_equal(r.values.numpy().view(np.uint32), ref["values"])
        assert np.array_equal(r.ranges.numpy().view(np.uint32), ref["ranges"])
