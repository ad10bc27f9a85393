"""Autotuner for the radix passes.

Times candidate settings of a context's tuning knobs on a representative
workload with CUDA events and keeps the fastest:

* tdgs_sort_pairs: the pass kernel variant (digit width 8..11, threads,
  keys per thread, blocks per SM) and CTAs per SM of the persistent grid;
* the fused frame / multi-view batch: widest tile digit (6, 8 or 12
  bits), CTAs per SM and the depth sort's digit width (8 or 11).

Results are stored as JSON keyed by workload shape (pair-count bucket and
key bits, or Gaussians/tiles buckets), so a server can apply the table
entry that matches each request.  Every setting yields identical results;
only speed differs.
"""
from __future__ import annotations

import json
import math
import os
import statistics
from typing import Callable

import torch

from . import tdgs

L2_FLUSH = 256 << 20
# Gaussians from which a frame's depth sort runs one launch per pass over
# all key bits (the only form the depth digit width knob reaches)
DEPTH_PER_PASS_MIN = 1 << 30


def _bucket(x: int) -> int:
    return 0 if x <= 1 else int(math.ceil(math.log2(x)))


def _time(fn: Callable[[], None], reps: int, flush: torch.Tensor, setup=None) -> float:
    stream = torch.cuda.current_stream()
    ts = []
    for i in range(reps + 1):
        if setup:
            setup()
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        if i:
            ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def tune_sort_pairs(ctx: tdgs.Context, keys: torch.Tensor, values: torch.Tensor, tile_bits: int,
                    flags: int = tdgs.SORT_DEPTH_POSITIVE, reps: int = 3) -> dict:
    """Best (sort_variant, ctas_per_sm) for sorting these pairs."""
    kw, vw = torch.empty_like(keys), torch.empty_like(values)
    ka, va = torch.empty_like(keys), torch.empty_like(values)
    flush = torch.empty(L2_FLUSH, dtype=torch.uint8, device=keys.device)

    def setup():
        kw.copy_(keys)
        vw.copy_(values)

    trials = []
    for v in range(len(tdgs.sort_variants())):
        for cps in (0, 1, 2):
            ctx.apply_tuning({"sort_variant": v, "ctas_per_sm": cps})
            ms = _time(lambda: ctx.sort_pairs(kw, vw, tile_bits, flags, ka, va), reps, flush, setup)
            trials.append(({"sort_variant": v, "ctas_per_sm": cps}, ms))
    ctx.apply_tuning({"sort_variant": -1, "ctas_per_sm": 0})
    ctx.sync()
    best, ms = min(trials, key=lambda x: x[1])
    return {"best": best, "ms": ms, "trials": [(t, round(m, 4)) for t, m in trials],
            "key": f"pairs:m{_bucket(keys.shape[0])}:tb{tile_bits}:f{flags}"}


def tune_views(ctx: tdgs.Context, views: list, reps: int = 3) -> dict:
    """Best (tile_digit_bits, ctas_per_sm, depth_digit_bits) for a batch of
    views [(records, width, height)] (one view = one frame)."""
    flush = torch.empty(L2_FLUSH, dtype=torch.uint8, device=views[0][0].device)
    n = sum(int(v[0].shape[0]) for v in views)
    # the depth digit width only reaches the per-pass depth sort (2^30
    # Gaussians or more); below that the built-in choice stands
    dbit_choices = (11, 8) if n >= DEPTH_PER_PASS_MIN else (0,)
    trials = []
    for bits in (12, 8, 6):
        for cps in (0, 1, 2, 3):
            for dbits in dbit_choices:
                knobs = {"tile_digit_bits": bits, "ctas_per_sm": cps, "depth_digit_bits": dbits}
                ctx.apply_tuning(knobs)
                ms = _time(lambda: ctx.sort_views(views), reps, flush)
                trials.append((knobs, ms))
    ctx.apply_tuning({"tile_digit_bits": 0, "ctas_per_sm": 0, "depth_digit_bits": 0})
    ctx.sync()
    best, ms = min(trials, key=lambda x: x[1])
    t = sum(tdgs.num_tiles(v[1], v[2]) for v in views)
    return {"best": best, "ms": ms, "trials": [(tt, round(m, 4)) for tt, m in trials],
            "key": f"views:n{_bucket(n)}:t{_bucket(t)}:v{len(views)}"}


class Table:
    """JSON table of tuned knobs, keyed by workload shape."""

    def __init__(self, path: str):
        self.path = path
        self.entries = json.load(open(path)) if os.path.exists(path) else {}

    def record(self, result: dict):
        self.entries[result["key"]] = {"knobs": result["best"], "ms": result["ms"]}

    def save(self):
        os.makedirs(os.path.dirname(os.path.abspath(self.path)), exist_ok=True)
        json.dump(self.entries, open(self.path, "w"), indent=1, sort_keys=True)

    def knobs_for_views(self, views) -> dict | None:
        n = sum(int(v[0].shape[0]) for v in views)
        t = sum(tdgs.num_tiles(v[1], v[2]) for v in views)
        e = self.entries.get(f"views:n{_bucket(n)}:t{_bucket(t)}:v{len(views)}")
        return e["knobs"] if e else None

    def knobs_for_pairs(self, m: int, tile_bits: int, flags: int) -> dict | None:
        e = self.entries.get(f"pairs:m{_bucket(m)}:tb{tile_bits}:f{flags}")
        return e["knobs"] if e else None
