"""Continuous-batching request server for the tile depth sort.

Frames (views) arrive as requests.  Each request is admitted against an
HBM budget (its estimated device footprint); admitted requests wait in a
queue; every slot (one worker thread, one library context, one CUDA stream
and device-resident buffers reused from batch to batch) takes all queued
requests up to a batch limit the moment it is free and sorts them as one
multi-view batch.  While one slot's batch runs, newly arrived requests are
admitted and picked up by the next free slot, so host work, host-to-device
copies and kernels of different batches overlap.  Latency is completion
minus arrival.

Batching changes nothing in the results: a view sorted in a batch is
byte-identical to the same view sorted alone (the library's multi-view
call keeps local tile ids and per-view lists).  If a batch fails (for
example one request carries an invalid Gaussian), its requests are retried
one by one so that only the offending request fails.

The execution of a batch is a callable, so the scheduling logic can run
without a GPU (tests use a fake executor).
"""
from __future__ import annotations

import collections
import concurrent.futures as cf
import dataclasses
import threading
import time
from typing import Callable, Optional, Sequence

import numpy as np


@dataclasses.dataclass
class Request:
    rid: int
    records: object          # host tensor / array of (n, 4) int32 Gaussian records
    n: int
    width: int
    height: int
    est_bytes: int
    arrival: float
    future: cf.Future
    started: float = 0.0


@dataclasses.dataclass
class Result:
    rid: int
    m: int                   # Gaussian-tile pairs
    latency_s: float
    batch_size: int
    keys: object = None      # filled when the server keeps results
    values: object = None
    ranges: object = None
    checksum: int = 0


def estimate_bytes(n: int, width: int, height: int, pairs_per_gaussian: float = 24.0) -> int:
    """Conservative device footprint of one request: its records (16 B),
    the per-Gaussian sort buffers (24 B), and per pair the two packed
    stream buffers, the final keys and values (<= 28 B)."""
    tiles = ((width + 15) // 16) * ((height + 15) // 16)
    m = int(n * pairs_per_gaussian)
    return 16 * n + 24 * n + 28 * m + 24 * tiles


Executor = Callable[[int, Sequence[Request]], Sequence[Result]]
Policy = Callable[[Sequence[Request], Request], bool]


def _bits(x: int) -> int:
    return 0 if x <= 1 else int(x - 1).bit_length()


def narrow_batches(batch: Sequence[Request], nxt: Request) -> bool:
    """A request joins a batch only while the batch stays cheap to sort
    together: the packed (tile, depth rank) element fits 32 bits and the
    tile ids need at most 16 bits (two 8-bit tile passes).  Larger
    combinations cost more per pair than the launch overhead they save,
    so such requests run in a batch of their own."""
    n = sum(r.n for r in batch) + nxt.n
    t = sum(((r.width + 15) // 16) * ((r.height + 15) // 16) for r in batch)
    t += ((nxt.width + 15) // 16) * ((nxt.height + 15) // 16)
    return _bits(n) + _bits(t) <= 32 and _bits(t) <= 16


class Server:
    """Admission by HBM budget + continuous batching over `slots` workers.

    executor(slot, batch) sorts one batch and returns one Result per
    request (in order); it raises on failure."""

    def __init__(self, executor: Executor, slots: int = 2, hbm_budget: int = 40 << 30,
                 max_batch: int = 32, batching: bool = True, policy: Optional[Policy] = None):
        self.executor = executor
        self.policy = policy
        self.hbm_budget = int(hbm_budget)
        self.max_batch = max_batch if batching else 1
        self.cv = threading.Condition()
        self.waiting: collections.deque[Request] = collections.deque()   # not yet admitted
        self.queued: collections.deque[Request] = collections.deque()    # admitted, not started
        self.in_flight_bytes = 0
        self.max_in_flight_bytes = 0
        self.closed = False
        self.batches: list[int] = []
        self.workers = [threading.Thread(target=self._work, args=(s,), daemon=True)
                        for s in range(slots)]
        for w in self.workers:
            w.start()

    # ---------------------------------------------------------------- API
    def submit(self, rid: int, records, n: int, width: int, height: int,
               est_bytes: Optional[int] = None) -> cf.Future:
        fut: cf.Future = cf.Future()
        est = estimate_bytes(n, width, height) if est_bytes is None else int(est_bytes)
        req = Request(rid, records, n, width, height, est, time.perf_counter(), fut)
        with self.cv:
            if self.closed:
                raise RuntimeError("server is closed")
            if est > self.hbm_budget:
                fut.set_exception(MemoryError(
                    f"request {rid} needs {est} B, above the {self.hbm_budget} B HBM budget"))
                return fut
            self.waiting.append(req)
            self._admit()
            self.cv.notify_all()
        return fut

    def close(self, timeout: float = 60.0):
        with self.cv:
            self.closed = True
            self.cv.notify_all()
        for w in self.workers:
            w.join(timeout)

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------ internal
    def _admit(self):
        # FIFO admission: the head waits until it fits, so large requests
        # are not starved by smaller ones behind them.
        while self.waiting and self.in_flight_bytes + self.waiting[0].est_bytes <= self.hbm_budget:
            r = self.waiting.popleft()
            self.in_flight_bytes += r.est_bytes
            self.max_in_flight_bytes = max(self.max_in_flight_bytes, self.in_flight_bytes)
            self.queued.append(r)

    def _take(self) -> list[Request]:
        with self.cv:
            while not self.queued and not (self.closed and not self.waiting):
                self.cv.wait()
            if not self.queued:
                return []
            batch = [self.queued.popleft()]
            while (self.queued and len(batch) < self.max_batch
                   and (self.policy is None or self.policy(batch, self.queued[0]))):
                batch.append(self.queued.popleft())
            return batch

    def _release(self, batch: Sequence[Request]):
        with self.cv:
            for r in batch:
                self.in_flight_bytes -= r.est_bytes
            self._admit()
            self.cv.notify_all()

    def _run(self, slot: int, batch: list[Request]):
        t0 = time.perf_counter()
        for r in batch:
            r.started = t0
        try:
            results = self.executor(slot, batch)
            for r, res in zip(batch, results):
                r.future.set_result(res)
        except Exception as e:  # isolate the failing request(s)
            if len(batch) == 1:
                batch[0].future.set_exception(e)
            else:
                for r in batch:
                    try:
                        r.future.set_result(self.executor(slot, [r])[0])
                    except Exception as e1:
                        r.future.set_exception(e1)

    def _work(self, slot: int):
        while True:
            batch = self._take()
            if not batch:
                return
            self.batches.append(len(batch))
            try:
                self._run(slot, batch)
            finally:
                self._release(batch)


# ------------------------------------------------------------- GPU executor
class GpuExecutor:
    """Runs a batch with the library's multi-view sort on a per-slot
    context and stream.  Device record buffers are kept per slot and grown
    on demand, so steady-state serving allocates nothing."""

    def __init__(self, device: int = 0, slots: int = 2, keep_results: bool = False):
        import torch

        from . import tdgs
        self.torch = torch
        self.tdgs = tdgs
        self.device = torch.device("cuda", device)
        self.keep = keep_results
        self.ctx = [tdgs.Context(device) for _ in range(slots)]
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        self.pool: list[list] = [[] for _ in range(slots)]  # resident record buffers

    def _buffer(self, slot: int, i: int, n: int):
        torch = self.torch
        pool = self.pool[slot]
        while len(pool) <= i:
            pool.append(torch.empty((0, 4), dtype=torch.int32, device=self.device))
        if pool[i].shape[0] < n:
            pool[i] = torch.empty((max(n, int(pool[i].shape[0] * 1.25)), 4), dtype=torch.int32,
                                  device=self.device)
        return pool[i][:n]

    def __call__(self, slot: int, batch: Sequence[Request]) -> list[Result]:
        torch = self.torch
        ctx = self.ctx[slot]
        with torch.cuda.stream(self.streams[slot]):
            views = []
            for i, r in enumerate(batch):
                d = self._buffer(slot, i, r.n)
                if r.n:
                    d.copy_(r.records, non_blocking=True)
                views.append((d, r.width, r.height))
            out = ctx.sort_views(views, copy=self.keep)
            self.streams[slot].synchronize()
        t = time.perf_counter()
        res = []
        for r, (k, v, rg, m) in zip(batch, out):
            rr = Result(r.rid, m, t - r.arrival, len(batch))
            if self.keep:
                rr.keys, rr.values, rr.ranges = k, v, rg
            res.append(rr)
        return res

    def close(self):
        for c in self.ctx:
            c.close()


def percentile(xs: Sequence[float], q: float) -> float:
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else float("nan")
