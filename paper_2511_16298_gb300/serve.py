"""Continuous-batching request server for the tile depth sort.

Frames (views) arrive as requests and wait in a queue; every slot (one
worker thread, one library context, one CUDA stream and device-resident
buffers reused from batch to batch) takes queued requests the moment it is
free and sorts them as one multi-view batch.  While one slot's batch runs,
newly arrived requests queue up and are picked up by the next free slot,
so host work, copies and kernels of different batches overlap.  Latency is
completion minus arrival.

Device memory: the HBM budget is split evenly over the slots.  A slot's
buffers grow to fit the largest batch it has run and stay resident, so a
slot never takes a batch whose estimated footprint exceeds its share; the
slots' resident memory (their high-water marks) thus stays within the
budget.  A request larger than a share is refused.

Which queued requests run together is decided by a batching policy; the
cost model below (per-batch overhead against per-pair cost, measured on
the device) joins a request to a batch only when running them together is
cheaper than running them apart.

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


def _tiles(r: Request) -> int:
    return ((r.width + 15) // 16) * ((r.height + 15) // 16)


def narrow_elements(n: int, tiles: int) -> bool:
    """Whether a batch of n Gaussians over `tiles` tiles (all views) sorts
    with 32-bit packed (tile, depth rank) elements and at most two 8-bit
    tile passes -- the library's cheaper per-pair form."""
    return _bits(n) + _bits(tiles) <= 32 and _bits(tiles) <= 16


@dataclasses.dataclass
class CostModel:
    """Device time of one batch: overhead_s per batch (launches, the host
    wait for the pair count, the copies' fixed costs) plus per pair the
    cost of the element form the batch sorts with, plus per Gaussian.
    Pair counts are estimated from Gaussian counts."""
    overhead_s: float = 100e-6
    pair_s_narrow: float = 20e-12   # per pair, 32-bit elements
    pair_s_wide: float = 45e-12     # per pair, 64-bit elements
    gaussian_s: float = 60e-12      # per Gaussian (depth sort, duplication)
    pairs_per_gaussian: float = 12.0

    def cost(self, batch: Sequence[Request]) -> float:
        n = sum(r.n for r in batch)
        t = sum(_tiles(r) for r in batch)
        per_pair = self.pair_s_narrow if narrow_elements(n, t) else self.pair_s_wide
        return self.overhead_s + n * (self.gaussian_s + self.pairs_per_gaussian * per_pair)

    def joins(self, batch: Sequence[Request], nxt: Request) -> bool:
        """Run nxt in this batch if that is cheaper than running it alone."""
        return self.cost(list(batch) + [nxt]) <= self.cost(batch) + self.cost([nxt])


def narrow_batches(batch: Sequence[Request], nxt: Request) -> bool:
    """Join only while the batch keeps the 32-bit element form."""
    n = sum(r.n for r in batch) + nxt.n
    return narrow_elements(n, sum(_tiles(r) for r in batch) + _tiles(nxt))


class Server:
    """Continuous batching over `slots` workers within an HBM budget.

    executor(slot, batch) sorts one batch and returns one Result per
    request (in order); it raises on failure.  The budget is split evenly
    over the slots; a slot takes queued requests in arrival order while
    their estimated footprint fits its share and the policy accepts them."""

    def __init__(self, executor: Executor, slots: int = 2, hbm_budget: int = 40 << 30,
                 max_batch: int = 32, batching: bool = True, policy: Optional[Policy] = None):
        self.executor = executor
        self.policy = policy
        self.hbm_budget = int(hbm_budget)
        self.share = self.hbm_budget // slots
        self.max_batch = max_batch if batching else 1
        self.cv = threading.Condition()
        self.queued: collections.deque[Request] = collections.deque()
        # per slot: estimated footprint of the largest batch it has run --
        # the high-water mark its resident buffers grow to
        self.resident = [0] * slots
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
            if est > self.share:
                fut.set_exception(MemoryError(
                    f"request {rid} needs {est} B, above a slot's {self.share} B share of the "
                    f"{self.hbm_budget} B HBM budget"))
                return fut
            self.queued.append(req)
            self.cv.notify_all()
        return fut

    def resident_bytes(self) -> int:
        """Estimated device memory the slots hold (their high-water marks)."""
        with self.cv:
            return sum(self.resident)

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
    def _take(self, slot: int) -> list[Request]:
        with self.cv:
            while not self.queued and not self.closed:
                self.cv.wait()
            if not self.queued:
                return []
            batch = [self.queued.popleft()]
            foot = batch[0].est_bytes
            while (self.queued and len(batch) < self.max_batch
                   and foot + self.queued[0].est_bytes <= self.share
                   and (self.policy is None or self.policy(batch, self.queued[0]))):
                foot += self.queued[0].est_bytes
                batch.append(self.queued.popleft())
            self.resident[slot] = max(self.resident[slot], foot)
            return batch

    def _run(self, slot: int, batch: list[Request]):
        t0 = time.perf_counter()
        for r in batch:
            r.started = t0
        try:
            if getattr(self.executor, "completes_each", False):
                # the executor hands over each request's result as soon as it
                # is ready (before the rest of its batch)
                def done(i: int, res: Result):
                    batch[i].future.set_result(res)

                results = self.executor(slot, batch, done)
            else:
                results = self.executor(slot, batch)
                for r, res in zip(batch, results):
                    r.future.set_result(res)
        except Exception as e:  # isolate the failing request(s)
            if len(batch) == 1:
                batch[0].future.set_exception(e)
            else:
                for r in batch:
                    if r.future.done():
                        continue
                    try:
                        r.future.set_result(self.executor(slot, [r])[0])
                    except Exception as e1:
                        r.future.set_exception(e1)

    def _work(self, slot: int):
        while True:
            batch = self._take(slot)
            if not batch:
                return
            self.batches.append(len(batch))
            self._run(slot, batch)


# ------------------------------------------------------------- GPU executor
DEFAULT_KNOBS = {"tile_digit_bits": 0, "ctas_per_sm": 0, "depth_digit_bits": 0}


class GpuExecutor:
    """Runs a batch with the library's multi-view sort on a per-slot
    context and stream.  Device record buffers are kept per slot and grown
    on demand, so steady-state serving allocates nothing.

    download=True copies every view's sorted keys, values and ranges into
    pinned host memory (per-slot staging, grown on demand) before the
    latency clock stops: a served request is complete when its result is in
    host memory.  The views of a batch download smallest first, in chunks
    (so two slots' copies interleave), and each request completes -- its
    future is resolved -- as soon as its own download is done, not when the
    whole batch is.  Those host tensors are reused by the slot's next batch.
    keep_results=True instead keeps device copies (for tests).  With a
    tuning table (autotune.Table), the knobs stored for the batch's shape
    are applied to the slot's context before it runs."""

    def __init__(self, device: int = 0, slots: int = 2, keep_results: bool = False,
                 download: bool = False, table=None):
        import torch

        from . import tdgs
        self.torch = torch
        self.tdgs = tdgs
        self.device = torch.device("cuda", device)
        self.keep = keep_results
        self.download = download
        self.table = table
        self.ctx = [tdgs.Context(device) for _ in range(slots)]
        self.streams = [torch.cuda.Stream(self.device) for _ in range(slots)]
        self.pool: list[list] = [[] for _ in range(slots)]       # resident record buffers
        self.host_pool: list[list] = [[] for _ in range(slots)]  # pinned result staging
        self.knobs: list = [None] * slots
        self.tuned_batches = 0

    def _buffer(self, slot: int, i: int, n: int):
        torch = self.torch
        pool = self.pool[slot]
        while len(pool) <= i:
            pool.append(torch.empty((0, 4), dtype=torch.int32, device=self.device))
        if pool[i].shape[0] < n:
            pool[i] = torch.empty((max(n, int(pool[i].shape[0] * 1.25)), 4), dtype=torch.int32,
                                  device=self.device)
        return pool[i][:n]

    def _host(self, slot: int, i: int, m: int, tiles: int):
        torch = self.torch
        pool = self.host_pool[slot]
        while len(pool) <= i:
            pool.append([torch.empty(0, dtype=torch.int64).pin_memory(),
                         torch.empty(0, dtype=torch.int32).pin_memory(),
                         torch.empty((0, 2), dtype=torch.int32).pin_memory()])
        e = pool[i]
        if e[0].shape[0] < m:
            cap = max(m, int(e[0].shape[0] * 1.25))
            e[0] = torch.empty(cap, dtype=torch.int64).pin_memory()
            e[1] = torch.empty(cap, dtype=torch.int32).pin_memory()
        if e[2].shape[0] < tiles:
            e[2] = torch.empty((max(tiles, int(e[2].shape[0] * 1.25)), 2), dtype=torch.int32).pin_memory()
        return e[0][:m], e[1][:m], e[2][:tiles]

    def reserve(self, slot: int, batch: Sequence[Request], pairs_per_gaussian: float = 16.0):
        """Grow the slot's host staging for a batch like this one ahead of
        time (pinned allocations are slow)."""
        for i, r in enumerate(batch):
            self._host(slot, i, int(r.n * pairs_per_gaussian), _tiles(r))

    completes_each = True
    CHUNK = 1 << 20  # pairs per download copy (8 MB of keys)

    def __call__(self, slot: int, batch: Sequence[Request], done=None) -> list[Result]:
        torch = self.torch
        ctx = self.ctx[slot]
        with torch.cuda.stream(self.streams[slot]):
            views = []
            for i, r in enumerate(batch):
                d = self._buffer(slot, i, r.n)
                if r.n:
                    d.copy_(r.records, non_blocking=True)
                views.append((d, r.width, r.height))
            if self.table is not None:
                knobs = self.table.knobs_for_views(views)
                if knobs:
                    self.tuned_batches += 1
                want = knobs or DEFAULT_KNOBS
                if want != self.knobs[slot]:
                    ctx.apply_tuning(want)
                    self.knobs[slot] = want
            out = ctx.sort_views(views, copy=self.keep)
            order = sorted(range(len(batch)), key=lambda i: out[i][3])  # smallest first
            host = [None] * len(batch)
            events = []
            for i in order:
                k, v, rg, m = out[i]
                if self.download:
                    hk, hv, hr = self._host(slot, i, m, rg.shape[0])
                    for a in range(0, m, self.CHUNK):
                        b = min(m, a + self.CHUNK)
                        hk[a:b].copy_(k[a:b], non_blocking=True)
                        hv[a:b].copy_(v[a:b], non_blocking=True)
                    hr.copy_(rg, non_blocking=True)
                    host[i] = (hk, hv, hr)
                ev = torch.cuda.Event()
                ev.record(self.streams[slot])
                events.append((i, ev))
        res: list = [None] * len(batch)
        for i, ev in events:
            ev.synchronize()
            t = time.perf_counter()
            r = batch[i]
            k, v, rg, m = out[i]
            rr = Result(r.rid, m, t - r.arrival, len(batch))
            if self.keep:
                rr.keys, rr.values, rr.ranges = k, v, rg
            elif self.download:
                rr.keys, rr.values, rr.ranges = host[i]
            res[i] = rr
            if done is not None:
                done(i, rr)
        return res

    def calibrate(self, batches: Sequence[Sequence[Request]], reps: int = 3) -> CostModel:
        """Fit the cost model's overhead and per-pair costs to measured
        batch times (slot 0, results downloaded as when serving): the
        narrow and wide per-pair costs from the batches of each form, the
        overhead from the intercept."""
        rows = []
        for b in batches:
            self(0, b)
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter()
                res = self(0, b)
                ts.append(time.perf_counter() - t0)
            pairs = sum(r.m for r in res)
            n = sum(r.n for r in b)
            narrow = narrow_elements(n, sum(_tiles(r) for r in b))
            rows.append((narrow, n, pairs, float(np.median(ts))))
        cm = CostModel()
        cm.pairs_per_gaussian = sum(p for _, _, p, _ in rows) / max(1, sum(n for _, n, _, _ in rows))
        # least squares t = overhead + pairs * per_pair(form), Gaussian cost folded into per_pair
        a = np.array([[1.0, p if nr else 0.0, 0.0 if nr else p] for nr, _, p, _ in rows])
        y = np.array([t for *_, t in rows])
        coef, *_ = np.linalg.lstsq(a, y, rcond=None)
        cm.overhead_s = max(float(coef[0]), 0.0)
        if any(nr for nr, *_ in rows):
            cm.pair_s_narrow = max(float(coef[1]), 1e-13)
        if any(not nr for nr, *_ in rows):
            cm.pair_s_wide = max(float(coef[2]), 1e-13)
        cm.gaussian_s = 0.0
        return cm

    def close(self):
        for c in self.ctx:
            c.close()


def percentile(xs: Sequence[float], q: float) -> float:
    return float(np.percentile(np.asarray(xs, dtype=np.float64), q)) if len(xs) else float("nan")
