"""Serving scheduler logic on the CPU (fake executor, no GPU)."""
import threading
import time

import pytest

from paper_2511_16298_gb300 import serve


class FakeExec:
    def __init__(self, delay=0.01, fail_rid=None):
        self.delay = delay
        self.fail_rid = fail_rid
        self.calls = []
        self.lock = threading.Lock()

    def __call__(self, slot, batch):
        with self.lock:
            self.calls.append((slot, [r.rid for r in batch]))
        if self.fail_rid is not None and any(r.rid == self.fail_rid for r in batch):
            raise ValueError(f"bad request {self.fail_rid}")
        time.sleep(self.delay)
        t = time.perf_counter()
        return [serve.Result(r.rid, r.n * 3, t - r.arrival, len(batch)) for r in batch]


def test_all_requests_complete_in_order_of_results():
    ex = FakeExec()
    with serve.Server(ex, slots=2, hbm_budget=1 << 40, max_batch=8) as s:
        futs = [s.submit(i, None, 100 + i, 64, 64) for i in range(50)]
        res = [f.result(timeout=10) for f in futs]
    assert [r.rid for r in res] == list(range(50))
    assert [r.m for r in res] == [3 * (100 + i) for i in range(50)]
    assert max(s.batches) > 1  # requests that queued up were batched


def test_batching_off_runs_one_at_a_time():
    ex = FakeExec(delay=0.001)
    with serve.Server(ex, slots=1, hbm_budget=1 << 40, batching=False) as s:
        futs = [s.submit(i, None, 10, 16, 16) for i in range(20)]
        [f.result(timeout=10) for f in futs]
    assert all(len(b) == 1 for _, b in ex.calls)


def test_budget_is_never_exceeded_and_fifo():
    ex = FakeExec(delay=0.005)
    est = 1000
    with serve.Server(ex, slots=3, hbm_budget=2500, max_batch=8) as s:
        futs = [s.submit(i, None, 10, 16, 16, est_bytes=est) for i in range(30)]
        [f.result(timeout=20) for f in futs]
    assert s.max_in_flight_bytes <= 2500
    started = [rid for _, b in ex.calls for rid in b]
    assert started == sorted(started)  # admitted and started in arrival order
    assert s.in_flight_bytes == 0


def test_oversized_request_is_rejected():
    ex = FakeExec()
    with serve.Server(ex, slots=1, hbm_budget=1000) as s:
        f = s.submit(0, None, 10, 16, 16, est_bytes=5000)
        ok = s.submit(1, None, 10, 16, 16, est_bytes=500)
        with pytest.raises(MemoryError):
            f.result(timeout=5)
        assert ok.result(timeout=5).rid == 1


def test_failing_request_is_isolated():
    ex = FakeExec(delay=0.02, fail_rid=7)
    with serve.Server(ex, slots=1, hbm_budget=1 << 40, max_batch=16) as s:
        futs = [s.submit(i, None, 10, 16, 16) for i in range(16)]
        outs = []
        for f in futs:
            try:
                outs.append(f.result(timeout=10).rid)
            except ValueError:
                outs.append("failed")
    assert outs[7] == "failed"
    assert [o for i, o in enumerate(outs) if i != 7] == [i for i in range(16) if i != 7]


def test_estimate_grows_with_size():
    a = serve.estimate_bytes(100_000, 640, 360)
    b = serve.estimate_bytes(3_000_000, 1920, 1080)
    assert 0 < a < b


def test_narrow_policy():
    mk = lambda n, w, h: serve.Request(0, None, n, w, h, 0, 0.0, None)
    small = [mk(100_000, 640, 360)]
    assert serve.narrow_batches(small, mk(100_000, 640, 360))        # 18 + 11 bits
    assert not serve.narrow_batches([mk(3_000_000, 1920, 1080)], mk(200_000, 640, 360))
    ex = FakeExec(delay=0.002)
    with serve.Server(ex, slots=1, hbm_budget=1 << 40, max_batch=16,
                      policy=lambda b, r: len(b) < 3) as s:
        futs = [s.submit(i, None, 10, 16, 16) for i in range(12)]
        [f.result(timeout=10) for f in futs]
    assert max(len(b) for _, b in ex.calls) <= 3
