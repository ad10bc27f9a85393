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
    with serve.Server(ex, slots=3, hbm_budget=3000, max_batch=8) as s:
        futs = [s.submit(i, None, 10, 16, 16, est_bytes=est) for i in range(30)]
        [f.result(timeout=20) for f in futs]
    assert s.resident_bytes() <= 3000
    assert all(len(b) == 1 for _, b in ex.calls)  # a share holds one such request
    started = [rid for _, b in ex.calls for rid in b]
    assert started == sorted(started)  # started in arrival order


def test_resident_high_water_stays_within_budget():
    """Slots keep buffers sized for the largest batch they ran; the sum of
    those high-water marks never exceeds the budget, whatever the mix."""
    import random
    rnd = random.Random(4)
    ex = FakeExec(delay=0.001)
    budget = 10_000
    with serve.Server(ex, slots=2, hbm_budget=budget, max_batch=16) as s:
        futs = [s.submit(i, None, 10, 16, 16, est_bytes=rnd.randint(100, 5000)) for i in range(200)]
        [f.result(timeout=30) for f in futs]
        assert all(r <= s.share for r in s.resident)
        assert s.resident_bytes() <= budget
    seen = {}
    for slot, b in ex.calls:
        seen.setdefault(slot, []).append(len(b))
    assert max(len(b) for _, b in ex.calls) > 1


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


def test_cost_model_batches_small_and_keeps_wide_apart():
    mk = lambda n, w, h: serve.Request(0, None, n, w, h, 0, 0.0, None)
    cm = serve.CostModel(overhead_s=100e-6, pair_s_narrow=20e-12, pair_s_wide=45e-12, gaussian_s=0.0,
                         pairs_per_gaussian=12.0)
    small = mk(100_000, 640, 360)
    # small frames: the per-batch overhead saved outweighs nothing -> join
    assert cm.joins([small, small], small)
    # a 3M-Gaussian 1080p frame already sorts with 64-bit elements: a small
    # frame joins it for its own pairs' extra cost (60 us) < the 100 us saved
    big = mk(3_000_000, 1920, 1080)
    assert not serve.narrow_elements(3_000_000, 8160)
    assert cm.joins([big], mk(200_000, 640, 360))
    # two 1M-Gaussian 720p frames are each 32-bit alone but 64-bit together:
    # 24M pairs x 25 ps extra (0.6 ms) outweigh the 0.1 ms saved -> apart
    one = mk(1_000_000, 1280, 720)
    assert serve.narrow_elements(1_000_000, 3600) and not serve.narrow_elements(2_000_000, 7200)
    assert not cm.joins([one], one)
    # the policy is a plain callable for the server
    ex = FakeExec(delay=0.002)
    with serve.Server(ex, slots=1, hbm_budget=1 << 40, max_batch=16, policy=cm.joins) as s:
        futs = [s.submit(i, None, 100_000, 640, 360) for i in range(12)]
        [f.result(timeout=10) for f in futs]
    assert max(len(b) for _, b in ex.calls) > 1


def test_executor_completing_each_request_early():
    """An executor that hands over each result as it is ready resolves that
    request's future before the rest of its batch is done."""
    gate = threading.Event()

    class EachExec:
        completes_each = True

        def __call__(self, slot, batch, done=None):
            out = []
            for i, r in enumerate(batch):
                res = serve.Result(r.rid, r.n, 0.0, len(batch))
                out.append(res)
                if done is not None:
                    done(i, res)
                if i == 0:
                    assert gate.wait(5)  # the rest of the batch waits for the test
            return out

    with serve.Server(EachExec(), slots=1, hbm_budget=1 << 40, max_batch=8) as s:
        blocker = s.submit(99, None, 1, 16, 16)
        futs = [s.submit(i, None, 10 + i, 16, 16) for i in range(3)]
        assert blocker.result(timeout=5).rid == 99  # done before the gate opens
        gate.set()
        assert [f.result(timeout=5).rid for f in futs] == [0, 1, 2]
