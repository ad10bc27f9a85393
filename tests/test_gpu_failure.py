"""Failure detection without a GPU fault: a cross-block wait that runs out
(one block waits at the radix passes' grid barrier for a block that never
arrives) ends by its iteration bound, latches TDGS_ERR_TIMEOUT, is reported
by the next sync, and leaves the context usable."""
import time

import numpy as np
import pytest

from paper_2511_16298_gb300 import synth
from paper_2511_16298_gb300 import tdgs as T

pytestmark = pytest.mark.gpu


def test_barrier_wait_runs_out_and_context_recovers(oracle):
    from paper_2511_16298_gb300 import build
    build.build()
    with T.Context(0) as ctx:
        t0 = time.perf_counter()
        ctx.diag_barrier_timeout()
        with pytest.raises(T.TdgsError) as e:
            ctx.sync()
        waited = time.perf_counter() - t0
        assert e.value.status == T.TIMEOUT
        assert waited < 30.0  # bounded: ends by the iteration limit
        ctx.sync()  # the error was cleared
        fr = synth.frame_small(2, n=3000, width=200, height=120)
        k, v, r, m = ctx.sort_frame(T.records_to_tensor(fr.gaussians, "cuda:0"), fr.width, fr.height, copy=True)
        ref = oracle.sort_frame(fr.gaussians, fr.width, fr.height)
        assert m == ref["m"]
        assert np.array_equal(v.cpu().numpy().view(np.uint32), ref["values"])
        assert np.array_equal(r.cpu().numpy().view(np.uint32), ref["ranges"])
