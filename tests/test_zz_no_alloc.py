"""tdgs_scan_noalloc -- the scan for callers that cannot allocate device
memory (code running under CUDA graph capture, real-time loops that must
not reach the allocator, plugins whose memory belongs to a host
application).  Its scratch is a fixed device array inside the library; the
test calls it through the C ABI twice in a row (the second call must not
see the first one's leftovers) and compares with tdgs_scan, bit for bit
(integer results), and checks the size limit.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def test_scan_noalloc_matches_scan():
    from paper_2511_16298_gb300 import build
    build.build()
    from paper_2511_16298_gb300 import tdgs as T
    L = T.lib()
    rng = np.random.default_rng(42)
    with T.Context(0) as ctx:
        for n in (3_000_001, 5000):  # two calls in a row, the second smaller
            c = torch.from_numpy(rng.integers(0, 1500, size=n).astype(np.int32)).to(DEV)
            ref_off, ref_tot = ctx.scan(c)
            ctx.sync()
            off = torch.full((n,), -1, dtype=torch.int32, device=DEV)
            tot = torch.full((1,), -1, dtype=torch.int32, device=DEV)
            err = torch.full((1,), -1, dtype=torch.int32, device=DEV)
            st = L.tdgs_scan_noalloc(ctypes.c_void_p(c.data_ptr()), n, ctypes.c_void_p(off.data_ptr()),
                                     ctypes.c_void_p(tot.data_ptr()), ctypes.c_void_p(err.data_ptr()),
                                     ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert st == T.OK
            torch.cuda.synchronize()
            assert torch.equal(off, ref_off)
            assert torch.equal(tot, ref_tot)
            assert int(err.item()) == 0


def test_scan_noalloc_limits():
    from paper_2511_16298_gb300 import tdgs as T
    L = T.lib()
    c = torch.zeros(4, dtype=torch.int32, device=DEV)
    assert L.tdgs_scan_noalloc(ctypes.c_void_p(c.data_ptr()), (1 << 24) + 1, ctypes.c_void_p(c.data_ptr()),
                               None, None, None) == T.INVALID_ARGUMENT
    # overflow is reported through the error word
    big = torch.full((5000,), 1 << 20, dtype=torch.int32, device=DEV)
    off, tot, err = T.scan_noalloc(big)
    torch.cuda.synchronize()
    assert int(err.item()) == T.OVERFLOW and int(tot.item()) == -1
