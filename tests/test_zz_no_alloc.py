"""tdgs_scan_noalloc -- the scan for callers that cannot allocate device
memory (real-time loops that must not reach the device allocator, plugins
whose device memory belongs to a host application).  Its scratch is a fixed
device array inside the library.  The tests call it through the C ABI, two
calls in a row (the second must not see the first one's leftovers), and
compare its offsets and total with both tdgs_scan and the CPU oracle's scan
bit for bit (integer results); they also cover n == 0, NULL total/error
pointers and the size limit.  Collected last on purpose: if this file fails,
a run stopped at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
DEV = "cuda:0"


def _call(L, c, n, off, tot, err):
    p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None  # noqa: E731
    return L.tdgs_scan_noalloc(p(c), n, p(off), p(tot), p(err),
                               ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_scan_noalloc_matches_scan_and_oracle():
    from oracle import oracle as O
    from paper_2511_16298_gb300 import build
    build.build()
    from paper_2511_16298_gb300 import tdgs as T
    L = T.lib()
    rng = np.random.default_rng(42)
    with T.Context(0) as ctx:
        for n in (3_000_001, 5000):  # two calls in a row, the second smaller
            host = rng.integers(0, 1500, size=n).astype(np.uint32)
            st_o, off_o, tot_o = O.scan(host)
            assert st_o == 0
            c = torch.from_numpy(host.view(np.int32)).to(DEV)
            ref_off, ref_tot = ctx.scan(c)
            ctx.sync()
            off = torch.full((n,), -1, dtype=torch.int32, device=DEV)
            tot = torch.full((1,), -1, dtype=torch.int32, device=DEV)
            err = torch.full((1,), -1, dtype=torch.int32, device=DEV)
            assert _call(L, c, n, off, tot, err) == T.OK
            torch.cuda.synchronize()
            assert torch.equal(off, ref_off)
            assert torch.equal(tot, ref_tot)
            assert np.array_equal(off.cpu().numpy().view(np.uint32), off_o)
            assert int(tot.cpu().numpy().view(np.uint32)[0]) == tot_o
            assert int(err.item()) == 0


def test_scan_noalloc_empty_and_null_outputs():
    from oracle import oracle as O
    from paper_2511_16298_gb300 import tdgs as T
    L = T.lib()
    tot = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    err = torch.full((1,), -1, dtype=torch.int32, device=DEV)
    assert _call(L, None, 0, None, tot, err) == T.OK
    torch.cuda.synchronize()
    assert int(tot.item()) == 0 and int(err.item()) == 0
    # offsets only: total and error pointers are NULL
    host = np.random.default_rng(3).integers(0, 40, size=70_000).astype(np.uint32)
    c = torch.from_numpy(host.view(np.int32)).to(DEV)
    off = torch.full((len(host),), -1, dtype=torch.int32, device=DEV)
    assert _call(L, c, len(host), off, None, None) == T.OK
    torch.cuda.synchronize()
    _, off_o, _ = O.scan(host)
    assert np.array_equal(off.cpu().numpy().view(np.uint32), off_o)


def test_scan_noalloc_limits():
    from paper_2511_16298_gb300 import tdgs as T
    L = T.lib()
    c = torch.zeros(4, dtype=torch.int32, device=DEV)
    assert _call(L, c, (1 << 24) + 1, c, None, None) == T.INVALID_ARGUMENT
    # overflow is reported through the error word
    big = torch.full((5000,), 1 << 20, dtype=torch.int32, device=DEV)
    off, tot, err = T.scan_noalloc(big)
    torch.cuda.synchronize()
    assert int(err.item()) == T.OVERFLOW and int(tot.item()) == -1
