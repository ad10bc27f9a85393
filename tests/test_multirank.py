"""The replica path of the benchmark on two CPU ranks (gloo): each rank sorts
its own frame, so the only cross-rank step is combining the timings -- the
slowest rank's time and the sum of the pairs all ranks sorted."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank: int, world: int, port: int, out):
    import torch.distributed as dist

    import bench
    from paper_2511_16298_gb300 import synth
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seconds = [0.5, 2.0][rank]
        pairs = [1000.0, 3000.0][rank]
        t, u = bench.combine_ranks(dist, seconds, pairs, "cpu")
        # replicas: every rank's frame comes from its own seed
        fr = synth.frame_small(seed=rank, n=200)
        dist.barrier()
        out.put((rank, t, u, float(fr.gaussians["x"][0])))
    finally:
        dist.destroy_process_group()


def test_combine_ranks_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    for rank, t, u, _ in res:
        assert t == 2.0 and u == 4000.0
    assert res[0][3] != res[1][3]  # different frames per rank


def test_combine_ranks_single_process():
    import bench
    assert bench.combine_ranks(None, 1.5, 10.0, "cpu") == (1.5, 10.0)
