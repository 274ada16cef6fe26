"""Multi-rank host logic of the benchmark on CPU: two `gloo` ranks reduce
their timings to the maximum and report the whole-job rate (weak scaling).
No GPU is involved; the renderers themselves are independent per rank."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update({"WORLD_SIZE": str(ws), "RANK": str(rank), "LOCAL_RANK": str(rank)})
    assert bench._dist() == (ws, rank, rank)
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=ws)
    try:
        # rank r is slow in column r: the reduction must take each column's maximum
        local = [1.0 + 3.0 * (rank == 0), 2.0 + 5.0 * (rank == 1), -1.0 if rank == 1 else 4.0]
        got = bench.max_over_ranks(local, ws)
        out[rank] = got
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_to_the_slowest():
    import torch.multiprocessing as mp
    ws = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()   # no fork of a multi-threaded process
    out = mgr.dict()
    mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
    assert out[0] == out[1] == [4.0, 7.0, 4.0]


def test_whole_job_rate_is_weak_scaling():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job_rate(1, 0.25) == pytest.approx(4000.0)
    # two ranks, each one frame per 0.25 ms step (max over ranks): 8000 frames/s
    assert bench.whole_job_rate(2, 0.25) == pytest.approx(8000.0)
    assert bench.max_over_ranks([1.5, 2.5], 1) == [1.5, 2.5]
