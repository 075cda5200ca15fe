"""The replica path of bench.py on CPU: two gloo ranks combine their
per-rank timings (max) and throughputs (sum) the way the benchmark does
under torchrun, and a single process passes its values through."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_setup(None)
    ms = 3.0 + 2.0 * rank                 # rank 1 is the slower one
    rate = 100.0 * (rank + 1)
    out[rank] = (ws, r, local, bench.across_ranks(ms, "max", dist, device="cpu"),
                 bench.across_ranks(rate, "sum", dist, device="cpu"))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_combine_like_the_benchmark():
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(timeout=120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][:3] == (2, 0, 0) and res[1][:3] == (2, 1, 1)
    for r in (0, 1):
        assert res[r][3] == pytest.approx(5.0)     # max of 3 ms and 5 ms
        assert res[r][4] == pytest.approx(300.0)   # 100/s + 200/s


def test_single_process_passes_values_through():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.across_ranks(4.5, "max") == 4.5
    assert bench.across_ranks(7.0, "sum") == 7.0
