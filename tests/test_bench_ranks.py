"""The multi-process path of bench.py on CPU (gloo, world size 2): each rank
gets its own seeds, the timed region is the slowest rank's, and the job
throughput counts every rank's images. No GPU and no data-path collective."""
from __future__ import annotations

import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    r, w, lr = bench.rank_info()
    t_local = 100.0 + 50.0 * rank  # rank 1 is slower
    t_max = bench.max_over_ranks(t_local, w)
    q.put((r, w, lr, bench.rank_seeds(r), t_max, bench.job_throughput(256, 3, w, t_max / 1e3)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_timing_and_seeds():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, w0, l0, s0, t0, v0), (r1, w1, l1, s1, t1, v1) = res
    assert (r0, r1, w0, w1, l0, l1) == (0, 1, 2, 2, 0, 1)
    assert t0 == t1 == 150.0                      # both ranks report the slowest rank's time
    assert v0 == v1 == pytest.approx(256 * 3 * 2 / 0.150)
    assert s0["ctx_seed"] != s1["ctx_seed"] and s0["image_seed"] != s1["image_seed"]
    assert s0["weight_seed"] == s1["weight_seed"]  # one model, independent inputs


def test_single_rank_defaults():
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_throughput(256, 2, 1, 0.5) == 1024.0
