"""The multi-rank timing path with two gloo ranks on the CPU: every rank
does its own work (independent cubes, nothing exchanged on the data path);
the job's rate is all ranks' units over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist
    from paper_1609_03782_gb300 import ranks
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, lr = ranks.world_info()
        ranks.barrier()
        secs = 1.0 + rank          # rank 1 is the slower one
        units = 100.0 * (rank + 1)
        out.put((r, w, lr, ranks.max_over_ranks(secs), ranks.sum_over_ranks(units),
                 ranks.job_rate(units, secs)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
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
    for r, (rank, world, local, mx, sm, rate) in enumerate(res):
        assert (rank, world, local) == (r, 2, r)
        assert mx == 2.0 and sm == 300.0 and rate == pytest.approx(150.0)


def test_single_process_is_identity():
    from paper_1609_03782_gb300 import ranks
    assert ranks.max_over_ranks(3.5) == 3.5
    assert ranks.job_rate(10.0, 2.0) == 5.0
