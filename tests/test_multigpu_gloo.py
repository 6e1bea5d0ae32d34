"""The N > 1 host path of the benchmark on CPU: two gloo ranks agree on the job's step time (the
maximum over ranks) and on the whole-job value of replicated workloads."""
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


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t = 0.010 + 0.005 * rank  # ranks finish at different times
    tmax = bench.max_over_ranks(t)
    out[rank] = (tmax, bench.job_value(816000 * 20, world, tmax))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_max_step_time():
    ctx = mp.get_context("spawn")
    world, port = 2, _free_port()
    with ctx.Manager() as mgr:
        out = mgr.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == pytest.approx(0.015)
    assert res[0][1] == pytest.approx(816000 * 20 * 2 / 0.015 / 1e6)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(0.02) == 0.02
    assert bench.job_value(1_000_000, 1, 0.5) == pytest.approx(2.0)
