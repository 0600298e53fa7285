"""The benchmark's whole-job figures across ranks (bench.job_totals), on the CPU: two gloo ranks,
each with its own timed-region length and units of work, both obtain the slowest rank's time and
the units summed over the ranks; one rank gets its own figures back."""
import os
import socket

import torch.multiprocessing as mp


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, out):
    import torch.distributed as dist

    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=2)
    try:
        dist.barrier()
        out[rank] = bench.job_totals(1.5 + rank, 100.0 * (rank + 1), 2)
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_job_totals_over_two_gloo_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0] == res[1] == (2.5, 300.0)


def test_job_totals_of_one_rank():
    import bench

    assert bench.job_totals(3.0, 7.0, 1) == (3.0, 7.0)
