"""The multi-rank path of bench.py on CPU: two ranks over gloo (127.0.0.1).  On GPUs the
job runs one replica of the workload per rank (the path shards into independent
problems; no collective on the data path); what crosses ranks is the barrier around
the timed region, the maximum of the ranks' times, and rank 0 alone printing (and
alone running the oracle arm).  This checks that logic without a GPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench.dist_env()
        assert (w, r, local) == (world, rank, rank)
        bench.barrier()
        slowest = bench.max_over_ranks(torch, 1.0 + rank)        # rank 1 is the slow one
        rate = bench.whole_job_rate(100.0, 4, w, slowest)
        # the oracle arm: every rank but 0 returns at once without work
        ran_reference = False
        if rank != 0:
            class A:   # noqa: E306  (the arguments the arm reads)
                steps, warmup = 1, 0
            assert bench.run_reference(A()) is None
            ran_reference = True
        with open(os.path.join(out_dir, "rank%d.txt" % rank), "w") as f:
            f.write("%r %r %r" % (slowest, rate, ran_reference))
    finally:
        dist.destroy_process_group()


def test_two_ranks_over_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as tmp
    world, port = 2, _free_port()
    tmp.start_processes(_rank, args=(world, port, str(tmp_path)), nprocs=world, start_method="spawn",
                        join=True)
    r0 = open(tmp_path / "rank0.txt").read().split()
    r1 = open(tmp_path / "rank1.txt").read().split()
    # both ranks see the slowest rank's time; the job rate counts both replicas
    assert float(r0[0]) == float(r1[0]) == 2.0
    assert float(r0[1]) == float(r1[1]) == 100.0 * 4 * 2 / 2.0
    assert r1[2] == "True"
