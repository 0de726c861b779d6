"""The multi-GPU path is replicas only: every rank solves its own shots and
the job time is the max over ranks.  This covers that host logic with two
gloo ranks on the CPU (no GPU, no collective on the data path)."""

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    from paper_2308_06152_gb300 import workloads as wl
    nodes = bench.rank_sources(wl.centre_cluster(641, 641, 16), rank)
    t = bench.max_over_ranks(1.5 + rank, world)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, f"r{rank}.txt"), "w") as fh:
        fh.write(repr((nodes, t)))


def test_two_gloo_replicas(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2,
                       join=True, start_method="spawn")
    res = [eval(open(tmp_path / f"r{r}.txt").read()) for r in range(2)]
    (n0, t0), (n1, t1) = res
    assert t0 == t1 == 2.5                     # max over ranks
    assert len(n0) == len(n1) == 16 and set(n0).isdisjoint(n1)
    assert all(0 <= i < 641 and 0 <= j < 641 for (i, j) in n0 + n1)
