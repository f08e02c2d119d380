"""Host logic of the multi-GPU replicas path, exercised with gloo ranks on the CPU."""
import os
import socket

import pytest

from paper_1303_1377_gb300.replicas import aggregate, rhs_slice


def test_rhs_slice_partitions_the_batch():
    for n in (1, 5, 12, 13):
        for world in (1, 2, 3, 8):
            got = [i for r in range(world) for i in rhs_slice(n, r, world)]
            assert got == list(range(n))
            sizes = [len(rhs_slice(n, r, world)) for r in range(world)]
            assert max(sizes) - min(sizes) <= 1


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r "took" 100 + 50 r ms for 12 solves
    val, ms, units = aggregate(100.0 + 50.0 * rank, 12.0, dist=dist)
    dist.barrier()
    q.put((rank, val, ms, units))
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    torch = pytest.importorskip("torch")
    mp = torch.multiprocessing.get_context("spawn")
    q = mp.Queue()
    port = _free_port()
    procs = [mp.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, val, ms, units in res:
        assert ms == 150.0 and units == 24.0
        assert abs(val - 24.0 / 0.15) < 1e-9


def test_aggregate_single_process():
    assert aggregate(500.0, 12.0) == (24.0, 500.0, 12.0)
