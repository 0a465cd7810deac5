"""The benchmark's multi-rank path (replicas, one per GPU) on CPU: two gloo
ranks take the maximum of their timings, as the benchmark does over NCCL."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
mp = pytest.importorskip("torch.multiprocessing")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [10.0 + rank, 5.0 - rank, 7.0 * (rank + 1)]
        out[rank] = bench.max_over_ranks(mine, world, torch.device("cpu"))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_maximum():
    world, port = 2, _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(world, port, out), nprocs=world, join=True,
                           start_method="spawn")
        got = dict(out)
    want = [11.0, 5.0, 14.0]
    assert got[0] == want and got[1] == want


def test_single_rank_is_a_no_op():
    import bench
    assert bench.max_over_ranks([1, 2.5], 1, None) == [1.0, 2.5]


def test_power_law_extrapolation_is_exact_on_a_power_law():
    import bench
    t = lambda n: 2e-9 * n ** 1.5
    est, b = bench.power_law(100_000, t(100_000), 200_000, t(200_000), 1_000_000)
    assert abs(b - 1.5) < 1e-12 and abs(est - t(1_000_000)) < 1e-9 * t(1_000_000)


def test_host_info_names_cores_and_cpu():
    import bench
    hi = bench.host_info()
    assert hi["nproc"] == os.cpu_count() and hi["machine"]
