"""The N > 1 path of bench.py (independent replicas, one per GPU) on the CPU:
two gloo ranks reduce their timings and particle-step counts exactly as the
benchmark does (slowest rank's time, summed particle-steps)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, local = bench._dist()
    assert (ws, r, local) == (world, rank, rank)
    ms, pushed = bench.reduce_over_ranks(10.0 + rank, 1000 * (rank + 1), ws)
    dist.barrier()
    out[rank] = (ms, pushed)
    dist.destroy_process_group()


def test_two_rank_reduction_matches_bench_contract():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        assert out[rank] == (11.0, 3000.0)  # max time, summed particle-steps


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_over_ranks(5.0, 7, 1) == (5.0, 7.0)


def test_bench_reaches_the_start_step_in_the_run_state():
    import bench
    # shorter than the window: the run is replayed from its empty box
    assert bench._prerun_steps(900, 1536, False) == 900
    # longer: nx steps after a load at rest flush every loaded particle out
    assert bench._prerun_steps(4500, 2048, False) == 2048
    assert bench._prerun_steps(0, 128, False) == 0
    assert bench._prerun_steps(900, 1536, True) == 0  # --cold-start
