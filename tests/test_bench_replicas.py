"""Host logic of the multi-GPU benchmark (replicas, no collective on the data path), on CPU.

Each rank solves its own sweep cells; the only collectives are the timing barrier and the
max-over-ranks reduction of the timed region. Run here as world-size-2 `gloo` process groups.
"""
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8, 9, 12])
def test_rank_cells_partition_the_sweep(world):
    """Ranks own disjoint cells that together cover the nine (one cell each beyond nine)."""
    per_rank = [bench.rank_cells(r, world) for r in range(world)]
    assert all(per_rank)
    if world <= 9:
        flat = sorted(c for cells in per_rank for c in cells)
        assert flat == list(range(9))
    else:
        assert all(len(c) == 1 for c in per_rank)
        assert sorted({c[0] for c in per_rank}) == list(range(9))
    assert bench.rank_cells(0, 1, 3) == [0, 1, 2]


def test_throughput_counts_every_rank():
    assert bench.throughput(1, 9, 1000.0) == pytest.approx(9.0)
    assert bench.throughput(4, 9, 2000.0) == pytest.approx(18.0)


def _worker(rank, world, port, times, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        m = bench.max_over_ranks(times[rank], dist, "cpu")
        out[rank] = (m, bench.rank_cells(rank, world))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_world_size_2():
    """Both ranks see the slower rank's time, as the JSON line's value requires."""
    import torch.multiprocessing as mp
    world = 2
    times = [123.5, 456.25]
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_worker, args=(world, _free_port(), times, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == max(times)
    assert sorted(res[0][1] + res[1][1]) == list(range(9))


def test_max_over_ranks_without_process_group():
    assert bench.max_over_ranks(7.5) == 7.5


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    """Under torchrun the reference arm (the oracle) runs on rank 0; other ranks return."""
    called = []
    monkeypatch.setattr(bench, "cpu_baseline", lambda *a, **k: called.append(1))

    class Args:
        warmup, steps = 1, 1
    bench.run_reference(Args(), 1, 2)
    assert called == []
