"""Host logic of bench.py's multi-GPU run, on CPU.

The method has no data-path collective (every problem is independent, so
N GPUs run N replicas); the only cross-rank step is the aggregation of the
timed region: the slowest rank's time and the sum of the units all ranks
processed.  It runs here as two gloo ranks on 127.0.0.1."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, l = bench.dist_env()
        elapsed, units = bench.aggregate_over_ranks(dist, 10.0 * (rank + 1), 1e6 * (rank + 1))
        q.put((r, w, elapsed, units))
    finally:
        dist.destroy_process_group()


def test_two_replicas_aggregate_slowest_time_and_all_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, world, elapsed, units) in enumerate(out):
        assert (rank, world) == (r, 2)
        assert elapsed == 20.0            # the slower rank
        assert units == 3e6               # both ranks' work


def test_single_process_aggregate_is_identity():
    assert bench.aggregate_over_ranks(None, 1.5, 42.0) == (1.5, 42.0)


@pytest.mark.parametrize("s,launches", [(2, 2), (3, 3), (4, 3), (5, 4), (20, 11), (21, 12)])
def test_two_stage_launch_count(s, launches):
    """Two-stage schedule: stage 1, pairs (j, j+1) while j + 1 < s, then the
    remaining stages one by one (the last one writes T in place)."""
    assert bench.stage_launches_per_step(5, s) == launches
    assert bench.stage_launches_per_step(0, s) == s
