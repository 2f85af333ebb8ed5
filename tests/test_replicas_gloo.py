"""Host logic of the multi-GPU form (independent replicas, one per rank), run
as two gloo ranks on the CPU: the only cross-rank exchange is the whole-job
aggregation of the benchmark (units summed, time of the slowest rank), and
every rank draws replicas of its own."""
import os
import socket
import sys

import numpy as np
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    import workloads

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        units, ms = bench.aggregate(100.0 * (rank + 1), 10.0 + rank)
        reps = workloads.batch_replicas(2, first=2 * rank)
        out[rank] = (units, ms, [int(r["seed"]) for r in reps], [int(r["sites"][0]) for r in reps])
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_and_replica_seeds():
    world = 2
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        units, ms, seeds, first_sites = res[r]
        assert units == 300.0  # 100 + 200: every rank's units
        assert ms == 11.0  # the slower rank's time
    assert res[0][2] == [2000, 2001] and res[1][2] == [2002, 2003]
    assert res[0][3] != res[1][3]


def test_single_process_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.aggregate(5.0, 2.0) == (5.0, 2.0)
    # downward levels 2-4 in one launch plus levels 5 and 6, propose, finalize, select, record, move, 2 accept
    assert bench.launches_per_step(6) == 10
    assert np.isclose(bench.step_bytes(256, 6, 1 << 20, 12), 6 * (1 << 20) * 12 + 32768 * 512 * 16 + 32768 * 91 * 8)
