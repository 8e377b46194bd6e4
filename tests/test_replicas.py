"""Multi-process (world size 2, gloo on CPU) checks of the replica logic that
bench.py uses for N > 1 GPUs: each rank solves its own energy point, the job
time is the slowest rank's, the job rate counts every rank's points, and the
shares of independent points partition the set."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2601_04904_gb300 import replicas  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        r, w, local = replicas.env()
        per_rank_time = 1.0 + rank  # rank 1 is the slower one
        t = replicas.max_over_ranks(per_rank_time, dist)
        dist.barrier()
        out[rank] = {"env": (r, w, local), "t": t, "rate": replicas.job_rate(w, 3, t),
                     "energy": replicas.energy_of(r), "seed": replicas.rhs_seed(r),
                     "shard": list(replicas.shard(10, r, w))}
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_gloo():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0]["env"] == (0, 2, 0) and res[1]["env"] == (1, 2, 1)
    # both ranks see the slowest rank's time; the rate counts both ranks' points
    assert res[0]["t"] == res[1]["t"] == 2.0
    assert res[0]["rate"] == res[1]["rate"] == 2 * 3 / 2.0
    # rank 0 keeps the benchmark's energy; the replicas solve different points
    assert res[0]["energy"] == 0.3 and res[1]["energy"] != 0.3 and -1.0 <= res[1]["energy"] <= 1.0
    assert res[0]["seed"] != res[1]["seed"]
    # shares of independent points: disjoint, contiguous, covering
    assert sorted(res[0]["shard"] + res[1]["shard"]) == list(range(10))
    assert not set(res[0]["shard"]) & set(res[1]["shard"])


@pytest.mark.parametrize("n,world", [(0, 3), (1, 4), (7, 3), (256, 8), (255, 8)])
def test_shard_partition(n, world):
    parts = [list(replicas.shard(n, r, world)) for r in range(world)]
    assert sum(parts, []) == list(range(n))
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 1


def test_single_process_reduction_is_identity():
    assert replicas.max_over_ranks(1.5) == 1.5
    assert replicas.job_rate(1, 4, 2.0) == 2.0
