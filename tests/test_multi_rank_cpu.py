"""The N > 1 path of bench.py on CPU: two gloo ranks (no GPU).

Instances are independent, so ranks shard the batch with disjoint seeds and
exchange nothing but the slowest rank's time (weak scaling)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as tdist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    tdist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    wl = bench.WORKLOADS["n256_beta20"]
    seeds = bench.rank_seeds(wl, rank, 4)
    local_ms = 100.0 * (rank + 1)
    mx = bench.reduce_max(local_ms)
    gathered = [None] * world
    tdist.all_gather_object(gathered, seeds)
    q.put((rank, mx, gathered, bench.job_value(4, world, 2, mx)))
    tdist.destroy_process_group()


def test_two_gloo_ranks_shard_and_reduce():
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, gathered, value in out:
        assert mx == 200.0                       # slowest rank's time
        s0, s1 = set(gathered[0]), set(gathered[1])
        assert len(s0) == 4 and len(s1) == 4 and not (s0 & s1)
        assert value == pytest.approx(4 * 2 * 2 / 0.2)


def test_single_process_reduce_is_identity():
    import bench
    assert bench.reduce_max(3.5) == 3.5
