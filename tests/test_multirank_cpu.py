"""The multi-rank bench logic on CPU with the gloo backend (world size 2):
ranks own disjoint streams and the reported time is the slowest rank's.
The streams shard with no data exchange, so nothing else crosses ranks."""
import os
import socket

import numpy as np
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


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seeds = bench.rank_seeds(rank)
    gathered = [None] * world
    dist.all_gather_object(gathered, (int(seeds[0]), int(seeds[-1]), int(seeds.size)))
    t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
    q.put((rank, gathered, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_streams_and_take_the_slowest_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, gathered, t in out:
        assert t == pytest.approx(2.5)
        (a0, a1, an), (b0, b1, bn) = gathered
        assert an == bn == 16384
        assert a1 < b0  # disjoint, consecutive seed ranges
        assert b0 == a0 + 16384


def test_bench_gpus_flag_launches_ranks():
    """`bench.py --gpus 2` without an outer launcher starts two ranks (here
    in its launcher-check mode, gloo, no GPU work): rank 0 sees both, their
    seeds are disjoint, and the time is the slowest rank's."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items()
           if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK", "MASTER_ADDR", "MASTER_PORT")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--rank-check"],
                       capture_output=True, text=True, timeout=300, env=env, cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads([l for l in r.stdout.splitlines() if l.startswith("{")][-1])
    assert line["n_gpus"] == 2 and line["requested"] == 2
    ranks = sorted(line["ranks"])
    assert [x[0] for x in ranks] == [0, 1]
    (_, a0, a1, an), (_, b0, b1, bn) = ranks
    assert an == bn == 16384 and a1 < b0 and b0 == a0 + 16384
    assert line["max_ms"] == pytest.approx(2.0)
