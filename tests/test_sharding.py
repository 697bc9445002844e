"""Host logic of multi-GPU runs (CPU): the scene split between ranks and the timing
reduction, the latter with two gloo processes on 127.0.0.1."""
import os
import socket

import pytest

from paper_2403_11156_gb300 import scenes
from paper_2403_11156_gb300.sharding import reduce_timing, shard_scenes


def test_split_covers_every_scene_once_and_balances():
    sizes = scenes.batch_scene_sizes()
    for world in (1, 2, 3, 4, 8):
        parts = shard_scenes(sizes, world)
        flat = sorted(k for p in parts for k in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[k] for k in p) for p in parts]
        # greedy bound: no rank exceeds the mean by more than the largest scene
        assert max(loads) - sum(loads) / world <= max(sizes)
    assert shard_scenes([5, 1, 4], 2) == [[0], [1, 2]]
    assert shard_scenes([], 2) == [[], []]
    with pytest.raises(ValueError):
        shard_scenes([1], 0)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sizes = scenes.batch_scene_sizes()
        mine = shard_scenes(sizes, world)[rank]
        units = float(sum(sizes[k] for k in mine))
        ms, total = reduce_timing(10.0 + rank, units, world)
        out.put((rank, ms, total, mine))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_timing():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sizes = scenes.batch_scene_sizes()
    for rank, ms, total, mine in res:
        assert ms == 11.0                      # slowest rank
        assert total == float(sum(sizes))      # every scene stepped once
    assert sorted(res[0][3] + res[1][3]) == list(range(len(sizes)))
    assert reduce_timing(3.0, 7.0, 1) == (3.0, 7.0)
