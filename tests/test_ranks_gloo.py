"""The multi-process host path on CPU: two gloo ranks agree on the work split
and on the slowest rank's time, as bench.py's one-process-per-GPU runs do."""
import os
import socket

import pytest

from paper_2403_03571_gb300 import ranks

torch = pytest.importorskip("torch")


def test_shard_covers_units_once():
    for count in (0, 1, 7, 256, 1000):
        for world in (1, 2, 3, 8):
            parts = [ranks.shard(count, r, world) for r in range(world)]
            flat = [u for p in parts for u in p]
            assert flat == list(range(count))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
    with pytest.raises(ValueError):
        ranks.shard(5, 2, 2)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, w, lr = ranks.rank_world()
    mine = ranks.shard(256, r, w)
    slowest = ranks.max_over_ranks(10.0 + r)
    total = ranks.sum_over_ranks(len(mine))
    dist.barrier()
    out.put((r, w, lr, mine[0], len(mine), slowest, total))
    dist.destroy_process_group()


def test_two_gloo_ranks_agree():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[:3] for r in res] == [(0, 2, 0), (1, 2, 1)]
    assert [(r[3], r[4]) for r in res] == [(0, 128), (128, 128)]
    assert all(r[5] == 11.0 for r in res)      # slowest rank's time everywhere
    assert all(r[6] == 256.0 for r in res)     # units of the whole job


def test_single_process_defaults(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert ranks.rank_world() == (0, 1, 0)
    assert ranks.max_over_ranks(3.5) == 3.5
    assert ranks.sum_over_ranks(2.0) == 2.0
