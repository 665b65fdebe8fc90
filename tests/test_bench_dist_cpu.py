"""The multi-rank logic of bench.py on CPU: two gloo ranks (world size 2) shard independent
units, gather their records and take the maximum time over ranks, as bench.py does under
torchrun on N GPUs."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = list(bench.shard(11, world, rank))
    rec = [{"seed": s, "rank": rank} for s in mine]
    allrec = bench.gather_records(rec, world)
    t = bench.max_over_ranks(float(rank + 1) * 1.5, world)
    out[rank] = {"mine": mine, "seeds": [x["seed"] for x in allrec],
                 "owners": [x["rank"] for x in allrec], "max": t}
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_gather_and_max():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert sorted(res[0]["mine"] + res[1]["mine"]) == list(range(11))
    assert not set(res[0]["mine"]) & set(res[1]["mine"])
    for r in range(world):
        assert res[r]["seeds"] == list(range(11))
        assert res[r]["owners"] == [s % 2 for s in range(11)]
        assert res[r]["max"] == 3.0


def test_single_rank_paths_need_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert list(bench.shard(5, 1, 0)) == [0, 1, 2, 3, 4]
    assert bench.gather_records([{"seed": 2}, {"seed": 1}], 1) == [{"seed": 1}, {"seed": 2}]
    assert bench.max_over_ranks(4.5, 1) == 4.5
