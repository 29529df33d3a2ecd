"""Sharding a batch's instance list over ranks (host logic, CPU): the partition covers
every instance exactly once and balances the updates per step, every rank computes the
same one, and the host gather returns each rank's per-instance results in global order
(gloo, world size 2)."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from paper_1702_01335_gb300.lbs import Instance  # noqa: E402
from paper_1702_01335_gb300.shard import cost, gather, partition, shard  # noqa: E402


def _sweep():
    return [Instance(**p) for p in W.sweep(64, W.SWEEP_SEED)]


@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_partition_covers_once_and_balances(world):
    inst = _sweep()
    parts = partition(inst, world)
    assert len(parts) == world
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(inst)))
    assert all(p == sorted(p) for p in parts)
    loads = [sum(cost(inst[i]) for i in p) for p in parts]
    mean = sum(loads) / world
    assert max(loads) <= mean + max(cost(i) for i in inst)  # the rule's bound
    assert [shard(inst, r, world) for r in range(world)] == parts


def test_partition_edge_cases():
    inst = [Instance(Nz=32), Instance(Nz=64), Instance(Nz=32)]
    assert partition(inst, 1) == [[0, 1, 2]]
    # more ranks than instances: some ranks own nothing; largest first, ties by index
    assert partition(inst, 4) == [[1], [0], [2], []]
    assert partition([], 3) == [[], [], []]
    # equal weights: round robin in index order
    same = [Instance()] * 6
    assert partition(same, 3) == [[0, 3], [1, 4], [2, 5]]
    with pytest.raises(ValueError):
        partition(inst, 0)
    with pytest.raises(ValueError):
        shard(inst, 2, 2)


def test_gather_single_rank_and_checks():
    assert gather(["a", "b"], [1, 0], 2) == ["b", "a"]
    with pytest.raises(ValueError):
        gather(["a"], [0], 2)          # instance 1 owned by nobody
    with pytest.raises(ValueError):
        gather(["a", "b"], [0, 0], 2)  # owned twice
    with pytest.raises(ValueError):
        gather(["a"], [0, 1], 2)       # one result per index


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        inst = _sweep()
        idx = shard(inst, rank, world)
        local = [(i, cost(inst[i]), rank) for i in idx]  # a per-instance result
        q.put((rank, idx, gather(local, idx, len(inst), dist)))
    finally:
        dist.destroy_process_group()


def test_gather_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = dict()
    for _ in ps:
        r, idx, out = q.get(timeout=120)
        got[r] = (idx, out)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    inst = _sweep()
    owner = {i: r for r in (0, 1) for i in got[r][0]}
    assert sorted(owner) == list(range(len(inst)))
    for r in (0, 1):
        out = got[r][1]
        assert [o[0] for o in out] == list(range(len(inst)))
        assert all(o[1] == cost(inst[o[0]]) and o[2] == owner[o[0]] for o in out)
