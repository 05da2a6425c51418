"""The multi-process path of bench.py on CPU: two gloo ranks split a global batch by sample
(disjoint shares that cover it, no collective on the data) and agree on the max of their
timings."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    from paper_2504_01302_b300 import shard, synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        th, sid = synth.workload_thetas(3, world * 16, 8)
        mine_th, mine_sid = shard.shard(th, sid, rank, world)
        shares = [None] * world
        dist.all_gather_object(shares, (mine_th, mine_sid))
        t = shard.max_over_ranks(10.0 + rank, dist)
        q.put((rank, shares, t, th, sid))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_the_batch():
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, shares, t, th, sid in out:
        assert t == 11.0  # max over ranks
        got_th = np.concatenate([s[0] for s in shares])
        got_sid = np.concatenate([s[1] for s in shares])
        assert np.array_equal(got_th, th) and np.array_equal(got_sid, sid)
        assert shares[0][0].shape[0] == shares[1][0].shape[0] == 16


def test_uneven_split_is_refused():
    from paper_2504_01302_b300 import shard
    with pytest.raises(ValueError):
        shard.shard(np.zeros((5, 20)), np.zeros(5, np.int32), 0, 2)
