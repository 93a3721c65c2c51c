"""The multi-rank bench path on CPU (gloo, world size 2): each rank gets its
own shard of generator streams (distinct generator IDs and seeds, so no two
ranks produce the same numbers; no data-path collective), the job time is
the max over ranks, and each rank's shard checks out against the oracle."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        import oracle as O
        wl = bench.workload("c2s", rank)
        ids = torch.tensor([g.gen_id for g in wl.gens], dtype=torch.int64)
        seeds = torch.tensor([g.seed for g in wl.gens], dtype=torch.int64)
        got_ids = [torch.zeros_like(ids) for _ in range(world)]
        got_seeds = [torch.zeros_like(seeds) for _ in range(world)]
        dist.all_gather(got_ids, ids)
        dist.all_gather(got_seeds, seeds)
        slowest = bench.max_over_ranks(torch, dist, 10.0 + rank, "cpu")
        # this rank's first generator, a short prefix, from the oracle
        g = wl.gens[0]
        p = O.params_draw(g.mexp, g.param_seed, g.id)
        head = O.generate(p, O.seed_state(p, g.gen_id, g.seed), 64, 0)
        heads = [torch.zeros(64, dtype=torch.int64) for _ in range(world)]
        dist.all_gather(heads, torch.from_numpy(head.astype(np.int64)))
        q.put((rank, [t.tolist() for t in got_ids], [t.tolist() for t in got_seeds], slowest,
               [h.tolist() for h in heads]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_shard_generators_and_take_the_max_time():
    import oracle as O
    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ids, seeds, slowest, heads in res:
        assert slowest == 11.0                           # max over ranks
        assert not set(ids[0]) & set(ids[1])             # disjoint generator IDs
        assert len(set(ids[0])) == len(ids[0]) // 3      # three dtype instances per set on each rank
        assert seeds[0] != seeds[1]
        assert heads[0] != heads[1]                      # the shards are different streams
