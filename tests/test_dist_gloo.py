"""N > 1 path on CPU with the gloo backend (world size 2): the systems of a
batch are sharded by cell count with no data-path collective; each rank
solves its share (here with the oracle, as no GPU is involved) and only the
per-system results and the max time are exchanged.  The union of the shards
must reproduce the single-process results exactly."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2009_13916_gb300.dist import partition_by_weight


def test_partition_covers_and_balances():
    rng = np.random.default_rng(3)
    w = rng.integers(16, 49, size=37) ** 3
    for world in (1, 2, 3, 8):
        ranges = [partition_by_weight(w, world, r) for r in range(world)]
        assert ranges[0][0] == 0 and ranges[-1][1] == len(w)
        for a, b in zip(ranges, ranges[1:]):
            assert a[1] == b[0]
        loads = [w[s:e].sum() for s, e in ranges]
        # contiguous ranges: each boundary sits within half an item of its target
        assert max(loads) - min(loads) <= 2 * w.max()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist

    import oracle as O
    import workloads as W
    from paper_2009_13916_gb300.dist import gather_objects, max_over_ranks
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sizes = [4, 6, 5, 7, 3]
    w = [n ** 3 for n in sizes]
    s, e = partition_by_weight(w, world, rank)
    mine = {}
    for i in range(s, e):
        sysd = W.config4_system(200 + i, sizes[i])
        r = O.edfa_pipeline(sysd, mode="nbr")
        mine[i] = (r["iters"], float(r["true_rel"]))
    allres = gather_objects(mine)
    tmax = max_over_ranks(float(rank + 1) * 1.5)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, allres, tmax))


def test_two_ranks_shard_batch_with_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle as O
    import workloads as W
    sizes = [4, 6, 5, 7, 3]
    ref = {}
    for i, n in enumerate(sizes):
        r = O.edfa_pipeline(W.config4_system(200 + i, n), mode="nbr")
        ref[i] = (r["iters"], float(r["true_rel"]))
    for rank, allres, tmax in out:
        merged = {}
        for d in allres:
            assert not (set(d) & set(merged))
            merged.update(d)
        assert merged == ref
        assert tmax == 3.0
