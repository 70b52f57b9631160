"""The multi-GPU path on CPU: two gloo ranks, no GPU.

Each rank answers its own share of the queries with the oracle; gathered on
rank 0 the results equal a single-process run (queries are independent, so
sharding changes nothing), and the timing reduction takes the slowest rank."""
import os

import numpy as np
import pytest
import torch.multiprocessing as mp


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import oracle
    import rrsynth
    from paper_2502_13245_gb300 import multi
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg = rrsynth.small_config("mr", n=1500, nq=41, d=32, R=16, L=32, n_centres=6, fam_cap=100, seed=21)
        ds = rrsynth.make_dataset(cfg)
        oi = oracle.Index(ds.X, ds.adj, ds.start)
        lo, hi = multi.shard_bounds(len(ds.Q), world, rank)
        ids, _, _ = oracle.range_search(oi, ds.Q[lo:hi], ds.radius, "greedy_es", beam=16)
        gathered = [None] * world
        dist.all_gather_object(gathered, (lo, hi, [x.tolist() for x in ids]))
        mx = multi.reduce_max(10.0 + rank)
        if rank == 0:
            q.put((gathered, mx))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process():
    import socket

    import oracle
    import rrsynth
    from paper_2502_13245_gb300 import multi
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    gathered, mx = q.get(timeout=300)
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    assert mx == 11.0
    cfg = rrsynth.small_config("mr", n=1500, nq=41, d=32, R=16, L=32, n_centres=6, fam_cap=100, seed=21)
    ds = rrsynth.make_dataset(cfg)
    oi = oracle.Index(ds.X, ds.adj, ds.start)
    ref, _, _ = oracle.range_search(oi, ds.Q, ds.radius, "greedy_es", beam=16)
    merged = [None] * len(ds.Q)
    covered = 0
    for lo, hi, lists in gathered:
        assert hi - lo == len(lists)
        covered += hi - lo
        for k, lst in enumerate(lists):
            merged[lo + k] = lst
    assert covered == len(ds.Q)
    for a, b in zip(merged, ref):
        assert a == b.tolist()


@pytest.mark.parametrize("nq,world", [(10, 3), (7, 8), (0, 2), (100, 4)])
def test_shard_bounds_partition(nq, world):
    from paper_2502_13245_gb300 import multi
    parts = [multi.shard_bounds(nq, world, r) for r in range(world)]
    assert parts[0][0] == 0 and parts[-1][1] == nq
    for (a, b), (c, d) in zip(parts, parts[1:]):
        assert b == c and b >= a
    sizes = [b - a for a, b in parts]
    assert max(sizes) - min(sizes) <= 1
    assert multi.job_throughput(10, 4, 100.0) == pytest.approx(400.0)
    assert len({multi.rank_query_seed(5, r) for r in range(8)}) == 8
