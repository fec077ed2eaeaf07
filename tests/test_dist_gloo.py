"""Multi-rank host logic of bench.py on CPU: two gloo ranks.

The solve path has no collective (ensembles are independent; each rank
solves its own samples), so what needs checking with world size 2 is the
host side: disjoint, covering sample shards; the max-over-ranks timing;
the whole-job throughput; and the reference arm doing its work on rank 0
only.  No GPU is used.
"""
import multiprocessing as mp
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    try:
        import torch
        import torch.distributed as dist
        import bench
        dist.init_process_group("gloo", rank=rank, world_size=world)
        w, r, _ = bench.dist_setup()
        per_rank, s = 64, 32
        xi = bench.rank_xi(r, per_rank, s)
        first = bench.shard_first_sample(r, per_rank)
        # every rank sees every shard's first sample index (all-gather)
        firsts = [torch.zeros(1, dtype=torch.int64) for _ in range(w)]
        dist.all_gather(firsts, torch.tensor([first], dtype=torch.int64))
        # each rank reports its own time; all must agree on the slowest
        ms = bench.max_over_ranks(100.0 + 50.0 * r, w)
        value = bench.job_throughput(w, 3, per_rank, ms)
        # the reference arm: rank 0 does the work, the others return at once
        bench.cpu_baseline_run = lambda ns=None, nthreads=None: {
            "value": 1.0, "unit": bench.UNIT, "cores": 1, "kind": "oracle", "sample": "stub", "seconds": 1.0}

        class A:
            steps, warmup, s, spmv = 1, 0, 32, "dfv"
        ref = bench.main_reference(A())
        dist.barrier()
        dist.destroy_process_group()
        q.put((r, w, xi, [int(f) for f in firsts], ms, value, ref is not None))
    except Exception as e:  # report instead of hanging the parent
        q.put((rank, "error", repr(e)))


def test_two_gloo_ranks_shard_and_time():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
    assert all(p.exitcode == 0 for p in procs)
    for item in res:
        assert item[1] != "error", item
    res = sorted(res, key=lambda t: t[0])
    import bench
    from paper_1511_03703_gb300 import inputs
    xs_all = inputs.kl_samples(inputs.SEED_SCALE, 0, world * 64, bench.M_KL)
    for r, w, xi, firsts, ms, value, did_ref in res:
        assert w == world and firsts == [0, 64]
        # rank r's ensembles hold samples r*64 .. r*64+63, commuted layout
        expect = np.stack([inputs.ensemble_layout(b) for b in xs_all[r * 64:(r + 1) * 64].reshape(2, 32, -1)])
        assert np.array_equal(xi, expect)
        assert ms == 150.0                      # the slowest rank's time on every rank
        assert value == pytest.approx(world * 3 * 64 / 0.150)
        assert did_ref == (r == 0)
