"""The multi-GPU path is replicas only: each rank runs its own queries on
its own copy of the graph, with a barrier and a max over ranks around the
timed region and no data-path collective.  This checks that host logic of
bench.py with two gloo ranks on the CPU (127.0.0.1 rendezvous)."""
import multiprocessing as mp
import os
import socket

import pytest


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank: int, world: int, port: int, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    w, r, _ = bench.dist_setup()
    bench.barrier(w)
    slowest = bench.max_over_ranks(10.0 * (r + 1), w)
    g, seeds, tune_seeds = bench.workload(r, side=64, k=16)
    bench.barrier(w)
    dist.destroy_process_group()
    out.put((r, w, slowest, g.n, seeds.tolist(), tune_seeds.tolist()))


def test_two_replicas_over_gloo():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        results = sorted(out.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert all(p.exitcode == 0 for p in procs)
    (r0, w0, m0, n0, s0, t0), (r1, w1, m1, n1, s1, t1) = results
    assert (r0, r1) == (0, 1) and w0 == w1 == 2
    assert m0 == m1 == 20.0                 # both ranks see the slowest rank's time
    assert n0 == n1 == 64 * 64              # the same graph on every replica
    assert len(s0) == len(s1) == 16 and s0 != s1   # own queries of the same size
    assert len(set(s1)) == 16 and all(0 <= v < n1 for v in s1)
    # the autotuner's sample is another seed set of the same size
    assert len(t0) == len(t1) == 16 and t0 != s0 and t1 != s1 and t0 != t1


def test_single_process_needs_no_process_group(monkeypatch):
    for key in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(key, raising=False)
    import bench
    assert bench.dist_setup() == (1, 0, 0)
    assert bench.max_over_ranks(3.5, 1) == 3.5
    bench.barrier(1)
