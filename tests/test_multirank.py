"""Multi-rank host logic of bench.py on CPU: two gloo ranks, one process each.
Each rank maps its own snapshot (distinct seeds: weak scaling, no data-path
collective), the job's time is the slowest rank's, and only rank 0 prints."""
import importlib.util
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    b = _bench()
    r, w, local = b.dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        seed = b.rank_seed(20240426 + 2, r)
        ms = b.max_over_ranks(10.0 + 5.0 * r, w)          # rank 1 is the slow one
        seeds = [None] * w
        dist.all_gather_object(seeds, seed)
        printed = b.emit({"rank": r}, r)
        q.put((r, ms, seeds, printed))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, ms0, seeds0, pr0), (r1, ms1, seeds1, pr1) = out
    assert ms0 == ms1 == 15.0                 # max over ranks, seen by both
    assert seeds0 == seeds1 and seeds0[0] != seeds0[1]
    assert pr0 is True and pr1 is False       # one JSON line, from rank 0


def test_single_rank_defaults():
    b = _bench()
    assert b.max_over_ranks(3.5, 1) == 3.5
    assert b.rank_seed(7, 0) == 7
