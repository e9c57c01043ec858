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


# ----------------------------------------------------------------- one snapshot split over ranks

def _split_rank(rank, world, port, q):
    """One rank of the split: its shard of cells, its halo of particles, the
    oracle's mapping of the shard (a stand-in for the rank's GPU), the total
    mass all-reduced and the cell masses gathered on rank 0."""
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import sys
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    import synth
    from paper_2404_17084_gb300 import shard
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p = synth.lognormal_particles(1200, 20240426 + 9, ngrid=32)
        g = synth.voronoi(p.pos(), nthreads=1)
        h, _ = oracle.solve_h(p.x, p.y, p.z, oracle.particle_h_guess(oracle.Tree(p.x, p.y, p.z, p.m)), nthreads=1)
        sh = shard.make_shard(g, p.pos(), h, rank, world)
        a = sh.particles
        r = oracle.map_cells(sh.grid, p.x[a], p.y[a], p.z[a], p.m[a], h[a], nthreads=1)
        total = torch.tensor([float(r["mass"].sum())], dtype=torch.float64)
        dist.all_reduce(total)
        parts = [None] * world
        dist.all_gather_object(parts, (sh.cells.tolist(), r["mass"].tolist(), len(a)))
        q.put((rank, float(total.item()), parts))
    finally:
        dist.destroy_process_group()


def test_snapshot_split_over_two_gloo_ranks_is_exact():
    """Cells split by the Morton order of their sites, particles replicated
    where their support can reach a rank's cells: each rank's cell masses
    equal the single-rank mapping's bit for bit, every cell is mapped once,
    and the all-reduced total matches the single-rank total."""
    import sys
    sys.path.insert(0, ROOT)
    import numpy as np
    import oracle
    import synth
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_split_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    out = sorted(q.get(timeout=300) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = synth.lognormal_particles(1200, 20240426 + 9, ngrid=32)
    g = synth.voronoi(p.pos(), nthreads=1)
    h, _ = oracle.solve_h(p.x, p.y, p.z, oracle.particle_h_guess(oracle.Tree(p.x, p.y, p.z, p.m)), nthreads=1)
    ref = oracle.map_cells(g, p.x, p.y, p.z, p.m, h, nthreads=1)["mass"]
    (_, tot0, parts0), (_, tot1, parts1) = out
    assert tot0 == tot1 and abs(tot0 - ref.sum()) < 1e-14 * ref.sum()
    assert parts0 == parts1
    seen = np.zeros(g.ncell, int)
    for cells, mass, nhalo in parts0:
        cells = np.array(cells)
        seen[cells] += 1
        assert np.array_equal(np.array(mass), ref[cells])  # bit for bit
        assert 0 < nhalo < p.n                             # a halo, not the whole set
    assert np.all(seen == 1)
