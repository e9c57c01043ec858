"""Batched mapping (many uneven snapshots in one persistent launch): every
snapshot's result equals the single-snapshot mapping of the same input, bit
for bit (each cell is computed by one warp in a fixed order, whatever the
launch), and the FP64 build matches the oracle."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import lib, dev_particles, gpu_map, oracle_h, rel_err, sample_cells

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def snapshots():
    """Six snapshots, 2^9..2^12 particles, uniform and clumpy (sigma 1-2)."""
    out = []
    for spec in synth.batch_specs(6, synth.BASE_SEED + 4, 9.0, 12.0):
        p = synth.batch_particles(spec)
        g = synth.voronoi(p.pos())
        h, _ = oracle_h(p)
        out.append((spec, p, g, h))
    return out


def run_batch(snaps, precision, autotune=0, repeat=1):
    L = lib()
    ctx = L.map_init(L.map_config_default(precision=precision, autotune=autotune))
    try:
        handles, parts, keep, mass = [], [], [], []
        for _, p, g, h in snaps:
            handles.append(L.map_grid_upload(ctx, L.grid_to_device(g)))
            t = dev_particles(p, h)
            keep.append(t)
            parts.append(L.make_particles(*t))
            mass.append(torch.full((g.ncell,), -1.0, dtype=torch.float64, device="cuda"))
        totals = torch.zeros(len(snaps), dtype=torch.float64, device="cuda")
        runs = []
        for _ in range(repeat):
            L.map_batch(ctx, parts, handles, mass, totals=totals)
            torch.cuda.synchronize()
            runs.append(([m.cpu().numpy().copy() for m in mass], totals.cpu().numpy().copy()))
        st = L.map_get_stats(ctx)
        tune = L.map_get_autotune(ctx)
        return runs, st, tune
    finally:
        L.map_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_single(snapshots, precision):
    runs, st, _ = run_batch(snapshots, precision)
    masses, totals = runs[0]
    n_pairs = 0
    for j, (_, p, g, h) in enumerate(snapshots):
        single = gpu_map(g, p, h, precision)
        assert np.array_equal(masses[j], single["mass"]), j
        assert totals[j] == pytest.approx(single["total"], rel=1e-14, abs=0)
        n_pairs += single["n_pairs"]
    assert st.n_pairs == n_pairs
    assert st.total_mass == pytest.approx(float(np.sum(totals)), rel=1e-14)


def test_batch_autotune_and_replay(snapshots):
    """The autotuner times every pair of a work-item size (3) and a launch
    shape (4) and keeps one; each shape launches as many CTAs per SM as it
    names, all resident at once.  Replays of the captured graph give the same
    bits; another shape or item size (a separate compilation, other groups of
    a cell's pairs) agrees to FP32 rounding."""
    L = lib()
    ref, _, _ = run_batch(snapshots, 1)
    runs, _, (chosen, ms) = run_batch(snapshots, 1, autotune=1, repeat=3)
    assert len(ms) == len(L.AUTOTUNE_SHAPES) * len(L.AUTOTUNE_ITEM_TARGETS) == 12
    ctx = L.map_init(L.map_config_default())
    try:
        shapes = L.map_autotune_shapes(ctx)
    finally:
        L.map_destroy(ctx)
    assert [(s["warps_per_cta"], s["ctas_per_sm"]) for s in shapes] == [(4, 5), (4, 4), (2, 9), (8, 2)]
    assert all(0 < s["registers"] <= 65536 // (32 * s["warps_per_cta"] * s["ctas_per_sm"]) for s in shapes)
    assert 0 <= chosen < len(ms) and all(t > 0 for t in ms)
    for masses, totals in runs[1:]:
        for a, b in zip(masses, runs[0][0]):
            assert np.array_equal(a, b)
        assert np.array_equal(totals, runs[0][1])
    worst = max(rel_err(a, b).max() for a, b in zip(runs[0][0], ref[0][0]))
    assert worst < 1e-6, worst


def test_batch_fp64_vs_oracle(snapshots):
    runs, _, _ = run_batch(snapshots, 0)
    masses, _ = runs[0]
    for j in (0, len(snapshots) - 1):
        _, p, g, h = snapshots[j]
        cells = sample_cells(g.ncell, 60, j)
        ref = oracle.map_cells(g, p.x, p.y, p.z, p.m, h, cells=cells)
        assert rel_err(masses[j][cells], ref["mass"]).max() < 1e-9


@pytest.mark.parametrize("precision", [0, 1])
def test_solve_h_batch_equals_single(snapshots, precision):
    """solve_h_batch (the sets solved by the context's workers, several at
    once) gives every set the h and routes of solve_h on it alone, bit for
    bit."""
    L = lib()
    ctx = L.map_init(L.map_config_default(precision=precision))
    try:
        sets = [dev_particles(p) for _, p, _, _ in snapshots]
        routes = [torch.empty(p.n, dtype=torch.int32, device="cuda") for _, p, _, _ in snapshots]
        L.solve_h_batch(ctx, [L.make_particles(x, y, z, None, h) for x, y, z, _, h in sets], routes)
        torch.cuda.synchronize()
        got = [(t[4].cpu().numpy().copy(), r.cpu().numpy().copy()) for t, r in zip(sets, routes)]
        for j, (x, y, z, _, _) in enumerate(sets):
            h1 = torch.empty_like(x)
            r1 = torch.empty_like(routes[j])
            L.solve_h(ctx, L.make_particles(x, y, z, None, h1), r1)
            torch.cuda.synchronize()
            assert np.array_equal(got[j][0], h1.cpu().numpy()), j
            assert np.array_equal(got[j][1], r1.cpu().numpy()), j
    finally:
        L.map_destroy(ctx)


@pytest.mark.parametrize("precision", [1, 0])
def test_batch_whole_step_graph(snapshots, precision):
    """After an eager call the whole step (validation, octrees, pair lists,
    work items, the integral launch, the sums) is captured once; calls on the
    same buffers replay it, computing from the buffers' current values: new
    positions give the single-snapshot results on those positions bit for
    bit; lists that outgrow their buffers (h raised) fall back to the eager
    step and capture anew; an invalid particle is refused."""
    L = lib()
    ctx = L.map_init(L.map_config_default(precision=precision))
    try:
        handles, parts, keep, mass = [], [], [], []
        for _, p, g, h in snapshots:
            handles.append(L.map_grid_upload(ctx, L.grid_to_device(g)))
            t = dev_particles(p, h)
            keep.append(t)
            parts.append(L.make_particles(*t))
            mass.append(torch.full((g.ncell,), -1.0, dtype=torch.float64, device="cuda"))
        totals = torch.zeros(len(snapshots), dtype=torch.float64, device="cuda")

        def call():
            L.map_batch(ctx, parts, handles, mass, totals=totals)
            torch.cuda.synchronize()
            return [m.cpu().numpy().copy() for m in mass], totals.cpu().numpy().copy()

        first, t1 = call()
        assert L.map_batch_graph_stats(ctx) == (1, 0, 0)
        for m in mass:
            m.fill_(-1.0)
        again, t2 = call()
        assert L.map_batch_graph_stats(ctx) == (1, 1, 0)
        for a, b in zip(first, again):
            assert np.array_equal(a, b)
        assert np.array_equal(t1, t2)
        assert L.map_get_stats(ctx).n_pairs == sum(gpu_map(g, p, h, precision)["n_pairs"] for _, p, g, h in snapshots)

        # new positions in the same buffers: moved by up to 1e-3, kept in the cube
        rng = np.random.default_rng(5)
        moved = []
        for (_, p, g, h), t in zip(snapshots, keep):
            q = synth.Particles(*(np.clip(c + rng.uniform(-1e-3, 1e-3, p.n), 0.0, 1.0) for c in (p.x, p.y, p.z)), p.m)
            for dst, src in zip(t[:3], (q.x, q.y, q.z)):
                dst.copy_(torch.as_tensor(src, device="cuda"))
            moved.append(q)
        got, _ = call()
        assert L.map_batch_graph_stats(ctx) == (1, 2, 0)
        for j, (_, p, g, h) in enumerate(snapshots):
            assert np.array_equal(got[j], gpu_map(g, moved[j], h, precision)["mass"]), j

        # h raised 1.6x: about 4x the pairs, beyond the captured buffers
        for t in keep:
            t[4].mul_(1.6)
        grown, _ = call()
        assert L.map_batch_graph_stats(ctx) == (2, 2, 1)
        for j, (_, p, g, h) in enumerate(snapshots):
            assert np.array_equal(grown[j], gpu_map(g, moved[j], 1.6 * h, precision)["mass"]), j

        # an invalid particle: refused by the replay, the graph kept
        keep[0][4][0] = float("nan")
        with pytest.raises(L.MapError) as e:
            call()
        assert e.value.code == L.MAP_EINVAL
        keep[0][4][0] = float(1.6 * snapshots[0][3][0])
        again2, _ = call()
        assert L.map_batch_graph_stats(ctx) == (2, 3, 1)  # the refused call counts as no replay
        for a, b in zip(grown, again2):
            assert np.array_equal(a, b)
    finally:
        L.map_destroy(ctx)


def test_solve_h_batch_graph_replay(snapshots):
    """solve_h_batch captures its step after the first call; a call on the
    same buffers with moved positions replays it and gives solve_h's h and
    routes on the moved sets, bit for bit; an out-of-cube position is
    refused by the replay."""
    L = lib()
    ctx = L.map_init(L.map_config_default(precision=1))
    try:
        sets = [dev_particles(p) for _, p, _, _ in snapshots]
        routes = [torch.empty(p.n, dtype=torch.int32, device="cuda") for _, p, _, _ in snapshots]
        hp = [L.make_particles(x, y, z, None, h) for x, y, z, _, h in sets]
        L.solve_h_batch(ctx, hp, routes)
        assert L.solve_h_batch_graph_stats(ctx) == (1, 0)
        rng = np.random.default_rng(7)
        for (x, y, z, _, _), (_, p, _, _) in zip(sets, snapshots):
            for t in (x, y, z):
                t.copy_(torch.clamp(t + torch.as_tensor(rng.uniform(-1e-3, 1e-3, p.n), device="cuda"), 0.0, 1.0))
        L.solve_h_batch(ctx, hp, routes)
        torch.cuda.synchronize()
        assert L.solve_h_batch_graph_stats(ctx) == (1, 1)
        got = [(t[4].cpu().numpy().copy(), r.cpu().numpy().copy()) for t, r in zip(sets, routes)]
        ref_ctx = L.map_init(L.map_config_default(precision=1))
        try:
            for j, (x, y, z, _, _) in enumerate(sets):
                h1 = torch.empty_like(x)
                r1 = torch.empty_like(routes[j])
                L.solve_h(ref_ctx, L.make_particles(x, y, z, None, h1), r1)
                torch.cuda.synchronize()
                assert np.array_equal(got[j][0], h1.cpu().numpy()), j
                assert np.array_equal(got[j][1], r1.cpu().numpy()), j
        finally:
            L.map_destroy(ref_ctx)
        sets[1][0][3] = 1.5
        with pytest.raises(L.MapError) as e:
            L.solve_h_batch(ctx, hp, routes)
        assert e.value.code == L.MAP_EINVAL
    finally:
        L.map_destroy(ctx)
