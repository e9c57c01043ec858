"""GPU parity of the table variant (MAP_TABLE, the paper's production route of
Section II-B): pyramid integrals interpolated in a pre-computed table.

The oracle runs the same algorithm (oracle.set_table: the same nodes, exact
trilinear interpolation in FP64).  The GPU interpolates with the texture
unit, whose weights carry 8 fractional bits: each lookup may differ from the
exact trilinear value by up to 3 * 2^-9 of the largest difference between
neighbouring nodes, a fraction of the interpolation error itself.  Gates,
per pair integral: the GPU's distance to the oracle's table variant is at
most half the oracle's own distance to the exact integrals (mean and 99th
percentile), and the GPU's distance to the exact integrals is within 20% of
the oracle's.  Pair lists are the exact rule's, bit for bit; the interior
particles' sum_i f_ai stays within the 0.6% the paper quotes for its table.
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import gpu_map, lib, oracle_h

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def uniform4096():
    p = synth.uniform_particles(4096, synth.BASE_SEED + 1)
    g = synth.voronoi(p.pos())
    h, _ = oracle_h(p)
    ex = oracle.map_cells(g, p.x, p.y, p.z, p.m, h)
    return p, g, h, ex


@pytest.mark.parametrize("n", [33, 64])
def test_table_variant_vs_oracle(uniform4096, n):
    p, g, h, ex = uniform4096
    L = lib()
    ctx = L.map_init(L.map_config_default(precision=L.MAP_TABLE, table_n=n))
    try:
        gt = gpu_map(g, p, h, L.MAP_TABLE, ctx=ctx)
    finally:
        L.map_destroy(ctx)
    try:
        oracle.set_table(n)
        ot = oracle.map_cells(g, p.x, p.y, p.z, p.m, h, off=ex["off"], idx=ex["idx"])
    finally:
        oracle.set_table(0)
    assert gt["status"] == 0
    assert np.array_equal(gt["off"], ex["off"]) and np.array_equal(gt["idx"], ex["idx"])
    d_go = np.abs(gt["frac"] - ot["frac"])
    d_oe = np.abs(ot["frac"] - ex["frac"])
    d_ge = np.abs(gt["frac"] - ex["frac"])
    assert d_go.mean() < 0.5 * d_oe.mean(), (d_go.mean(), d_oe.mean())
    assert np.percentile(d_go, 99) < 0.5 * np.percentile(d_oe, 99)
    assert d_ge.mean() < 1.2 * d_oe.mean() and np.percentile(d_ge, 99) < 1.2 * np.percentile(d_oe, 99)
    # mass conservation of the interior particles, against the paper's 0.6%
    pos = p.pos()
    interior = np.all((pos >= 2 * h[:, None]) & (pos <= 1 - 2 * h[:, None]), axis=1)
    tot = np.zeros(p.n)
    np.add.at(tot, gt["idx"], gt["frac"])
    assert np.abs(tot[interior] - 1).max() < 0.006
    # the cell masses are the sums of the pair integrals
    m_from_pairs = np.zeros(g.ncell)
    np.add.at(m_from_pairs, np.repeat(np.arange(g.ncell), np.diff(gt["off"])), p.m[gt["idx"]] * gt["frac"])
    assert np.max(np.abs(gt["mass"] - m_from_pairs) / m_from_pairs) < 1e-12


def test_table_variant_batch_equals_single(uniform4096):
    """Batches run the table variant too, with the same bits per snapshot."""
    p, g, h, _ = uniform4096
    import torch
    from gpu_helpers import dev_particles
    L = lib()
    ctx = L.map_init(L.map_config_default(precision=L.MAP_TABLE))
    try:
        single = gpu_map(g, p, h, L.MAP_TABLE, ctx=ctx)
        hd = L.map_grid_upload(ctx, L.grid_to_device(g))
        t = dev_particles(p, h)
        mass = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
        L.map_batch(ctx, [L.make_particles(*t)], [hd], [mass])
        torch.cuda.synchronize()
        assert np.array_equal(mass.cpu().numpy(), single["mass"])
    finally:
        L.map_destroy(ctx)


def test_table_n_out_of_range():
    L = lib()
    for n in (1, 513):
        with pytest.raises(L.MapError):
            L.map_init(L.map_config_default(precision=L.MAP_TABLE, table_n=n))
