"""Parity at the full size the bench times: the clumpy cloud of 2^20 equal-mass
particles on its 2^20-cell clipped Voronoi grid, mapped in the bench's launch
configuration (autotuned mixed build, then the FP64 build), checked on a
seeded sample of outputs the oracle computes one by one:

* h of sampled particles against the oracle's h solve (Eq. 7-9) on the same
  positions (mixed: FP32 sums, 1e-6; FP64: 1e-9);
* the pair lists of sampled cells, bit for bit, against the oracle's
  brute-force pair rule on each build's own h;
* the cell masses of those cells against the oracle's FP64 integrals on the
  same h (mixed 1e-5, FP64 1e-9, relative to each cell's mass);
* the reported total against the sum of the cell masses.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import lib, sample_cells

pytestmark = pytest.mark.gpu

N = 1 << 20
TOL_MASS = {1: 1e-5, 0: 1e-9}
TOL_H = {1: 1e-6, 0: 1e-9}


@pytest.fixture(scope="module")
def snapshot():
    p = synth.lognormal_particles(N, synth.BASE_SEED + 2, sigma=1.5)
    g = synth.voronoi(p.pos())
    return p, g


@pytest.mark.parametrize("precision", [1, 0])
def test_full_size_sampled_outputs(snapshot, precision):
    p, g = snapshot
    L = lib()
    ctx = L.map_init(L.map_config_default(precision=precision, autotune=1))
    try:
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        x, y, z, m = t(p.x), t(p.y), t(p.z), t(p.m)
        h = torch.empty_like(x)
        handle = L.map_grid_upload(ctx, L.grid_to_device(g))
        mass = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
        L.solve_h(ctx, L.make_particles(x, y, z, None, h))
        L.map_particles_to_cells(ctx, L.make_particles(x, y, z, m, h), handle, mass)
        st = L.map_get_stats(ctx)
        cells = sample_cells(g.ncell, 48, 11 + precision)
        off, idx, _ = L.map_copy_pairs(ctx, g.ncell)
        torch.cuda.synchronize()
        hh = h.cpu().numpy()
        got_mass = mass.cpu().numpy()
        offh = off.cpu().numpy()
        lists = [idx[offh[c]:offh[c + 1]].cpu().numpy() for c in cells]
    finally:
        L.map_destroy(ctx)

    # h of sampled particles against the oracle's solve on the same positions
    tree = oracle.Tree(p.x, p.y, p.z, p.m)
    h0 = oracle.particle_h_guess(tree)
    parts = sample_cells(N, 48, 21 + precision)
    h_ref, _ = oracle.solve_h(p.x, p.y, p.z, h0, targets=parts)
    assert np.max(np.abs(hh[parts] - h_ref) / h_ref) < TOL_H[precision]

    # pair lists and masses of sampled cells on the build's own h
    ref = oracle.map_cells(g, p.x, p.y, p.z, p.m, hh, cells=cells)
    for k, c in enumerate(cells):
        assert np.array_equal(lists[k], ref["idx"][ref["off"][k]:ref["off"][k + 1]]), c
    err = np.abs(got_mass[cells] - ref["mass"]) / np.abs(ref["mass"])
    assert err.max() < TOL_MASS[precision], (err.max(), cells[np.argmax(err)])
    assert st.n_pairs == offh[-1]
    assert abs(st.total_mass - got_mass.sum()) < 1e-12 * got_mass.sum()
