"""GPU parity of the inverse mapping (Eq. 4), through the C ABI.

Gates: on the GPU's own pair list the result equals the sequential sum with
one rounding per term (acc <- RN(acc + v_i f_ai) in ascending cell order,
evaluated exactly in rationals) bit for bit; against the oracle's
own pair integrals, per particle |err| <= tol * sum_i |v_i| f_ai with the
forward mapping's per-cell gates (FP64 1e-9, mixed 1e-5); the mass-weighted
totals agree (sum_a m_a out_a = sum_i v_i M_i) to the total-mass gates.
"""
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import dev_particles, lib, oracle_h

pytestmark = pytest.mark.gpu

TOL = {0: (1e-9, 1e-12), 1: (1e-5, 1e-7)}


def fused_sums(off, idx, frac, v, particles):
    """For each listed particle: acc <- RN(acc + v_i f_ai) over its pairs in
    ascending cell order from +0, each step exact in rationals and rounded
    once (float() of a Fraction rounds to nearest even)."""
    cell = np.repeat(np.arange(len(off) - 1), np.diff(off))
    out = []
    for a in particles:
        acc = 0.0
        for k in np.flatnonzero(idx == a):  # CSR by cell: ascending cell order
            acc = float(Fraction(acc) + Fraction(float(v[cell[k]])) * Fraction(float(frac[k])))
        out.append(acc)
    return np.array(out)


def map_and_invert(g, p, h, precision, values, copy_first=False):
    """Map, then carry every array in `values` back to the particles.  Returns
    (list of particle arrays, off, idx, frac, cell masses)."""
    L = lib()
    ctx = L.map_init(L.map_config_default(precision=precision))
    try:
        handle = L.map_grid_upload(ctx, L.grid_to_device(g))
        x, y, z, m, hh = dev_particles(p, h)
        mass = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
        L.map_particles_to_cells(ctx, L.make_particles(x, y, z, m, hh), handle, mass)
        if copy_first:
            off, idx, frac = L.map_copy_pairs(ctx, g.ncell)
        outs = []
        for v in values:
            cv = torch.as_tensor(v, dtype=torch.float64, device="cuda")
            pv = torch.full((p.n,), -1.0, dtype=torch.float64, device="cuda")
            L.map_cells_to_particles(ctx, cv, pv)
            outs.append(pv)
        if not copy_first:
            off, idx, frac = L.map_copy_pairs(ctx, g.ncell)
        torch.cuda.synchronize()
        return ([o.cpu().numpy() for o in outs], off.cpu().numpy(), idx.cpu().numpy(), frac.cpu().numpy(),
                mass.cpu().numpy())
    finally:
        L.map_destroy(ctx)


@pytest.fixture(scope="module")
def ragged():
    """3001 particles (not a multiple of the 32 a warp sums), oracle h, one
    particle with h = 0.45 (listed by most cells: its terms span several
    staged chunks) and one with a tiny support."""
    p = synth.uniform_particles(3001, synth.BASE_SEED + 31)
    g = synth.voronoi(p.pos())
    h, _ = oracle_h(p)
    h[17] = 0.45
    h[2000] = 1e-5
    ref = oracle.map_cells(g, p.x, p.y, p.z, p.m, h)
    rng = np.random.default_rng(8)
    values = [rng.random(g.ncell), np.full(g.ncell, 0.5), rng.uniform(-1, 1, g.ncell)]
    return p, g, h, ref, values


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("copy_first", [False, True])
def test_inverse_equals_the_fused_sequential_sum(ragged, precision, copy_first):
    """Bit for bit the sequential fused sum over the same pairs (sampled
    particles, including the longest list, a one-pair list and the last
    particle), whether the particle-major index is built from the
    walk-ordered lists (first) or from the sorted ones (after
    map_copy_pairs); later calls reuse the index.  Every particle agrees with
    the plain numpy sum of rounded products to the rounding of the products."""
    p, g, h, _, values = ragged
    outs, off, idx, frac, _ = map_and_invert(g, p, h, precision, values, copy_first)
    count = np.bincount(idx, minlength=p.n)
    assert count[17] > 512 and count[2000] == 1
    sample = np.concatenate([[17, 2000, p.n - 1], np.random.default_rng(1).choice(p.n, 120, replace=False)])
    for v, got in zip(values, outs):
        want = fused_sums(off, idx, frac, v, sample)
        assert np.array_equal(got[sample], want), sample[got[sample] != want][:5]
        plain = oracle.inverse_map(off, idx, frac, v, p.n)
        scale = oracle.inverse_map(off, idx, frac, np.abs(v), p.n)
        assert np.all(np.abs(got - plain) <= 1e-13 * scale)


@pytest.mark.parametrize("precision", [0, 1])
def test_inverse_vs_oracle(ragged, precision):
    p, g, h, ref, values = ragged
    outs, _, _, _, mass = map_and_invert(g, p, h, precision, values)
    tol, tot_tol = TOL[precision]
    for v, got in zip(values, outs):
        want = oracle.inverse_map(ref["off"], ref["idx"], ref["frac"], v, p.n)
        scale = oracle.inverse_map(ref["off"], ref["idx"], ref["frac"], np.abs(v), p.n)
        err = np.abs(got - want) / np.maximum(scale, 1e-300)
        assert err.max() < tol, (err.max(), np.argmax(err))
        # the ionised mass is the same on the particles and on the grid
        lhs, rhs = np.dot(p.m, got), np.dot(v, mass)
        assert abs(lhs - rhs) < tot_tol * np.dot(np.abs(v), mass), (lhs, rhs)
    # interior particles: the weights sum to 1, a constant comes back unchanged
    pos = p.pos()
    interior = np.all((pos >= 2 * h[:, None]) & (pos <= 1 - 2 * h[:, None]), axis=1)
    assert interior.sum() > 100
    assert np.max(np.abs(outs[1][interior] - 0.5)) < (1e-12 if precision == 0 else 1e-6)


@pytest.mark.parametrize("precision", [0, 1])
def test_inverse_clumpy_sampled_particles(precision):
    """Clumpy-cloud field, 2^16 particles: sampled particles against the
    oracle's single-pair integrals over every cell within reach of the
    particle's support (|r_a - s_i| < 2 h_a + R_i; farther cells give 0)."""
    p = synth.lognormal_particles(1 << 16, synth.BASE_SEED + 2)
    g = synth.voronoi(p.pos())
    h, _ = oracle_h(p)
    v = np.random.default_rng(4).random(g.ncell)
    (got,), _, _, _, _ = map_and_invert(g, p, h, precision, [v])
    _, rad = oracle.cell_geometry(g)
    rng = np.random.default_rng(6)
    sample = rng.choice(p.n, 150, replace=False)
    pos = p.pos()
    for a in sample:
        d = np.linalg.norm(g.site - pos[a], axis=1)
        cells = np.flatnonzero(d < 2 * h[a] + rad).astype(np.int64)
        k = len(cells)
        r = oracle.map_cells(g, p.x, p.y, p.z, p.m, h, cells=cells, off=np.arange(k + 1, dtype=np.int64),
                             idx=np.full(k, a, np.int32))
        want = float(np.dot(v[cells], r["frac"]))
        scale = float(np.dot(np.abs(v[cells]), r["frac"]))
        assert abs(got[a] - want) <= TOL[precision][0] * scale, (a, got[a], want)


def test_inverse_errors():
    """A wrong particle count, a batch context (no per-pair integrals kept)
    and a context that has not mapped are refused with MAP_EINVAL."""
    L = lib()
    p = synth.uniform_particles(300, 3)
    g = synth.voronoi(p.pos())
    h, _ = oracle_h(p)
    ctx = L.map_init(L.map_config_default(precision=1))
    try:
        cv = torch.zeros(g.ncell, dtype=torch.float64, device="cuda")
        with pytest.raises(L.MapError) as e:
            L.map_cells_to_particles(ctx, cv, torch.empty(p.n, dtype=torch.float64, device="cuda"))
        assert e.value.code == L.MAP_EINVAL
        handle = L.map_grid_upload(ctx, L.grid_to_device(g))
        x, y, z, m, hh = dev_particles(p, h)
        mass = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
        parts = L.make_particles(x, y, z, m, hh)
        L.map_particles_to_cells(ctx, parts, handle, mass)
        with pytest.raises(L.MapError) as e:
            L.map_cells_to_particles(ctx, cv, torch.empty(p.n - 1, dtype=torch.float64, device="cuda"))
        assert e.value.code == L.MAP_EINVAL
        out = torch.empty(p.n, dtype=torch.float64, device="cuda")
        L.map_cells_to_particles(ctx, cv, out)
        torch.cuda.synchronize()
        assert torch.all(out == 0)
        L.map_batch(ctx, [parts], [handle], [mass])
        with pytest.raises(L.MapError) as e:
            L.map_cells_to_particles(ctx, cv, out)
        assert e.value.code == L.MAP_EINVAL
    finally:
        L.map_destroy(ctx)
