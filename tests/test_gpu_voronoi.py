"""GPU grid construction (Section II-A: merging, Lloyd iterations, clipped
Voronoi cells) against the oracle's brute-force construction.

Gates: the same cell count and per-cell face count; per cell, volumes equal
to 1e-13 of the mean cell volume and every vertex within 1e-12 of a vertex
of the oracle's cell (the two clip in different orders, so vertices agree to
rounding); after Lloyd iterations the sites agree to 1e-12; merging keeps
exactly the oracle's sites.  A mapping on the device-built grid equals the
mapping on the same grid uploaded from the host to the FP64 gates.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import gpu_map, lib, oracle_h, rel_err

pytestmark = pytest.mark.gpu


class HostGrid:
    def __init__(self, d):
        for k, v in d.items():
            setattr(self, k, v.cpu().numpy())

    @property
    def ncell(self):
        return len(self.cell_face_off) - 1


def gpu_build(sites, lloyd=0, merge_tol=0.0, precision=0):
    L = lib()
    ctx = L.map_init(L.map_config_default(precision=precision))
    try:
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        kept = torch.empty(len(sites), dtype=torch.int64, device="cuda")
        hd, nk = L.map_grid_build(ctx, t(sites[:, 0]), t(sites[:, 1]), t(sites[:, 2]), lloyd, merge_tol, kept)
        g = HostGrid(L.map_grid_copy(ctx, hd))
        torch.cuda.synchronize()
        return g, kept[:nk].cpu().numpy()
    finally:
        L.map_destroy(ctx)


def compare_cells(g, ref, tol_v=1e-12):
    assert g.ncell == ref.ncell
    assert np.array_equal(np.diff(g.cell_face_off), np.diff(ref.cell_face_off))
    v1, _ = oracle.cell_geometry(g)
    v2, _ = oracle.cell_geometry(ref)
    assert np.max(np.abs(v1 - v2)) < 1e-13 / g.ncell
    a = np.stack([g.vx, g.vy, g.vz], 1)
    b = np.stack([ref.vx, ref.vy, ref.vz], 1)
    for c in range(g.ncell):
        fa, fb = g.cell_face_off[c], g.cell_face_off[c + 1]
        ia = np.unique(g.face_vert[g.face_vert_off[fa]:g.face_vert_off[fb]])
        ra, rb = ref.cell_face_off[c], ref.cell_face_off[c + 1]
        ib = np.unique(ref.face_vert[ref.face_vert_off[ra]:ref.face_vert_off[rb]])
        assert len(ia) == len(ib), c
        d = np.linalg.norm(a[ia][:, None, :] - b[ib][None, :, :], axis=2).min(axis=1)
        assert d.max() < tol_v, (c, d.max())


@pytest.mark.parametrize("case", ["uniform", "lattice", "clumpy"])
def test_cells_match_oracle(case):
    pts = {"uniform": synth.uniform_particles(300, 5).pos(), "lattice": synth.lattice_particles(5).pos(),
           "clumpy": synth.lognormal_particles(1500, 7, ngrid=32).pos()}[case]
    g, kept = gpu_build(pts)
    assert np.array_equal(kept, np.arange(len(pts)))
    assert np.array_equal(g.site, pts)
    compare_cells(g, oracle.voronoi_cells(pts))


def test_lloyd_and_merge_match_oracle():
    p = synth.uniform_particles(200, 17).pos()
    sites = np.concatenate([p, p[:7] + 2e-9, p[40:42] - 1e-9])
    g, kept = gpu_build(sites, lloyd=2, merge_tol=1e-8)
    ref, ref_kept = oracle.build_grid(sites, lloyd=2, merge_tol=1e-8)
    assert np.array_equal(kept, ref_kept) and len(kept) == 200
    assert np.max(np.abs(g.site - ref.site)) < 1e-12
    compare_cells(g, ref, tol_v=1e-11)


def test_mapping_on_device_built_grid():
    """The device-built grid serves the mapping directly; its result equals
    the mapping on the host-built grid of the same sites (FP64 gates)."""
    p = synth.uniform_particles(2048, synth.BASE_SEED + 41)
    h, _ = oracle_h(p)
    L = lib()
    ctx = L.map_init(L.map_config_default(precision=0))
    try:
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
        x, y, z, m, hh = t(p.x), t(p.y), t(p.z), t(p.m), t(h)
        hd, nk = L.map_grid_build(ctx, x, y, z, 0, 0.0)
        mass = torch.empty(nk, dtype=torch.float64, device="cuda")
        L.map_particles_to_cells(ctx, L.make_particles(x, y, z, m, hh), hd, mass)
        torch.cuda.synchronize()
        got = mass.cpu().numpy()
    finally:
        L.map_destroy(ctx)
    ref = gpu_map(synth.voronoi(p.pos()), p, h, 0)
    assert rel_err(got, ref["mass"]).max() < 1e-9


def test_build_errors():
    L = lib()
    ctx = L.map_init(L.map_config_default())
    try:
        bad = torch.tensor([0.5, 1.5], dtype=torch.float64, device="cuda")
        ok = torch.tensor([0.5, 0.25], dtype=torch.float64, device="cuda")
        with pytest.raises(L.MapError) as e:
            L.map_grid_build(ctx, bad, ok, ok, 0, 0.0)
        assert e.value.code == L.MAP_EINVAL
        with pytest.raises(L.MapError):
            L.map_grid_build(ctx, ok, ok, ok, -1, 0.0)
    finally:
        L.map_destroy(ctx)


def test_cells_match_oracle_16k_clumpy_sampled():
    """A larger clumpy site set (2^14 sites, log-normal field): 200 sampled
    cells against the oracle's cells built for those sites alone (each
    against all sites): face counts, vertices and volumes as above."""
    sites = synth.lognormal_particles(1 << 14, 71, ngrid=64).pos()
    g, kept = gpu_build(sites)
    assert np.array_equal(kept, np.arange(len(sites)))
    which = np.sort(np.random.default_rng(3).choice(len(sites), 200, replace=False))
    ref = oracle.VoronoiGrid(oracle.voronoi_cells_of(sites, which), sites[which])
    # the GPU grid restricted to the same cells (vertex arrays shared)
    sub = HostGrid({})
    cfo, fvo = g.cell_face_off, g.face_vert_off
    faces = np.concatenate([np.arange(cfo[c], cfo[c + 1]) for c in which])
    sub.cell_face_off = np.concatenate([[0], np.cumsum(np.diff(cfo)[which])]).astype(np.int64)
    nl = fvo[faces + 1] - fvo[faces]
    sub.face_vert_off = np.concatenate([[0], np.cumsum(nl)]).astype(np.int64)
    sub.face_vert = np.concatenate([g.face_vert[fvo[f]:fvo[f + 1]] for f in faces]).astype(np.int32)
    sub.face_plane = g.face_plane.reshape(-1, 4)[faces]
    sub.vx, sub.vy, sub.vz, sub.site = g.vx, g.vy, g.vz, g.site.reshape(-1, 3)[which]
    compare_cells(sub, ref, tol_v=1e-12)


def test_full_size_build_sampled_cells():
    """The bench's tessellation at full size: the 2^20 clumpy snapshot's
    positions, sites merged below 1e-6 of the mean spacing, 5 Lloyd
    iterations, the final cells.  32 sampled cells of the GPU grid against
    the oracle's cells of the same final sites (each built against all of
    them): face counts, vertices and volumes as above."""
    n = 1 << 20
    pos = synth.lognormal_particles(n, synth.BASE_SEED + 2, sigma=1.5).pos()
    g, kept = gpu_build(pos, lloyd=5, merge_tol=1e-6 * n ** (-1.0 / 3.0))
    sites = g.site.reshape(-1, 3)
    assert len(sites) == len(kept) > 0.99 * n
    which = np.sort(np.random.default_rng(13).choice(len(sites), 32, replace=False))
    ref = oracle.VoronoiGrid(oracle.voronoi_cells_of(sites, which), sites[which])
    sub = HostGrid({})
    cfo, fvo = g.cell_face_off, g.face_vert_off
    faces = np.concatenate([np.arange(cfo[c], cfo[c + 1]) for c in which])
    sub.cell_face_off = np.concatenate([[0], np.cumsum(np.diff(cfo)[which])]).astype(np.int64)
    nl = fvo[faces + 1] - fvo[faces]
    sub.face_vert_off = np.concatenate([[0], np.cumsum(nl)]).astype(np.int64)
    sub.face_vert = np.concatenate([g.face_vert[fvo[f]:fvo[f + 1]] for f in faces]).astype(np.int32)
    sub.face_plane = g.face_plane.reshape(-1, 4)[faces]
    sub.vx, sub.vy, sub.vz, sub.site = g.vx, g.vy, g.vz, sites[which]
    compare_cells(sub, ref, tol_v=1e-12)
