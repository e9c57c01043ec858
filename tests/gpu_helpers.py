"""Shared helpers for the GPU parity tests (calls go through the C ABI)."""
import numpy as np
import torch

import oracle
import synth


def lib():
    import paper_2404_17084_gb300 as L
    return L


def dev_particles(p, h=None):
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")
    x, y, z, m = t(p.x), t(p.y), t(p.z), t(p.m)
    hh = t(h) if h is not None else torch.empty_like(x)
    return x, y, z, m, hh


def gpu_map(grid, p, h, precision, ctx=None):
    """Map on the GPU; returns dict(mass, rho, vol, off, idx, frac, stats) as numpy."""
    L = lib()
    own = ctx is None
    if own:
        ctx = L.map_init(L.map_config_default(precision=precision))
    try:
        handle = L.map_grid_upload(ctx, L.grid_to_device(grid))
        x, y, z, m, hh = dev_particles(p, h)
        nc = grid.ncell
        mass = torch.empty(nc, dtype=torch.float64, device="cuda")
        rho = torch.empty_like(mass)
        vol = torch.empty_like(mass)
        L.map_particles_to_cells(ctx, L.make_particles(x, y, z, m, hh), handle, mass, rho, vol)
        off, idx, frac = L.map_copy_pairs(ctx, nc)
        st = L.map_get_stats(ctx)
        torch.cuda.synchronize()
        out = dict(mass=mass.cpu().numpy(), rho=rho.cpu().numpy(), vol=vol.cpu().numpy(), off=off.cpu().numpy(),
                   idx=idx.cpu().numpy(), frac=frac.cpu().numpy(), n_pairs=st.n_pairs, total=st.total_mass,
                   terms=st.n_edge_terms, status=st.status)
        L.map_grid_release(ctx, handle)
        return out
    finally:
        if own:
            L.map_destroy(ctx)


def oracle_h(p, hfact=oracle.HFACT):
    t = oracle.Tree(p.x, p.y, p.z, p.m)
    h0 = oracle.particle_h_guess(t, hfact)
    h, route = oracle.solve_h(p.x, p.y, p.z, h0, hfact=hfact)
    return h, route


def rel_err(a, b, floor_frac=1e-12):
    """Per-cell relative error with an absolute floor at floor_frac * max|b|."""
    scale = np.maximum(np.abs(b), floor_frac * np.max(np.abs(b)))
    return np.abs(a - b) / scale


def sample_cells(ncell, k, seed):
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(ncell, size=min(k, ncell), replace=False)).astype(np.int64)
