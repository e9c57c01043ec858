"""Failure handling on the host side of the C ABI: bad particles, a corrupted
grid and a memory budget below one request are refused with the documented
status codes, and the context stays usable.  Every bad input here is caught
by the library's validation (host checks, or bounds-checked validation
kernels that read only inside the arrays' declared sizes) before any kernel
indexes memory with it."""
import numpy as np
import pytest
import torch

import oracle
import synth
from gpu_helpers import lib, dev_particles, oracle_h, rel_err

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def small():
    p = synth.uniform_particles(512, synth.BASE_SEED + 11)
    g = synth.voronoi(p.pos())
    h, _ = oracle_h(p)
    return p, g, h


def _code(fn):
    L = lib()
    with pytest.raises(L.MapError) as e:
        fn()
    return e.value.code


def _map(L, ctx, g, p, h, handle=None):
    handle = L.map_grid_upload(ctx, L.grid_to_device(g)) if handle is None else handle
    x, y, z, m, hh = dev_particles(p, h)
    mass = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
    L.map_particles_to_cells(ctx, L.make_particles(x, y, z, m, hh), handle, mass)
    torch.cuda.synchronize()
    return handle, mass


@pytest.mark.parametrize("bad", ["h_nan", "h_zero", "h_negative", "x_outside", "z_nan"])
def test_bad_particles_rejected(small, bad):
    L = lib()
    p, g, h = small
    ctx = L.map_init(L.map_config_default(precision=1))
    try:
        handle, ref = _map(L, ctx, g, p, h)
        x, y, z, m, hh = dev_particles(p, h)
        if bad == "h_nan":
            hh[17] = float("nan")
        elif bad == "h_zero":
            hh[3] = 0.0
        elif bad == "h_negative":
            hh[200] = -0.01
        elif bad == "x_outside":
            x[5] = 1.5
        else:
            z[9] = float("nan")
        mass = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
        code = _code(lambda: L.map_particles_to_cells(ctx, L.make_particles(x, y, z, m, hh), handle, mass))
        assert code == L.MAP_EINVAL
        if bad in ("x_outside", "z_nan"):
            # solve_h reads positions only: it refuses the same positions
            hs = torch.empty_like(x)
            assert _code(lambda: L.solve_h(ctx, L.make_particles(x, y, z, None, hs))) == L.MAP_EINVAL
        # the context still maps the good particles, to the same bits
        _, again = _map(L, ctx, g, p, h, handle)
        assert torch.equal(again, ref)
    finally:
        L.map_destroy(ctx)


@pytest.mark.parametrize("bad", ["face_vert_range", "face_vert_negative", "cfo_non_monotone", "cfo_last",
                                 "fvo_short_loop"])
def test_corrupted_grid_rejected(small, bad):
    L = lib()
    p, g, h = small
    ctx = L.map_init(L.map_config_default(precision=1))
    try:
        d = L.grid_to_device(g)
        if bad == "face_vert_range":
            d["face_vert"][123] = g.vx.shape[0]  # one past the last vertex
        elif bad == "face_vert_negative":
            d["face_vert"][7] = -1
        elif bad == "cfo_non_monotone":
            d["cell_face_off"][10] = d["cell_face_off"][12] + 1
        elif bad == "cfo_last":
            d["cell_face_off"][-1] -= 1
        else:
            d["face_vert_off"][40] = d["face_vert_off"][39] + 2  # a two-vertex loop
        assert _code(lambda: L.map_grid_upload(ctx, d)) == L.MAP_EINVAL
        # the good grid still uploads and maps
        _, mass = _map(L, ctx, g, p, h)
        assert np.isfinite(mass.cpu().numpy()).all()
    finally:
        L.map_destroy(ctx)


def test_budget_below_one_request(small):
    L = lib()
    p, g, h = small
    ctx = L.map_init(L.map_config_default(precision=1, hbm_budget=64 << 10))
    try:
        assert _code(lambda: L.map_grid_upload(ctx, L.grid_to_device(g))) == L.MAP_ENOMEM
    finally:
        L.map_destroy(ctx)
    # a context with room maps the same input afterwards
    ctx = L.map_init(L.map_config_default(precision=1))
    try:
        _, mass = _map(L, ctx, g, p, h)
        ref = oracle.map_cells(g, p.x, p.y, p.z, p.m, h)
        assert rel_err(mass.cpu().numpy(), ref["mass"]).max() < 1e-5
    finally:
        L.map_destroy(ctx)
