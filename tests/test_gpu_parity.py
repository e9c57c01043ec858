"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Gates (per cell, relative to the oracle, absolute floor at 1e-12 of the
largest cell mass): FP64 build 1e-9, mixed build 1e-5; total mass 1e-12 and
1e-7; pair lists bit-equal; smoothing lengths 1e-9 relative in the FP64 build
and 1e-6 relative in the mixed build, whose h solve sums the kernel in FP32 and
stops Newton at |dh|/h < 1e-6 (h to ~1e-7; the mapping's 1e-5 gate holds on
either build's h).
"""
import numpy as np
import pytest

import oracle
import synth
from gpu_helpers import gpu_map, oracle_h, rel_err, sample_cells, lib, dev_particles

pytestmark = pytest.mark.gpu

TOL = {0: (1e-9, 1e-12), 1: (1e-5, 1e-7)}


@pytest.fixture(scope="module")
def uniform4096():
    """Plain Exact mapping workload: 4096 equal-mass particles uniform in the cube."""
    p = synth.uniform_particles(4096, synth.BASE_SEED + 1)
    g = synth.voronoi(p.pos())
    h, route = oracle_h(p)
    ref = oracle.map_cells(g, p.x, p.y, p.z, p.m, h)
    return p, g, h, route, ref


@pytest.mark.parametrize("precision", [0, 1])
def test_uniform4096_all_cells(uniform4096, precision):
    p, g, h, _, ref = uniform4096
    out = gpu_map(g, p, h, precision)
    assert out["status"] == 0
    # pair lists: bit-equal
    assert np.array_equal(out["off"], ref["off"])
    assert np.array_equal(out["idx"], ref["idx"])
    cell_tol, tot_tol = TOL[precision]
    e = rel_err(out["mass"], ref["mass"])
    assert e.max() < cell_tol, (precision, e.max(), np.percentile(e, 99))
    assert abs(out["total"] - ref["mass"].sum()) < tot_tol * ref["mass"].sum()
    assert np.max(np.abs(out["vol"] - ref["vol"]) / ref["vol"]) < 1e-12
    assert np.max(np.abs(out["rho"] / ref["rho"] - 1)) < cell_tol * 1.01 + 1e-12
    # per-pair integrals: FP64 closed form ~1e-14 per edge term; the mixed build's
    # FP32 edge terms carry <= 4e-8 each (inner closed form 2.4e-8, middle
    # Gauss-Legendre 3.5e-8, geometry 1e-7 h), and a pair sums ~50 of them
    fe = np.abs(out["frac"] - ref["frac"])
    assert fe.max() < (1e-11 if precision == 0 else 5e-6), fe.max()


def test_uniform4096_mass_conservation(uniform4096):
    """Interior particles: sum_i f_ai = 1 on the GPU too (mixed build)."""
    p, g, h, _, _ = uniform4096
    out = gpu_map(g, p, h, 1)
    tot = np.zeros(p.n)
    np.add.at(tot, out["idx"], out["frac"])
    pos = p.pos()
    interior = np.all((pos >= 2 * h[:, None]) & (pos <= 1 - 2 * h[:, None]), axis=1)
    assert interior.sum() > 100
    assert np.max(np.abs(tot[interior] - 1)) < 1e-6


@pytest.mark.parametrize("precision", [0, 1])
def test_count_work(uniform4096, precision):
    """count_work = 1 runs the counting compilation of the integral kernel:
    its tally is positive (zeros without it) and both compilations meet the
    build's gate against the oracle and agree with each other."""
    p, g, h, _, ref = uniform4096
    L = lib()
    res = {}
    for cw in (0, 1):
        ctx = L.map_init(L.map_config_default(precision=precision, count_work=cw))
        try:
            out = gpu_map(g, p, h, precision, ctx=ctx)
            work, _ = L.map_get_work(ctx)
        finally:
            L.map_destroy(ctx)
        assert out["status"] == 0
        assert rel_err(out["mass"], ref["mass"]).max() < TOL[precision][0]
        res[cw] = (out, work)
    assert res[0][0]["terms"] == 0 and all(v == 0 for v in res[0][1].values())
    w, terms = res[1][1], res[1][0]["terms"]
    assert w["face_tests"] > 0 and 0 < terms <= w["edge_records"]
    assert w["mid_intervals"] > 0 and w["outer_intervals"] > 0
    assert rel_err(res[1][0]["mass"], res[0][0]["mass"]).max() < (1e-12 if precision == 0 else 1e-6)


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-6)])
def test_solve_h_uniform4096(uniform4096, precision, tol):
    """FP64 build: Newton to 1e-10 in FP64 sums.  Mixed build: FP32 sums on
    hi/lo-split coordinates, Newton to 1e-6, h to ~1e-7 relative."""
    p, g, h_ref, route_ref, _ = uniform4096
    L = lib()
    ctx = L.map_init(L.map_config_default(precision=precision))
    try:
        x, y, z, m, hh = dev_particles(p)
        route = __import__("torch").empty(p.n, dtype=__import__("torch").int32, device="cuda")
        L.solve_h(ctx, L.make_particles(x, y, z, None, hh), route)
        h = hh.cpu().numpy()
        r = route.cpu().numpy()
    finally:
        L.map_destroy(ctx)
    assert np.array_equal(r, route_ref)
    assert np.max(np.abs(h / h_ref - 1)) < tol


@pytest.fixture(scope="module")
def clumpy():
    """Clumpy-cloud workload at reduced size: 2^16 particles from the log-normal field."""
    p = synth.lognormal_particles(1 << 16, synth.BASE_SEED + 2)
    g = synth.voronoi(p.pos())
    h, route = oracle_h(p)
    cells = sample_cells(g.ncell, 400, 5)
    ref = oracle.map_cells(g, p.x, p.y, p.z, p.m, h, cells=cells)
    return p, g, h, cells, ref, route


@pytest.mark.parametrize("precision", [0, 1])
def test_clumpy_sampled_cells(clumpy, precision):
    p, g, h, cells, ref, _ = clumpy
    out = gpu_map(g, p, h, precision)
    for k, c in enumerate(cells):
        a = out["idx"][out["off"][c]:out["off"][c + 1]]
        b = ref["idx"][ref["off"][k]:ref["off"][k + 1]]
        assert np.array_equal(a, b), c
    cell_tol, _ = TOL[precision]
    e = rel_err(out["mass"][cells], ref["mass"], floor_frac=1e-12)
    assert e.max() < cell_tol, (e.max(), np.percentile(e, 99))


@pytest.mark.parametrize("precision,tol", [(0, 1e-9), (1, 1e-6)])
def test_solve_h_clumpy(clumpy, precision, tol):
    """Clumpy set: a wide spread of h, some particles whose Newton iterates
    leave [h0/16, 16 h0] and finish by bisection (route 1)."""
    p, _, h_ref, _, _, route_ref = clumpy
    assert np.count_nonzero(route_ref == 1) > 0
    L = lib()
    ctx = L.map_init(L.map_config_default(precision=precision))
    try:
        x, y, z, m, hh = dev_particles(p)
        route = __import__("torch").empty(p.n, dtype=__import__("torch").int32, device="cuda")
        L.solve_h(ctx, L.make_particles(x, y, z, None, hh), route)
        h = hh.cpu().numpy()
        r = route.cpu().numpy()
    finally:
        L.map_destroy(ctx)
    assert np.array_equal(r, route_ref), np.nonzero(r != route_ref)
    assert np.max(np.abs(h / h_ref - 1)) < tol


def test_edge_cases_tiny_and_huge_support():
    """One particle (one cell = the cube); a few particles whose supports cover
    the whole cube; particles with tiny supports inside their own cells."""
    rng = np.random.default_rng(3)
    # one particle: the whole support inside the cube -> M = m
    p1 = synth.Particles(np.array([0.5]), np.array([0.5]), np.array([0.5]), np.array([2.0]))
    g1 = synth.voronoi(p1.pos())
    for prec in (0, 1):
        out = gpu_map(g1, p1, np.array([0.2]), prec)
        assert out["n_pairs"] == 1
        assert abs(out["mass"][0] - 2.0) < 1e-12
    # ragged: 37 particles, supports larger than the cube
    p2 = synth.uniform_particles(37, 99)
    g2 = synth.voronoi(p2.pos())
    h2 = rng.uniform(0.6, 1.5, 37)
    ref = oracle.map_cells(g2, p2.x, p2.y, p2.z, p2.m, h2)
    for prec in (0, 1):
        out = gpu_map(g2, p2, h2, prec)
        assert np.array_equal(out["idx"], ref["idx"])
        assert rel_err(out["mass"], ref["mass"]).max() < TOL[prec][0]
    # tiny supports: each cell holds its own particle's mass, except where a
    # site lies within 2h of a wall (one does here, 1.4e-6 away) and mass
    # leaves the cube
    p3 = synth.uniform_particles(200, 5)
    g3 = synth.voronoi(p3.pos())
    h3 = np.full(200, 1e-5)
    ref3 = oracle.map_cells(g3, p3.x, p3.y, p3.z, p3.m, h3)
    for prec in (0, 1):
        out = gpu_map(g3, p3, h3, prec)
        assert out["n_pairs"] == 200
        assert rel_err(out["mass"], ref3["mass"]).max() < TOL[prec][0]
        whole = np.abs(ref3["mass"] / p3.m - 1) < 1e-9
        assert whole.sum() >= 190 and np.all(out["mass"][whole] == p3.m[whole])


def test_particles_on_face_planes():
    """Lattice sites with extra particles placed exactly on shared faces: the
    mapping stays continuous (each such particle splits between its cells)."""
    n = 6
    lat = synth.lattice_particles(n)
    g = synth.voronoi(lat.pos())
    extra = np.array([[3.0 / n, 2.5 / n, 2.5 / n], [3.0 / n, 3.0 / n, 2.5 / n]])
    pos = np.concatenate([lat.pos(), extra])
    m = np.full(len(pos), 1.0 / len(pos))
    p = synth.Particles(pos[:, 0].copy(), pos[:, 1].copy(), pos[:, 2].copy(), m)
    h = np.full(len(pos), 1.3 / n)
    ref = oracle.map_cells(g, p.x, p.y, p.z, p.m, h)
    for prec in (0, 1):
        out = gpu_map(g, p, h, prec)
        assert np.array_equal(out["idx"], ref["idx"])
        assert rel_err(out["mass"], ref["mass"]).max() < TOL[prec][0]


def test_few_large_cells():
    """Many particles per cell (64 here): the pair list comes from the
    warp-per-cell walk and cells span several work items; lists bit-equal,
    masses within the gates."""
    lat = synth.lattice_particles(4, jitter=0.3, seed=7)
    g = synth.voronoi(lat.pos())
    p = synth.uniform_particles(4096, synth.BASE_SEED + 7)
    h, _ = oracle_h(p)
    ref = oracle.map_cells(g, p.x, p.y, p.z, p.m, h)
    assert np.diff(ref["off"]).max() > 256  # some cells overflow the 256-pair row
    for prec in (0, 1):
        out = gpu_map(g, p, h, prec)
        assert np.array_equal(out["off"], ref["off"])
        assert np.array_equal(out["idx"], ref["idx"])
        assert np.abs(out["frac"] - ref["frac"]).max() < (1e-11 if prec == 0 else 5e-6)
        assert rel_err(out["mass"], ref["mass"]).max() < TOL[prec][0]
        assert abs(out["total"] - ref["mass"].sum()) < TOL[prec][1] * ref["mass"].sum()


def test_lists_longer_than_the_shared_memory_sort():
    """8 cells for 4096 particles: lists of more than 1024 pairs, which the
    library segmented sort orders (with f_ai alongside) when they are read;
    lists bit-equal, per-pair integrals and masses within the gates."""
    lat = synth.lattice_particles(2, jitter=0.2, seed=11)
    g = synth.voronoi(lat.pos())
    p = synth.uniform_particles(4096, synth.BASE_SEED + 11)
    h, _ = oracle_h(p)
    ref = oracle.map_cells(g, p.x, p.y, p.z, p.m, h)
    assert np.diff(ref["off"]).max() > 1024
    for prec in (0, 1):
        out = gpu_map(g, p, h, prec)
        assert np.array_equal(out["off"], ref["off"])
        assert np.array_equal(out["idx"], ref["idx"])
        assert np.abs(out["frac"] - ref["frac"]).max() < (1e-11 if prec == 0 else 5e-6)
        assert rel_err(out["mass"], ref["mass"]).max() < TOL[prec][0]


def test_grid_upload_from_pinned_host_and_reuse(uniform4096):
    """map_grid_upload takes page-locked host arrays as well as device arrays
    (the same prepared grid, so bit-equal volumes and masses), and a grid
    uploaded after a release reuses the released buffers with the same result."""
    import torch
    p, g, h, _, _ = uniform4096
    L = lib()
    ctx = L.map_init(L.map_config_default(precision=1))
    try:
        x, y, z, m, hh = dev_particles(p, h)
        res = []
        for src in ("device", "pinned", "device"):
            if src == "device":
                gd = L.grid_to_device(g)
            else:
                gd = {k: v.cpu().pin_memory() for k, v in L.grid_to_device(g).items()}
            handle = L.map_grid_upload(ctx, gd)
            mass = torch.empty(g.ncell, dtype=torch.float64, device="cuda")
            vol = torch.empty_like(mass)
            L.map_particles_to_cells(ctx, L.make_particles(x, y, z, m, hh), handle, mass, None, vol)
            torch.cuda.synchronize()
            res.append((mass.cpu().numpy(), vol.cpu().numpy()))
            L.map_grid_release(ctx, handle)
    finally:
        L.map_destroy(ctx)
    for a, b in res[1:]:
        assert np.array_equal(a, res[0][0]) and np.array_equal(b, res[0][1])


@pytest.mark.parametrize("precision", [0, 1])
def test_particles_on_face_planes(precision):
    """Particles on the face planes of the grid: the midpoints of neighbouring
    sites (on their bisector plane up to rounding) and points 1e-9 and 1e-6
    off it (h is about 0.1 here, so all within the 1e-4 h where the mixed
    build decides the face's side and distance in FP64).  Every cell against
    the oracle, at the build's gate."""
    sites = synth.uniform_particles(300, synth.BASE_SEED + 13)
    g = synth.voronoi(sites.pos())
    pos = sites.pos()
    rng = np.random.default_rng(8)
    pts = []
    for f in rng.choice(len(g.face_nb), 400, replace=False):
        nb = g.face_nb[f]
        if nb < 0:
            continue
        c = int(np.searchsorted(g.cell_face_off, f, side="right") - 1)
        mid = 0.5 * (pos[c] + pos[nb])
        n = g.face_plane[f][:3]
        for off in (0.0, 1e-9, -1e-6):
            pts.append(np.clip(mid + off * n, 0.0, 1.0))
    pts = np.array(pts)
    p = synth.Particles(pts[:, 0].copy(), pts[:, 1].copy(), pts[:, 2].copy(), np.full(len(pts), 1.0 / len(pts)))
    h, _ = oracle_h(p)
    out = gpu_map(g, p, h, precision)
    ref = oracle.map_cells(g, p.x, p.y, p.z, p.m, h)
    assert np.array_equal(out["idx"], ref["idx"])
    cell_tol, tot_tol = TOL[precision]
    assert rel_err(out["mass"], ref["mass"]).max() < cell_tol
    assert abs(out["total"] - ref["mass"].sum()) < tot_tol * ref["mass"].sum()
