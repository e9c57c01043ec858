"""Pins for the FP64 oracle against facts that do not come from the oracle.

Each check uses an independent route: direct numerical integration of the
kernel's definition, closed values, exact invariants (mass conservation,
translation symmetry, scale invariance), or brute-force ray casting over the
cell.  A dropped term, a wrong sign or a transposed operand anywhere in the
oracle's decomposition fails at least one of them.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate

import oracle
import synth

HERE = os.path.dirname(os.path.abspath(__file__))


# ----------------------------------------------------------------- test-side kernel definition
# The M4 cubic spline, support 2h, sigma = 1/pi (Section III-C names the kernel;
# the formula is the standard one).  Written here independently of the oracle.
def w_def(q):
    q = np.asarray(q, dtype=float)
    return np.where(q < 1, 1 - 1.5 * q**2 + 0.75 * q**3, np.where(q < 2, 0.25 * (2 - q) ** 3, 0.0))


def W_def(r, h=1.0):
    return w_def(np.asarray(r) / h) / (math.pi * h**3)


# exact radial mass per steradian, int_0^u W(r,1) r^2 dr, via numpy polynomial antiderivatives
_P_in = np.polynomial.Polynomial([1, 0, -1.5, 0.75]) * np.polynomial.Polynomial([0, 0, 1]) / math.pi
_P_out = np.polynomial.Polynomial([2, -1]) ** 3 * 0.25 * np.polynomial.Polynomial([0, 0, 1]) / math.pi
_A_in = _P_in.integ()
_A_out = _P_out.integ()


def Fr_def(u):
    u = np.asarray(u, dtype=float)
    m1 = _A_in(1.0) - _A_in(0.0)
    m2 = m1 + _A_out(2.0) - _A_out(1.0)
    return np.where(u < 1, _A_in(np.minimum(u, 1)) - _A_in(0.0),
                    np.where(u < 2, m1 + _A_out(np.clip(u, 1, 2)) - _A_out(1.0), m2))


def load_golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "kernel_constants.txt")) as fh:
        for line in fh:
            line = line.split("#")[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


# ----------------------------------------------------------------- helpers: hand-built cells

class OneCellGrid:
    """A single convex cell given as faces (planes + CCW vertex loops)."""

    def __init__(self, verts, loops, site):
        verts = np.asarray(verts, float)
        self.vx, self.vy, self.vz = verts[:, 0].copy(), verts[:, 1].copy(), verts[:, 2].copy()
        self.cell_face_off = np.array([0, len(loops)], np.int64)
        fvo = [0]
        fv = []
        planes = []
        for lp in loops:
            fv += list(lp)
            fvo.append(len(fv))
            p = verts[list(lp)]
            a = np.zeros(3)
            for k in range(len(p)):
                a += np.cross(p[k], p[(k + 1) % len(p)])
            n = a / np.linalg.norm(a)
            planes.append([n[0], n[1], n[2], float(n @ p[0])])
        self.face_vert_off = np.array(fvo, np.int64)
        self.face_vert = np.array(fv, np.int32)
        self.face_plane = np.array(planes, float)
        self.site = np.asarray(site, float).reshape(1, 3)

    @property
    def ncell(self):
        return 1


def box_cell(lo, hi):
    lo = np.asarray(lo, float)
    hi = np.asarray(hi, float)
    v = [[(hi if i & 1 else lo)[0], (hi if i & 2 else lo)[1], (hi if i & 4 else lo)[2]] for i in range(8)]
    loops = [[1, 3, 7, 5], [0, 4, 6, 2], [2, 6, 7, 3], [0, 1, 5, 4], [4, 5, 7, 6], [0, 2, 3, 1]]
    return OneCellGrid(v, loops, 0.5 * (lo + hi))


def frac_one(grid, pos, h):
    r = oracle.map_cells(grid, [pos[0]], [pos[1]], [pos[2]], [1.0], [h], cells=[0],
                         off=np.array([0, 1], np.int64), idx=np.array([0], np.int32), nthreads=1)
    return float(r["frac"][0])


# ----------------------------------------------------------------- kernel pins

def test_kernel_normalisation_and_golden_masses():
    g = load_golden()
    tot = integrate.quad(lambda r: 4 * math.pi * r * r * W_def(r), 0, 2, points=[1])[0]
    assert abs(tot - 1.0) < 1e-13
    assert abs(4 * math.pi * oracle.F(1.0) - g["mass_within_h"]) < 1e-15
    assert abs(4 * math.pi * oracle.F(2.0) - g["mass_within_2h"]) < 1e-15
    for u in (0.0, 0.1, 0.37, 0.99, 1.0, 1.5, 1.99, 2.0, 3.0):
        ref = integrate.quad(lambda r: r * r * W_def(r), 0, min(u, 2.0), points=[1] if u > 1 else None)[0]
        assert abs(oracle.F(u) - ref) < 1e-15, u


def test_H_continuity_and_derivative():
    for b in (1.0, 2.0):
        assert abs(oracle.H(b - 1e-13) - oracle.H(b + 1e-13)) < 1e-12
    for u in (0.2, 0.7, 1.3, 1.8, 2.5, 4.0):
        d = 1e-6
        fd = (oracle.H(u + d) - oracle.H(u - d)) / (2 * d)
        assert abs(fd - oracle.F(u) / u**2) < 1e-9, u


# ----------------------------------------------------------------- vertex pyramid pins

@pytest.mark.parametrize("r0,R0,phi", [(0.3, 0.4, 0.9), (1.2, 0.5, 1.2), (0.05, 1.5, 0.3),
                                       (0.8, 0.1, 1.45), (1.7, 0.2, 0.7), (0.5, 2.5, 0.2)])
def test_wedge_matches_3d_integral(r0, R0, phi):
    """I(r0,R0,phi) against a direct volume integral over the pyramid: points
    lam*(rho cos t, rho sin t, r0), lam in [0,1], rho in [0, R0 sec t], t in [0, phi];
    dV = lam^2 rho r0 dlam drho dt."""
    def inner(t):
        rmax = R0 / math.cos(t)

        def f2(rho):
            L = math.sqrt(rho * rho + r0 * r0)
            # int_0^1 W(lam L) lam^2 dlam = (1/L^3) int_0^L W(r) r^2 dr
            return rho * r0 * float(Fr_def(L)) / L**3
        return integrate.quad(f2, 0, rmax, epsabs=1e-14, epsrel=1e-12, limit=200)[0]
    ref = integrate.quad(inner, 0, phi, epsabs=1e-14, epsrel=1e-12, limit=200)[0]
    assert abs(oracle.wedge(r0, R0, phi) - ref) < 1e-11


@pytest.mark.parametrize("r0,R0,phi", [(2.0, 0.5, 1.0), (2.7, 1.3, 0.4), (5.0, 0.01, 1.5)])
def test_wedge_beyond_support_is_solid_angle(r0, R0, phi):
    omega = phi - math.asin(r0 * math.sin(phi) / math.hypot(r0, R0))
    assert abs(oracle.wedge(r0, R0, phi) - omega / (4 * math.pi)) < 1e-15


def test_cube_containing_support_gives_one():
    g = box_cell([-2.5, -2.5, -2.5], [2.5, 2.5, 2.5])
    assert abs(frac_one(g, [0.0, 0.0, 0.0], 1.0) - 1.0) < 1e-13
    # off-centre but the whole support still inside
    assert abs(frac_one(g, [0.3, -0.2, 0.4], 1.0) - 1.0) < 1e-13


@pytest.mark.parametrize("d", [0.0, 0.05, 0.4, 0.999, 1.0, 1.3, 1.95])
def test_halfspace_mass(d):
    """Box with one face at distance d, all others beyond the support:
    f = 1 - P(d), P(d) = int_d^2 2 pi r (r - d) W(r) dr (cap areas)."""
    P = integrate.quad(lambda r: 2 * math.pi * r * (r - d) * W_def(r), d, 2, points=[1] if d < 1 else None,
                       epsabs=1e-15)[0]
    g = box_cell([-5, -5, -5], [5, 5, d])
    f = frac_one(g, [0.0, 0.0, 0.0], 1.0)
    if d == 0.0:
        assert abs(P - load_golden()["halfspace_mass_d0"]) < 1e-14
    assert abs(f - (1.0 - P)) < 1e-12, (d, f, 1 - P)
    # particle outside the box, mirrored: mass inside is P(d)
    g2 = box_cell([-5, -5, d], [5, 5, 5])
    assert abs(frac_one(g2, [0.0, 0.0, 0.0], 1.0) - P) < 1e-12


def test_scale_invariance():
    g = box_cell([0.1, -0.3, -0.2], [0.9, 0.4, 0.6])
    f1 = frac_one(g, [0.35, 0.05, 0.9], 0.4)
    lam = 3.7
    g2 = box_cell(np.array([0.1, -0.3, -0.2]) * lam, np.array([0.9, 0.4, 0.6]) * lam)
    f2 = frac_one(g2, np.array([0.35, 0.05, 0.9]) * lam, 0.4 * lam)
    assert f1 > 1e-3
    assert abs(f1 - f2) < 1e-13


# ----------------------------------------------------------------- brute force: ray casting

def raycast_fraction(planes, pos, h, nmu=700, nphi=1400):
    """f = int dOmega [Fr(t_out/h) - Fr(t_in/h)] over rays from the particle
    through the convex cell {x : n.x <= d} (h = 1 units after scaling)."""
    mu, wmu = np.polynomial.legendre.leggauss(nmu)
    ph = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    st = np.sqrt(1 - mu**2)
    om = np.stack([st[:, None] * np.cos(ph)[None, :], st[:, None] * np.sin(ph)[None, :],
                   np.broadcast_to(mu[:, None], (nmu, nphi))], -1).reshape(-1, 3)
    wts = (wmu[:, None] * np.full(nphi, 2 * math.pi / nphi)[None, :]).ravel()
    tin = np.zeros(len(om))
    tout = np.full(len(om), np.inf)
    for nx, ny, nz, d in planes:
        n = np.array([nx, ny, nz])
        num = d - n @ pos
        den = om @ n
        with np.errstate(divide="ignore", invalid="ignore"):
            t = num / den
        pos_den = den > 0
        neg_den = den < 0
        tout = np.where(pos_den, np.minimum(tout, t), tout)
        tin = np.where(neg_den, np.maximum(tin, t), tin)
        if num < 0:
            tout = np.where(den == 0, -1.0, tout)
    tout = np.minimum(tout, 1e3)
    ok = tout > tin
    val = np.where(ok, Fr_def(tout / h) - Fr_def(tin / h), 0.0)
    return float(np.sum(val * wts))


def test_raycast_brute_force_small_voronoi():
    rng = np.random.default_rng(11)
    pts = rng.random((10, 3))
    grid = synth.voronoi(pts, nthreads=1)
    parts = rng.random((6, 3))
    hs = rng.uniform(0.1, 0.35, 6)
    worst = 0.0
    for c in range(grid.ncell):
        f0, f1 = grid.cell_face_off[c], grid.cell_face_off[c + 1]
        planes = grid.face_plane[f0:f1]
        for a in range(len(parts)):
            ref = raycast_fraction(planes, parts[a], hs[a])
            r = oracle.map_cells(grid, parts[:, 0], parts[:, 1], parts[:, 2], np.ones(6), hs, cells=[c],
                                 off=np.array([0, 1], np.int64), idx=np.array([a], np.int32), nthreads=1)
            worst = max(worst, abs(r["frac"][0] - ref))
    assert worst < 2e-4, worst


# ----------------------------------------------------------------- invariants on Voronoi grids

def test_cell_volumes_tile_the_cube():
    p = synth.uniform_particles(300, 5)
    g = synth.voronoi(p.pos(), nthreads=1)
    vol, rad = oracle.cell_geometry(g)
    assert abs(vol.sum() - 1.0) < 1e-13
    assert np.all(vol > 0) and np.all(rad > 0)


def test_mass_conservation_interior_particles():
    """sum_i f_ai = 1 for every particle whose support lies inside the cube."""
    p = synth.uniform_particles(512, 7)
    g = synth.voronoi(p.pos(), nthreads=1)
    h = np.full(p.n, 0.15)
    res = oracle.map_cells(g, p.x, p.y, p.z, p.m, h)
    tot = np.zeros(p.n)
    np.add.at(tot, res["idx"], res["frac"])
    pos = p.pos()
    interior = np.all((pos >= 2 * h[:, None]) & (pos <= 1 - 2 * h[:, None]), axis=1)
    assert interior.sum() >= 10
    assert np.max(np.abs(tot[interior] - 1.0)) < 1e-11
    # particles near the walls lose mass outside the cube, never gain
    assert np.all(tot <= 1.0 + 1e-11)


def test_lattice_uniform_density():
    """Cubic lattice, equal masses and h: every cell farther than 4h from the
    walls holds exactly one particle's mass (translation symmetry), so rho = m/V."""
    n = 12
    p = synth.lattice_particles(n)
    g = synth.voronoi(p.pos(), nthreads=1)
    h = np.full(p.n, 1.2 / n)
    site = g.site
    far = np.all((site > 4 * h[0]) & (site < 1 - 4 * h[0]), axis=1)
    cells = np.nonzero(far)[0]
    assert len(cells) >= 8
    res = oracle.map_cells(g, p.x, p.y, p.z, p.m, h, cells=cells)
    assert np.max(np.abs(res["mass"] / p.m[0] - 1.0)) < 1e-11
    assert np.max(np.abs(res["rho"] * res["vol"] / p.m[0] - 1.0)) < 1e-11
    assert np.max(np.abs(res["vol"] * n**3 - 1.0)) < 1e-11


def test_pair_rule_is_conservative():
    """Every particle with nonzero f_ai is listed: compare the pair list against
    brute-force f over ALL particles for a few cells."""
    p = synth.uniform_particles(200, 3)
    g = synth.voronoi(p.pos(), nthreads=1)
    h = np.full(p.n, 0.12)
    cells = np.array([0, 17, 99], np.int64)
    off, idx = oracle.pair_lists(g, p.x, p.y, p.z, h, cells)
    for k, c in enumerate(cells):
        listed = set(idx[off[k]:off[k + 1]].tolist())
        allidx = np.arange(p.n, dtype=np.int32)
        r = oracle.map_cells(g, p.x, p.y, p.z, p.m, h, cells=[c], off=np.array([0, p.n], np.int64), idx=allidx)
        nz = set(np.nonzero(np.abs(r["frac"]) > 1e-15)[0].tolist())
        assert nz <= listed


# ----------------------------------------------------------------- smoothing lengths

def test_h_solve_residual_and_lattice_value():
    n = 10
    p = synth.lattice_particles(n, jitter=0.2, seed=1)
    pos = p.pos()
    tree = oracle.Tree(p.x, p.y, p.z, p.m)
    h0 = oracle.particle_h_guess(tree)
    targets = np.arange(p.n)
    h, route = oracle.solve_h(p.x, p.y, p.z, h0, targets)
    assert np.all(route == 0)
    # independent residual: brute-force number density with the test's kernel
    for a in (0, 123, 555, 999):
        r = np.linalg.norm(pos - pos[a], axis=1)
        nn = np.sum(W_def(r, h[a]))
        assert abs(h[a] - 1.2 * nn ** (-1.0 / 3.0)) < 1e-9 * h[a]
    # an interior particle of an unjittered lattice: h close to 1.2 x spacing
    q = synth.lattice_particles(n)
    hq, _ = oracle.solve_h(q.x, q.y, q.z, np.full(q.n, 0.1), [555])
    assert abs(hq[0] * n / 1.2 - 1.0) < 0.05


def g_def(pos, a, h, hfact=1.2):
    """The residual of Eq. (7) at h, from the test-side kernel: h - hfact n^(-1/3)."""
    r = np.linalg.norm(pos - pos[a], axis=1)
    return h - hfact * np.sum(W_def(r, h)) ** (-1.0 / 3.0)


def test_h_solve_estimate_route_isolated_particle():
    """Section III-C's last resort.  A particle with no neighbour within 2h
    anywhere in [h0/16, 16 h0] sees only its self term, n(h) = W(0, h) =
    1/(pi h^3), so g(h) = h (1 - hfact pi^(1/3)) < 0 for hfact = 1.2: Newton
    leaves the bracket (its step lands on h = 0), bisection finds no sign
    change, and the solve must return the estimate h0 itself (route 2)."""
    x, y, z = np.array([0.1, 0.9]), np.array([0.1, 0.9]), np.array([0.1, 0.9])
    h0 = 0.01  # 2 x 16 h0 = 0.32, well short of the other particle at 1.39
    assert 1.2 * math.pi ** (1.0 / 3.0) > 1.0
    h, route = oracle.solve_h(x, y, z, np.array([h0]), [0])
    assert route[0] == 2 and h[0] == h0
    # a root that exists but lies below the bracket: h0 far too large on a
    # dense lattice, g > 0 at both ends of [h0/16, 16 h0] (test-side g)
    q = synth.lattice_particles(10)
    pos = q.pos()
    h0 = 10.0
    assert g_def(pos, 555, h0 / 16) > 0 and g_def(pos, 555, 16 * h0) > 0
    h, route = oracle.solve_h(q.x, q.y, q.z, np.array([h0]), [555])
    assert route[0] == 2 and h[0] == h0


@pytest.mark.parametrize("jitter,h0_over_dx", [(0.0, 0.3), (0.2, 0.2)])
def test_h_solve_bisection_route_against_brentq(jitter, h0_over_dx):
    """Newton leaves [h0/16, 16 h0] while a root exists there: the guess h0 is
    so small that no neighbour lies within 2 h0 (spacing dx, nearest
    neighbour >= (1 - 2 jitter) dx > 2 h0), so the first Newton step lands on
    h = 0.  The solve must then bisect (route 1) to the unique root of
    g(h) = h - 1.2 n(h)^(-1/3) (g/h is non-decreasing since n h^3 =
    sum_b w(r_b/h)/pi is), which scipy's brentq finds here on the test-side
    number density."""
    from scipy.optimize import brentq
    nside = 10
    q = synth.lattice_particles(nside, jitter=jitter, seed=4)
    pos = q.pos()
    dx = 1.0 / nside
    targets = [555, 444]
    h0 = np.full(len(targets), h0_over_dx * dx)
    for a in targets:
        r = np.linalg.norm(pos - pos[a], axis=1)
        assert np.sort(r)[1] > 2 * h0[0]
    h, route = oracle.solve_h(q.x, q.y, q.z, h0, targets)
    assert np.all(route == 1)
    for k, a in enumerate(targets):
        lo, hi = h0[k] / 16, 16 * h0[k]
        assert g_def(pos, a, lo) < 0 < g_def(pos, a, hi)
        root = brentq(lambda v: g_def(pos, a, v), lo, hi, xtol=1e-16, rtol=1e-15)
        assert abs(h[k] / root - 1) < 1e-10


def test_pseudo_h0_and_member_rules():
    """Eq. (9) and the member set of the pseudo-particle solve (Section
    III-C), against quantities computed here from the particles alone:
      * one accepted node and nothing else (the root, seen from a far source
        with a wide opening angle): its member set is the root alone, so the
        solve cannot find a root and returns Eq. (9)'s guess
        h0 = hfact * 2 * s_node, s_node = largest distance from the centre of
        mass (numpy) to a particle;
      * a node of size 0 (five coincident particles, leaf capacity 4, so the
        octree splits down to the deepest level) starts from the h of its
        lowest-index particle;
      * the member set is the accepted nodes plus the opened leaves, one
        point each at its centre of mass: every node (solved by Newton or by
        bisection) meets Eq. (7) over those points with the test-side
        kernel."""
    p = synth.uniform_particles(300, 41)
    pos = p.pos()
    t = oracle.Tree(p.x, p.y, p.z, p.m)
    acc, opened = t.walk(np.array([50.0, 50.0, 50.0]), 1e9)
    assert list(acc) == [0] and len(opened) == 0
    members, tgt = oracle.pseudo_members(t, acc, opened)
    assert list(members) == [0] and list(tgt) == [0]
    com = pos.mean(axis=0)  # equal masses
    s_node = np.linalg.norm(pos - com, axis=1).max()
    hn, route = oracle.pseudo_h(t, acc, opened, np.full(p.n, 0.05))
    assert route[0] == 2 and abs(hn[0] / (1.2 * 2 * s_node) - 1) < 1e-13

    a = np.array([0.2, 0.3, 0.4])
    b = np.array([0.7, 0.8, 0.6])
    pts = np.concatenate([np.repeat(a[None], 5, 0), np.repeat(b[None], 5, 0)])
    perm = np.random.default_rng(3).permutation(10)
    pts = pts[perm]
    hin = np.linspace(0.01, 0.1, 10)
    tc = oracle.Tree(pts[:, 0], pts[:, 1], pts[:, 2], np.full(10, 0.1), leaf_size=4)
    zero = np.nonzero((tc.size == 0) & (tc.leaf == 1) & (tc.count == 5))[0]
    assert len(zero) == 2
    h0 = oracle.pseudo_h0(tc, zero, hin)
    for k, nid in enumerate(zero):
        group = np.nonzero(np.all(pts == pts[tc.particles_of(nid)[0]], axis=1))[0]
        assert h0[k] == hin[group.min()]

    q = synth.lognormal_particles(3000, 17, ngrid=32)
    tq = oracle.Tree(q.x, q.y, q.z, q.m)
    src = q.pos()[7]
    acc, opened = tq.walk(src, 0.5)
    assert len(acc) > 20 and len(opened) > 0
    members, tgt = oracle.pseudo_members(tq, acc, opened)
    assert np.array_equal(members, np.sort(np.concatenate([acc, opened])))
    assert np.array_equal(members[tgt], acc)
    hq = np.full(q.n, 0.02)
    hn, route = oracle.pseudo_h(tq, acc, opened, hq)
    mpos = tq.com[members]
    assert np.all(route != 2) and np.sum(route == 0) > 0.5 * len(acc)
    for k in range(len(acc)):
        r = np.linalg.norm(mpos - tq.com[acc[k]], axis=1)
        assert abs(hn[k] - 1.2 * np.sum(W_def(r, hn[k])) ** (-1.0 / 3.0)) < 1e-9 * hn[k]


# ----------------------------------------------------------------- octree and walk

def test_octree_invariants_and_walk_partition():
    p = synth.lognormal_particles(4000, 9, ngrid=32)
    t = oracle.Tree(p.x, p.y, p.z, p.m, 16)
    assert abs(t.mass[0] - 1.0) < 1e-15
    leaves = np.nonzero(t.leaf)[0]
    assert t.count[leaves].sum() == p.n
    assert np.all(t.count[leaves] <= 16)
    # children labels: parent = label >> 3
    for nid in np.nonzero(t.leaf == 0)[0][:200]:
        fc, nc = t.first_child[nid], t.nchild[nid]
        assert np.all(t.label[fc:fc + nc] >> 3 == t.label[nid])
        assert abs(t.mass[fc:fc + nc].sum() - t.mass[nid]) < 1e-13
    # size = distance from the centre of mass to the furthest particle
    for nid in (0, leaves[0], leaves[-1]):
        idx = t.particles_of(nid)
        d = np.sqrt(((p.pos()[idx] - t.com[nid]) ** 2).sum(1)).max()
        assert abs(d - t.size[nid]) < 1e-14
    src = p.pos()[17]
    for theta in (0.3, 0.5, 0.9):
        acc, opened = t.walk(src, theta)
        covered = np.concatenate([t.particles_of(i) for i in np.concatenate([acc, opened])])
        assert len(covered) == p.n and len(np.unique(covered)) == p.n
        m = t.mass[acc].sum() + sum(p.m[t.particles_of(i)].sum() for i in opened)
        assert abs(m - p.m.sum()) < 1e-12
        for i in acc:
            r = np.linalg.norm(t.com[i] - src)
            assert t.size[i] <= theta * r
    # theta -> 0 opens everything down to particles
    acc, opened = t.walk(src, 0.0)
    assert np.all(t.size[acc] == 0.0)
    assert sum(int(t.count[i]) for i in opened) + sum(int(t.count[i]) for i in acc) == p.n


def _walk_output(t, acc, opened):
    """Particle sets of the accepted nodes and the extracted particles."""
    parts = np.concatenate([t.particles_of(i) for i in opened]) if len(opened) else np.zeros(0, np.int64)
    return parts


def test_walk_controls_geometry():
    """Section III-B's thresholds, checked on the particles themselves (not on
    the walk's own bounding-sphere test): every particle within r_part of a
    source comes out as an individual particle; no pseudo-particle coarser
    than a leaf holds a particle within r_leaf of a source; with several
    sources each source's neighbourhood is resolved; the output still
    partitions the particles and conserves mass."""
    p = synth.lognormal_particles(6000, 13, ngrid=32)
    t = oracle.Tree(p.x, p.y, p.z, p.m, 16)
    pos = p.pos()
    srcs = np.array([pos[17], pos[4001]])
    for r_part, r_leaf in ((0.05, 0.05), (0.05, 0.15), (0.0, 0.2), (0.1, 0.3)):
        acc, opened = t.walk(srcs, 0.5, r_part=r_part, r_leaf=r_leaf)
        parts = _walk_output(t, acc, opened)
        covered = np.concatenate([t.particles_of(i) for i in np.concatenate([acc, opened])])
        assert len(covered) == p.n and len(np.unique(covered)) == p.n
        assert abs(t.mass[acc].sum() + p.m[parts].sum() - p.m.sum()) < 1e-12
        d = np.min(np.linalg.norm(pos[:, None, :] - srcs[None, :, :], axis=2), axis=1)
        assert np.all(np.isin(np.nonzero(d < r_part)[0], parts))
        for i in acc:
            if not t.leaf[i]:
                assert d[t.particles_of(i)].min() >= r_leaf, (r_part, r_leaf, i)
        # more resolution near the sources than the plain walk gives
        acc0, opened0 = t.walk(srcs, 0.5)
        assert len(acc) + len(parts) >= len(acc0) + len(_walk_output(t, acc0, opened0))
    # r_part covering the cube: every particle alone; r_leaf covering it with
    # a theta that opens nothing by itself: exactly the leaves
    acc, opened = t.walk(srcs[0], 0.5, r_part=2.0)
    assert len(acc) == 0 and len(_walk_output(t, acc, opened)) == p.n
    acc, opened = t.walk(srcs[0], 1e9, r_leaf=2.0)
    assert len(opened) == 0 and np.array_equal(np.sort(acc), np.nonzero(t.leaf)[0])


def test_walk_region_memory():
    """A region recorded in an earlier step (centre, radius, smallest size
    reached there): every pseudo-particle whose centre of mass lies inside it
    is no larger than that size, unless it is a single particle or a leaf
    that cannot be opened further than its particles; outside, the walk is the
    plain one."""
    p = synth.lognormal_particles(6000, 13, ngrid=32)
    t = oracle.Tree(p.x, p.y, p.z, p.m, 16)
    src = p.pos()[17]
    acc0, opened0 = t.walk(src, 0.5)
    # the region: a large accepted node of the plain walk, refined to a size
    # a quarter of its own
    big = acc0[np.argmax(t.size[acc0])]
    region = np.array([[*t.com[big], t.size[big], 0.25 * t.size[big]]])
    acc, opened = t.walk(src, 0.5, regions=region)
    inside = np.linalg.norm(t.com[acc] - t.com[big], axis=1) < t.size[big]
    assert inside.sum() > 1
    assert np.all(t.size[acc][inside] <= 0.25 * t.size[big])
    assert big not in set(acc.tolist())
    # nodes away from the region are untouched
    far0 = {int(i) for i in acc0 if np.linalg.norm(t.com[i] - t.com[big]) > 3 * t.size[big]}
    assert far0 <= set(acc.tolist())
    covered = np.concatenate([t.particles_of(i) for i in np.concatenate([acc, opened])])
    assert len(covered) == p.n and len(np.unique(covered)) == p.n


# ----------------------------------------------------------------- inverse mapping (Eq. 4)

def test_inverse_map_octants_by_symmetry():
    """Eight octant cells (a 2x2x2 lattice of sites).  The kernel is
    spherically symmetric, so a particle where k cell boundaries meet puts the
    same share of its support into each cell it touches, and the share the
    cube's walls cut off is fixed by symmetry too: at the cube's centre 1/8 in
    every cell, on an edge between two cells 1/2 each, on a wall 1/2 of the
    support inside the cube, at a corner 1/8.  Eq. 4 must then return those
    weighted means of the cell values."""
    sites = synth.lattice_particles(2)
    g = synth.voronoi(sites.pos(), nthreads=1)
    v = np.array([0.9, 0.1, 0.35, 0.6, 0.05, 0.8, 0.45, 0.2])  # cell k = 4 ix + 2 iy + iz
    pos = np.array([[0.5, 0.5, 0.5],    # all eight cells, 1/8 each
                    [0.5, 0.5, 0.2],    # the four cells with iz = 0, 1/4 each
                    [0.5, 0.2, 0.2],    # cells (0,0,0) and (1,0,0), 1/2 each
                    [0.2, 0.2, 0.2],    # cell (0,0,0) alone
                    [0.0, 0.0, 0.0],    # cube corner: 1/8 of the support, in cell (0,0,0)
                    [0.0, 0.5, 0.5],    # wall x = 0 at the cells' common edge: 1/8 in each ix = 0 cell
                    [0.5, 0.5, 1.0]])   # wall z = 1: 1/8 in each iz = 1 cell
    want = np.array([v.mean(), v[[0, 2, 4, 6]].mean(), (v[0] + v[4]) / 2, v[0], v[0] / 8,
                     v[[0, 1, 2, 3]].sum() / 8, v[[1, 3, 5, 7]].sum() / 8])
    h = np.full(len(pos), 0.1)
    res = oracle.map_cells(g, pos[:, 0], pos[:, 1], pos[:, 2], np.ones(len(pos)), h, nthreads=1)
    got = oracle.inverse_map(res["off"], res["idx"], res["frac"], v, len(pos))
    assert np.max(np.abs(got - want)) < 1e-12, got - want


def test_inverse_map_constant_and_linear_fields():
    """Cubic lattice, particles at the sites: a constant cell value comes back
    unchanged on every particle whose support lies inside the cube (the
    weights sum to 1, Eq. 1-3 mass conservation); a linear field x_i of the
    sites comes back as the particle's own x (the lattice is symmetric about
    every site, so the weights' first moment is the particle position)."""
    n = 8
    p = synth.lattice_particles(n)
    g = synth.voronoi(p.pos(), nthreads=1)
    h = np.full(p.n, 1.2 / n)
    res = oracle.map_cells(g, p.x, p.y, p.z, p.m, h)
    interior = np.all((p.pos() >= 2 * h[:, None]) & (p.pos() <= 1 - 2 * h[:, None]), axis=1)
    assert interior.sum() >= 8
    const = oracle.inverse_map(res["off"], res["idx"], res["frac"], np.full(g.ncell, 0.37), p.n)
    assert np.max(np.abs(const[interior] - 0.37)) < 1e-12
    assert np.all(const <= 0.37 + 1e-12)  # wall particles lose weight outside the cube
    lin = oracle.inverse_map(res["off"], res["idx"], res["frac"], g.site[:, 0], p.n)
    assert np.max(np.abs(lin[interior] - p.x[interior])) < 1e-12


def test_inverse_map_conserves_the_weighted_total():
    """sum_a m_a f_ion,a = sum_i f_ion,i M_i (the ionised mass is the same on
    the particles and on the grid), with M_i the oracle's cell masses from
    its own long double sums; a random field on a random Voronoi grid."""
    p = synth.uniform_particles(400, 11)
    g = synth.voronoi(p.pos(), nthreads=1)
    rng = np.random.default_rng(3)
    m = rng.uniform(0.5, 1.5, p.n) / p.n
    h = rng.uniform(0.06, 0.14, p.n)
    res = oracle.map_cells(g, p.x, p.y, p.z, m, h)
    f_ion = rng.random(g.ncell)
    got = oracle.inverse_map(res["off"], res["idx"], res["frac"], f_ion, p.n)
    assert abs(np.dot(m, got) - np.dot(f_ion, res["mass"])) < 1e-13
    # every term is non-negative, so no particle exceeds the largest value
    assert np.all(got >= 0) and np.all(got <= f_ion.max() * (1 + 1e-12))


def test_inverse_map_brute_force_tiny():
    """Four particles, 27 cells: the sum written out as a double loop over
    particles and cells with f_ai taken one pair at a time from the oracle's
    single-pair integral, against the pair-list sum (tolerance: the order of
    the additions)."""
    p = synth.uniform_particles(27, 21)
    g = synth.voronoi(p.pos(), nthreads=1)
    pos = np.array([[0.3, 0.4, 0.5], [0.05, 0.9, 0.5], [0.7, 0.2, 0.8], [0.5, 0.5, 0.5]])
    h = np.array([0.2, 0.15, 0.1, 0.3])
    v = np.random.default_rng(5).random(g.ncell)
    res = oracle.map_cells(g, pos[:, 0], pos[:, 1], pos[:, 2], np.ones(4), h, nthreads=1)
    got = oracle.inverse_map(res["off"], res["idx"], res["frac"], v, 4)
    for a in range(4):
        acc = 0.0
        for i in range(g.ncell):
            r = oracle.map_cells(g, pos[a:a + 1, 0], pos[a:a + 1, 1], pos[a:a + 1, 2], [1.0], h[a:a + 1],
                                 cells=[i], off=np.array([0, 1], np.int64), idx=np.array([0], np.int32),
                                 nthreads=1)
            acc += v[i] * r["frac"][0]
        assert abs(got[a] - acc) < 1e-14 * max(1.0, abs(acc)), (a, got[a], acc)


# ----------------------------------------------------------------- table variant (Section II-B)

def test_table_wedge_nodes_convergence_and_box():
    """The interpolated pyramid integral equals the exact one at the table's
    nodes, its mean error over random points falls by about 4 per halving of
    the spacing (second order, as trilinear interpolation of a smooth
    function must), and outside the table's box it is the exact value."""
    try:
        mean_err = []
        rng = np.random.default_rng(1)
        pts = [(r0, rng.uniform(0, 1) * math.sqrt(4 - r0 * r0), rng.uniform(0, 1.55))
               for r0 in rng.uniform(0, 2, 1500)]
        for n in (17, 33, 65):
            oracle.set_table(n)
            for i, j, k in ((3, 5, 7), (n - 2, 1, n // 2), (1, n - 2, n - 3)):
                r0 = 2.0 * i / (n - 1)
                R0 = math.sqrt(4 - r0 * r0) * j / (n - 1)
                phi = 0.5 * math.pi * k / (n - 1)
                assert abs(oracle.wedge_table(r0, R0, phi) - oracle.wedge(r0, R0, phi)) < 1e-15
            mean_err.append(np.mean([abs(oracle.wedge_table(*q) - oracle.wedge(*q)) for q in pts]))
            for q in ((2.0, 0.3, 0.7), (2.5, 0.1, 0.2), (1.0, 1.8, 0.4), (0.3, 2.5, 1.2)):
                assert oracle.wedge_table(*q) == oracle.wedge(*q)
        assert mean_err[0] / mean_err[1] > 3.0 and mean_err[1] / mean_err[2] > 3.0, mean_err
    finally:
        oracle.set_table(0)


def test_table_mapping_mass_conservation():
    """Pair integrals from the table variant: off, the mapping is the exact
    one bit for bit; on, the interior particles' sum_i f_ai departs from 1 by
    less than the 0.6% the paper quotes for its table already at 33 nodes per
    axis, and the departure shrinks as the table is refined."""
    p = synth.uniform_particles(512, 7)
    g = synth.voronoi(p.pos(), nthreads=1)
    h = np.full(p.n, 0.15)
    ex = oracle.map_cells(g, p.x, p.y, p.z, p.m, h)
    pos = p.pos()
    interior = np.all((pos >= 2 * h[:, None]) & (pos <= 1 - 2 * h[:, None]), axis=1)
    dev = []
    try:
        for n in (17, 33, 65):
            oracle.set_table(n)
            r = oracle.map_cells(g, p.x, p.y, p.z, p.m, h, off=ex["off"], idx=ex["idx"])
            tot = np.zeros(p.n)
            np.add.at(tot, r["idx"], r["frac"])
            dev.append(np.abs(tot[interior] - 1).max())
        oracle.set_table(0)
        again = oracle.map_cells(g, p.x, p.y, p.z, p.m, h, off=ex["off"], idx=ex["idx"])
        assert np.array_equal(again["frac"], ex["frac"])
    finally:
        oracle.set_table(0)
    assert dev[1] < 0.006 and dev[0] > dev[1] > dev[2], dev


# ----------------------------------------------------------------- grid construction (Section II-A)

def test_voronoi_oracle_against_definition_and_qhull():
    """The oracle's clipped Voronoi cells: volumes tile the cube; every vertex
    of a cell is no farther from its site than from any other site (the
    defining property) and lies on at least three of the cell's face planes;
    cells untouched by the walls have exactly Qhull's Voronoi vertices
    (scipy.spatial.Voronoi); a cubic lattice gives cubes."""
    spatial = pytest.importorskip("scipy.spatial")
    p = synth.uniform_particles(150, 23)
    sites = p.pos()
    g = oracle.voronoi_cells(sites)
    vol, _ = oracle.cell_geometry(g)
    assert abs(vol.sum() - 1.0) < 1e-13 and np.all(vol > 0)
    v = np.stack([g.vx, g.vy, g.vz], 1)
    qh = spatial.Voronoi(sites)
    n_checked = 0
    for c in range(g.ncell):
        fb, fe = g.cell_face_off[c], g.cell_face_off[c + 1]
        ids = np.unique(g.face_vert[g.face_vert_off[fb]:g.face_vert_off[fe]])
        cv = v[ids]
        d_own = np.linalg.norm(cv - sites[c], axis=1)
        d_all = np.linalg.norm(cv[:, None, :] - sites[None, :, :], axis=2).min(axis=1)
        assert np.all(d_own <= d_all + 1e-12)
        pl = g.face_plane[fb:fe]
        on = np.abs(cv @ pl[:, :3].T - pl[:, 3]) < 1e-12
        assert np.all(on.sum(axis=1) >= 3)
        region = qh.regions[qh.point_region[c]]
        if -1 in region or np.any(g.face_nb[fb:fe] < 0):
            continue
        # the same vertices both ways, as positions: a degenerate vertex
        # (four or more planes through one point) may be listed twice by one
        # side, so both sets are compared up to that, never skipped
        qv = qh.vertices[region]
        dq = np.linalg.norm(qv[:, None, :] - cv[None, :, :], axis=2)
        assert dq.min(axis=1).max() < 1e-10 and dq.min(axis=0).max() < 1e-10
        n_checked += 1
    assert n_checked >= 10
    lat = oracle.voronoi_cells(synth.lattice_particles(3).pos())
    lv, _ = oracle.cell_geometry(lat)
    assert np.max(np.abs(lv * 27 - 1)) < 1e-13 and np.all(np.diff(lat.cell_face_off) == 6)


def cell_by_vertex_enumeration(sites, i, k0=20):
    """The clipped Voronoi cell of site i written from its definition alone,
    with no clipping: the points x of [0,1]^3 with
    (s_j - s_i).x <= (s_j - s_i).s_i + |s_j - s_i|^2 / 2 for every j.  Its
    vertices are the points where three of those planes (or the cube's walls)
    meet and every constraint holds.  Candidate planes start with the k0
    nearest sites and grow until every site nearer than 2 R (R the largest
    vertex distance found) is among them: a site at distance D puts its
    plane at D/2 from s_i, so farther sites cannot cut the cell.  Returns
    (vertices, plane ids of the facets), plane ids as the oracle's face_nb
    (site index, or -1-w for the walls x<=1, x>=0, y<=1, y>=0, z<=1, z>=0)."""
    from itertools import combinations
    s = sites[i]
    dist = np.linalg.norm(sites - s, axis=1)
    order = np.argsort(dist)[1:]
    eye = np.eye(3)
    wallN = np.array([eye[0], -eye[0], eye[1], -eye[1], eye[2], -eye[2]])
    wallB = np.array([1.0, 0.0, 1.0, 0.0, 1.0, 0.0])
    wallId = -1 - np.arange(6)
    allA = sites[order] - s
    allN = np.concatenate([allA, wallN])
    allB = np.concatenate([allA @ s + 0.5 * np.sum(allA * allA, 1), wallB])
    k = k0
    while True:
        k = min(k, len(order))
        N = np.concatenate([allN[:k], wallN])
        B = np.concatenate([allB[:k], wallB])
        ids = np.concatenate([order[:k], wallId])
        tri = np.array(list(combinations(range(len(N)), 3)))
        M = N[tri]
        det = np.linalg.det(M)
        ok = np.abs(det) > 1e-14
        X = np.linalg.solve(M[ok], B[tri[ok]][..., None])[..., 0]
        # the cell of the candidate planes alone, which contains the true cell
        feas = np.all(N @ X.T <= (B + 1e-12 * np.linalg.norm(N, axis=1))[:, None], axis=0)
        V = X[feas]
        R = np.linalg.norm(V - s, axis=1).max()
        if k == len(order) or dist[order[k]] >= 2 * R + 1e-12:
            break
        k *= 2
    # distinct vertices, and the planes holding three or more of them (facets)
    keep = []
    for v in V:
        if not keep or np.min(np.linalg.norm(np.array(keep) - v, axis=1)) > 1e-10:
            keep.append(v)
    V = np.array(keep)
    Nk = np.concatenate([allN[:k], wallN])
    Bk = np.concatenate([allB[:k], wallB])
    on = np.abs(V @ Nk.T - Bk) < 1e-11 * np.linalg.norm(Nk, axis=1)
    facets = ids[on.sum(axis=0) >= 3]
    return V, np.sort(facets)


@pytest.mark.parametrize("kind", ["uniform", "clumpy"])
def test_voronoi_cells_against_vertex_enumeration(kind):
    """Every sampled cell of the oracle, wall cells included, against the
    cell built above from the definition by vertex enumeration (no clipping,
    no ordering, no welding): the same vertices both ways, the same
    neighbours and walls face for face, and the volume of the convex hull of
    the enumerated vertices (Qhull)."""
    spatial = pytest.importorskip("scipy.spatial")
    if kind == "uniform":
        sites = synth.uniform_particles(150, 29).pos()
    else:
        sites = synth.lognormal_particles(400, 31, ngrid=32).pos()
    g = oracle.voronoi_cells(sites)
    vol, rad = oracle.cell_geometry(g)
    v = np.stack([g.vx, g.vy, g.vz], 1)
    # cells whose enumeration stays small (at most 60 sites within twice the
    # cell's radius: C(66, 3) plane triples); the choice does not enter the check
    near = np.array([np.sum(np.linalg.norm(sites - sites[c], axis=1) < 2 * rad[c]) for c in range(g.ncell)])
    pool = np.nonzero(near <= 61)[0]
    cells = np.random.default_rng(5).choice(pool, min(40, len(pool)), replace=False)
    assert len(cells) >= 30
    n_wall = 0
    for c in cells:
        V, facets = cell_by_vertex_enumeration(sites, c)
        fb, fe = g.cell_face_off[c], g.cell_face_off[c + 1]
        cv = v[np.unique(g.face_vert[g.face_vert_off[fb]:g.face_vert_off[fe]])]
        d = np.linalg.norm(V[:, None, :] - cv[None, :, :], axis=2)
        assert d.min(axis=1).max() < 1e-10 and d.min(axis=0).max() < 1e-10, c
        assert np.array_equal(np.sort(g.face_nb[fb:fe]), facets), c
        assert abs(spatial.ConvexHull(V).volume - vol[c]) < 1e-12 * max(vol[c], 1e-3), c
        n_wall += int(np.any(facets < 0))
    assert n_wall >= 5


def test_centroids_lloyd_and_merge():
    """Cell centroids: the volume-weighted mean of the centroids is the cube's
    centre (0.5, 0.5, 0.5) exactly; a lattice is a fixed point of the Lloyd
    step (centroids = sites).  Lloyd iterations keep the cells tiling the
    cube and make the cell volumes more even.  Merging drops exactly the
    sites within tol of an earlier site."""
    p = synth.uniform_particles(120, 31)
    g = oracle.voronoi_cells(p.pos())
    vol, _ = oracle.cell_geometry(g)
    cen = oracle.cell_centroids(g)
    assert np.max(np.abs((vol[:, None] * cen).sum(0) - 0.5)) < 1e-13
    lat = synth.lattice_particles(3)
    assert np.max(np.abs(oracle.cell_centroids(oracle.voronoi_cells(lat.pos())) - lat.pos())) < 1e-13
    g2, keep = oracle.build_grid(p.pos(), lloyd=3)
    v2, _ = oracle.cell_geometry(g2)
    assert len(keep) == p.n and abs(v2.sum() - 1) < 1e-13
    assert np.std(v2) < 0.7 * np.std(vol)
    sites = np.concatenate([p.pos(), p.pos()[:10] + 1e-9, p.pos()[5:8] + 0.3e-9])
    kept = oracle.merge_sites(sites, 1e-8)
    assert np.array_equal(kept, np.arange(p.n))
    d = np.linalg.norm(sites[:, None, :] - sites[None, :, :], axis=2)
    for i in range(len(sites)):
        assert (i in set(kept.tolist())) == (not np.any(d[i, :i] < 1e-8))
