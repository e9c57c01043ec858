"""FP64 CPU oracle for the Exact SPH -> Voronoi mapping (test infrastructure).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg may import this package; the CUDA library never does, and this
package never imports the CUDA library.  The arithmetic lives in
``exactmap_oracle.c`` (plain C, FP64, compiled with FMA contraction off);
this module only marshals numpy arrays into it.

Routes (see the C file's header for the full statement):
  * pair integral f_ai: signed vertex-pyramid decomposition (Section II-B)
    with each pyramid integral I(r0, R0, phi) evaluated by adaptive
    Gauss-Kronrod quadrature of its 1-D reduction;
  * cell mass and density: Eq. (1)-(3), long double sums;
  * inverse mapping: Eq. (4), a plain numpy sum over the pair list;
  * table variant: pyramid integrals interpolated trilinearly in a table of I
    (set_table), the paper's production route;
  * smoothing lengths: Eq. (7)-(9), Newton -> bisection -> estimate;
  * pseudo-particle smoothing lengths: the same solve over the accepted
    nodes and opened leaves (Section III-C) from the Eq. (9) guess;
  * octree, adaptive walk: Section III-A/B, Eq. (5).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "exactmap_oracle.c")
_SO = os.path.join(_HERE, "_exactmap_oracle.so")

HFACT = 1.2
LEAF_SIZE = 16


def build(verbose: bool = False) -> str:
    if os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", _SO, "-lm"]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    return _SO


_lib = None
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_D = ctypes.c_double
_INT = ctypes.c_int


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        for name in ("or_w", "or_dw", "or_F", "or_H"):
            getattr(lib, name).restype = _D
            getattr(lib, name).argtypes = [_D]
        lib.or_W.restype = _D
        lib.or_W.argtypes = [_D, _D]
        lib.or_wedge.restype = _D
        lib.or_wedge.argtypes = [_D, _D, _D]
        lib.or_wedge_table.argtypes = [_D, _D, _D]
        lib.or_wedge_table.restype = _D
        lib.or_table_set.argtypes = [_INT]
        lib.or_table_set.restype = None
        grid8 = [_P] * 8
        lib.or_pair_count.argtypes = grid8 + [_P, _I64, _P, _P, _P, _P, _I64, _P, _INT]
        lib.or_pair_fill.argtypes = grid8 + [_P, _I64, _P, _P, _P, _P, _I64, _P, _P, _INT]
        lib.or_map_cells.argtypes = grid8 + [_P, _I64, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _P, _INT]
        lib.or_cell_geometry.argtypes = grid8 + [_I64, _P, _P]
        lib.or_solve_h.argtypes = [_P, _P, _P, _I64, _P, _I64, _P, _D, _P, _P, _INT]
        lib.or_number_density.argtypes = [_P, _P, _P, _I64, _P, _I64, _P, _P, _INT]
        lib.or_tree_build.restype = _I64
        lib.or_tree_build.argtypes = [_P, _P, _P, _P, _I64, _INT]
        lib.or_tree_nodes.argtypes = [_P] * 11
        lib.or_tree_free.argtypes = []
        _lib = lib
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


def _nthreads(n):
    return int(n) if n else (os.cpu_count() or 1)


# ----------------------------------------------------------------- kernel

def w(q: float) -> float:
    return _load().or_w(q)


def W(r: float, h: float) -> float:
    return _load().or_W(r, h)


def F(u: float) -> float:
    """int_0^u W(r,1) r^2 dr; 4 pi F(u) is the kernel mass inside u."""
    return _load().or_F(u)


def H(u: float) -> float:
    return _load().or_H(u)


def set_table(n: int) -> None:
    """Table variant (Section II-B's production route): n nodes per axis of
    I over r0 in [0, 2], rho = R0 / sqrt(4 - r0^2) in [0, 1], phi in
    [0, pi/2], interpolated trilinearly by wedge_table and by map_cells while
    it is set; n = 0 drops it (exact pyramid integrals again)."""
    _load().or_table_set(int(n))


def wedge_table(r0: float, R0: float, phi: float) -> float:
    return _load().or_wedge_table(r0, R0, phi)


def wedge(r0: float, R0: float, phi: float) -> float:
    """Vertex-pyramid integral I(r0, R0, phi) in units of h (Section II-B)."""
    return _load().or_wedge(r0, R0, phi)


# ----------------------------------------------------------------- grids

def _garr(grid):
    return (
        np.ascontiguousarray(grid.cell_face_off, np.int64),
        np.ascontiguousarray(grid.face_vert_off, np.int64),
        np.ascontiguousarray(grid.face_vert, np.int32),
        np.ascontiguousarray(grid.face_plane, np.float64),
        np.ascontiguousarray(grid.vx, np.float64),
        np.ascontiguousarray(grid.vy, np.float64),
        np.ascontiguousarray(grid.vz, np.float64),
        np.ascontiguousarray(grid.site, np.float64),
    )


def cell_geometry(grid):
    """(volume, radius) of every cell; radius R_i = max vertex distance from the site."""
    lib = _load()
    g = _garr(grid)
    n = grid.ncell
    vol = np.empty(n)
    rad = np.empty(n)
    lib.or_cell_geometry(*[_ptr(a) for a in g], n, _ptr(vol), _ptr(rad))
    return vol, rad


def pair_lists(grid, x, y, z, h, cells=None, nthreads=None):
    """Pair lists (CSR by the listed cells, ascending particle index) by brute force."""
    lib = _load()
    g = _garr(grid)
    cells = np.arange(grid.ncell, dtype=np.int64) if cells is None else np.ascontiguousarray(cells, np.int64)
    x, y, z, h = (np.ascontiguousarray(v, np.float64) for v in (x, y, z, h))
    cnt = np.zeros(len(cells), np.int64)
    nt = _nthreads(nthreads)
    lib.or_pair_count(*[_ptr(a) for a in g], _ptr(cells), len(cells), _ptr(x), _ptr(y), _ptr(z), _ptr(h),
                      len(x), _ptr(cnt), nt)
    off = np.zeros(len(cells) + 1, np.int64)
    np.cumsum(cnt, out=off[1:])
    idx = np.empty(int(off[-1]), np.int32)
    lib.or_pair_fill(*[_ptr(a) for a in g], _ptr(cells), len(cells), _ptr(x), _ptr(y), _ptr(z), _ptr(h),
                     len(x), _ptr(off), _ptr(idx), nt)
    return off, idx


def map_cells(grid, x, y, z, m, h, cells=None, off=None, idx=None, want_frac=True, nthreads=None):
    """Pair integrals, cell masses, volumes and densities for the listed cells.

    Returns dict(off, idx, frac, mass, vol, rho, cells)."""
    lib = _load()
    g = _garr(grid)
    cells = np.arange(grid.ncell, dtype=np.int64) if cells is None else np.ascontiguousarray(cells, np.int64)
    x, y, z, m, h = (np.ascontiguousarray(v, np.float64) for v in (x, y, z, m, h))
    if off is None:
        off, idx = pair_lists(grid, x, y, z, h, cells, nthreads)
    frac = np.empty(len(idx)) if want_frac else None
    mass = np.empty(len(cells))
    vol = np.empty(len(cells))
    rho = np.empty(len(cells))
    lib.or_map_cells(*[_ptr(a) for a in g], _ptr(cells), len(cells), _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(h),
                     _ptr(off), _ptr(idx), _ptr(frac), _ptr(mass), _ptr(vol), _ptr(rho), _nthreads(nthreads))
    return dict(cells=cells, off=off, idx=idx, frac=frac, mass=mass, vol=vol, rho=rho)


def inverse_map(off, idx, frac, cell_value, n):
    """Eq. (4): out[a] = sum over the pairs (i, a) of cell_value[i] * f_ai.

    off, idx, frac: a cell-major pair list (off[k]..off[k+1] are the pairs of
    the k-th listed cell, whose value is cell_value[k]); n particles.  Each
    product is rounded once; np.add.at adds them into each particle's slot
    one at a time in list order, from +0."""
    off = np.asarray(off, np.int64)
    cell = np.repeat(np.arange(len(off) - 1), np.diff(off))
    terms = np.asarray(cell_value, np.float64)[cell] * np.asarray(frac, np.float64)
    out = np.zeros(n)
    np.add.at(out, np.asarray(idx, np.int64), terms)
    return out


# ----------------------------------------------------------------- smoothing lengths

def number_density(x, y, z, h, targets=None, nthreads=None):
    lib = _load()
    x, y, z = (np.ascontiguousarray(v, np.float64) for v in (x, y, z))
    targets = np.arange(len(x), dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
    h = np.ascontiguousarray(np.broadcast_to(h, targets.shape), np.float64)
    out = np.empty(len(targets))
    lib.or_number_density(_ptr(x), _ptr(y), _ptr(z), len(x), _ptr(targets), len(targets), _ptr(h), _ptr(out),
                          _nthreads(nthreads))
    return out


def solve_h(x, y, z, h0, targets=None, hfact=HFACT, nthreads=None):
    """Solve h = hfact n(h)^(-1/3) (Eq. 7-8) for the targets; returns (h, route)."""
    lib = _load()
    x, y, z = (np.ascontiguousarray(v, np.float64) for v in (x, y, z))
    targets = np.arange(len(x), dtype=np.int64) if targets is None else np.ascontiguousarray(targets, np.int64)
    h0 = np.ascontiguousarray(h0, np.float64)
    h = np.empty(len(targets))
    route = np.empty(len(targets), np.int32)
    lib.or_solve_h(_ptr(x), _ptr(y), _ptr(z), len(x), _ptr(targets), len(targets), _ptr(h0), hfact, _ptr(h),
                   _ptr(route), _nthreads(nthreads))
    return h, route


# ----------------------------------------------------------------- octree / walk

class Tree:
    """Octree arrays (one entry per node, depth-first creation order)."""

    def __init__(self, x, y, z, m, leaf_size=LEAF_SIZE):
        lib = _load()
        x, y, z, m = (np.ascontiguousarray(v, np.float64) for v in (x, y, z, m))
        n = lib.or_tree_build(_ptr(x), _ptr(y), _ptr(z), _ptr(m), len(x), leaf_size)
        self.label = np.empty(n, np.int64)
        self.level = np.empty(n, np.int32)
        self.count = np.empty(n, np.int64)
        self.mass = np.empty(n)
        self.com = np.empty((n, 3))
        self.size = np.empty(n)
        self.leaf = np.empty(n, np.int32)
        self.first_child = np.empty(n, np.int64)
        self.nchild = np.empty(n, np.int64)
        self.pbegin = np.empty(n, np.int64)
        self.order = np.empty(len(x), np.int64)
        lib.or_tree_nodes(*[_ptr(a) for a in (self.label, self.level, self.count, self.mass, self.com, self.size,
                                              self.leaf, self.first_child, self.nchild, self.pbegin, self.order)])
        self.nnodes = int(n)

    def walk(self, src, theta, r_part=0.0, r_leaf=0.0, regions=None):
        """Adaptive walk (Section III-B).  A node is opened when, for some source
        (src: one point or k x 3):
          * Eq. (5): r_node = 0 or s_node^2 > theta^2 r_node^2;
          * its bounding sphere (centre of mass, radius s_node) reaches within
            r_part of the source: r_node < r_part + s_node;
          * it is not a leaf and its bounding sphere reaches within r_leaf:
            r_node < r_leaf + s_node (in the annulus at least leaves);
        or when, for some recorded region (cx, cy, cz, R, s_min) of an earlier
        step, its centre of mass lies within R of the region's centre and
        s_node > s_min.  Distances are compared squared, r^2 < (r_x + s)^2,
        each product and sum rounded once.  An opened leaf yields its
        particles.  Depth-first, children in octant order.  Returns (accepted
        node ids, opened leaf ids)."""
        srcs = np.asarray(src, np.float64).reshape(-1, 3)
        regs = np.zeros((0, 5)) if regions is None else np.asarray(regions, np.float64).reshape(-1, 5)
        acc, opened = [], []
        stack = [0]
        while stack:
            nid = stack.pop()
            s = float(self.size[nid])
            leaf = bool(self.leaf[nid])
            op = False
            for sx, sy, sz in srcs:
                dx = float(self.com[nid, 0]) - sx
                dy = float(self.com[nid, 1]) - sy
                dz = float(self.com[nid, 2]) - sz
                r2 = (dx * dx + dy * dy) + dz * dz
                tp = r_part + s
                tl = r_leaf + s
                if r2 == 0.0 or s * s > theta * theta * r2:
                    op = True
                elif r_part > 0.0 and r2 < tp * tp:
                    op = True
                elif not leaf and r_leaf > 0.0 and r2 < tl * tl:
                    op = True
            for cx, cy, cz, rad, smin in regs:
                dx = float(self.com[nid, 0]) - cx
                dy = float(self.com[nid, 1]) - cy
                dz = float(self.com[nid, 2]) - cz
                if (dx * dx + dy * dy) + dz * dz < rad * rad and s > smin:
                    op = True
            if not op:
                acc.append(nid)
            elif leaf:
                opened.append(nid)
            else:
                fc, nc = int(self.first_child[nid]), int(self.nchild[nid])
                stack.extend(range(fc + nc - 1, fc - 1, -1))
        return np.array(acc, np.int64), np.array(opened, np.int64)

    def particles_of(self, node):
        b = self.pbegin[node]
        return np.sort(self.order[b: b + self.count[node]])

    def leaf_of_particles(self):
        """For every particle, the index of the leaf node holding it."""
        out = np.empty(len(self.order), np.int64)
        for nid in np.nonzero(self.leaf)[0]:
            b = self.pbegin[nid]
            out[self.order[b: b + self.count[nid]]] = nid
        return out


def pseudo_members(tree: "Tree", acc, opened):
    """The node set of the pseudo-particle h solve (Section III-C): the
    accepted nodes and the opened leaves, which stand in for their particles
    as one point each (their centre of mass).  Returns the member node ids in
    ascending order and the position of each accepted node in that list."""
    acc = np.asarray(acc, np.int64)
    members = np.sort(np.concatenate([acc, np.asarray(opened, np.int64)]))
    return members, np.searchsorted(members, acc)


def pseudo_h0(tree: "Tree", nodes, h, hfact=HFACT):
    """Eq. (9): the initial guess of a node's smoothing length is hfact times
    twice its size s_node.  A node of size 0 (coincident particles) has no
    such scale; it starts from the h of its first particle (lowest index)."""
    nodes = np.asarray(nodes, np.int64)
    first = np.array([tree.particles_of(i)[0] for i in nodes], np.int64)
    return np.where(tree.size[nodes] > 0, hfact * 2.0 * tree.size[nodes], np.asarray(h, np.float64)[first])


def pseudo_h(tree: "Tree", acc, opened, h, hfact=HFACT, nthreads=None):
    """Smoothing lengths of the accepted nodes (Section III-C, Eq. 7-9): the
    solve of solve_h over the member set of pseudo_members, from the Eq. (9)
    guess of pseudo_h0.  Returns (h, route) per accepted node, in the order
    of acc."""
    members, targets = pseudo_members(tree, acc, opened)
    pos = tree.com[members]
    h0 = pseudo_h0(tree, acc, h, hfact)
    return solve_h(pos[:, 0], pos[:, 1], pos[:, 2], h0, targets, hfact=hfact, nthreads=nthreads)


def particle_h_guess(tree: "Tree", hfact=HFACT):
    """Initial guess for full-resolution particles: hfact * (leaf cube volume /
    leaf count)^(1/3), the number-density estimate of the octree leaf that
    holds the particle."""
    leaf = tree.leaf_of_particles()
    side = np.ldexp(1.0, -tree.level[leaf].astype(np.int64))
    return hfact * side / np.cbrt(tree.count[leaf].astype(np.float64))


# ----------------------------------------------------------------- grid construction (Section II-A)

class VoronoiGrid:
    """Clipped Voronoi grid in the CSR layout the mapping reads (cell ->
    faces -> vertex loops CCW from outside; planes (n, d) with unit outward n;
    face_nb = neighbour site, or -1-w for cube wall w in the order x<=1,
    x>=0, y<=1, y>=0, z<=1, z>=0)."""

    def __init__(self, cells, site):
        cfo, fvo, fv, nb, pl, vs = [0], [0], [], [], [], []
        for verts, faces, planes, nbs in cells:
            base = sum(len(v) for v in vs)
            vs.append(verts)
            for loop, plane, b in zip(faces, planes, nbs):
                fv.extend(base + k for k in loop)
                fvo.append(len(fv))
                pl.append(plane)
                nb.append(b)
            cfo.append(len(fvo) - 1)
        v = np.concatenate(vs) if vs else np.zeros((0, 3))
        self.cell_face_off = np.array(cfo, np.int64)
        self.face_vert_off = np.array(fvo, np.int64)
        self.face_vert = np.array(fv, np.int32)
        self.face_nb = np.array(nb, np.int32)
        self.face_plane = np.array(pl, np.float64).reshape(-1, 4)
        self.vx, self.vy, self.vz = (np.ascontiguousarray(v[:, k]) for k in range(3))
        self.site = np.ascontiguousarray(site, np.float64).reshape(-1, 3)

    @property
    def ncell(self):
        return len(self.cell_face_off) - 1

    @property
    def nface(self):
        return len(self.face_vert_off) - 1


def _clip_cell(verts, faces, planes, nbs, n, d, nb):
    """Keep the part of a convex polyhedron with n.x <= d (vertices relative to
    the site).  Each face loop is clipped in turn (a vertex within a relative
    1e-13 of the plane counts as on it); the new face collects the vertices on
    the plane, ordered by angle around their mean."""
    scale = math.sqrt(max(float(np.max(np.sum(verts * verts, axis=1))), 1e-300))
    tol = 1e-13 * scale
    s = verts @ n - d
    if s.max() <= tol:
        return verts, faces, planes, nbs
    cls = np.where(s < -tol, -1, np.where(s > tol, 1, 0))
    new_v = [verts[i] for i in range(len(verts)) if cls[i] <= 0]
    remap = {}
    for i in range(len(verts)):
        if cls[i] <= 0:
            remap[i] = len(remap)
    on = {remap[i] for i in range(len(verts)) if cls[i] == 0}
    cut = {}

    def cut_vertex(a, b):
        key = (min(a, b), max(a, b))
        if key not in cut:
            t = s[a] / (s[a] - s[b])
            new_v.append(verts[a] + (verts[b] - verts[a]) * t)
            cut[key] = len(new_v) - 1
            on.add(cut[key])
        return cut[key]

    nf, npl, nnb = [], [], []
    for loop, plane, b in zip(faces, planes, nbs):
        out = []
        for k in range(len(loop)):
            a, c = loop[k], loop[(k + 1) % len(loop)]
            if cls[a] <= 0:
                out.append(remap[a])
            if cls[a] * cls[c] < 0:
                out.append(cut_vertex(a, c))
        o2 = []
        for q in out:
            if not o2 or o2[-1] != q:
                o2.append(q)
        while len(o2) > 1 and o2[0] == o2[-1]:
            o2.pop()
        if len(o2) >= 3:
            nf.append(o2)
            npl.append(plane)
            nnb.append(b)
    new_v = np.array(new_v)
    if len(on) >= 3:
        ids = sorted(on)
        c = new_v[ids].mean(axis=0)
        a = np.array([1.0, 0, 0]) if abs(n[0]) < 0.6 else np.array([0, 1.0, 0])
        u1 = np.cross(n, a)
        u1 /= np.linalg.norm(u1)
        u2 = np.cross(n, u1)
        ang = [math.atan2(float((new_v[i] - c) @ u2), float((new_v[i] - c) @ u1)) for i in ids]
        nf.append([i for _, i in sorted(zip(ang, ids))])
        npl.append((n, d))
        nnb.append(nb)
    used = sorted({q for loop in nf for q in loop})
    ren = {q: k for k, q in enumerate(used)}
    return new_v[used], [[ren[q] for q in loop] for loop in nf], npl, nnb


def _voronoi_cell(sites, i):
    """The cell of site i: the cube cut by the bisector plane of every other
    site, nearest first, a site at distance D being skipped once D/2 is at
    least the cell's largest vertex radius (its plane cannot reach the cell).
    Vertices within a relative 1e-11 of each other are welded and faces left
    with fewer than three vertices dropped.  Returns (vertices, loops,
    planes, neighbours) with absolute vertices."""
    s = sites[i]
    lo, hi = -s, 1.0 - s
    verts = np.array([[hi[0] if k & 1 else lo[0], hi[1] if k & 2 else lo[1], hi[2] if k & 4 else lo[2]]
                      for k in range(8)])
    faces = [[1, 3, 7, 5], [0, 4, 6, 2], [2, 6, 7, 3], [0, 1, 5, 4], [4, 5, 7, 6], [0, 2, 3, 1]]
    axes = [np.array(v, float) for v in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1))]
    planes = [(axes[w], float(hi[w // 2] if w % 2 == 0 else -lo[w // 2])) for w in range(6)]
    nbs = [-1 - w for w in range(6)]
    d2 = np.sum((sites - s) ** 2, axis=1)
    for j in np.argsort(d2, kind="stable"):
        if j == i or d2[j] <= 0.0:
            continue
        if d2[j] >= 4.0 * float(np.max(np.sum(verts * verts, axis=1))):
            break
        dd = sites[j] - s
        ln = math.sqrt(d2[j])
        verts, faces, planes, nbs = _clip_cell(verts, faces, planes, nbs, dd / ln, 0.5 * ln, int(j))
    scale = math.sqrt(max(float(np.max(np.sum(verts * verts, axis=1))), 1e-300))
    rep = list(range(len(verts)))
    for a in range(len(verts)):
        for b in range(a):
            if rep[b] == b and np.sum((verts[a] - verts[b]) ** 2) < (1e-11 * scale) ** 2:
                rep[a] = b
                break
    keep = []
    for loop, plane, b in zip(faces, planes, nbs):
        o = []
        for q in loop:
            if not o or o[-1] != rep[q]:
                o.append(rep[q])
        while len(o) > 1 and o[0] == o[-1]:
            o.pop()
        if len(o) >= 3:
            keep.append((o, plane, b))
    used = sorted({q for o, _, _ in keep for q in o})
    ren = {q: k for k, q in enumerate(used)}
    out_faces, out_planes, out_nb = [], [], []
    for o, (nv, _), b in keep:
        out_faces.append([ren[q] for q in o])
        if b < 0:
            dabs = 1.0 if (-1 - b) % 2 == 0 else 0.0
        else:
            dabs = float(nv @ (0.5 * (s + sites[b])))
        out_planes.append([nv[0], nv[1], nv[2], dabs])
        out_nb.append(b)
    return verts[used] + s, out_faces, out_planes, out_nb


def voronoi_cells_of(sites, which):
    """The cells of the listed sites only (each against all sites)."""
    sites = np.asarray(sites, np.float64).reshape(-1, 3)
    return [_voronoi_cell(sites, int(i)) for i in which]


def voronoi_cells(sites):
    """The Voronoi cell of every site, clipped to the unit cube (Section
    II-A), as a VoronoiGrid.  Plain numpy, for small site counts."""
    sites = np.asarray(sites, np.float64).reshape(-1, 3)
    return VoronoiGrid([_voronoi_cell(sites, i) for i in range(len(sites))], sites)


def cell_centroids(grid):
    """Centroid of every cell: the volume-weighted mean of the tetrahedra
    (site, fan triangle of a face)."""
    out = np.empty((grid.ncell, 3))
    v = np.stack([grid.vx, grid.vy, grid.vz], 1)
    for c in range(grid.ncell):
        s = grid.site[c]
        tv, tc = 0.0, np.zeros(3)
        for f in range(grid.cell_face_off[c], grid.cell_face_off[c + 1]):
            loop = grid.face_vert[grid.face_vert_off[f]:grid.face_vert_off[f + 1]]
            a = v[loop[0]]
            for k in range(1, len(loop) - 1):
                b, e = v[loop[k]], v[loop[k + 1]]
                vol = float(np.dot(a - s, np.cross(b - s, e - s))) / 6.0
                tv += vol
                tc += vol * (s + a + b + e) / 4.0
        out[c] = tc / tv
    return out


def merge_sites(sites, tol):
    """Indices of the sites kept when tightly packed cells are merged
    (Section II-A footnote): a site within tol of any earlier site is
    dropped."""
    sites = np.asarray(sites, np.float64).reshape(-1, 3)
    keep = []
    for i in range(len(sites)):
        d2 = np.sum((sites[:i] - sites[i]) ** 2, axis=1)
        if not np.any(d2 < tol * tol):
            keep.append(i)
    return np.array(keep, np.int64)


def build_grid(sites, lloyd=5, merge_tol=0.0):
    """Grid construction of Section II-A: merge tightly packed sites, then
    `lloyd` Lloyd iterations (each site moved to its cell's centroid), then
    the Voronoi cells of the final sites.  Returns (grid, kept indices)."""
    sites = np.asarray(sites, np.float64).reshape(-1, 3)
    keep = merge_sites(sites, merge_tol) if merge_tol > 0 else np.arange(len(sites))
    s = sites[keep]
    for _ in range(lloyd):
        s = cell_centroids(voronoi_cells(s))
    return voronoi_cells(s), keep
