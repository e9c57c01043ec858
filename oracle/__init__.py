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
  * octree, adaptive walk: Section III-A/B, Eq. (5).
"""
from __future__ import annotations

import ctypes
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


def particle_h_guess(tree: "Tree", hfact=HFACT):
    """Initial guess for full-resolution particles: hfact * (leaf cube volume /
    leaf count)^(1/3), the number-density estimate of the octree leaf that
    holds the particle."""
    leaf = tree.leaf_of_particles()
    side = np.ldexp(1.0, -tree.level[leaf].astype(np.int64))
    return hfact * side / np.cbrt(tree.count[leaf].astype(np.float64))
