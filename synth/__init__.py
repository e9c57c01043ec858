"""Seeded synthetic inputs for the Exact SPH -> Voronoi mapping.

This module generates *inputs only*: particle positions and masses, and the
clipped Voronoi grid those particles generate (Section II-A: the particles
are the generating sites of the grid).  It contains none of the mapping's
arithmetic (kernel integrals, pair rules, smoothing lengths), so that the
CUDA library and the CPU oracle can both consume it without sharing any of
the method.

Workloads (stand-ins for the paper's Starbench uniform medium and turbulent
cloud snapshots, which are not available):

* ``uniform_particles`` -- equal-mass particles uniform in the unit cube.
* ``lognormal_particles`` -- equal-mass particles sampled from a log-normal
  density field exp(g), g a Gaussian random field with P(k) ~ k^slope on a
  periodic n^3 grid, scaled to a given standard deviation.
* ``voronoi`` -- the Voronoi tessellation of the sites, clipped to the cube.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_voronoi.so")

BASE_SEED = 20240426


def build(verbose: bool = False) -> str:
    """Compile the Voronoi generator (host C++, OpenMP) in place."""
    src = os.path.join(_HERE, "voronoi.cpp")
    if os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-fPIC", "-shared", src, "-o", _SO]
    if verbose:
        print(" ".join(cmd))
    subprocess.check_call(cmd)
    return _SO


_lib = None


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        lib.vor_build.restype = ctypes.c_void_p
        lib.vor_build.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int,
                                  ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                  ctypes.POINTER(ctypes.c_int64)]
        lib.vor_fill.restype = None
        lib.vor_fill.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 8
        _lib = lib
    return _lib


@dataclass
class Particles:
    """Structure-of-arrays particle set (float64)."""
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    m: np.ndarray

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    def pos(self) -> np.ndarray:
        return np.stack([self.x, self.y, self.z], axis=1)


@dataclass
class Grid:
    """Clipped Voronoi grid in CSR form (see voronoi.cpp for the layout)."""
    cell_face_off: np.ndarray  # int64 [ncell+1]
    face_vert_off: np.ndarray  # int64 [nface+1]
    face_vert: np.ndarray      # int32 [nloop]
    face_nb: np.ndarray        # int32 [nface]
    face_plane: np.ndarray     # float64 [nface,4] (nx,ny,nz,d), n unit outward
    vx: np.ndarray             # float64 [nvert]
    vy: np.ndarray
    vz: np.ndarray
    site: np.ndarray           # float64 [ncell,3]

    @property
    def ncell(self) -> int:
        return int(self.cell_face_off.shape[0] - 1)

    @property
    def nface(self) -> int:
        return int(self.face_vert_off.shape[0] - 1)

    def nbytes(self) -> int:
        """Bytes of the CSR arrays a mapping call reads (face_nb excluded)."""
        return int(sum(a.nbytes for a in (self.cell_face_off, self.face_vert_off, self.face_vert, self.face_plane,
                                          self.vx, self.vy, self.vz, self.site)))


def rng_for(config: int, salt: int = 0) -> np.random.Generator:
    return np.random.default_rng(BASE_SEED + config + 1000 * salt)


def uniform_particles(n: int, seed: int) -> Particles:
    rng = np.random.default_rng(seed)
    p = rng.random((n, 3))
    m = np.full(n, 1.0 / n)
    return Particles(p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), m)


def gaussian_random_field(ngrid: int, slope: float, rng: np.random.Generator) -> np.ndarray:
    """Periodic GRF: white noise filtered by sqrt(P(k)), P ~ k^slope, k=0 removed."""
    noise = rng.standard_normal((ngrid, ngrid, ngrid))
    fk = np.fft.rfftn(noise)
    kx = np.fft.fftfreq(ngrid) * ngrid
    kz = np.fft.rfftfreq(ngrid) * ngrid
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2
    amp = np.zeros_like(k2)
    nz = k2 > 0
    amp[nz] = k2[nz] ** (slope / 4.0)  # sqrt(P) = k^(slope/2) = (k^2)^(slope/4)
    g = np.fft.irfftn(fk * amp, s=(ngrid, ngrid, ngrid), axes=(0, 1, 2))
    return g


def lognormal_particles(n: int, seed: int, sigma: float = 1.5, ngrid: int = 128,
                        slope: float = -4.0) -> Particles:
    """Equal-mass particles sampled from rho ~ exp(g), std(g) = sigma."""
    rng = np.random.default_rng(seed)
    g = gaussian_random_field(ngrid, slope, rng)
    g = (g - g.mean()) / g.std() * sigma
    rho = np.exp(g).ravel()
    prob = rho / rho.sum()
    vox = rng.choice(rho.size, size=n, p=prob)
    iz = vox % ngrid
    iy = (vox // ngrid) % ngrid
    ix = vox // (ngrid * ngrid)
    u = rng.random((n, 3))
    x = (ix + u[:, 0]) / ngrid
    y = (iy + u[:, 1]) / ngrid
    z = (iz + u[:, 2]) / ngrid
    m = np.full(n, 1.0 / n)
    return Particles(x, y, z, m)


def batch_specs(nsnap: int, seed: int, log2_lo: float = 10.0, log2_hi: float = 18.0):
    """Uneven batch of independent snapshots: particle counts log-uniform in
    [2^log2_lo, 2^log2_hi]; half uniform, half log-normal clumpy with
    sigma_ln_rho uniform in [1, 2].  Returns (n, kind, sigma, seed) tuples."""
    rng = np.random.default_rng(seed)
    n = np.exp(rng.uniform(log2_lo * np.log(2.0), log2_hi * np.log(2.0), nsnap)).astype(np.int64)
    kind = np.array(["uniform", "clumpy"] * ((nsnap + 1) // 2))[:nsnap]
    rng.shuffle(kind)
    sigma = rng.uniform(1.0, 2.0, nsnap)
    seeds = rng.integers(1, 2**31, nsnap)
    return [(int(n[j]), str(kind[j]), float(sigma[j]), int(seeds[j])) for j in range(nsnap)]


def batch_particles(spec) -> Particles:
    """The particles of one batch_specs entry (clumpy fields on a 64^3 grid)."""
    n, kind, sigma, seed = spec
    if kind == "uniform":
        return uniform_particles(n, seed)
    return lognormal_particles(n, seed, sigma=sigma, ngrid=64)


def lattice_particles(nside: int, jitter: float = 0.0, seed: int = 0) -> Particles:
    """Cubic lattice of nside^3 equal-mass particles at cell centres."""
    g = (np.arange(nside) + 0.5) / nside
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    p = np.stack([x.ravel(), y.ravel(), z.ravel()], 1)
    if jitter:
        p = p + np.random.default_rng(seed).uniform(-jitter, jitter, p.shape) / nside
    n = p.shape[0]
    return Particles(p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(), np.full(n, 1.0 / n))


def dedupe_sites(pos: np.ndarray, rel_tol: float = 1e-6) -> np.ndarray:
    """Indices of sites to keep: drops a site closer than rel_tol * mean spacing
    to an earlier kept site (the tight-cell merge of Section II-A's footnote)."""
    n = pos.shape[0]
    if n == 0:
        return np.zeros(0, np.int64)
    tol = rel_tol * (1.0 / max(n, 1)) ** (1.0 / 3.0)
    q = np.floor(pos / max(tol, 1e-300)).astype(np.int64)
    keep = np.ones(n, bool)
    seen = {}
    for i in range(n):
        key = (int(q[i, 0]), int(q[i, 1]), int(q[i, 2]))
        hit = False
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    j = seen.get((key[0] + dx, key[1] + dy, key[2] + dz))
                    if j is not None and np.sum((pos[i] - pos[j]) ** 2) < tol * tol:
                        hit = True
        if hit:
            keep[i] = False
        else:
            seen[key] = i
    return np.nonzero(keep)[0]


def voronoi(sites: np.ndarray, nthreads: int | None = None) -> Grid:
    """Voronoi tessellation of ``sites`` (float64 [n,3] in [0,1)^3), clipped to the cube."""
    lib = _load()
    pts = np.ascontiguousarray(sites, dtype=np.float64)
    n = pts.shape[0]
    if nthreads is None:
        nthreads = os.cpu_count() or 1
    nf = ctypes.c_int64(); nl = ctypes.c_int64(); nv = ctypes.c_int64()
    h = lib.vor_build(pts.ctypes.data, n, nthreads, ctypes.byref(nf), ctypes.byref(nl), ctypes.byref(nv))
    cfo = np.empty(n + 1, np.int64)
    fvo = np.empty(nf.value + 1, np.int64)
    fv = np.empty(nl.value, np.int32)
    fnb = np.empty(nf.value, np.int32)
    fpl = np.empty((nf.value, 4), np.float64)
    vx = np.empty(nv.value, np.float64)
    vy = np.empty(nv.value, np.float64)
    vz = np.empty(nv.value, np.float64)
    lib.vor_fill(h, cfo.ctypes.data, fvo.ctypes.data, fv.ctypes.data, fnb.ctypes.data,
                 fpl.ctypes.data, vx.ctypes.data, vy.ctypes.data, vz.ctypes.data)
    return Grid(cfo, fvo, fv, fnb, fpl, vx, vy, vz, pts.copy())
