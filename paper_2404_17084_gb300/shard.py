"""One snapshot split over several ranks (one process per GPU).

Every cell's mass M_i = sum_a m_a f_ai (Eq. 1-3) depends only on the cell and
the particles whose support can reach it, so the cells of one snapshot split
into independent shards:

  * cells are ordered by the Morton key of their sites and cut into
    contiguous ranges of about equal estimated cost (pairs ~ the particles
    within each cell's reach), one range per rank, so that each shard is a
    compact region of the cube;
  * a rank keeps every particle whose support may reach one of its cells
    (the halo): |r_a - s_i| < 2 h_a + R_i for some cell i of the shard, the
    first test of the pair rule, so the shard's pair lists are exactly the
    full snapshot's lists for those cells, in the same order (particles keep
    their relative order);
  * each rank maps its shard; the only collective is one all-reduce of the
    total mass (and a gather of the cell masses where a caller wants them on
    one rank).

This module is host logic (numpy and scipy's k-d tree): it cuts a grid and
a particle set into the shard a rank maps with the same entry points as a
whole snapshot.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


def morton_keys(pos: np.ndarray, bits: int = 21) -> np.ndarray:
    """63-bit Morton keys of points in the unit cube (x the most significant
    axis of each triple)."""
    c = np.clip((np.asarray(pos, np.float64) * (1 << bits)).astype(np.int64), 0, (1 << bits) - 1).astype(np.uint64)
    key = np.zeros(len(c), np.uint64)
    for b in range(bits):
        for ax in range(3):
            key |= ((c[:, ax] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + 2 - ax)
    return key


def cell_radius(grid) -> np.ndarray:
    """R_i: the largest distance from a cell's site to its vertices."""
    v = np.stack([grid.vx, grid.vy, grid.vz], 1)
    cfo, fvo, fv = grid.cell_face_off, grid.face_vert_off, grid.face_vert
    out = np.empty(len(cfo) - 1)
    for c in range(len(out)):
        ids = fv[fvo[cfo[c]]:fvo[cfo[c + 1]]]
        out[c] = np.sqrt(((v[ids] - grid.site[c]) ** 2).sum(1).max())
    return out


def partition_cells(grid, nranks: int, weight=None) -> list:
    """Cells of each rank: contiguous ranges of the sites' Morton order with
    about equal total weight (default: one per cell).  Every cell is in
    exactly one range; ranges are sorted by cell index."""
    order = np.argsort(morton_keys(grid.site), kind="stable")
    w = np.ones(len(order)) if weight is None else np.asarray(weight, np.float64)[order]
    cum = np.cumsum(w)
    cuts = np.searchsorted(cum, cum[-1] * np.arange(1, nranks) / nranks, side="left")
    return [np.sort(part) for part in np.split(order, cuts)]


@dataclass
class ShardGrid:
    """A grid restricted to some cells (CSR re-based; the vertex arrays are
    shared with the full grid, so face_vert keeps its values)."""
    cell_face_off: np.ndarray
    face_vert_off: np.ndarray
    face_vert: np.ndarray
    face_plane: np.ndarray
    vx: np.ndarray
    vy: np.ndarray
    vz: np.ndarray
    site: np.ndarray

    @property
    def ncell(self) -> int:
        return len(self.cell_face_off) - 1

    @property
    def nface(self) -> int:
        return len(self.face_vert_off) - 1


def shard_grid(grid, cells: np.ndarray) -> ShardGrid:
    cfo, fvo = grid.cell_face_off, grid.face_vert_off
    faces = np.concatenate([np.arange(cfo[c], cfo[c + 1]) for c in cells]) if len(cells) else np.zeros(0, np.int64)
    nf = np.diff(cfo)[cells]
    new_cfo = np.concatenate([[0], np.cumsum(nf)]).astype(np.int64)
    nl = (fvo[faces + 1] - fvo[faces]) if len(faces) else np.zeros(0, np.int64)
    new_fvo = np.concatenate([[0], np.cumsum(nl)]).astype(np.int64)
    loops = np.concatenate([np.arange(fvo[f], fvo[f + 1]) for f in faces]) if len(faces) else np.zeros(0, np.int64)
    return ShardGrid(new_cfo, new_fvo, np.asarray(grid.face_vert)[loops].astype(np.int32),
                     np.asarray(grid.face_plane)[faces], grid.vx, grid.vy, grid.vz, np.asarray(grid.site)[cells])


def halo(grid, cells: np.ndarray, pos: np.ndarray, h: np.ndarray, radius=None) -> np.ndarray:
    """Indices (ascending) of the particles whose support may reach one of
    the cells: |r_a - s_i| < 2 h_a + R_i for some cell i -- the pair rule's
    first test, so no listed pair of those cells is left out."""
    from scipy.spatial import cKDTree
    if len(cells) == 0:
        return np.zeros(0, np.int64)
    R = cell_radius(grid)[cells] if radius is None else np.asarray(radius)[cells]
    site = np.asarray(grid.site)[cells]
    tree = cKDTree(site)
    reach = 2.0 * np.asarray(h) + R.max()
    cand = tree.query_ball_point(pos, reach * (1.0 + 1e-12) + 1e-15)
    keep = np.zeros(len(pos), bool)
    for a, near in enumerate(cand):
        if near:
            d = np.linalg.norm(site[near] - pos[a], axis=1)
            keep[a] = bool(np.any(d < 2.0 * h[a] + R[near]))
    return np.nonzero(keep)[0]


@dataclass
class Shard:
    cells: np.ndarray      # the rank's cells (indices into the full grid)
    grid: ShardGrid        # those cells
    particles: np.ndarray  # the halo (indices into the full particle set, ascending)


def make_shard(grid, pos: np.ndarray, h: np.ndarray, rank: int, nranks: int, weight=None) -> Shard:
    """The shard of `rank` among `nranks`: its cells, their grid and the
    particles that can reach them."""
    cells = partition_cells(grid, nranks, weight)[rank]
    return Shard(cells, shard_grid(grid, cells), halo(grid, cells, pos, h))
