"""Uniform octree and interaction lists (oracle, test infrastructure).

Sec. 3.3: space is partitioned by an octree whose smallest box delta is
larger than the near-field cutoff r_c; pairs of elements in touching leaf
boxes are near (entries computed directly), all others are reached through
multipole/local expansions and translations.

Readings used here (the paper does not spell them out):
  * root = bounding cube of all vertices: centre = centre of the bounding box,
    side = largest extent x (1 + 1e-6);
  * an element belongs to the leaf containing its centroid; box coordinates
    are floor((c - origin) / delta_L), clamped to [0, 2^L - 1];
  * leaf level L = min(first level >= 2 whose fullest leaf holds <= leaf_max
    elements, deepest level with delta_l > r_c);
  * U-list of a leaf: non-empty leaves at Chebyshev distance <= 1 (itself
    included);  V-list of a box at level l >= 2: non-empty boxes at level l
    that are not adjacent to it but whose parents are adjacent (or equal).
Boxes are identified by their Morton key (bits of x, y, z interleaved with
x in the lowest bit).
"""
from __future__ import annotations

import numpy as np


def morton(ix, iy, iz, level):
    """Morton key of integer box coordinates at `level`: bit b of x, y, z at
    key bits 3b, 3b+1, 3b+2 (the box numbering of the octree of Sec. 3.3)."""
    key = np.zeros(np.shape(ix), dtype=np.int64)
    for b in range(level):
        key |= ((np.asarray(ix, np.int64) >> b) & 1) << (3 * b)
        key |= ((np.asarray(iy, np.int64) >> b) & 1) << (3 * b + 1)
        key |= ((np.asarray(iz, np.int64) >> b) & 1) << (3 * b + 2)
    return key


def demorton(key, level):
    """Inverse of morton: the integer box coordinates of a key."""
    key = np.asarray(key, np.int64)
    ix = np.zeros(key.shape, np.int64)
    iy = np.zeros(key.shape, np.int64)
    iz = np.zeros(key.shape, np.int64)
    for b in range(level):
        ix |= ((key >> (3 * b)) & 1) << b
        iy |= ((key >> (3 * b + 1)) & 1) << b
        iz |= ((key >> (3 * b + 2)) & 1) << b
    return ix, iy, iz


def bounding_cube(verts):
    """Root box: the cube around the vertices' bounding box, its side the
    largest extent times (1 + 1e-6) so that no vertex lies on the far face
    (a reading: the paper does not fix the root box)."""
    v = np.asarray(verts, float)
    lo = v.min(axis=0)
    hi = v.max(axis=0)
    side = float((hi - lo).max()) * (1.0 + 1e-6)
    centre = 0.5 * (lo + hi)
    return centre - 0.5 * side, side


def box_coords(points, origin, side, level):
    """Integer coordinates of the box containing each point at `level`
    (clipped to the grid)."""
    nb = 1 << level
    delta = side / nb
    c = np.floor((np.asarray(points, float) - origin[None, :]) / delta).astype(np.int64)
    return np.clip(c, 0, nb - 1)


def choose_leaf_level(centroids, origin, side, rc, leaf_max, max_level=20):
    """Leaf level (a reading: the paper gives no rule): the first level >= 2
    where no box holds more than leaf_max centroids, but not deeper than the
    last level whose box side still exceeds the near-field radius rc."""
    l_rc = 0
    while side / (1 << (l_rc + 1)) > rc and l_rc + 1 <= max_level:
        l_rc += 1
    l_occ = max_level
    for lev in range(2, max_level + 1):
        c = box_coords(centroids, origin, side, lev)
        key = morton(c[:, 0], c[:, 1], c[:, 2], lev)
        _, counts = np.unique(key, return_counts=True)
        if counts.max() <= leaf_max:
            l_occ = lev
            break
    return min(l_occ, l_rc)


class Octree:
    """Uniform-depth octree of the element centroids (Sec. 3.3): elements
    sorted by leaf Morton key (perm), leaf ranges, and the occupied boxes of
    every level."""

    def __init__(self, verts, centroids, rc, leaf_max=64, level=None):
        self.origin, self.side = bounding_cube(verts)
        cen = np.asarray(centroids, float)
        self.L = choose_leaf_level(cen, self.origin, self.side, rc, leaf_max) if level is None else level
        L = self.L
        c = box_coords(cen, self.origin, self.side, L)
        self.elem_key = morton(c[:, 0], c[:, 1], c[:, 2], L)
        self.perm = np.lexsort((np.arange(cen.shape[0]), self.elem_key))  # stable by index
        sk = self.elem_key[self.perm]
        self.leaf_keys, self.leaf_start, self.leaf_count = np.unique(
            sk, return_index=True, return_counts=True)
        self.levels = {}
        for lev in range(L, -1, -1):
            self.levels[lev] = np.unique(self.leaf_keys >> (3 * (L - lev)))

    def delta(self, lev):
        """Box side at level lev."""
        return self.side / (1 << lev)

    def centers(self, lev):
        """Centres of the occupied boxes of level lev, in key order."""
        ix, iy, iz = demorton(self.levels[lev], lev)
        d = self.delta(lev)
        return self.origin[None, :] + (np.stack([ix, iy, iz], 1) + 0.5) * d

    def _coords(self, lev):
        ix, iy, iz = demorton(self.levels[lev], lev)
        return np.stack([ix, iy, iz], 1)

    def ulist(self):
        """(target leaf index, source leaf index) pairs, sorted."""
        c = self._coords(self.L)
        d = np.abs(c[:, None, :] - c[None, :, :]).max(axis=2)
        t, s = np.nonzero(d <= 1)
        return np.stack([t, s], 1)

    def vlist(self, lev):
        """(target box index, source box index) pairs at level lev, sorted."""
        c = self._coords(lev)
        d = np.abs(c[:, None, :] - c[None, :, :]).max(axis=2)
        pc = c >> 1
        dp = np.abs(pc[:, None, :] - pc[None, :, :]).max(axis=2)
        t, s = np.nonzero((d > 1) & (dp <= 1))
        return np.stack([t, s], 1)

    def parent_index(self, lev):
        """For each box at level lev (>0), index of its parent at lev-1."""
        keys = self.levels[lev] >> 3
        return np.searchsorted(self.levels[lev - 1], keys)
