"""Nested triangle-mesh hierarchy by uniform refinement (oracle; test infrastructure only).

Section 2.2 of the paper builds the hierarchy V_1 c V_2 c V_3 c V_4 by
subdividing every triangle of a coarse grid into four, so that a grid with N
elements refined k times has M = 4^k N elements.  The paper does not fix an
indexing; the one used here (and required bit-for-bit of the CUDA library) is:

* the vertices of level l are the first N_l vertices of level l+1, unchanged;
* every edge (a, b) of level l, a < b, gets the new vertex N_l + (rank of the
  key (a, b) among all edges of level l in ascending lexicographic order),
  placed at 0.5 * (x_a + x_b), 0.5 * (y_a + y_b);
* triangle t = (a, b, c) with edge midpoints m_ab, m_bc, m_ca has children
  4t+0 = (a, m_ab, m_ca), 4t+1 = (m_ab, b, m_bc), 4t+2 = (m_ca, m_bc, c),
  4t+3 = (m_ab, m_bc, m_ca), all counter-clockwise when t is;
* a new vertex on a boundary edge (an edge of exactly one triangle) gets the
  bitwise AND of its end points' boundary flags; on an interior edge, 0.

Parity: pinned by tests/test_oracle_mesh.py (counts, Euler characteristic,
area, orientation, and equality with the structured mesh of half spacing).
"""

from dataclasses import dataclass

import numpy as np


def unique_edges(tri):
    """Edges of a triangle list.

    Returns (ends, count, tri_edge): ``ends`` is (E, 2) with ends[:,0] < ends[:,1]
    in ascending lexicographic order, ``count`` the number of triangles on each
    edge, and ``tri_edge`` (T, 3) the edge ids of sides (a,b), (b,c), (c,a).
    """
    tri = np.asarray(tri, dtype=np.int64)
    T = tri.shape[0]
    sides = np.concatenate([tri[:, [0, 1]], tri[:, [1, 2]], tri[:, [2, 0]]])
    lo = sides.min(axis=1)
    hi = sides.max(axis=1)
    key = (lo << 32) | hi
    ukey, inverse, count = np.unique(key, return_inverse=True, return_counts=True)
    ends = np.stack([ukey >> 32, ukey & 0xFFFFFFFF], axis=1)
    tri_edge = inverse.reshape(3, T).T
    return ends, count, tri_edge


def refine(xy, tri, tag):
    """One uniform 1 -> 4 refinement with the indexing described in the module docstring.

    Returns (xy_fine, tri_fine, tag_fine, parents) where ``parents`` (E, 2) holds
    the two coarse end points of each new vertex N + e.
    """
    xy = np.asarray(xy, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int64)
    N = xy.shape[0]
    ends, count, te = unique_edges(tri)
    a, b = ends[:, 0], ends[:, 1]
    mid = 0.5 * (xy[a] + xy[b])
    xy_f = np.concatenate([xy, mid])
    bnd = count == 1
    tag_new = np.where(bnd, np.asarray(tag)[a] & np.asarray(tag)[b], 0).astype(np.uint8)
    tag_f = np.concatenate([np.asarray(tag, dtype=np.uint8), tag_new])
    m_ab, m_bc, m_ca = N + te[:, 0], N + te[:, 1], N + te[:, 2]
    A, B, C = tri[:, 0], tri[:, 1], tri[:, 2]
    kids = np.empty((tri.shape[0], 4, 3), dtype=np.int64)
    kids[:, 0] = np.stack([A, m_ab, m_ca], 1)
    kids[:, 1] = np.stack([m_ab, B, m_bc], 1)
    kids[:, 2] = np.stack([m_ca, m_bc, C], 1)
    kids[:, 3] = np.stack([m_ab, m_bc, m_ca], 1)
    return xy_f, kids.reshape(-1, 3).astype(np.int32), tag_f, ends.astype(np.int32)


def csr_pattern(n_vert, tri):
    """Vertex adjacency of a triangle mesh as CSR (diagonal included, columns ascending)."""
    tri = np.asarray(tri, dtype=np.int64)
    r = np.repeat(tri, 3, axis=1).ravel()
    c = np.tile(tri, (1, 3)).ravel()
    key = np.unique((r << 32) | c)
    rows = key >> 32
    cols = key & 0xFFFFFFFF
    rowptr = np.zeros(n_vert + 1, dtype=np.int64)
    np.add.at(rowptr, rows + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr.astype(np.int32), cols.astype(np.int32)


@dataclass
class Level:
    xy: np.ndarray
    tri: np.ndarray
    tag: np.ndarray
    parents: np.ndarray      # (N_l - N_{l-1}, 2) end points of the vertices added at this level
    rowptr: np.ndarray
    col: np.ndarray

    @property
    def n_vert(self):
        return int(self.xy.shape[0])

    @property
    def n_tri(self):
        return int(self.tri.shape[0])


def build_hierarchy(xy, tri, tag, n_levels):
    """Levels 0..n_levels: level 0 is the base mesh, level l+1 = refine(level l)."""
    xy = np.asarray(xy, dtype=np.float64)
    tri = np.asarray(tri, dtype=np.int32)
    tag = np.asarray(tag, dtype=np.uint8)
    rp, cl = csr_pattern(xy.shape[0], tri)
    levels = [Level(xy, tri, tag, np.zeros((0, 2), np.int32), rp, cl)]
    for _ in range(n_levels):
        L = levels[-1]
        xf, tf, gf, par = refine(L.xy, L.tri, L.tag)
        rp, cl = csr_pattern(xf.shape[0], tf)
        levels.append(Level(xf, tf, gf, par, rp, cl))
    return levels
