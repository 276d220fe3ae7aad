"""Pins of the oracle's nested refinement (Section 2.2: each triangle split into four)."""

import numpy as np

from workloads import square_mesh, crisscross_mesh, channel_cylinder_mesh, VEL_DIR, PHI_ZERO
from oracle.mesh import refine, build_hierarchy, unique_edges, csr_pattern


def _area2(xy, tri):
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    return (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1])


def test_single_triangle_by_hand():
    # worked by hand: edges (0,1),(0,2),(1,2) -> new vertices 3,4,5
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2]])
    tag = np.array([VEL_DIR, VEL_DIR | PHI_ZERO, PHI_ZERO], dtype=np.uint8)
    xf, tf, gf, par = refine(xy, tri, tag)
    assert np.array_equal(xf[3:], [[0.5, 0.0], [0.0, 0.5], [0.5, 0.5]])
    # a=0,b=1,c=2: m_ab=3, m_bc=5, m_ca=4
    assert np.array_equal(tf, [[0, 3, 4], [3, 1, 5], [4, 5, 2], [3, 5, 4]])
    assert np.array_equal(par, [[0, 1], [0, 2], [1, 2]])
    # all three edges are boundary edges: AND of the end flags
    assert list(gf[3:]) == [VEL_DIR & (VEL_DIR | PHI_ZERO), VEL_DIR & PHI_ZERO, (VEL_DIR | PHI_ZERO) & PHI_ZERO]


def test_counts_euler_orientation_area():
    for base, holes in ((square_mesh(4), 0), (crisscross_mesh(3), 0)):
        levels = build_hierarchy(base.xy, base.tri, base.tag, 3)
        for l in range(3):
            L0, L1 = levels[l], levels[l + 1]
            ends, count, _ = unique_edges(L0.tri)
            assert L1.n_tri == 4 * L0.n_tri
            assert L1.n_vert == L0.n_vert + ends.shape[0]
            assert L0.n_vert - ends.shape[0] + L0.n_tri == 1 - holes
            # coarse vertices are an unchanged prefix
            assert np.array_equal(L1.xy[:L0.n_vert], L0.xy)
            assert np.array_equal(L1.tag[:L0.n_vert], L0.tag)
            a0 = _area2(L0.xy, L0.tri)
            a1 = _area2(L1.xy, L1.tri).reshape(-1, 4)
            assert (a1 > 0).all()
            np.testing.assert_allclose(a1.sum(axis=1), a0, rtol=1e-14, atol=0)
            np.testing.assert_allclose(a1, np.repeat(a0[:, None] / 4, 4, 1), rtol=1e-12)


def test_refined_square_equals_half_spacing_mesh():
    # red refinement of the diagonal-split mesh is the diagonal-split mesh of half spacing
    for n in (2, 4, 8):
        xf, tf, gf, _ = refine(*(lambda m: (m.xy, m.tri, m.tag))(square_mesh(n)))
        ref = square_mesh(2 * n)

        def tri_set(xy, tri):
            return {tuple(sorted(map(tuple, xy[t]))) for t in tri}

        assert tri_set(xf, tf) == tri_set(ref.xy, ref.tri)
        flags = {tuple(p): g for p, g in zip(ref.xy, ref.tag)}
        assert all(flags[tuple(p)] == g for p, g in zip(xf, gf))


def test_channel_hierarchy_topology_and_flags():
    base = channel_cylinder_mesh(seed=3, h=0.05)
    levels = build_hierarchy(base.xy, base.tri, base.tag, 2)
    L = base.meta["L"]
    for lev in levels:
        ends, count, _ = unique_edges(lev.tri)
        assert lev.n_vert - ends.shape[0] + lev.n_tri == 0          # one hole
        x, y = lev.xy[:, 0], lev.xy[:, 1]
        outflow_inner = (x == L) & (y > 0) & (y < base.meta["H"])
        assert (lev.tag[outflow_inner] == PHI_ZERO).all()
        corners = (x == L) & ((y == 0) | (y == base.meta["H"]))
        assert (lev.tag[corners] == VEL_DIR | PHI_ZERO).all()
        assert ((lev.tag[(x == 0.0)] == VEL_DIR)).all()
        # boundary vertices = end points of edges with one triangle
        bnd = np.zeros(lev.n_vert, bool)
        bnd[ends[count == 1].ravel()] = True
        assert np.array_equal(bnd, lev.tag != 0)


def test_csr_pattern_is_vertex_adjacency():
    m = crisscross_mesh(2)
    rp, col = csr_pattern(m.n_vert, m.tri)
    adj = [set() for _ in range(m.n_vert)]
    for t in m.tri:
        for a in t:
            adj[a].update(int(b) for b in t)
    for i in range(m.n_vert):
        assert list(col[rp[i]:rp[i + 1]]) == sorted(adj[i])
