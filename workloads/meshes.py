"""Seeded base-mesh generators (inputs only; no part of the method).

Every generator returns a :class:`BaseMesh` whose triangles are counter-clockwise
and whose vertex flags mark the boundary parts (see the package docstring).
The meshes follow the workloads of the paper's Section 3 (unit square
Taylor-Green domain, Section 3.1) and the benchmark workloads built on them
(lid-driven cavity, channel with a cylinder).
"""

from dataclasses import dataclass, field

import numpy as np

VEL_DIR = 1
PHI_ZERO = 2


@dataclass
class BaseMesh:
    xy: np.ndarray            # (n_vert, 2) float64
    tri: np.ndarray           # (n_tri, 3) int32, counter-clockwise
    tag: np.ndarray           # (n_vert,) uint8, VEL_DIR | PHI_ZERO flags
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def n_vert(self):
        return int(self.xy.shape[0])

    @property
    def n_tri(self):
        return int(self.tri.shape[0])


def _signed_area2(xy, tri):
    a, b, c = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    return (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (c[:, 0] - a[:, 0]) * (b[:, 1] - a[:, 1])


def _grid_coords(n, lo, hi):
    # i/n is exact for power-of-two n, so refined midpoints land on the grid exactly
    return lo + (hi - lo) * (np.arange(n + 1, dtype=np.float64) / n)


def square_mesh(n, x0=0.0, x1=1.0, y0=0.0, y1=1.0, boundary_flags=VEL_DIR):
    """n x n squares, each split by its (i,j)-(i+1,j+1) diagonal into two triangles.

    Vertex (i, j) has index i + (n+1) j; square (i, j) gives triangles
    [(i,j),(i+1,j),(i+1,j+1)] and [(i,j),(i+1,j+1),(i,j+1)] in that order.
    All boundary vertices get ``boundary_flags``.
    """
    xs, ys = _grid_coords(n, x0, x1), _grid_coords(n, y0, y1)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    xy = np.stack([X.ravel(), Y.ravel()], axis=1)
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i, j = i.ravel(), j.ravel()
    v00 = i + (n + 1) * j
    v10, v11, v01 = v00 + 1, v00 + (n + 1) + 1, v00 + (n + 1)
    tri = np.empty((2 * n * n, 3), dtype=np.int32)
    tri[0::2] = np.stack([v00, v10, v11], axis=1)
    tri[1::2] = np.stack([v00, v11, v01], axis=1)
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    on_b = (ii.ravel() == 0) | (ii.ravel() == n) | (jj.ravel() == 0) | (jj.ravel() == n)
    tag = np.where(on_b, boundary_flags, 0).astype(np.uint8)
    return BaseMesh(xy, tri, tag, name="square%d" % n,
                    meta={"area": (x1 - x0) * (y1 - y0), "n": n})


def crisscross_mesh(n, x0=0.0, x1=1.0, y0=0.0, y1=1.0, boundary_flags=VEL_DIR):
    """n x n squares, each split into four triangles through its centre.

    This gives the 4 * 4^j element counts of the paper's square-domain tables
    (1024, 4096, 16384, 65536 elements in Tables 1-4).  Grid vertices come first
    (i + (n+1) j), then square centres (i + n j).
    """
    xs, ys = _grid_coords(n, x0, x1), _grid_coords(n, y0, y1)
    X, Y = np.meshgrid(xs, ys, indexing="xy")
    grid = np.stack([X.ravel(), Y.ravel()], axis=1)
    cx = 0.5 * (xs[:-1] + xs[1:])
    cy = 0.5 * (ys[:-1] + ys[1:])
    CX, CY = np.meshgrid(cx, cy, indexing="xy")
    cen = np.stack([CX.ravel(), CY.ravel()], axis=1)
    xy = np.concatenate([grid, cen])
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i, j = i.ravel(), j.ravel()
    v00 = i + (n + 1) * j
    v10, v11, v01 = v00 + 1, v00 + (n + 1) + 1, v00 + (n + 1)
    c = (n + 1) ** 2 + i + n * j
    tri = np.empty((4 * n * n, 3), dtype=np.int32)
    tri[0::4] = np.stack([v00, v10, c], axis=1)
    tri[1::4] = np.stack([v10, v11, c], axis=1)
    tri[2::4] = np.stack([v11, v01, c], axis=1)
    tri[3::4] = np.stack([v01, v00, c], axis=1)
    ii, jj = np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="xy")
    on_b = (ii.ravel() == 0) | (ii.ravel() == n) | (jj.ravel() == 0) | (jj.ravel() == n)
    tag = np.concatenate([np.where(on_b, boundary_flags, 0),
                          np.zeros(n * n, dtype=np.int64)]).astype(np.uint8)
    return BaseMesh(xy, tri, tag, name="crisscross%d" % n,
                    meta={"area": (x1 - x0) * (y1 - y0), "n": n})


def _morton_key(p, lo, hi, bits=16):
    q = ((p - lo) / (hi - lo) * ((1 << bits) - 1)).astype(np.uint64)
    key = np.zeros(p.shape[0], dtype=np.uint64)
    for b in range(bits):
        key |= ((q[:, 0] >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b)
        key |= ((q[:, 1] >> np.uint64(b)) & np.uint64(1)) << np.uint64(2 * b + 1)
    return key


def _poisson_disk(rng, h, inside, fixed, lo, hi, k=30):
    """Bridson's dart throwing: points >= h apart (and >= h from ``fixed``)."""
    cell = h / np.sqrt(2.0)
    gw = int(np.ceil((hi[0] - lo[0]) / cell)) + 1
    gh = int(np.ceil((hi[1] - lo[1]) / cell)) + 1
    grid = -np.ones((gh + 6, gw + 6), dtype=np.int64)   # 3-cell pad on every side
    pts = [p for p in fixed]

    def gidx(p):
        return int((p[1] - lo[1]) / cell) + 3, int((p[0] - lo[0]) / cell) + 3

    def far_enough(cands):
        ok = np.ones(len(cands), dtype=bool)
        for n, c in enumerate(cands):
            gy, gx = gidx(c)
            # 7x7 cells: also sees a boundary point displaced into a neighbouring cell
            nb = grid[gy - 3:gy + 4, gx - 3:gx + 4].ravel()
            nb = nb[nb >= 0]
            if nb.size:
                d2 = ((parr[nb] - c) ** 2).sum(axis=1)
                if d2.min() < h * h:
                    ok[n] = False
        return ok

    # fixed (boundary) points go into the grid but never into the active list;
    # two boundary points may share a cell, so keep a side list for those
    extra = []
    for n, p in enumerate(fixed):
        gy, gx = gidx(p)
        if grid[gy, gx] < 0:
            grid[gy, gx] = n
        else:
            extra.append(n)
    parr = np.array(pts, dtype=np.float64)
    if extra:
        # put overflowing boundary points into any free neighbouring cell slot
        for n in extra:
            gy, gx = gidx(parr[n])
            placed = False
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    if not placed and grid[gy + dy, gx + dx] < 0:
                        grid[gy + dy, gx + dx] = n
                        placed = True
            if not placed:
                raise RuntimeError("boundary points too dense for the sampling grid")
    # start from a random interior point
    while True:
        p0 = lo + rng.random(2) * (hi - lo)
        if inside(p0[None, :])[0] and far_enough(p0[None, :])[0]:
            break
    cap = len(pts) + int(4.0 * np.prod(hi - lo) / (h * h)) + 16
    buf = np.empty((cap, 2), dtype=np.float64)
    buf[:len(pts)] = parr
    npts = len(pts)
    buf[npts] = p0
    parr = buf
    active = [npts]
    npts += 1
    gy, gx = gidx(p0)
    grid[gy, gx] = npts - 1
    while active:
        a = active[rng.integers(len(active))]
        r = h * (1.0 + rng.random(k))
        th = 2.0 * np.pi * rng.random(k)
        cands = parr[a] + np.stack([r * np.cos(th), r * np.sin(th)], axis=1)
        keep = inside(cands)
        found = False
        for c in cands[keep]:
            if far_enough(c[None, :])[0]:
                parr[npts] = c
                gy, gx = gidx(c)
                grid[gy, gx] = npts
                active.append(npts)
                npts += 1
                found = True
                break
        if not found:
            active.remove(a)
    return parr[:npts].copy()


def channel_cylinder_mesh(seed=0, h=0.0084, L=2.2, H=0.41, xc=0.2, yc=0.2, r=0.05):
    """Channel [0,L]x[0,H] minus a disk, from a seeded Poisson-disk point set.

    Boundary points sit at spacing ~h on the four sides and on a polygon of the
    cylinder; interior points come from Bridson's sampling with radius h.  The
    triangulation is the Delaunay triangulation (scipy/qhull) with the triangles
    inside the polygon removed.  Flags: inflow (x=0), walls (y=0, y=H) and
    cylinder get VEL_DIR; the outflow (x=L) gets PHI_ZERO; the two outflow
    corners get both.  The default h gives about 16k triangles (8.3k vertices).
    r = 0 gives the plain channel (no cylinder).
    """
    from scipy.spatial import Delaunay

    rng = np.random.default_rng(seed)
    nx = max(2, int(round(L / h)))
    ny = max(2, int(round(H / h)))
    xs = L * (np.arange(nx + 1) / nx)
    ys = H * (np.arange(ny + 1) / ny)
    bottom = np.stack([xs, np.zeros_like(xs)], 1)
    top = np.stack([xs, np.full_like(xs, H)], 1)
    left = np.stack([np.zeros(ny - 1), ys[1:-1]], 1)
    right = np.stack([np.full(ny - 1, L), ys[1:-1]], 1)
    nc = max(8, int(round(2.0 * np.pi * r / h))) if r > 0 else 0
    th = 2.0 * np.pi * np.arange(nc) / nc
    cyl = np.stack([xc + r * np.cos(th), yc + r * np.sin(th)], 1)
    fixed = np.concatenate([bottom, top, left, right, cyl])
    ftag = np.concatenate([
        np.where(xs == L, VEL_DIR | PHI_ZERO, VEL_DIR),
        np.where(xs == L, VEL_DIR | PHI_ZERO, VEL_DIR),
        np.full(ny - 1, VEL_DIR), np.full(ny - 1, PHI_ZERO), np.full(nc, VEL_DIR),
    ]).astype(np.uint8)
    cyl_idx = np.arange(len(fixed) - nc, len(fixed))

    def inside(p):
        return ((p[:, 0] > 0.0) & (p[:, 0] < L) & (p[:, 1] > 0.0) & (p[:, 1] < H)
                & ((p[:, 0] - xc) ** 2 + (p[:, 1] - yc) ** 2 > r * r))

    lo, hi = np.array([0.0, 0.0]), np.array([L, H])
    pts = _poisson_disk(rng, h, inside, list(fixed), lo, hi)
    tag = np.concatenate([ftag, np.zeros(len(pts) - len(fixed), dtype=np.uint8)])
    # spatially coherent vertex order (Morton) for memory locality of the hierarchy
    order = np.argsort(_morton_key(pts, lo, hi), kind="stable")
    inv = np.empty_like(order)
    inv[order] = np.arange(len(order))
    pts, tag, cyl_idx = pts[order], tag[order], inv[cyl_idx]
    d = Delaunay(pts)
    tri = d.simplices.astype(np.int64)
    cen = pts[tri].mean(axis=1)
    if nc:
        keep = (cen[:, 0] - xc) ** 2 + (cen[:, 1] - yc) ** 2 > r * r
        tri = tri[keep]
    a2 = _signed_area2(pts, tri)
    flip = a2 < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    a2 = np.abs(a2)
    if a2.min() <= 1e-10 * h * h:
        raise RuntimeError("degenerate triangle in channel mesh (seed %d)" % seed)
    # every cylinder polygon edge must be a mesh edge (the hole is then exact)
    ekeys = set()
    for e in ((0, 1), (1, 2), (2, 0)):
        lo_ = np.minimum(tri[:, e[0]], tri[:, e[1]])
        hi_ = np.maximum(tri[:, e[0]], tri[:, e[1]])
        ekeys.update((lo_ * len(pts) + hi_).tolist())
    for i in range(nc):
        u, v = cyl_idx[i], cyl_idx[(i + 1) % nc]
        if min(u, v) * len(pts) + max(u, v) not in ekeys:
            raise RuntimeError("cylinder edge missing from Delaunay mesh (seed %d)" % seed)
    used = np.zeros(len(pts), dtype=bool)
    used[tri.ravel()] = True
    if not used.all():
        raise RuntimeError("unused vertex in channel mesh (seed %d)" % seed)
    # triangles in Morton order of their centroids
    cen = pts[tri].mean(axis=1)
    tri = tri[np.argsort(_morton_key(cen, lo, hi), kind="stable")]
    area = L * H - (0.5 * nc * r * r * np.sin(2.0 * np.pi / nc) if nc else 0.0)
    return BaseMesh(pts.astype(np.float64), tri.astype(np.int32), tag,
                    name="channel_seed%d" % seed,
                    meta={"area": area, "h": h, "L": L, "H": H, "xc": xc, "yc": yc,
                          "r": r, "n_cyl": nc, "seed": seed})


def open_square_mesh(n):
    """The open-boundary vortex domain of Section 3.2: [0,1]^2 as n x n squares of four
    triangles (crisscross_mesh), velocity Dirichlet data on x = 1, y = 0 and y = 1, the
    traction boundary on the y-axis x = 0 (PHI_ZERO; its two corners carry both flags)."""
    m = crisscross_mesh(n, boundary_flags=0)
    x, y = m.xy[:, 0], m.xy[:, 1]
    tag = np.zeros(m.n_vert, np.uint8)
    tag[(x == 1.0) | (y == 0.0) | (y == 1.0)] |= VEL_DIR
    tag[x == 0.0] |= PHI_ZERO
    m.tag = tag
    m.name = "open_square%d" % n
    return m


def disk_mesh(n_boundary=96, n_interior=1105, r=0.5):
    """The disk of Section 3.3 (x^2 + y^2 < r^2) as an unstructured Delaunay mesh: n_boundary
    vertices on the circle and n_interior vertices inside on a Vogel (golden-angle) spiral,
    so that a triangulation of the convex boundary polygon has exactly
    2 (n_boundary + n_interior) - n_boundary - 2 triangles.  The defaults give the paper's
    Fig. 1 counts: 1201 vertices and 2304 triangles, refined once 4705 / 9216, twice 18,625 /
    36,864.  Every boundary vertex carries VEL_DIR (Dirichlet data on the whole boundary)."""
    from scipy.spatial import Delaunay

    th = 2.0 * np.pi * np.arange(n_boundary) / n_boundary
    bnd = np.stack([r * np.cos(th), r * np.sin(th)], 1)
    # interior radius capped a bit inside the circle, spacing comparable to the boundary's
    k = np.arange(n_interior) + 0.5
    rho = (r - 0.5 * np.pi * r / n_boundary) * np.sqrt(k / n_interior)
    phi = k * np.pi * (3.0 - np.sqrt(5.0))
    inner = np.stack([rho * np.cos(phi), rho * np.sin(phi)], 1)
    pts = np.concatenate([bnd, inner])
    tri = Delaunay(pts).simplices.astype(np.int64)
    a2 = _signed_area2(pts, tri)
    flip = a2 < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    if np.abs(a2).min() <= 1e-12:
        raise RuntimeError("degenerate triangle in the disk mesh")
    tag = np.zeros(len(pts), np.uint8)
    tag[:n_boundary] = VEL_DIR
    area = 0.5 * n_boundary * r * r * np.sin(2.0 * np.pi / n_boundary)
    return BaseMesh(pts.astype(np.float64), tri.astype(np.int32), tag, name="disk%d" % len(pts),
                    meta={"area": area, "r": r, "n_boundary": n_boundary})
