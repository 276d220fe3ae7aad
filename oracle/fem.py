"""P1 finite-element operators and grid transfers (oracle; test infrastructure only).

Section 2.1 of the paper discretises velocity and pressure with piecewise-linear
(P1/P1) Galerkin elements (Eqs. 17-20).  With psi_i the hat function of vertex
i, |T| the area of triangle T and g_i = grad psi_i on T (constant), the exact
element integrals are

* mass            M_ij  = int psi_i psi_j          = |T|/12 (1 + delta_ij)
* stiffness       K_ij  = int grad psi_i . grad psi_j = |T| g_i . g_j
* first derivative Cx_ij = int psi_i d/dx psi_j    = |T|/3 g_j,x   (Cy likewise)
* convection      N_ij  = int psi_i (w . grad psi_j) = |T|/12 (W_T + w_i) . g_j,
  W_T the sum of w over the three vertices of T (w linear on T).

The paper's operators follow as L_v = K / Re, L_p = -K, D = [Cx Cy] and
G = [Cx; Cy] (a reading of Eqs. 17-20: the signs make Eq. 18 the weak form
of Eq. 12 with the Neumann condition of Eq. 13).  The coarse operators of
Eq. 23 are the same formulas on the coarse triangles (Section 2.2).

Grid transfers (Section 2.2, Eqs. 22 and 24): restriction is pure injection at
coincident vertices (the first N_c vertices, by the nested indexing), and
prolongation copies coincident vertices and sets every edge-midpoint vertex to
the mean of the two coarse end values, one level at a time.

Parity: element formulas pinned against an independent quadrature rule and
against closed-form integrals in tests/test_oracle_fem.py; transfers pinned by
exactness on linear fields and R P = I.
"""

import numpy as np
import scipy.sparse as sp


def geometry(xy, tri):
    """Areas |T| (T,) and hat-function gradients g (T, 3, 2) of every triangle."""
    p = np.asarray(xy, dtype=np.float64)[np.asarray(tri)]
    x0, y0 = p[:, 0, 0], p[:, 0, 1]
    x1, y1 = p[:, 1, 0], p[:, 1, 1]
    x2, y2 = p[:, 2, 0], p[:, 2, 1]
    det = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0)
    area = 0.5 * det
    g = np.empty((p.shape[0], 3, 2))
    g[:, 0, 0], g[:, 0, 1] = (y1 - y2) / det, (x2 - x1) / det
    g[:, 1, 0], g[:, 1, 1] = (y2 - y0) / det, (x0 - x2) / det
    g[:, 2, 0], g[:, 2, 1] = (y0 - y1) / det, (x1 - x0) / det
    return area, g


def assemble(n, tri, Ke):
    """Sum element matrices Ke (T, 3, 3) into an n x n CSR matrix (duplicates added)."""
    tri = np.asarray(tri, dtype=np.int64)
    rows = np.repeat(tri, 3, axis=1).ravel()
    cols = np.tile(tri, (1, 3)).ravel()
    A = sp.coo_matrix((Ke.reshape(-1), (rows, cols)), shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A


def element_mass(area):
    base = np.array([[2.0, 1.0, 1.0], [1.0, 2.0, 1.0], [1.0, 1.0, 2.0]])
    return area[:, None, None] / 12.0 * base[None]


def element_stiffness(area, g):
    return area[:, None, None] * np.einsum("tid,tjd->tij", g, g)


def element_deriv(area, g, d):
    """Ce_ij = |T|/3 * g_j[d]  (row i, column j), d = 0 for x, 1 for y."""
    return np.repeat((area[:, None] / 3.0 * g[:, :, d])[:, None, :], 3, axis=1)


def element_convection(area, g, tri, w):
    """Ne_ij = |T|/12 (W_T + w_i) . g_j for a P1 advecting field w (n, 2)."""
    wt = np.asarray(w)[np.asarray(tri)]                  # (T, 3, 2)
    W = wt.sum(axis=1)                                   # (T, 2)
    coef = area[:, None, None] / 12.0 * (W[:, None, :] + wt)   # (T, 3[i], 2)
    return np.einsum("tid,tjd->tij", coef, g)


def static_operators(xy, tri):
    """M, K, Cx, Cy of one level as CSR matrices."""
    n = np.asarray(xy).shape[0]
    area, g = geometry(xy, tri)
    return {
        "M": assemble(n, tri, element_mass(area)),
        "K": assemble(n, tri, element_stiffness(area, g)),
        "Cx": assemble(n, tri, element_deriv(area, g, 0)),
        "Cy": assemble(n, tri, element_deriv(area, g, 1)),
    }


def convection_operator(xy, tri, w):
    n = np.asarray(xy).shape[0]
    area, g = geometry(xy, tri)
    return assemble(n, tri, element_convection(area, g, tri, w))


def inject(u_fine, n_coarse):
    """Restriction by injection (Eq. 22): coarse vertices are the first n_coarse fine ones."""
    return np.array(u_fine[:n_coarse], copy=True)


def prolong_one(phi_c, parents):
    """One level of Eq. 24: copy coincident vertices, average the two ends at midpoints."""
    phi_c = np.asarray(phi_c, dtype=np.float64)
    mid = 0.5 * (phi_c[parents[:, 0]] + phi_c[parents[:, 1]])
    return np.concatenate([phi_c, mid])


def restrict_t_one(y_f, parents, n_coarse):
    """Transpose of one prolongation level: y_c[i] = y_f[i] + 1/2 (sum of y_f over the new
    vertices that have i as an end point of their edge)."""
    y_f = np.asarray(y_f, dtype=np.float64)
    y_c = np.array(y_f[:n_coarse], copy=True)
    new = y_f[n_coarse:]
    np.add.at(y_c, parents[:, 0], 0.5 * new)
    np.add.at(y_c, parents[:, 1], 0.5 * new)
    return y_c


def restrict_t(y_f, levels, l_from, l_to):
    """P^T from level l_from down to level l_to (< l_from): the transposed composition."""
    y = np.asarray(y_f, dtype=np.float64)
    for l in range(l_from, l_to, -1):
        y = restrict_t_one(y, levels[l].parents, levels[l - 1].n_vert)
    return y


def prolong(phi_c, levels, l_from, l_to):
    """Compose the one-level prolongations from level l_from up to level l_to."""
    phi = np.asarray(phi_c, dtype=np.float64)
    for l in range(l_from + 1, l_to + 1):
        phi = prolong_one(phi, levels[l].parents)
    return phi
