"""Pins of the oracle's P1 operators and grid transfers (Section 2.1 Eqs. 17-20, Section 2.2)."""

import numpy as np
import pytest

from workloads import square_mesh, crisscross_mesh, channel_cylinder_mesh, PHI_ZERO
from oracle import fem
from oracle.mesh import build_hierarchy
from oracle.cgp import CGPOracle

# Dunavant's 7-point rule, exact for polynomials of degree 5 on a triangle
# (barycentric points, weights summing to 1)
_A1, _B1, _W1 = 0.059715871789770, 0.470142064105115, 0.132394152788506
_A2, _B2, _W2 = 0.797426985353087, 0.101286507323456, 0.125939180544827
QP = np.array([[1 / 3, 1 / 3, 1 / 3],
               [_A1, _B1, _B1], [_B1, _A1, _B1], [_B1, _B1, _A1],
               [_A2, _B2, _B2], [_B2, _A2, _B2], [_B2, _B2, _A2]])
QW = np.array([0.225, _W1, _W1, _W1, _W2, _W2, _W2])


def _quadrature_element(p, w):
    """Element matrices by quadrature; gradients from inverting the 3x3 Vandermonde."""
    V = np.column_stack([np.ones(3), p])
    coef = np.linalg.inv(V)             # column i: (a, bx, by) of hat function i
    grad = coef[1:, :].T                # (3, 2)
    area = 0.5 * abs(np.linalg.det(V))
    M = np.zeros((3, 3)); K = np.zeros((3, 3)); Cx = np.zeros((3, 3)); N = np.zeros((3, 3))
    for lam, wq in zip(QP, QW):
        wv = lam @ w                    # advecting field at the point
        for i in range(3):
            for j in range(3):
                M[i, j] += wq * area * lam[i] * lam[j]
                K[i, j] += wq * area * grad[i] @ grad[j]
                Cx[i, j] += wq * area * lam[i] * grad[j, 0]
                N[i, j] += wq * area * lam[i] * (wv @ grad[j])
    return M, K, Cx, N


def test_element_matrices_match_quadrature():
    rng = np.random.default_rng(1)
    for _ in range(20):
        p = rng.random((3, 2))
        d1, d2 = p[1] - p[0], p[2] - p[0]
        if d1[0] * d2[1] - d1[1] * d2[0] < 0:
            p = p[[0, 2, 1]]
        w = rng.standard_normal((3, 2))
        tri = np.array([[0, 1, 2]])
        area, g = fem.geometry(p, tri)
        M, K, Cx, N = _quadrature_element(p, w)
        np.testing.assert_allclose(fem.element_mass(area)[0], M, rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(fem.element_stiffness(area, g)[0], K, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(fem.element_deriv(area, g, 0)[0], Cx, rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(fem.element_convection(area, g, tri, w)[0], N, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("mk", [lambda: square_mesh(6), lambda: crisscross_mesh(5),
                                lambda: channel_cylinder_mesh(seed=1, h=0.05)])
def test_assembled_identities(mk):
    m = mk()
    ops = fem.static_operators(m.xy, m.tri)
    one = np.ones(m.n_vert)
    x, y = m.xy[:, 0], m.xy[:, 1]
    area = m.meta["area"]
    # zero row sums: derivatives of the constant 1 vanish
    for s in ("K", "Cx", "Cy"):
        assert np.abs(ops[s] @ one).max() < 1e-12 * max(1.0, abs(ops[s]).max())
    rng = np.random.default_rng(0)
    N = fem.convection_operator(m.xy, m.tri, rng.standard_normal((m.n_vert, 2)))
    assert np.abs(N @ one).max() < 1e-12 * abs(N).max()
    # total mass = |Omega|
    np.testing.assert_allclose(one @ (ops["M"] @ one), area, rtol=1e-12)
    # energy of a linear field: u^T K u = |Omega| |grad u|^2
    u = 0.3 * x - 1.7 * y
    np.testing.assert_allclose(u @ (ops["K"] @ u), area * (0.09 + 2.89), rtol=1e-12)
    # d/dx of x is 1: Cx x = int psi_i = row sums of M
    rs = ops["M"] @ one
    np.testing.assert_allclose(ops["Cx"] @ x, rs, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(ops["Cy"] @ y, rs, rtol=1e-12, atol=1e-15)
    # convection by a constant field w = (a, b) of the linear u: N u = (a ux + b uy) M 1
    Nc = fem.convection_operator(m.xy, m.tri, np.tile([[0.7, -0.2]], (m.n_vert, 1)))
    np.testing.assert_allclose(Nc @ u, (0.7 * 0.3 + 0.2 * 1.7) * rs, rtol=1e-11, atol=1e-14)


def _neumann_poisson_error(n):
    # -Lap phi = 2 pi^2 phi, phi = cos(pi x) cos(pi y): homogeneous Neumann on [0,1]^2
    base = square_mesh(n)
    base.tag[:] = 1                     # velocity-Dirichlet only: pure-Neumann phi
    o = CGPOracle(base, 0, 0, 1.0, 1.0, 0, 2)
    x, y = o.fine.xy[:, 0], o.fine.xy[:, 1]
    ex = np.cos(np.pi * x) * np.cos(np.pi * y)
    r = o.ops_c["M"] @ (2 * np.pi ** 2 * ex)
    r = r - r.sum() / r.size
    phi = o.poisson(r)
    m = o.mlump_c
    assert abs(m @ phi) < 1e-12                        # normalisation
    e = (phi - (m @ phi) / m.sum()) - (ex - (m @ ex) / m.sum())
    return np.sqrt(e @ (o.ops_c["M"] @ e))


def _dirichlet_poisson_error(n):
    # phi = sin(pi x) sin(pi y), phi = 0 on the whole boundary (PHI_ZERO everywhere there)
    base = square_mesh(n, boundary_flags=PHI_ZERO)
    o = CGPOracle(base, 0, 0, 1.0, 1.0, 0, 2)
    x, y = o.fine.xy[:, 0], o.fine.xy[:, 1]
    ex = np.sin(np.pi * x) * np.sin(np.pi * y)
    r = o.ops_c["M"] @ (2 * np.pi ** 2 * ex)
    r[o.phi0_mask] = 0.0
    phi = o.poisson(r)
    e = phi - ex
    return np.sqrt(e @ (o.ops_c["M"] @ e))


def test_poisson_second_order():
    for fn in (_neumann_poisson_error, _dirichlet_poisson_error):
        e = np.array([fn(n) for n in (8, 16, 32, 64)])
        rates = np.log2(e[:-1] / e[1:])
        assert (rates > 1.85).all() and (rates < 2.2).all(), rates


def test_pure_neumann_solve_matches_dense_pseudoinverse():
    base = crisscross_mesh(3)
    o = CGPOracle(base, 0, 0, 1.0, 1.0, 0, 2)
    rng = np.random.default_rng(5)
    r = rng.standard_normal(o.coarse.n_vert)
    r -= r.mean()
    phi = o.poisson(r)
    Kd = o.ops_c["K"].toarray()
    ref = np.linalg.pinv(Kd) @ r        # minimum-norm solution, then the same mean fix
    m = o.mlump_c
    ref -= (m @ ref) / m.sum()
    np.testing.assert_allclose(phi, ref, rtol=1e-10, atol=1e-12)
    np.testing.assert_allclose(Kd @ phi, r, atol=1e-12)


def test_prolongation_exact_on_linear_and_injection_inverse():
    for base in (square_mesh(3), channel_cylinder_mesh(seed=2, h=0.06)):
        levels = build_hierarchy(base.xy, base.tri, base.tag, 3)
        for lc in range(3):
            for lf in range(lc + 1, 4):
                xc = levels[lc].xy
                phic = 0.25 + 1.5 * xc[:, 0] - 0.75 * xc[:, 1]
                phif = fem.prolong(phic, levels, lc, lf)
                xf = levels[lf].xy
                np.testing.assert_allclose(phif, 0.25 + 1.5 * xf[:, 0] - 0.75 * xf[:, 1],
                                           rtol=0, atol=1e-14)
                rnd = np.random.default_rng(lc).standard_normal(xc.shape[0])
                back = fem.inject(fem.prolong(rnd, levels, lc, lf), xc.shape[0])
                assert np.array_equal(back, rnd)          # R P = I bit for bit


@pytest.mark.parametrize("k", [1, 2, 3])
def test_restriction_is_the_transpose_of_prolongation(k):
    # <P x, y> = <x, P^T y> for random coarse x and fine y, over k levels
    base = square_mesh(4)
    levels = build_hierarchy(base.xy, base.tri, base.tag, 3)
    rng = np.random.default_rng(k)
    x = rng.standard_normal(levels[3 - k].n_vert)
    y = rng.standard_normal(levels[3].n_vert)
    lhs = fem.prolong(x, levels, 3 - k, 3) @ y
    rhs = x @ fem.restrict_t(y, levels, 3, 3 - k)
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1.0)


@pytest.mark.parametrize("k", [1, 2])
def test_pt_rhs_equals_injection_for_prolonged_velocity(k):
    # nested P1 spaces: P^T Cx_f P = Cx_c (the coarse operators are the Galerkin products),
    # so for a fine velocity that is the prolongation of a coarse one the two restrictions
    # of Eq. 22 give the same coarse right-hand side
    from oracle.cgp import CGPOracle
    from oracle import flows
    base = channel_cylinder_mesh(seed=3, h=0.08)
    o_inj = CGPOracle(base, 2, k, 100.0, 0.01, 0, flows.BC_CHANNEL, bc_param=(0.3, 0.41, 0, 0))
    o_pt = CGPOracle(base, 2, k, 100.0, 0.01, 0, flows.BC_CHANNEL, bc_param=(0.3, 0.41, 0, 0),
                     levels=o_inj.levels, restrict_mode="pt")
    rng = np.random.default_rng(5)
    Uc = rng.standard_normal((o_inj.coarse.n_vert, 2))
    Uf = np.stack([fem.prolong(Uc[:, c], o_inj.levels, 2 - k, 2) for c in range(2)], 1)
    a, b = o_inj.coarse_rhs(Uf), o_pt.coarse_rhs(Uf)
    assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max()
    # on a general fine field they differ (the variant is not the paper's restriction)
    Ur = rng.standard_normal(Uf.shape)
    assert np.abs(o_inj.coarse_rhs(Ur) - o_pt.coarse_rhs(Ur)).max() > 1e-3 * np.abs(o_inj.coarse_rhs(Ur)).max()


@pytest.mark.parametrize("mk,levels", [(lambda: square_mesh(6), 1), (lambda: crisscross_mesh(4), 1),
                                       (lambda: channel_cylinder_mesh(seed=4, h=0.05), 1)])
def test_jacobi_scaled_mass_spectrum_in_wathen_interval(mk, levels):
    """The eigenvalues of D^{-1} M for the consistent P1 mass matrix lie in [1/2, 2] (every
    element matrix D_e^{-1} M_e has eigenvalues 1/2, 1/2, 2), and so do those of M with the
    Dirichlet rows and columns eliminated (identity rows plus a principal submatrix).  The
    mixed form's Chebyshev mass solves use exactly this interval; dense eigenvalues of the
    symmetric scaling D^{-1/2} M D^{-1/2} on small meshes check it."""
    from oracle.cgp import _symmetric_eliminate, VEL_DIR
    base = mk()
    lev = build_hierarchy(base.xy, base.tri, base.tag, levels)[levels]
    M = fem.static_operators(lev.xy, lev.tri)["M"]
    for A in (M, _symmetric_eliminate(M, (lev.tag & VEL_DIR) != 0)):
        A = A.toarray()
        d = 1.0 / np.sqrt(np.diag(A))
        w = np.linalg.eigvalsh(d[:, None] * A * d[None, :])
        assert w.min() >= 0.5 - 1e-12 and w.max() <= 2.0 + 1e-12, (w.min(), w.max())
        assert w.max() > 1.9 and w.min() < 0.6   # the bound is nearly attained: not a loose test
