"""The coarse-grid incremental pressure-projection time step (oracle; test infrastructure only).

Follows Section 2.2, Eqs. 21-26, in the paper's order, on the hierarchy of
oracle.mesh with the P1 operators of oracle.fem:

1. Eq. 21 -- momentum: (3/2 M + dt N(w) + dt/Re K) U~ = -dt G P^n + dt M F^{n+1}
   + 2 M U^n - 1/2 M U^{n-1}, w = 2 U^n - U^{n-1} (Eq. 5's extrapolation).
2. Eq. 22 -- restriction of U~ to the pressure level by injection.
3. Eq. 23 -- coarse Poisson: K_c Phi_c = -3/(2 dt) (Cx_c u~_c + Cy_c v~_c)
   (L_p = -K), with phi = 0 at PHI_ZERO vertices (Eq. 14).
4. Eq. 24 -- prolongation of Phi_c to the fine level, k one-level steps.
5. Eq. 25 -- correction: M U = M U~ - 2/3 dt G Phi_f.
6. Eq. 26 -- pressure: chi = 0 uses the algebraic update P += Phi_f (Section
   2.3); chi = 1 solves M_p (P^{n+1} - P^n - Phi_f) = -1/Re D U~ with the
   consistent M_p (Eq. 20, as Section 2.3 prefers), or the lumped Eq. 27.

Readings of points the paper leaves open (listed with the design notes):

* Dirichlet velocity rows of Eq. 21 are replaced by u_D(t^{n+1}) (row of the
  identity); Eq. 25 is solved only on the other rows (U = U~ = u_D on Gamma_D),
  i.e. with M's Dirichlet rows and columns replaced by the identity.
* The pressure term of Eq. 21 is taken in the weak form -int p div(psi), i.e.
  G P = -(Cx^T P, Cy^T P); this is what makes the traction condition of Eq. 4
  natural on an outflow boundary, and equals Cx P on every non-Dirichlet row of
  a pure-Dirichlet domain.  Eq. 25 uses G = (Cx, Cy).
* Pure-Neumann coarse Poisson problems (no PHI_ZERO vertex): the right-hand
  side is projected onto the range (r -= mean(r)) and the solution fixed by
  sum_i m_i Phi_i = 0 with m the lumped coarse mass (row sums of M_c).
* The mean of nothing else is touched: P carries whatever constant the
  Phi updates give.
* Traction data on the natural boundary Gamma_N (Eq. 11; nonzero only for the open-boundary
  vortex of Section 3.2).  Eq. 11 leaves the time level of its pressure open; it is read at
  t^{n+1}, -p^{n+1} n + grad u~ . n / Re = t^{n+1}, with p^{n+1} the pressure prescribed on
  Gamma_N.  The weak pressure term of Eq. 21 carries p^n, so Eq. 21's right-hand side gains
  dt * int_{Gamma_N} (t + (p^{n+1} - p^n) n) psi_i ds, the integrand interpolated linearly
  between the vertices of each boundary edge (the boundary mass matrix l/6 [[2, 1], [1, 2]]
  of the edge times the nodal values).  (With p^n in Eq. 11 the scheme stays first order in
  time there; at t^{n+1} the velocity error on the paper's mesh falls ~25x.)  Eq. 14 is read
  with the same data: phi = p(t^{n+1}) - p^n at the coarse Gamma_N vertices (lifted into the
  right-hand side of Eq. 23), so that the pressure follows the prescribed values; where no
  pressure is prescribed, phi = 0 there and t = 0 (the channel's outflow).

Solves use scipy's sparse LU (a library primitive), so each result is the
exact discrete solution up to rounding.

Pins (tests/test_oracle_step.py, tests/test_oracle_pins.py): Taylor-Green convergence;
uniform flow as a fixed point; chi = 1 minus chi = 0 equal to the Eq. 26 term; plane
Poiseuille flow in a channel with the traction-free outflow (a fixed point on the uniform
mesh, second-order convergence on unstructured ones); the change of Eq. 21's right-hand
side under P -> P + c against the outflow boundary integral; Eq. 27's lumped masses and
corrections against hand-worked values and linear fields.
"""

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem, flows
from .mesh import build_hierarchy, unique_edges

VEL_DIR, PHI_ZERO = 1, 2


def _dirichlet_replace(A, mask):
    """Rows in ``mask`` become rows of the identity (columns kept)."""
    keep = sp.diags((~mask).astype(np.float64))
    return (keep @ A + sp.diags(mask.astype(np.float64))).tocsc()


def _symmetric_eliminate(A, mask):
    """Rows and columns in ``mask`` become those of the identity."""
    keep = sp.diags((~mask).astype(np.float64))
    return (keep @ A @ keep + sp.diags(mask.astype(np.float64))).tocsc()


class CGPOracle:
    """State and operators of one CGP run.

    base: workloads.BaseMesh; n_levels: refinements giving the velocity level;
    k: coarsening levels of the pressure-increment mesh (0 = plain incremental
    scheme on the fine mesh).
    """

    def __init__(self, base, n_levels, k, Re, dt, chi, bc,
                 bc_param=(1.0, 0.0, 0.0, 0.0), mass_mode="consistent", levels=None, restrict_mode="inject"):
        if not 0 <= k <= n_levels:
            raise ValueError("need 0 <= k <= n_levels")
        self.levels = levels if levels is not None else build_hierarchy(base.xy, base.tri, base.tag, n_levels)
        self.lf, self.lc = n_levels, n_levels - k
        self.fine, self.coarse = self.levels[self.lf], self.levels[self.lc]
        self.Re, self.dt, self.chi, self.bc = float(Re), float(dt), int(chi), int(bc)
        self.bc_param = tuple(bc_param)
        self.restrict_mode = restrict_mode
        self.mass_mode = mass_mode
        f, c = self.fine, self.coarse
        self.ops_f = fem.static_operators(f.xy, f.tri)
        self.ops_c = fem.static_operators(c.xy, c.tri)
        self.dir_mask = (f.tag & VEL_DIR) != 0
        self.phi0_mask = (c.tag & PHI_ZERO) != 0
        self.pure_neumann = not self.phi0_mask.any()
        M = self.ops_f["M"]
        self.BN = self._natural_boundary_mass(f, (f.tag & PHI_ZERO) != 0)
        self.mlump_f = np.asarray(M.sum(axis=1)).ravel()
        self.mlump_c = np.asarray(self.ops_c["M"].sum(axis=1)).ravel()
        # factorisations of the constant systems
        self._lu_corr = spla.splu(_symmetric_eliminate(M, self.dir_mask))
        self._lu_mass = spla.splu(M.tocsc())
        Kc = self.ops_c["K"]
        if self.pure_neumann:
            m = sp.csr_matrix(self.mlump_c[None, :])
            B = sp.bmat([[Kc, m.T], [m, None]]).tocsc()
            self._lu_pois = spla.splu(B)
        else:
            self._lu_pois = spla.splu(_symmetric_eliminate(Kc, self.phi0_mask))
        self.U, self.Uprev, self.P = flows.initial_state(
            self.bc, f.xy, self.dir_mask, self.dt, self.Re, self.bc_param)
        self.t = 0.0
        self.n = 0

    @staticmethod
    def _natural_boundary_mass(lev, on_n):
        """int psi_i psi_j ds over the boundary edges (edges of one triangle) whose ends both
        lie on Gamma_N: l/6 (1 + delta_ij) per edge."""
        ends, count, _ = unique_edges(lev.tri)
        e = ends[(count == 1) & on_n[ends[:, 0]] & on_n[ends[:, 1]]]
        ell = np.hypot(*(lev.xy[e[:, 1]] - lev.xy[e[:, 0]]).T)
        rows = np.concatenate([e[:, 0], e[:, 1], e[:, 0], e[:, 1]])
        cols = np.concatenate([e[:, 0], e[:, 1], e[:, 1], e[:, 0]])
        vals = np.concatenate([ell / 3.0, ell / 3.0, ell / 6.0, ell / 6.0])
        n = lev.xy.shape[0]
        return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))

    # ---- individual steps (each follows one equation) ----
    def momentum(self, U, Uprev, P, t_new):
        """Eq. 21: the intermediate velocity U~ (n_f, 2)."""
        f, dt, Re = self.fine, self.dt, self.Re
        M, K, Cx, Cy = (self.ops_f[s] for s in ("M", "K", "Cx", "Cy"))
        w = 2.0 * U - Uprev
        N = fem.convection_operator(f.xy, f.tri, w)
        A = 1.5 * M + dt * N + (dt / Re) * K
        F = flows.body_force(self.bc, f.xy, t_new, Re, self.bc_param)
        hist = 2.0 * U - 0.5 * Uprev
        T = flows.traction(self.bc, f.xy, t_new, Re, self.bc_param)
        pn = flows.natural_pressure(self.bc, f.xy, t_new, Re, self.bc_param)
        if pn is not None:
            T = T + (pn - P)[:, None] * flows.natural_normal(self.bc, f.xy)
        bx = dt * (Cx.T @ P) + M @ (dt * F[:, 0] + hist[:, 0]) + dt * (self.BN @ T[:, 0])
        by = dt * (Cy.T @ P) + M @ (dt * F[:, 1] + hist[:, 1]) + dt * (self.BN @ T[:, 1])
        uD = flows.dirichlet_value(self.bc, f.xy, t_new, Re, self.bc_param)
        d = self.dir_mask
        bx[d], by[d] = uD[d, 0], uD[d, 1]
        lu = spla.splu(_dirichlet_replace(A.tocsr(), d))
        return np.stack([lu.solve(bx), lu.solve(by)], 1)

    def coarse_rhs(self, Ut, P=None, t_new=None):
        """Eqs. 22-23: inject U~ and form -3/(2 dt) (Cx_c u~_c + Cy_c v~_c).  restrict_mode
        "pt" (a variant, not the paper's): -3/(2 dt) P^T (Cx_f u~ + Cy_f v~), the fine
        divergence restricted by the transpose of the prolongation.  With a prescribed
        pressure on Gamma_N (P = P^n and t_new given), the phi = 0 rows carry g = p(t_new) - P^n
        and the other rows have K_c[:, Gamma_N] g moved to the right-hand side."""
        if self.restrict_mode == "pt":
            g = self.ops_f["Cx"] @ Ut[:, 0] + self.ops_f["Cy"] @ Ut[:, 1]
            r = -1.5 / self.dt * fem.restrict_t(g, self.levels, self.lf, self.lc)
        else:
            Uc = fem.inject(Ut, self.coarse.n_vert)
            r = -1.5 / self.dt * (self.ops_c["Cx"] @ Uc[:, 0] + self.ops_c["Cy"] @ Uc[:, 1])
        r[self.phi0_mask] = 0.0
        pn = None if t_new is None else flows.natural_pressure(self.bc, self.coarse.xy, t_new, self.Re, self.bc_param)
        if pn is not None and self.phi0_mask.any():
            g = np.where(self.phi0_mask, pn - P[:self.coarse.n_vert], 0.0)
            r = r - self.ops_c["K"] @ g
            r[self.phi0_mask] = g[self.phi0_mask]
        if self.pure_neumann:
            r = r - r.sum() / r.size
        return r

    def poisson(self, r):
        """Eq. 23: K_c Phi_c = r (with the readings in the module docstring)."""
        if self.pure_neumann:
            sol = self._lu_pois.solve(np.concatenate([r, [0.0]]))
            return sol[:-1]
        return self._lu_pois.solve(r)

    def prolong(self, phic):
        """Eq. 24."""
        return fem.prolong(phic, self.levels, self.lc, self.lf)

    def correct(self, Ut, phif):
        """Eq. 25: U = U~ + delta, M delta = -2/3 dt G Phi_f on non-Dirichlet rows."""
        g = -2.0 / 3.0 * self.dt * np.stack([self.ops_f["Cx"] @ phif, self.ops_f["Cy"] @ phif], 1)
        g[self.dir_mask] = 0.0
        if self.mass_mode == "lumped":
            delta = g / self.mlump_f[:, None]
            delta[self.dir_mask] = 0.0
        else:
            delta = np.stack([self._lu_corr.solve(g[:, 0]), self._lu_corr.solve(g[:, 1])], 1)
        return Ut + delta

    def pressure(self, P, phif, Ut):
        """Eq. 26 (chi = 0: the algebraic Eq. 16; chi = 1: Eq. 20, or Eq. 27 if lumped)."""
        if self.chi == 0:
            return P + phif
        div = self.ops_f["Cx"] @ Ut[:, 0] + self.ops_f["Cy"] @ Ut[:, 1]
        if self.mass_mode == "lumped":
            q = div / self.mlump_f
        else:
            q = self._lu_mass.solve(div)
        return P + phif - q / self.Re

    # ---- the whole step ----
    def step(self):
        t_new = self.t + self.dt
        Ut = self.momentum(self.U, self.Uprev, self.P, t_new)
        r = self.coarse_rhs(Ut, self.P, t_new)
        phic = self.poisson(r)
        phif = self.prolong(phic)
        U = self.correct(Ut, phif)
        P = self.pressure(self.P, phif, Ut)
        self.Uprev, self.U, self.P = self.U, U, P
        self.t, self.n = t_new, self.n + 1
        return {"Ut": Ut, "rc": r, "phic": phic, "phif": phif, "U": U, "P": P}

    def run(self, steps):
        out = None
        for _ in range(steps):
            out = self.step()
        return out

    def set_state(self, U, Uprev, P, t, n=0):
        self.U, self.Uprev, self.P = np.array(U, float), np.array(Uprev, float), np.array(P, float)
        self.t, self.n = float(t), int(n)
