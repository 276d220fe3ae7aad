"""The projection guess of the coarse solve (CGP_GUESS_PROJ; a form beyond the paper).

The guess is the Galerkin projection of the new increment onto the span of the last eight
increments: among the combinations of them it has the smallest K_c-norm error.  Checked
against the same projection formed on the host from the recorded increments and the
solver's own coarse matrix, then by what it buys: fewer coarse iterations than the
previous-increment guess for the same fields (the solve's tolerance judges both).
"""

import numpy as np
import pytest
import scipy.sparse as sp

from workloads import channel_cylinder_mesh

pytestmark = pytest.mark.gpu

COMMON = dict(chi=1, k=1, bc_kind=1, bc_param=(0.3, 0.41), tol_mom=1e-10, tol_poisson=1e-10, tol_mass=1e-12)


@pytest.fixture(scope="module")
def cg(lib):
    from paper_1812_00185_gb300 import binding
    return binding


def _coarse_matrix(cg, mesh, s, level):
    lev = mesh.level(level)
    K = sp.csr_matrix((s.matrix(cg.CGP_MAT_KC), lev["col"], lev["rowptr"]))
    z = (lev["tag"] & cg.CGP_PHI_ZERO) != 0
    keep = sp.diags((~z).astype(float))
    return (keep @ K @ keep + sp.diags(z.astype(float))).tocsr()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_projection_guess_is_the_best_combination_of_the_window(cg, precision):
    base = channel_cylinder_mesh(seed=7, h=0.04)
    mesh = cg.Mesh(base.xy, base.tri, base.tag, 2)
    s = cg.Solver(mesh, cg.make_params(1000.0, 0.002, guess=cg.CGP_GUESS_PROJ,
                                       precision=cg.CGP_MIXED if precision == "mixed" else cg.CGP_FP64, **COMMON))
    n, nc = 14, s.nc
    rhs, q, tgt = (np.zeros((n, nc)) for _ in range(3))
    cg.cgp_record_pairs(s.handle, n, rhs, q, tgt)
    K = _coarse_matrix(cg, mesh, s, 1)
    knorm = lambda e: float(np.sqrt(e @ (K @ e)))
    for k in range(2, n):
        X = tgt[max(0, k - 8):k].T                      # the window: the last (up to) 8 increments
        c = np.linalg.lstsq(X.T @ (K @ X), X.T @ rhs[k], rcond=1e-12)[0]
        best = X @ c
        e_gpu, e_best = knorm(tgt[k] - q[k]), knorm(tgt[k] - best)
        # the GPU guess lies in the window's span and is K-norm optimal there (its Galerkin
        # matrix comes from the stored right-hand sides, equal to K x_j up to the tolerance)
        resid_span = np.linalg.norm(q[k] - X @ np.linalg.lstsq(X, q[k], rcond=None)[0]) / np.linalg.norm(q[k])
        assert resid_span < 1e-8, (k, resid_span)
        assert e_gpu <= 1.01 * e_best + 1e-3 * knorm(tgt[k]), (k, e_gpu, e_best)
    s.close()
    mesh.close()


def test_projection_guess_saves_iterations(cg):
    base = channel_cylinder_mesh(seed=8, h=0.03)
    mesh = cg.Mesh(base.xy, base.tri, base.tag, 2)
    out = {}
    for guess in (cg.CGP_GUESS_ZERO, cg.CGP_GUESS_PREV, cg.CGP_GUESS_PROJ):
        s = cg.Solver(mesh, cg.make_params(1000.0, 0.002, guess=guess, precision=cg.CGP_MIXED, **COMMON))
        s.step(40)
        U, P, t, st, rc = s.fields()
        assert rc == 0
        out[guess] = (U, P, st["sum_it_poisson"])
        s.close()
    Up, Pp, it_prev = out[cg.CGP_GUESS_PREV]
    Uj, Pj, it_proj = out[cg.CGP_GUESS_PROJ]
    it_zero = out[cg.CGP_GUESS_ZERO][2]
    print("coarse iterations over 40 steps: zero %d, previous %d, projection %d" % (it_zero, it_prev, it_proj))
    assert np.linalg.norm(Uj - Up) / np.linalg.norm(Up) < 1e-7
    assert np.linalg.norm(Pj - Pp) / np.linalg.norm(Pp) < 1e-6
    assert it_proj < 0.95 * min(it_prev, it_zero), (it_zero, it_prev, it_proj)
    mesh.close()
