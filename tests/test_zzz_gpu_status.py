"""Statuses of the coarse solve under host-made faults (no GPU fault, trap or hang):
a right-hand side poisoned with a NaN ends the solve with CGP_ENONFINITE (and the next
solve with a finite right-hand side converges as usual), and an iteration cap ends it with
CGP_ENOTCONV and a finite iterate, and a bounded device wait that runs out (the
cgp_set_wait_test hook: each wait also awaits one signal that nothing sends, under a limit
of milliseconds) ends it with CGP_ETIMEOUT, after which the same solver converges again.
FP64 (register-resident grid solve, software grid barrier) and mixed form (one cluster,
FP32 inner, mbarrier waits) alike; pure-Neumann and Dirichlet coarse problems.  Collected
after the main suites, so a run stopping at the first failure has run them first."""

import numpy as np
import pytest

from workloads import square_mesh, channel_cylinder_mesh
from oracle import flows

pytestmark = pytest.mark.gpu


def _solver(cg, kind, precision, **kw):
    if kind == "neumann":
        base, bc, bp = square_mesh(16), flows.BC_CAVITY, (1.0, 0, 0, 0)
    else:
        base, bc, bp = channel_cylinder_mesh(seed=4, h=0.05), flows.BC_CHANNEL, (0.3, 0.41, 0, 0)
    m = cg.Mesh(base.xy, base.tri, base.tag, 2)
    prm = cg.make_params(100.0, 0.01, k=1, bc_kind=bc, bc_param=bp, guess=cg.CGP_GUESS_ZERO,
                         tol_poisson=1e-11, precision=precision, **kw)
    return m, cg.Solver(m, prm)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["neumann", "dirichlet"])
def test_nan_rhs_reports_nonfinite_then_recovers(lib, kind, precision):
    from paper_1812_00185_gb300 import binding as cg
    m, s = _solver(cg, kind, cg.CGP_FP64 if precision == "fp64" else cg.CGP_MIXED)
    nc = s.nc
    r = np.random.default_rng(3).standard_normal(nc)
    bad = r.copy()
    bad[::3] = np.nan          # many rows, so some lie outside the phi = 0 rows the solve zeroes
    with pytest.raises(cg.CgpError) as e:
        cg.cgp_poisson_solve(s.handle, bad)
    assert e.value.code == cg.CGP_ENONFINITE
    phi, it, rc = cg.cgp_poisson_solve(s.handle, r)
    assert rc == cg.CGP_OK and it > 0 and np.isfinite(phi).all()
    s.close()
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["neumann", "dirichlet"])
def test_iteration_cap_reports_notconv(lib, kind, precision):
    from paper_1812_00185_gb300 import binding as cg
    m, s = _solver(cg, kind, cg.CGP_FP64 if precision == "fp64" else cg.CGP_MIXED, max_it_poisson=1)
    r = np.random.default_rng(4).standard_normal(s.nc)
    phi, it, rc = cg.cgp_poisson_solve(s.handle, r)
    assert rc == cg.CGP_ENOTCONV
    assert np.isfinite(phi).all()
    s.close()
    m.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("kind", ["neumann", "dirichlet"])
def test_wait_that_runs_out_reports_timeout_then_recovers(lib, kind, precision):
    import time
    from paper_1812_00185_gb300 import binding as cg
    m, s = _solver(cg, kind, cg.CGP_FP64 if precision == "fp64" else cg.CGP_MIXED)
    want = cg.CGP_COARSE_PERSISTENT if precision == "fp64" else cg.CGP_COARSE_ONCHIP
    assert s.coarse_info()[0] == want
    r = np.random.default_rng(5).standard_normal(s.nc)
    cg.cgp_set_wait_test(s.handle, 1)
    t0 = time.time()
    with pytest.raises(cg.CgpError) as e:
        cg.cgp_poisson_solve(s.handle, r)
    assert e.value.code == cg.CGP_ETIMEOUT
    assert time.time() - t0 < 5.0          # the short limit, not the seconds-long one
    cg.cgp_set_wait_test(s.handle, 0)
    phi, it, rc = cg.cgp_poisson_solve(s.handle, r)
    assert rc == cg.CGP_OK and it > 0 and np.isfinite(phi).all()
    s.close()
    m.close()
