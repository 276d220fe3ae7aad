"""The Jobelin vortices of Sections 3.2-3.3 through the C ABI against the FP64 oracle.

* Open boundary (CGP_BC_JOBELIN_OPEN): [0,1]^2, traction data and the prescribed pressure
  on the y-axis (the traction integral added to Eq. 21, phi lifted in Eq. 23), standard and
  rotational forms, pressure increment one level coarser.
* Disk (CGP_BC_JOBELIN_DISK): unstructured disk mesh, velocity data on the whole boundary,
  rotational form (the paper's RCGP), pressure one level coarser; FP64 and mixed forms.
Both match the oracle element by element, and cgp_exact_fields gives the closed forms.
"""

import numpy as np
import pytest

from workloads import open_square_mesh, disk_mesh
from oracle.cgp import CGPOracle
from oracle import flows

pytestmark = pytest.mark.gpu

TIGHT = dict(tol_mom=1e-13, tol_poisson=1e-11, tol_mass=1e-14, max_it_poisson=50000)


@pytest.fixture(scope="module")
def cg(lib):
    from paper_1812_00185_gb300 import binding
    return binding


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("case", ["open_chi0", "open_chi1", "disk_fp64", "disk_mixed"])
def test_jobelin_vortex_matches_oracle(cg, case):
    if case.startswith("open"):
        base, lv, kind, chi, prec = open_square_mesh(4), 3, cg.CGP_BC_JOBELIN_OPEN, int(case[-1]), cg.CGP_FP64
    else:
        base, lv, kind, chi = disk_mesh(48, 260), 2, cg.CGP_BC_JOBELIN_DISK, 1
        prec = cg.CGP_MIXED if case.endswith("mixed") else cg.CGP_FP64
    Re, dt, steps = 10.0, 0.01, 8
    mesh = cg.Mesh(base.xy, base.tri, base.tag, lv)
    s = cg.Solver(mesh, cg.make_params(Re, dt, chi=chi, k=1, bc_kind=kind, precision=prec, **TIGHT))
    o = CGPOracle(base, lv, 1, Re, dt, chi, kind)
    U0, P0, _, _, _ = s.fields()
    Ue, Pe = flows.exact(kind, o.fine.xy, 0.0, Re)
    np.testing.assert_allclose(U0, Ue, atol=1e-15)
    Ug, Pg = cg.cgp_exact_fields(s.handle, 0.37)
    Ux, Px = flows.exact(kind, o.fine.xy, 0.37, Re)
    np.testing.assert_allclose(Ug, Ux, atol=1e-14)
    np.testing.assert_allclose(Pg, Px, atol=1e-14)
    s.step(steps)
    o.run(steps)
    U, P, t, st, rc = s.fields()
    assert rc == 0 and abs(t - o.t) < 1e-12
    tol = 1e-6 if prec == cg.CGP_MIXED else 1e-8
    assert rel(U, o.U) < tol and rel(P, o.P) < tol, (case, rel(U, o.U), rel(P, o.P))
    s.close()
    mesh.close()


def test_open_vortex_rejects_the_transposed_restriction(cg):
    base = open_square_mesh(2)
    mesh = cg.Mesh(base.xy, base.tri, base.tag, 1)
    with pytest.raises(cg.CgpError):
        cg.Solver(mesh, cg.make_params(10.0, 0.01, k=1, bc_kind=cg.CGP_BC_JOBELIN_OPEN,
                                       restrict_mode=cg.CGP_RESTRICT_PT))
    mesh.close()
