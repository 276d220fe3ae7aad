"""Batched instances: one graph per step, one persistent launch for all coarse solves."""

import numpy as np
import pytest

from workloads import square_mesh
from oracle.cgp import CGPOracle
from oracle import flows

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cg(lib):
    from paper_1812_00185_gb300 import binding
    return binding


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _instances(cg, specs, mixed):
    out = []
    for n_fine, k, Re in specs:
        base = square_mesh(n_fine >> k)
        mesh = cg.Mesh(base.xy, base.tri, base.tag, k)
        prm = cg.make_params(Re, 0.005, chi=1, k=k, tol_mom=1e-12, tol_poisson=1e-12, tol_mass=1e-13,
                             precision=cg.CGP_MIXED if mixed else cg.CGP_FP64, bc_kind=cg.CGP_BC_CAVITY)
        out.append((base, mesh, cg.Solver(mesh, prm), (n_fine, k, Re)))
    return out


@pytest.mark.parametrize("mixed", [False, True])
def test_batch_matches_oracle_per_instance(cg, mixed):
    specs = [(32, 2, 400.0), (16, 1, 100.0), (64, 3, 10.0), (16, 2, 250.0), (32, 1, 50.0)]
    inst = _instances(cg, specs, mixed)
    b = cg.cgp_batch_create([x[2] for x in inst])
    info = cg.cgp_batch_info(b)
    assert info["cluster_size"] in (1, 2, 4, 8) and info["threads"] in (256, 512, 1024) and info["trials_ms"]
    cg.cgp_batch_step(b, 4)
    for base, mesh, s, (n_fine, k, Re) in inst:
        U, P, t, st, rc = s.fields()
        assert rc == 0 and st["steps"] == 4
        o = CGPOracle(base, k, k, Re, 0.005, 1, flows.BC_CAVITY)
        o.run(4)
        assert rel(U, o.U) < 1e-8 and rel(P, o.P) < 1e-7, (n_fine, k, rel(U, o.U), rel(P, o.P))
    cg.cgp_batch_destroy(b)
    for x in inst:
        x[2].close()
        x[1].close()


def test_batch_equals_instances_run_alone(cg):
    # the same solvers advanced one by one give the same fields (each within the solver tolerance)
    specs = [(32, 1, 200.0), (16, 2, 30.0), (32, 3, 120.0)]
    a = _instances(cg, specs, False)
    b_ = _instances(cg, specs, False)
    batch = cg.cgp_batch_create([x[2] for x in a], cluster_size=2, threads=256)
    cg.cgp_batch_step(batch, 3)
    for (_, _, sa, _), (_, _, sb, _) in zip(a, b_):
        sb.step(3)
        Ua, Pa = sa.fields()[:2]
        Ub, Pb = sb.fields()[:2]
        assert rel(Ua, Ub) < 1e-9 and rel(Pa, Pb) < 1e-8
    cg.cgp_batch_destroy(batch)
    for x in a + b_:
        x[2].close()
        x[1].close()
