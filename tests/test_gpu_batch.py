"""Batched instances: the whole-step form (one persistent clustered launch runs every
instance's entire step) and the graph-branch form (one graph per step, one persistent
launch for all coarse solves), each against the oracle and against the other."""

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


@pytest.mark.parametrize("mode", ["whole", "branches"])
@pytest.mark.parametrize("mixed", [False, True])
def test_batch_matches_oracle_per_instance(cg, mixed, mode):
    specs = [(32, 2, 400.0), (16, 1, 100.0), (64, 3, 10.0), (16, 2, 250.0), (32, 1, 50.0)]
    inst = _instances(cg, specs, mixed)
    m = cg.CGP_BATCH_WHOLE_STEP if mode == "whole" else cg.CGP_BATCH_BRANCHES
    b = cg.cgp_batch_create([x[2] for x in inst], mode=m)
    assert cg.cgp_batch_mode(b) == m
    info = cg.cgp_batch_info(b)
    assert info["cluster_size"] in (1, 2, 4, 8) and info["threads"] in (256, 512, 1024) and info["trials_ms"]
    if mode == "whole":
        assert info["threads"] <= 512
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


def test_whole_step_is_the_default_and_matches_the_branch_form(cg):
    # uneven sizes and coarsening 1-3, FP32-inner coarse solves
    specs = [(64, 1, 120.0), (32, 3, 30.0), (16, 1, 300.0), (32, 2, 80.0)]
    out = {}
    for m in (None, cg.CGP_BATCH_BRANCHES):
        inst = _instances(cg, specs, True)
        b = cg.cgp_batch_create([x[2] for x in inst], mode=m)
        assert cg.cgp_batch_mode(b) == (cg.CGP_BATCH_WHOLE_STEP if m is None else cg.CGP_BATCH_BRANCHES)
        cg.cgp_batch_step(b, 3)
        out[m] = [x[2].fields() for x in inst]
        cg.cgp_batch_destroy(b)
        for x in inst:
            x[2].close()
            x[1].close()
    for (Uw, Pw, tw, sw, rw), (Ub, Pb, tb, sb, rb) in zip(out[None], out[cg.CGP_BATCH_BRANCHES]):
        assert rw == 0 and rb == 0 and tw == tb and sw["steps"] == sb["steps"] == 3
        assert rel(Uw, Ub) < 1e-9 and rel(Pw, Pb) < 1e-8


def test_whole_step_refuses_instances_it_cannot_run(cg):
    base = square_mesh(8)
    mesh = cg.Mesh(base.xy, base.tri, base.tag, 1)
    ok = cg.Solver(mesh, cg.make_params(100.0, 0.005, chi=1, k=1))
    pt = cg.Solver(mesh, cg.make_params(100.0, 0.005, chi=1, k=1, restrict_mode=cg.CGP_RESTRICT_PT))
    with pytest.raises(cg.CgpError):
        cg.cgp_batch_create([ok, pt], mode=cg.CGP_BATCH_WHOLE_STEP)
    b = cg.cgp_batch_create([ok, pt])            # the default falls back to the branch form
    assert cg.cgp_batch_mode(b) == cg.CGP_BATCH_BRANCHES
    cg.cgp_batch_destroy(b)
    ok.close(); pt.close(); mesh.close()
