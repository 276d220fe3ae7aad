"""GPU parity at the benchmarked sizes: the CUDA path against the FP64 oracle, element by
element, on the full workloads the benchmark times.

Each case advances the GPU solver a few steps from rest, reads its state, and then advances
both the GPU and the oracle (sparse direct solves, test infrastructure only) three more steps
from that same state.  Bounds: relative L2 of U and P within 1e-6 for the FP64 form and
1e-4 for the mixed (FP32-inner / FP64-outer) forms, at the workloads' own solver tolerance of
1e-8 (the same parameters the benchmark uses, from paper_1812_00185_gb300.forms).

* the channel with a cylinder, 1,018,560 fine triangles, pressure increment two levels
  coarser (32,489 vertices): the headline form (mixed + learned guess, the on-chip coarse
  solve with the subdomain coarse correction), the plain FP64 form, and the standard form
  (chi = 0) of the mixed solver;
* the 512 x 512 lid-driven cavity (524,288 triangles) with the pressure 1, 2 and 3 levels
  coarser, FP64 and mixed;
* the batched form: all 256 uneven cavity instances in one batch, three steps, and a seeded
  sample of 8 of them compared with the oracle one by one.
"""

import numpy as np
import pytest

from workloads import WORKLOADS, square_mesh, batch_instances
from oracle.cgp import CGPOracle
from oracle import flows

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

WARM, STEPS = 5, 3
BOUND = {"fp64": 1e-6, "mixed": 1e-4, "mixed_learned": 1e-4}


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


@pytest.fixture(scope="module")
def cg(lib):
    from paper_1812_00185_gb300 import binding
    return binding


def _state(cg, s):
    U, P, t, _, _ = s.fields()
    return U, s.vector(cg.CGP_VEC_UPREV), P, t, s.vector(cg.CGP_VEC_PHI_C)


def _advance_from(cg, mesh, prm, state, steps, net=None):
    s = cg.Solver(mesh, prm)
    if net is not None:
        cg.cgp_guess_set(s.handle, net)
    U, Up, P, t, phic = state
    s.set_fields(U, Up, P, t)
    s.set_vector(cg.CGP_VEC_PHI_C, phic)
    s.step(steps)
    out = s.fields()
    info = (s.coarse_info(), s.coarse_subdomains())
    s.close()
    return out, info


def _oracle_from(base, w, state, steps, chi=None, levels=None):
    o = CGPOracle(base, w.n_levels, w.k, w.Re, w.dt, w.chi if chi is None else chi, w.bc,
                  bc_param=w.bc_param, levels=levels)
    U, Up, P, t, _ = state
    o.set_state(U, Up, P, t)
    o.run(steps)
    return o


@pytest.fixture(scope="module")
def channel(cg):
    from paper_1812_00185_gb300.forms import workload_params, train_guess
    w = WORKLOADS["channel1m_k2"]
    base = w.base_mesh()
    mesh = cg.Mesh(base.xy, base.tri, base.tag, w.n_levels)
    params, info = train_guess(w)
    net = cg.cgp_mlp_create(mesh.handle, w.n_levels - w.k, 1)
    cg.cgp_mlp_set_params(net, params)
    s = cg.Solver(mesh, workload_params(w, "mixed_learned"))
    cg.cgp_guess_set(s.handle, net)
    s.step(WARM)
    state = _state(cg, s)
    s.close()
    o = _oracle_from(base, w, state, STEPS)
    yield {"w": w, "base": base, "mesh": mesh, "net": net, "state": state, "oracle": o}
    cg.cgp_mlp_destroy(net)
    mesh.close()


@pytest.mark.parametrize("form", ["mixed_learned", "fp64", "mixed"])
def test_channel1m_k2_matches_oracle(cg, channel, form):
    from paper_1812_00185_gb300.forms import workload_params
    w, o = channel["w"], channel["oracle"]
    net = channel["net"] if form == "mixed_learned" else None
    (U, P, t, st, rc), (coarse, nsub) = _advance_from(cg, channel["mesh"], workload_params(w, form),
                                                      channel["state"], STEPS, net)
    assert rc == 0 and st["res_poisson"] <= 1.0001 * w.tol_poisson
    assert abs(t - o.t) < 1e-12
    if form != "fp64":
        # the benchmarked coarse solve: one cluster, on chip, with the subdomain coarse correction
        assert coarse[0] == cg.CGP_COARSE_ONCHIP and nsub > 0, (coarse, nsub)
    if form == "mixed_learned":
        assert st["guess_used"] > 0
    eu, ep = rel(U, o.U), rel(P, o.P)
    print("channel1m_k2 %s: rel-L2 U %.3g, P %.3g" % (form, eu, ep))
    assert eu < BOUND[form] and ep < BOUND[form], (form, eu, ep)


def test_channel1m_k2_standard_form_matches_oracle(cg, channel):
    from paper_1812_00185_gb300.forms import workload_params
    w = channel["w"]
    o = _oracle_from(channel["base"], w, channel["state"], STEPS, chi=0, levels=channel["oracle"].levels)
    (U, P, t, st, rc), _ = _advance_from(cg, channel["mesh"], workload_params(w, "mixed", chi=0),
                                         channel["state"], STEPS)
    assert rc == 0
    eu, ep = rel(U, o.U), rel(P, o.P)
    print("channel1m_k2 mixed chi=0: rel-L2 U %.3g, P %.3g" % (eu, ep))
    assert eu < BOUND["mixed"] and ep < BOUND["mixed"], (eu, ep)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_cavity512_matches_oracle(cg, k):
    from paper_1812_00185_gb300.forms import workload_params
    w = WORKLOADS["cavity512_k%d" % k]
    base = w.base_mesh()
    mesh = cg.Mesh(base.xy, base.tri, base.tag, w.n_levels)
    s = cg.Solver(mesh, workload_params(w, "fp64"))
    s.step(WARM)
    state = _state(cg, s)
    s.close()
    o = _oracle_from(base, w, state, STEPS)
    for form in ("fp64", "mixed"):
        (U, P, t, st, rc), _ = _advance_from(cg, mesh, workload_params(w, form), state, STEPS)
        assert rc == 0 and abs(t - o.t) < 1e-12
        eu, ep = rel(U, o.U), rel(P, o.P)
        print("cavity512_k%d %s: rel-L2 U %.3g, P %.3g" % (k, form, eu, ep))
        assert eu < BOUND[form] and ep < BOUND[form], (k, form, eu, ep)
    mesh.close()


def test_batch256_sample_matches_oracle(cg):
    # all 256 instances of the batched workload in one batch, as the benchmark builds it
    specs = batch_instances(256)
    meshes, solvers = [], []
    for sp in specs:
        base = square_mesh(sp["n_fine"] >> sp["k"])
        m = cg.Mesh(base.xy, base.tri, base.tag, sp["k"])
        prm = cg.make_params(sp["Re"], 0.005, chi=1, k=sp["k"], tol_mom=1e-8, tol_poisson=1e-8, tol_mass=1e-10,
                             precision=cg.CGP_MIXED, bc_kind=cg.CGP_BC_CAVITY)
        meshes.append(m)
        solvers.append(cg.Solver(m, prm))
    b = cg.cgp_batch_create(solvers)
    cg.cgp_batch_step(b, STEPS)
    sample = np.random.default_rng(2024).choice(len(specs), size=8, replace=False)
    for i in sample:
        sp = specs[i]
        U, P, t, st, rc = solvers[i].fields()
        assert rc == 0 and st["steps"] == STEPS
        base = square_mesh(sp["n_fine"] >> sp["k"])
        o = CGPOracle(base, sp["k"], sp["k"], sp["Re"], 0.005, 1, flows.BC_CAVITY)
        o.run(STEPS)
        eu, ep = rel(U, o.U), rel(P, o.P)
        print("batch instance %d (%s): rel-L2 U %.3g, P %.3g" % (int(i), sp, eu, ep))
        assert eu < BOUND["mixed"] and ep < BOUND["mixed"], (int(i), sp, eu, ep)
    cg.cgp_batch_destroy(b)
    for s in solvers:
        s.close()
    for m in meshes:
        m.close()
