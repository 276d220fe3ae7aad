"""Pins of the oracle's time step (Section 2.2, Eqs. 21-26) against closed forms and the paper's trends."""

import numpy as np

from workloads import square_mesh, crisscross_mesh
from oracle import flows, norms
from oracle.cgp import CGPOracle
from oracle.mesh import build_hierarchy


def _tg_errors(o):
    ue, pe = flows.exact(o.bc, o.fine.xy, o.t, o.Re)
    M = o.ops_f["M"]
    return norms.l2(M, o.U - ue), norms.pressure_errors(M, o.P, pe)[0]


def test_taylor_green_velocity_second_order_in_space():
    # decaying Taylor-Green (Eqs. 28-30), plain incremental scheme (k = 0), small dt
    eu = []
    for n in (8, 16, 32):
        o = CGPOracle(square_mesh(n), 0, 0, Re=10.0, dt=0.0025, chi=1, bc=flows.BC_TG)
        o.run(20)
        eu.append(_tg_errors(o)[0])
    r = np.log2(np.array(eu[:-1]) / np.array(eu[1:]))
    assert (r > 1.8).all(), r


def test_periodic_forced_taylor_green_converges():
    # the body force of the periodic Taylor-Green makes it exact; errors fall at O(h^2)
    eu = []
    for n in (8, 16, 32):
        o = CGPOracle(square_mesh(n // 2), 1, 1, Re=100.0, dt=0.002, chi=1, bc=flows.BC_TG_PERIODIC)
        o.run(25)
        eu.append(_tg_errors(o)[0])
    r = np.log2(np.array(eu[:-1]) / np.array(eu[1:]))
    assert (r > 1.5).all(), r


def test_uniform_flow_is_a_fixed_point(monkeypatch):
    # u = const, p = const, f = 0 solves Eqs. 1-2; every discrete term must cancel
    c = np.array([0.3, -0.8])
    monkeypatch.setattr(flows, "dirichlet_value", lambda kind, xy, t, Re, bp=None: np.tile(c, (xy.shape[0], 1)))
    for chi in (0, 1):
        o = CGPOracle(crisscross_mesh(4), 2, 1, Re=50.0, dt=0.01, chi=chi, bc=flows.BC_CAVITY)
        U = np.tile(c, (o.fine.n_vert, 1))
        o.set_state(U, U, np.full(o.fine.n_vert, 2.5), 0.0)
        out = o.run(3)
        np.testing.assert_allclose(out["U"], U, atol=1e-12)
        np.testing.assert_allclose(out["phic"], 0.0, atol=1e-10)
        np.testing.assert_allclose(out["P"], 2.5, atol=1e-10)


def test_cgp_table_trends_standard_vs_rotational():
    # Tables 1-2 (Section 3.1): with the Poisson mesh two levels coarser (16384:1024)
    # the standard form (chi=0) loses pressure accuracy, the rotational form keeps it.
    base = crisscross_mesh(16)            # 1024 elements
    levels = build_hierarchy(base.xy, base.tri, base.tag, 2)   # 16384 elements
    err = {}
    for chi in (0, 1):
        for k in (0, 2):
            o = CGPOracle(None, 2, k, Re=10.0, dt=0.00125, chi=chi, bc=flows.BC_TG, levels=levels)
            o.run(80)                                           # to t = 0.1
            err[chi, k] = _tg_errors(o)
    assert err[0, 2][1] > 3.0 * err[0, 0][1]             # SCGP pressure error jumps
    assert err[1, 2][1] < 1.1 * err[1, 0][1]             # RCGP pressure error flat
    assert err[1, 2][0] < 1.05 * err[1, 0][0]            # RCGP velocity error flat


def test_rotational_equals_standard_plus_divergence_term():
    # Eq. 26: the two forms differ exactly by -1/Re M_p^{-1} D U~ in the pressure
    o0 = CGPOracle(square_mesh(8), 1, 1, Re=20.0, dt=0.01, chi=0, bc=flows.BC_TG)
    o1 = CGPOracle(square_mesh(8), 1, 1, Re=20.0, dt=0.01, chi=1, bc=flows.BC_TG)
    a, b = o0.step(), o1.step()
    np.testing.assert_array_equal(a["U"], b["U"])
    div = o1.ops_f["Cx"] @ b["Ut"][:, 0] + o1.ops_f["Cy"] @ b["Ut"][:, 1]
    np.testing.assert_allclose(o1.ops_f["M"] @ (a["P"] - b["P"]), div / 20.0, atol=1e-12)
