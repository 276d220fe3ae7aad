"""GPU parity: the CUDA path through the C ABI against the FP64 oracle."""

import numpy as np
import pytest
import scipy.sparse as sp

from workloads import square_mesh, crisscross_mesh, channel_cylinder_mesh, WORKLOADS
from oracle.mesh import build_hierarchy
from oracle.cgp import CGPOracle
from oracle import fem, flows

pytestmark = pytest.mark.gpu

# the coarse solve stops on the true FP64 residual, whose rounding floor is near 1e-13 relative
TIGHT = dict(tol_mom=1e-13, tol_poisson=1e-11, tol_mass=1e-14, max_it_poisson=50000)


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300)


@pytest.fixture(scope="module")
def cg(lib):
    from paper_1812_00185_gb300 import binding
    return binding


def _channel_small():
    return channel_cylinder_mesh(seed=4, h=0.05)


def _channel_small_fine():
    return channel_cylinder_mesh(seed=4, h=0.03)


@pytest.mark.parametrize("mk,levels", [(lambda: square_mesh(8), 3), (lambda: crisscross_mesh(5), 2),
                                       (_channel_small, 2)])
def test_mesh_hierarchy_bit_exact(cg, mk, levels):
    base = mk()
    ref = build_hierarchy(base.xy, base.tri, base.tag, levels)
    m = cg.Mesh(base.xy, base.tri, base.tag, levels)
    for l in range(levels + 1):
        g = m.level(l)
        r = ref[l]
        assert np.array_equal(g["xy"], r.xy), l
        assert np.array_equal(g["tri"], r.tri), l
        assert np.array_equal(g["tag"], r.tag), l
        assert np.array_equal(g["rowptr"], r.rowptr), l
        assert np.array_equal(g["col"], r.col), l
        if l > 0:
            assert np.array_equal(g["parents"], r.parents), l
    m.close()


def _csr(lev, vals):
    n = lev["rowptr"].shape[0] - 1
    return sp.csr_matrix((vals, lev["col"], lev["rowptr"]), shape=(n, n))


def test_static_operators_match(cg):
    base = _channel_small()
    m = cg.Mesh(base.xy, base.tri, base.tag, 2)
    s = cg.Solver(m, cg.make_params(20.0, 0.01, k=1, bc_kind=cg.CGP_BC_CHANNEL, bc_param=(0.3, 0.41)))
    o = CGPOracle(base, 2, 1, 20.0, 0.01, 1, flows.BC_CHANNEL, bc_param=(0.3, 0.41, 0, 0))
    F, C = m.level(2), m.level(1)
    for which, name, lev, ops in [(cg.CGP_MAT_M, "M", F, o.ops_f), (cg.CGP_MAT_K, "K", F, o.ops_f),
                                  (cg.CGP_MAT_CX, "Cx", F, o.ops_f), (cg.CGP_MAT_CY, "Cy", F, o.ops_f),
                                  (cg.CGP_MAT_KC, "K", C, o.ops_c), (cg.CGP_MAT_CXC, "Cx", C, o.ops_c),
                                  (cg.CGP_MAT_CYC, "Cy", C, o.ops_c)]:
        G = _csr(lev, s.matrix(which))
        R = ops[name]
        assert abs(G - R).max() <= 1e-13 * abs(R).max(), name
    s.close(); m.close()


def test_prolongation_bit_exact(cg):
    base = square_mesh(4)
    m = cg.Mesh(base.xy, base.tri, base.tag, 3)
    s = cg.Solver(m, cg.make_params(100.0, 0.01, k=3))
    levels = build_hierarchy(base.xy, base.tri, base.tag, 3)
    phic = np.random.default_rng(0).standard_normal(levels[0].n_vert)
    assert np.array_equal(cg.cgp_prolong(s.handle, phic), fem.prolong(phic, levels, 0, 3))
    s.close(); m.close()


@pytest.mark.parametrize("mode", ["kernels", "cluster", "persistent", "persistent_mem", "mixed", "mixed_jacobi",
                                  "mixed_cluster", "mixed_persistent"])
@pytest.mark.parametrize("kind", ["neumann", "dirichlet"])
def test_coarse_poisson_solve(cg, kind, mode):
    if kind == "neumann":
        base, bc, bp = square_mesh(16), flows.BC_CAVITY, (1.0, 0, 0, 0)
    else:
        base, bc, bp = _channel_small(), flows.BC_CHANNEL, (0.3, 0.41, 0, 0)
    m = cg.Mesh(base.xy, base.tri, base.tag, 2)
    extra = {"kernels": dict(coarse_mode=cg.CGP_COARSE_KERNELS), "cluster": dict(coarse_mode=cg.CGP_COARSE_CLUSTER),
             "persistent": dict(coarse_mode=cg.CGP_COARSE_PERSISTENT), "mixed": dict(precision=cg.CGP_MIXED),
             "mixed_jacobi": dict(precision=cg.CGP_MIXED, precond=cg.CGP_PRECOND_JACOBI),
             "persistent_mem": dict(coarse_mode=cg.CGP_COARSE_PERSISTENT_MEM),
             "mixed_cluster": dict(precision=cg.CGP_MIXED, coarse_mode=cg.CGP_COARSE_CLUSTER),
             "mixed_persistent": dict(precision=cg.CGP_MIXED, coarse_mode=cg.CGP_COARSE_PERSISTENT)}[mode]
    s = cg.Solver(m, cg.make_params(100.0, 0.01, k=1, bc_kind=bc, bc_param=bp, guess=cg.CGP_GUESS_ZERO,
                                    **TIGHT, **extra))
    kind = {"kernels": cg.CGP_COARSE_KERNELS, "cluster": cg.CGP_COARSE_CLUSTER, "persistent": cg.CGP_COARSE_PERSISTENT,
            "persistent_mem": cg.CGP_COARSE_PERSISTENT_MEM, "mixed": cg.CGP_COARSE_ONCHIP,
            "mixed_jacobi": cg.CGP_COARSE_ONCHIP,
            "mixed_cluster": cg.CGP_COARSE_CLUSTER, "mixed_persistent": cg.CGP_COARSE_PERSISTENT_MEM}[mode]
    assert s.coarse_info()[0] == kind
    o = CGPOracle(base, 2, 1, 100.0, 0.01, 0, bc, bc_param=bp)
    r = np.random.default_rng(1).standard_normal(o.coarse.n_vert)
    r[o.phi0_mask] = 0.0
    phi, it, rc = cg.cgp_poisson_solve(s.handle, r)
    rr = r - r.mean() if o.pure_neumann else r
    ref = o.poisson(rr)
    assert rc == 0 and 0 < it < 5000
    assert rel(phi, ref) < 1e-9
    s.close(); m.close()


def _pair(cg, base, n_levels, k, Re, dt, chi, bc, bp=(1.0, 0, 0, 0), use_graph=1, mass_mode=0, **kw):
    m = cg.Mesh(base.xy, base.tri, base.tag, n_levels)
    prm = cg.make_params(Re, dt, chi=chi, k=k, bc_kind=bc, bc_param=bp, use_graph=use_graph,
                         mass_mode=mass_mode, **{**TIGHT, **kw})
    s = cg.Solver(m, prm)
    o = CGPOracle(base, n_levels, k, Re, dt, chi, bc, bc_param=bp,
                  mass_mode="lumped" if mass_mode else "consistent")
    return m, s, o


def test_one_step_intermediates(cg):
    m, s, o = _pair(cg, square_mesh(16), 2, 1, 100.0, 0.01, 1, flows.BC_CAVITY)
    s.step(1)
    out = o.step()
    # iterative solves stopped at relative residual 1e-13 are within ~kappa * 1e-13 of
    # the oracle's direct solves; 1e-8 leaves two decades of margin on every piece
    assert rel(s.vector(cg.CGP_VEC_UTILDE), out["Ut"]) < 1e-8
    assert rel(s.vector(cg.CGP_VEC_RHS_C), out["rc"]) < 1e-8
    assert rel(s.vector(cg.CGP_VEC_PHI_C), out["phic"]) < 1e-8
    assert rel(s.vector(cg.CGP_VEC_PHI_F), out["phif"]) < 1e-8
    U, P, t, st, rc = s.fields()
    assert rc == 0 and t == o.t
    assert rel(U, out["U"]) < 1e-8 and rel(P, out["P"]) < 1e-8
    s.close(); m.close()


@pytest.mark.parametrize("form", ["fp64", "fp64_kernels", "fp64_cluster", "fp64_mem", "mixed", "mixed_grid"])
def test_cavity64_k1_full_run(cg, form):
    # 64x64 lid-driven cavity, Re 100, pressure on 32x32, 50 steps at tolerance 1e-10:
    # FP64 within 1e-6 of the oracle, FP32-inner/FP64-outer within 1e-4 (it lands far closer)
    w = WORKLOADS["cavity64_k1"]
    base = w.base_mesh()
    extra = {"fp64": {}, "fp64_kernels": dict(coarse_mode=cg.CGP_COARSE_KERNELS),
             "fp64_cluster": dict(coarse_mode=cg.CGP_COARSE_CLUSTER), "mixed": dict(precision=cg.CGP_MIXED),
             "mixed_grid": dict(precision=cg.CGP_MIXED, coarse_mode=cg.CGP_COARSE_PERSISTENT),
             "fp64_mem": dict(coarse_mode=cg.CGP_COARSE_PERSISTENT_MEM)}[form]
    m, s, o = _pair(cg, base, w.n_levels, w.k, w.Re, w.dt, w.chi, w.bc, tol_mom=w.tol_mom,
                    tol_poisson=w.tol_poisson, tol_mass=1e-12, **extra)
    s.step(w.steps)
    o.run(w.steps)
    U, P, t, st, rc = s.fields()
    assert rc == 0 and st["steps"] == w.steps
    tol = 1e-4 if form == "mixed" else 1e-6
    assert rel(U, o.U) < tol and rel(P, o.P) < tol, (rel(U, o.U), rel(P, o.P))
    s.close(); m.close()


@pytest.mark.parametrize("csize", [2, 4, 8, 16])
def test_cluster_sizes_agree(cg, csize):
    m, s, o = _pair(cg, square_mesh(16), 2, 1, 100.0, 0.01, 1, flows.BC_CAVITY, coarse_mode=cg.CGP_COARSE_CLUSTER,
                    cluster_size=csize)
    s.step(2)
    o.run(2)
    U, P, t, st, rc = s.fields()
    assert rc == 0 and rel(U, o.U) < 1e-8 and rel(P, o.P) < 1e-8
    s.close(); m.close()


@pytest.mark.parametrize("chi,mass", [(0, 0), (1, 0), (1, 1)])
def test_channel_and_forms(cg, chi, mass):
    m, s, o = _pair(cg, _channel_small(), 2, 1, 20.0, 0.005, chi, flows.BC_CHANNEL, bp=(0.3, 0.41, 0, 0),
                    mass_mode=mass)
    s.step(4)
    o.run(4)
    U, P, t, st, rc = s.fields()
    assert rc == 0
    assert rel(U, o.U) < 1e-8 and rel(P, o.P) < 1e-8, (rel(U, o.U), rel(P, o.P))
    s.close(); m.close()


def test_periodic_taylor_green(cg):
    m, s, o = _pair(cg, square_mesh(8), 2, 2, 100.0, 0.002, 1, flows.BC_TG_PERIODIC)
    s.step(5)
    o.run(5)
    U, P, t, st, rc = s.fields()
    assert rc == 0 and rel(U, o.U) < 1e-8 and rel(P, o.P) < 1e-8
    s.close(); m.close()


@pytest.mark.parametrize("mode", [1, 2, 3, 4])
def test_graph_replay_equals_eager_launches(cg, mode):
    res = []
    for g in (0, 1):
        m, s, _ = _pair(cg, square_mesh(8), 2, 1, 100.0, 0.01, 1, flows.BC_CAVITY, use_graph=g, coarse_mode=mode)
        s.step(3)
        U, P, t, st, rc = s.fields()
        res.append((U, P, st))
        s.close(); m.close()
    assert np.array_equal(res[0][0], res[1][0]) and np.array_equal(res[0][1], res[1][1])
    assert res[0][2]["sum_it_mom"] == res[1][2]["sum_it_mom"]


def test_checkpoint_resume_is_bitwise(cg):
    # 4 steps in one go == 2 steps, state saved, a fresh solver restored, 2 more steps
    m, s, _ = _pair(cg, square_mesh(8), 2, 1, 100.0, 0.01, 1, flows.BC_CAVITY)
    s.step(4)
    U4, P4, t4, _, _ = s.fields()
    m2, s2, _ = _pair(cg, square_mesh(8), 2, 1, 100.0, 0.01, 1, flows.BC_CAVITY)
    s2.step(2)
    U2, P2, t2, _, _ = s2.fields()
    ck = (U2, s2.vector(cg.CGP_VEC_UPREV), P2, t2, s2.vector(cg.CGP_VEC_PHI_C))
    m3, s3, _ = _pair(cg, square_mesh(8), 2, 1, 100.0, 0.01, 1, flows.BC_CAVITY)
    s3.set_fields(ck[0], ck[1], ck[2], ck[3])
    s3.set_vector(cg.CGP_VEC_PHI_C, ck[4])
    s3.step(2)
    U, P, t, _, _ = s3.fields()
    assert t == t4
    assert np.array_equal(U, U4) and np.array_equal(P, P4)
    for x in (s, s2, s3, m, m2, m3):
        x.close()


def test_mixed_onchip_cluster_solve_on_channel(cg):
    # the mixed form's FP32 inner solve held on chip by one cluster, on a mesh with phi = 0 rows
    m, s, o = _pair(cg, _channel_small(), 2, 1, 20.0, 0.005, 1, flows.BC_CHANNEL, bp=(0.3, 0.41, 0, 0),
                    precision=cg.CGP_MIXED, coarse_mode=cg.CGP_COARSE_ONCHIP)
    kind, ctas, cl = s.coarse_info()
    assert kind == cg.CGP_COARSE_ONCHIP and cl in (8, 16) and ctas == cl
    s.step(4)
    o.run(4)
    U, P, t, st, rc = s.fields()
    assert rc == 0
    assert rel(U, o.U) < 1e-6 and rel(P, o.P) < 1e-6, (rel(U, o.U), rel(P, o.P))
    s.close(); m.close()


def test_onchip_coarse_correction_cuts_iterations(cg):
    """The subdomain coarse correction of the on-chip solve (a preconditioner variant, not in
    the paper): the same solution as the oracle's direct solve of Eq. 23, in far fewer inner
    iterations than Jacobi alone, on a 10.5K-row coarse level with phi = 0 rows and a hole."""
    base = _channel_small_fine()
    bp = (0.3, 0.41, 0, 0)
    m = cg.Mesh(base.xy, base.tri, base.tag, 3)
    o = CGPOracle(base, 3, 1, 100.0, 0.01, 0, flows.BC_CHANNEL, bc_param=bp)
    r = np.random.default_rng(2).standard_normal(o.coarse.n_vert)
    r[o.phi0_mask] = 0.0
    ref = o.poisson(r)
    its = {}
    for pc in (cg.CGP_PRECOND_JACOBI, cg.CGP_PRECOND_COARSE):
        s = cg.Solver(m, cg.make_params(100.0, 0.01, k=1, bc_kind=flows.BC_CHANNEL, bc_param=bp,
                                        guess=cg.CGP_GUESS_ZERO, precision=cg.CGP_MIXED, precond=pc, **TIGHT))
        assert s.coarse_info()[0] == cg.CGP_COARSE_ONCHIP
        assert (s.coarse_subdomains() == 0) == (pc == cg.CGP_PRECOND_JACOBI)
        phi, it, rc = cg.cgp_poisson_solve(s.handle, r)
        assert rc == 0 and rel(phi, ref) < 1e-9, (pc, rc, rel(phi, ref))
        its[pc] = it
        s.close()
    assert its[cg.CGP_PRECOND_COARSE] < 0.5 * its[cg.CGP_PRECOND_JACOBI], its
    m.close()


def test_mixed_mass_solves_run_chebyshev_steps(cg):
    """The mixed form's mass-matrix solves (Eqs. 25-26) run fixed FP32 Chebyshev steps inside
    FP64 refinement (two sweeps of 12 steps each), and the steps still match the oracle."""
    m, s, o = _pair(cg, _channel_small(), 2, 1, 20.0, 0.005, 1, flows.BC_CHANNEL, bp=(0.3, 0.41, 0, 0),
                    precision=cg.CGP_MIXED)
    s.step(2)
    o.run(2)
    prof = cg.cgp_profile_step(s.handle)   # one more step, eager launches with events
    o.run(1)
    assert prof.get("cheb_corr", (0, 0.0))[0] == 24 and prof.get("cheb_mass", (0, 0.0))[0] == 24, prof
    U, P, t, st, rc = s.fields()
    assert rc == 0
    assert rel(U, o.U) < 1e-6 and rel(P, o.P) < 1e-6, (rel(U, o.U), rel(P, o.P))
    s.close(); m.close()


def test_coarse_solver_choice(cg):
    base = square_mesh(16)
    m = cg.Mesh(base.xy, base.tri, base.tag, 2)

    def info(**kw):
        s = cg.Solver(m, cg.make_params(100.0, 0.01, k=1, **kw))
        out = s.coarse_info()
        s.close()
        return out

    assert info(coarse_mode=cg.CGP_COARSE_KERNELS) == (cg.CGP_COARSE_KERNELS, 0, 0)
    k, n, c = info(coarse_mode=cg.CGP_COARSE_CLUSTER)
    assert k == cg.CGP_COARSE_CLUSTER and n == c and c in (2, 4, 8, 16)
    k, n, c = info()                                    # FP64 default: register-resident grid solve
    assert k == cg.CGP_COARSE_PERSISTENT and n > 0 and c == 0
    k, n, c = info(coarse_mode=cg.CGP_COARSE_PERSISTENT_MEM)
    assert k == cg.CGP_COARSE_PERSISTENT_MEM and n > 0 and c == 0
    k, n, c = info(precision=cg.CGP_MIXED)              # mixed default: on-chip cluster solve
    assert k == cg.CGP_COARSE_ONCHIP and n == c and c in (8, 16)
    s = cg.Solver(m, cg.make_params(100.0, 0.01, k=1, precision=cg.CGP_MIXED))
    assert s.coarse_subdomains() >= 16                  # ... with the subdomain coarse correction
    s.close()
    s = cg.Solver(m, cg.make_params(100.0, 0.01, k=1, precision=cg.CGP_MIXED, precond=cg.CGP_PRECOND_JACOBI))
    assert s.coarse_subdomains() == 0
    s.close()
    with pytest.raises(RuntimeError):
        info(precond=cg.CGP_PRECOND_COARSE)             # the coarse correction lives in the on-chip solve
    k, n, c = info(precision=cg.CGP_MIXED, coarse_mode=cg.CGP_COARSE_PERSISTENT)   # FP32 inner in memory
    assert k == cg.CGP_COARSE_PERSISTENT_MEM and n > 0 and c == 0
    with pytest.raises(RuntimeError):
        info(coarse_mode=cg.CGP_COARSE_ONCHIP)          # the on-chip solve is FP32: mixed form only
    with pytest.raises(RuntimeError):
        info(precision=cg.CGP_MIXED, coarse_mode=cg.CGP_COARSE_KERNELS)
    m.close()


def test_mixed_falls_back_to_fp64_coarse_when_off_chip(cg):
    # a coarse system larger than one cluster can hold: AUTO keeps the mixed form's FP32-inner
    # fine solves and runs the grid-wide FP64 coarse solve
    w = WORKLOADS["cavity512_k1"]
    base = w.base_mesh()
    m = cg.Mesh(base.xy, base.tri, base.tag, w.n_levels)
    s = cg.Solver(m, cg.make_params(w.Re, w.dt, chi=w.chi, k=w.k, precision=cg.CGP_MIXED))
    assert s.coarse_info()[0] in (cg.CGP_COARSE_PERSISTENT, cg.CGP_COARSE_PERSISTENT_MEM)
    ref = cg.Solver(m, cg.make_params(w.Re, w.dt, chi=w.chi, k=w.k, precision=cg.CGP_MIXED,
                                      coarse_mode=cg.CGP_COARSE_PERSISTENT))
    assert ref.coarse_info()[0] == cg.CGP_COARSE_PERSISTENT_MEM
    ref.close()
    s.step(2)
    U, P, t, st, rc = s.fields()
    assert rc == 0 and np.isfinite(U).all() and st["res_poisson"] <= 1.0001e-8
    s.close(); m.close()


def test_user_boundary_data_reproduce_the_built_in_kinds(cg):
    # CGP_BC_USER with the caller's arrays: the cavity lid gives the cavity run bit for bit;
    # per-step Taylor-Green-periodic data (Dirichlet values and body force at t^{n+1},
    # evaluated on the host) give the built-in kind to rounding
    base = square_mesh(8)
    m = cg.Mesh(base.xy, base.tri, base.tag, 2)
    F = m.level(2)
    xy = F["xy"]
    ref = cg.Solver(m, cg.make_params(100.0, 0.01, chi=1, k=1, **TIGHT))
    usr = cg.Solver(m, cg.make_params(100.0, 0.01, chi=1, k=1, bc_kind=cg.CGP_BC_USER, **TIGHT))
    U0, P0, t0, _, _ = ref.fields()
    lid = flows.dirichlet_value(flows.BC_CAVITY, xy, 0.0, 100.0)
    cg.cgp_set_dirichlet(usr.handle, lid)
    usr.set_fields(U0, U0, P0, t0)
    ref.step(5)
    usr.step(5)
    assert np.array_equal(ref.fields()[0], usr.fields()[0]) and np.array_equal(ref.fields()[1], usr.fields()[1])
    ref.close(); usr.close()
    Re, dt = 100.0, 0.005
    ref = cg.Solver(m, cg.make_params(Re, dt, chi=1, k=1, bc_kind=cg.CGP_BC_TG_PERIODIC, **TIGHT))
    usr = cg.Solver(m, cg.make_params(Re, dt, chi=1, k=1, bc_kind=cg.CGP_BC_USER, **TIGHT))
    U0, P0, t0, _, _ = ref.fields()
    usr.set_fields(U0, ref.vector(cg.CGP_VEC_UPREV), P0, t0)
    for n in range(6):
        t1 = (n + 1) * dt
        cg.cgp_set_dirichlet(usr.handle, flows.dirichlet_value(flows.BC_TG_PERIODIC, xy, t1, Re))
        cg.cgp_set_forcing(usr.handle, flows.body_force(flows.BC_TG_PERIODIC, xy, t1, Re))
        usr.step(1)
    ref.step(6)
    Ur, Pr = ref.fields()[:2]
    Uu, Pu = usr.fields()[:2]
    assert rel(Uu, Ur) < 1e-10 and rel(Pu, Pr) < 1e-8, (rel(Uu, Ur), rel(Pu, Pr))
    with pytest.raises(RuntimeError):
        cg.cgp_set_forcing(ref.handle, np.zeros((xy.shape[0], 2)))     # not a CGP_BC_USER solver
    ref.close(); usr.close(); m.close()


@pytest.mark.parametrize("case", ["cavity_k2", "channel_k1"])
def test_pt_restriction_full_run(cg, case):
    # restrict_mode PT (the fine divergence restricted by P^T) against the oracle's variant
    if case == "cavity_k2":
        base, lv, k, bc, bp = square_mesh(8), 2, 2, flows.BC_CAVITY, (1.0, 0, 0, 0)
    else:
        base, lv, k, bc, bp = _channel_small(), 2, 1, flows.BC_CHANNEL, (0.3, 0.41, 0, 0)
    m = cg.Mesh(base.xy, base.tri, base.tag, lv)
    s = cg.Solver(m, cg.make_params(100.0, 0.01, chi=1, k=k, bc_kind=bc, bc_param=bp,
                                    restrict_mode=cg.CGP_RESTRICT_PT, **TIGHT))
    o = CGPOracle(base, lv, k, 100.0, 0.01, 1, bc, bc_param=bp, restrict_mode="pt")
    s.step(1)
    out = o.step()
    assert rel(s.vector(cg.CGP_VEC_RHS_C), out["rc"]) < 1e-10
    s.step(4)
    o.run(4)
    U, P, t, st, rc = s.fields()
    assert rc == 0 and rel(U, o.U) < 1e-6 and rel(P, o.P) < 1e-6, (rel(U, o.U), rel(P, o.P))
    s.close(); m.close()
