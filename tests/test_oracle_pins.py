"""Pins of the oracle parts that the manufactured-solution tests cannot see (CPU only).

* The outflow reading of Eq. 21's pressure term (-dt G P^n in weak form, -int p div psi,
  which makes the traction of Eq. 4 vanish on the outflow) and the channel's inflow
  profile: plane Poiseuille flow u = 4 Umax y (H - y) / H^2, p = 8 Umax nu (L - x) / H^2 is
  an exact steady solution of the Navier-Stokes equations (Eqs. 1-2) whose do-nothing
  traction -p n + nu du/dn vanishes at x = L.  On the uniform two-triangle mesh its nodal
  interpolant is a fixed point of the whole discrete step (every row of Eqs. 21-26 holds
  exactly for a y-quadratic u and a linear p there); on unstructured meshes the step
  converges to it at second order in u.  A constant added to P changes Eq. 21's right-hand
  side by dt c times the boundary integral of psi_i n_x over the outflow, computed here from
  the edge lengths alone.
* Eq. 27, the lumped mass: m_i = integral of psi_i = sum over the triangles at i of |T|/3;
  for a linear Phi the lumped correction of Eq. 25 is exactly -2/3 dt grad Phi, and for a
  linear U~ the rotational term of Eq. 26 is exactly div U~ / Re (consistent and lumped
  alike, since M 1 = m); a two-triangle case worked by hand.
* Adam (Kingma and Ba, 2015, Algorithm 1), the optimiser of the learned guess: the first
  bias-corrected step moves every parameter by -lr g / (|g| + eps), and two steps on a
  scalar match values worked out exactly by hand.

The last test applies each plausible mistake (a sign, the strong form of the pressure
term, diag(M) for the row sums, Adam without bias correction) to a copy of the oracle's
source and checks that the pin above it fails.
"""

import importlib.util
import inspect
import sys

import numpy as np
import pytest

from workloads import square_mesh, channel_cylinder_mesh, BaseMesh, VEL_DIR, PHI_ZERO
import oracle.cgp
import oracle.mlp
from oracle import flows, norms

L_CH, H_CH = 2.0, 1.0


def _tag_channel(m, L, H):
    x, y = m.xy[:, 0], m.xy[:, 1]
    tag = np.zeros(m.n_vert, np.uint8)
    tag[(x == 0.0) | (y == 0.0) | (y == H)] |= VEL_DIR
    tag[x == L] |= PHI_ZERO
    m.tag = tag
    return m


def _poiseuille(xy, Re, L=L_CH, H=H_CH, Umax=1.0):
    x, y = xy[:, 0], xy[:, 1]
    U = np.stack([4.0 * Umax * y * (H - y) / H ** 2, np.zeros_like(y)], 1)
    P = 8.0 * Umax / (Re * H ** 2) * (L - x)
    return U, P


def _poiseuille_run(cgp, base, n_levels, k, chi, Re=1.0, steps=5, dt=0.01):
    o = cgp.CGPOracle(base, n_levels, k, Re, dt, chi, flows.BC_CHANNEL, bc_param=(1.0, H_CH, 0, 0))
    Ue, Pe = _poiseuille(o.fine.xy, Re)
    o.set_state(Ue, Ue, Pe, 0.0)
    o.run(steps)
    M = o.ops_f["M"]
    return norms.l2(M, o.U - Ue) / norms.l2(M, Ue), norms.l2(M, o.P - Pe) / norms.l2(M, Pe)


def _structured_channel():
    return _tag_channel(square_mesh(4, 0.0, L_CH, 0.0, H_CH), L_CH, H_CH)


def check_poiseuille_fixed_point(cgp):
    """Largest relative error of U and P after 5 steps from the Poiseuille interpolant."""
    worst = 0.0
    for k in (0, 1, 2):
        for chi in (0, 1):
            eu, ep = _poiseuille_run(cgp, _structured_channel(), 2, k, chi)
            worst = max(worst, eu, ep)
    return worst


def test_poiseuille_is_a_fixed_point_on_the_uniform_mesh():
    assert check_poiseuille_fixed_point(oracle.cgp) < 1e-12


@pytest.mark.parametrize("chi,k", [(0, 0), (0, 1), (1, 0), (1, 1)])
def test_poiseuille_converges_at_second_order_on_unstructured_meshes(chi, k):
    base = channel_cylinder_mesh(seed=3, h=0.2, L=L_CH, H=H_CH, r=0.0)
    e = np.array([_poiseuille_run(oracle.cgp, base, lv, k, chi, steps=20) for lv in (1, 2, 3)])
    rate = np.log2(e[:-1] / e[1:])
    # velocity O(h^2); pressure at least O(h) (P1 pressure with an O(h^2) velocity error)
    assert (rate[:, 0] > 1.8).all(), rate
    assert (rate[:, 1] > 1.0).all(), rate
    assert e[-1, 0] < 3e-3


def _outflow_boundary_integral(xy, L):
    """int over {x = L} of psi_i n_x ds for every vertex: half of each outflow edge's length
    to both of its ends (n_x = 1 there)."""
    on = np.flatnonzero(xy[:, 0] == L)
    on = on[np.argsort(xy[on, 1])]
    beta = np.zeros(xy.shape[0])
    for a, b in zip(on[:-1], on[1:]):
        ell = xy[b, 1] - xy[a, 1]
        beta[a] += 0.5 * ell
        beta[b] += 0.5 * ell
    return beta


def check_outflow_pressure_term(cgp):
    """Largest deviation of the change of Eq. 21's right-hand side under P -> P + c from
    dt c (boundary integral of psi n_x), relative to its size."""
    base = channel_cylinder_mesh(seed=3, h=0.2, L=L_CH, H=H_CH, r=0.0)
    Re, dt, c = 2.0, 0.05, 0.75
    o = cgp.CGPOracle(base, 1, 0, Re, dt, 0, flows.BC_CHANNEL, bc_param=(1.0, H_CH, 0, 0))
    n = o.fine.n_vert
    Z = np.zeros((n, 2))
    Pe = _poiseuille(o.fine.xy, Re)[1]
    # at rest the convection operator vanishes, so Eq. 21's matrix is 3/2 M + dt/Re K with
    # identity rows at the Dirichlet vertices (operators pinned in test_oracle_fem.py)
    d = o.dir_mask
    A = (1.5 * o.ops_f["M"] + (dt / Re) * o.ops_f["K"]).tolil()
    for i in np.flatnonzero(d):
        A.rows[i], A.data[i] = [int(i)], [1.0]
    A = A.tocsr()
    b0 = np.stack([A @ u for u in o.momentum(Z, Z, Pe, dt).T], 1)
    b1 = np.stack([A @ u for u in o.momentum(Z, Z, Pe + c, dt).T], 1)
    beta = _outflow_boundary_integral(o.fine.xy, L_CH)
    beta[d] = 0.0
    want = np.stack([dt * c * beta, np.zeros(n)], 1)
    return np.abs((b1 - b0) - want).max() / np.abs(want).max()


def test_outflow_pressure_term_is_the_weak_form():
    assert check_outflow_pressure_term(oracle.cgp) < 1e-10


def test_channel_inflow_profile():
    xy = np.array([[0.0, 0.0], [0.0, 0.1025], [0.0, 0.205], [0.0, 0.41], [0.5, 0.205]])
    uD = flows.dirichlet_value(flows.BC_CHANNEL, xy, 0.3, 20.0, (0.3, 0.41, 0, 0))
    # Umax at mid-height, 3/4 Umax at a quarter, zero at the walls; only x = 0 is inflow
    np.testing.assert_allclose(uD[:, 0], [0.0, 0.225, 0.3, 0.0, 0.0], rtol=0, atol=1e-15)
    assert not uD[:, 1].any()


# ---- Eq. 27 (lumped mass) ----

def _two_triangles():
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [1.0, 1.0], [0.0, 1.0]])
    tri = np.array([[0, 1, 2], [0, 2, 3]], np.int32)
    return BaseMesh(xy, tri, np.zeros(4, np.uint8))


def _lumped_oracle(cgp, base, n_levels=0, mass_mode="lumped", chi=1, Re=4.0, dt=0.3):
    return cgp.CGPOracle(base, n_levels, 0, Re, dt, chi, flows.BC_CAVITY, mass_mode=mass_mode)


def check_lumped_two_triangles(cgp):
    """Largest error of the lumped Eq. 25 / Eq. 27 results against the hand-worked values."""
    dt, Re = 0.3, 4.0
    o = _lumped_oracle(cgp, _two_triangles(), dt=dt, Re=Re)
    # integral of each hat function: vertices 0 and 2 lie in both triangles (area 1/2 each)
    err = np.abs(o.mlump_f - [1 / 3, 1 / 6, 1 / 3, 1 / 6]).max()
    # Phi = psi_3 = y - x on triangle (0,2,3), zero on (0,1,2): Cx Phi = -1/6, Cy Phi = 1/6
    # at vertices 0, 2, 3; the correction -2/3 dt (Cx Phi, Cy Phi) / m_i
    phi = np.array([0.0, 0.0, 0.0, 1.0])
    Ut = np.zeros((4, 2))
    want = dt * np.array([[1 / 3, -1 / 3], [0.0, 0.0], [1 / 3, -1 / 3], [2 / 3, -2 / 3]])
    err = max(err, np.abs(o.correct(Ut, phi) - want).max())
    # U~ = (psi_3, 0): div = Cx u = -1/6 at vertices 0, 2, 3; P1 = P + Phi - div / (m Re)
    Ut = np.array([[0.0, 0.0], [0.0, 0.0], [0.0, 0.0], [1.0, 0.0]])
    P = np.array([1.0, 2.0, 3.0, 4.0])
    want = P + phi - np.array([-0.5, 0.0, -0.5, -1.0]) / Re
    err = max(err, np.abs(o.pressure(P, phi, Ut) - want).max())
    return err


def test_lumped_mass_two_triangles_by_hand():
    assert check_lumped_two_triangles(oracle.cgp) < 1e-15


def test_lumped_mass_is_the_hat_function_integral():
    base = channel_cylinder_mesh(seed=5, h=0.08)
    o = _lumped_oracle(oracle.cgp, base, n_levels=1)
    xy, tri = o.fine.xy, o.fine.tri
    m = np.zeros(o.fine.n_vert)
    for a, b, c in tri:                       # shoelace area, a third to each corner
        area = 0.5 * abs((xy[b, 0] - xy[a, 0]) * (xy[c, 1] - xy[a, 1])
                         - (xy[c, 0] - xy[a, 0]) * (xy[b, 1] - xy[a, 1]))
        m[[a, b, c]] += area / 3.0
    np.testing.assert_allclose(o.mlump_f, m, rtol=1e-13)
    assert abs(o.mlump_f.sum() - base.meta["area"]) < 1e-12


@pytest.mark.parametrize("mass_mode", ["lumped", "consistent"])
def test_linear_fields_are_corrected_exactly(mass_mode):
    # a linear Phi: grad Phi = (a, b) everywhere, Cx Phi = a m, so M delta = -2/3 dt a m has
    # the constant solution (no Dirichlet rows here); a linear U~ has constant divergence d
    dt, Re = 0.01, 50.0
    base = square_mesh(4, 0.0, 1.0, 0.0, 1.0, boundary_flags=0)     # no boundary flags
    o = _lumped_oracle(oracle.cgp, base, n_levels=1, mass_mode=mass_mode, dt=dt, Re=Re)
    x, y = o.fine.xy[:, 0], o.fine.xy[:, 1]
    a, b = 0.7, -1.3
    phi = a * x + b * y + 0.25
    Ut = np.stack([2.0 * x - y, 0.5 * x + 3.0 * y], 1)      # div = 2 + 3
    U = o.correct(Ut, phi)
    np.testing.assert_allclose(U - Ut, np.broadcast_to(-2.0 / 3.0 * dt * np.array([a, b]), Ut.shape),
                               rtol=1e-11, atol=1e-14)
    P0 = np.sin(x)
    np.testing.assert_allclose(o.pressure(P0, phi, Ut), P0 + phi - 5.0 / Re, rtol=1e-12)


def test_lumped_correction_with_dirichlet_rows():
    # Dirichlet rows keep U~; every other row gets -2/3 dt grad Phi exactly (lumped: local)
    dt = 0.02
    base = _tag_channel(square_mesh(4, 0.0, L_CH, 0.0, H_CH), L_CH, H_CH)
    o = _lumped_oracle(oracle.cgp, base, n_levels=1, dt=dt)
    x, y = o.fine.xy[:, 0], o.fine.xy[:, 1]
    phi = 2.0 * x - 0.5 * y
    Ut = np.random.default_rng(0).standard_normal((o.fine.n_vert, 2))
    U = o.correct(Ut, phi)
    d = o.dir_mask
    assert d.any() and (~d).any()
    np.testing.assert_array_equal(U[d], Ut[d])
    np.testing.assert_allclose(U[~d] - Ut[~d], np.broadcast_to(-2.0 / 3.0 * dt * np.array([2.0, -0.5]),
                                                               (int((~d).sum()), 2)), rtol=1e-12, atol=1e-15)


# ---- Adam ----

def _adam_scalar(mlp, grads, lr, eps):
    W, b = [np.zeros((1, 1))], [np.zeros(1)]
    state = {"m": [np.zeros((1, 1)), np.zeros(1)], "v": [np.zeros((1, 1)), np.zeros(1)], "t": 0}
    out = []
    for g in grads:
        mlp.adam_step(W, b, [np.full((1, 1), g)], [np.full(1, g)], state, lr, eps=eps)
        out.append((W[0][0, 0], b[0][0]))
    return out


def check_adam(mlp):
    """Largest error of two scalar Adam steps against the values worked out by hand, and of
    a first step on a random tensor against -lr g / (|g| + eps)."""
    # g = 2 then -1, lr = 1/2, beta = (0.9, 0.999), eps = 0:
    #   m1 = 1/5, v1 = 1/250, m^ = 2, v^ = 4: step -1/2 * 2/2 = -1/2
    #   m2 = 2/25, v2 = 1249/250000, m^ = 8/19, v^ = 4996/1999: step -1/2 (8/19)/sqrt(4996/1999)
    (w1, b1), (w2, b2) = _adam_scalar(mlp, [2.0, -1.0], 0.5, 0.0)
    err = max(abs(w1 + 0.5), abs(b1 + 0.5), abs(w2 + 0.6331685198302013), abs(b2 + 0.6331685198302013))
    rng = np.random.default_rng(7)
    W = [rng.standard_normal((3, 4))]
    b = [rng.standard_normal(3)]
    gW = [rng.standard_normal((3, 4))]
    gb = [rng.standard_normal(3) * 1e-3]
    W0, b0 = W[0].copy(), b[0].copy()
    state = {"m": [np.zeros((3, 4)), np.zeros(3)], "v": [np.zeros((3, 4)), np.zeros(3)], "t": 0}
    lr, eps = 1e-2, 1e-8
    mlp.adam_step(W, b, gW, gb, state, lr, eps=eps)
    err = max(err, np.abs((W[0] - W0) + lr * gW[0] / (np.abs(gW[0]) + eps)).max() / lr,
              np.abs((b[0] - b0) + lr * gb[0] / (np.abs(gb[0]) + eps)).max() / lr)
    return err


def test_adam_matches_the_published_update():
    assert check_adam(oracle.mlp) < 1e-12


# ---- the pins bite: each plausible mistake, planted in a copy of the oracle, fails them ----

def _mutated(module, old, new):
    src = inspect.getsource(module)
    assert src.count(old) == 1, old
    name = module.__name__ + "_mutant"
    spec = importlib.util.spec_from_loader(name, loader=None)
    mod = importlib.util.module_from_spec(spec)
    mod.__package__ = module.__package__
    sys.modules[name] = mod
    try:
        exec(compile(src.replace(old, new), module.__file__ + " (mutant)", "exec"), mod.__dict__)
    finally:
        del sys.modules[name]
    return mod


@pytest.mark.parametrize("old,new,check,bound", [
    # sign of the pressure term of Eq. 21
    ("bx = dt * (Cx.T @ P)", "bx = -dt * (Cx.T @ P)", check_poiseuille_fixed_point, 1e-12),
    # strong form Cx P instead of the weak form -Cx^T P (differs only where P != 0 on the outflow)
    ("bx = dt * (Cx.T @ P)", "bx = -dt * (Cx @ P)", check_outflow_pressure_term, 1e-10),
    # the diagonal of M instead of its row sums in Eq. 27
    ('self.mlump_f = np.asarray(M.sum(axis=1)).ravel()', "self.mlump_f = M.diagonal().copy()",
     check_lumped_two_triangles, 1e-15),
])
def test_planted_oracle_mistakes_fail_their_pins(old, new, check, bound):
    assert check(oracle.cgp) < bound
    assert check(_mutated(oracle.cgp, old, new)) > 1e3 * bound


@pytest.mark.parametrize("old,new", [
    ("mh = m / (1 - beta1 ** t)", "mh = m"),                       # no bias correction of m
    ("vh = v / (1 - beta2 ** t)", "vh = v / (1 - beta1 ** t)"),    # beta1 where beta2 belongs
])
def test_planted_adam_mistakes_fail_their_pin(old, new):
    assert check_adam(oracle.mlp) < 1e-12
    assert check_adam(_mutated(oracle.mlp, old, new)) > 1e-6
