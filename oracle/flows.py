"""Boundary data, body forces and closed-form flows (oracle; test infrastructure only).

Problem statements used by the workloads:

* BC_CAVITY (0): lid-driven cavity on [0,1]^2.  u = (lid, 0) at vertices with
  y = 1 and 0 < x < 1, u = 0 on the rest of the boundary (corners included),
  f = 0, start from rest.  lid = bc_param[0].
* BC_CHANNEL (1): channel [0,L]x[0,H] with a cylinder.  u = (4 Umax y (H-y)/H^2, 0)
  at x = 0, u = 0 on walls and cylinder, traction-free outflow (Eq. 4 with
  t = 0), f = 0, start from rest with the inflow profile on the inlet.
  Umax = bc_param[0], H = bc_param[1].
* BC_TG (2): the Taylor-Green vortex of Section 3.1, Eqs. 28-30, f = 0.
* BC_TG_PERIODIC (3): Taylor-Green with amplitude g(t) = cos(2 pi t):
  u = g U0(x), p = g^2 P0(x) with U0, P0 the t = 0 Taylor-Green fields, and the
  body force f = (g' + 8 pi^2 g / Re) U0 that makes it an exact solution
  ((U0 . grad) U0 + grad P0 = 0 and -Lap U0 = 8 pi^2 U0).

Start of BDF2 (Eq. 5 needs u^{n-1}): where a closed form exists u^{-1} is the
exact field at t = -dt, otherwise u^{-1} = u^0.  p^0 is the exact pressure at
t = 0, or 0.
"""

import numpy as np

BC_CAVITY, BC_CHANNEL, BC_TG, BC_TG_PERIODIC = 0, 1, 2, 3


def _tg_shape(x, y):
    u = -np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y)
    v = np.sin(2 * np.pi * x) * np.cos(2 * np.pi * y)
    p = -(np.cos(4 * np.pi * x) + np.cos(4 * np.pi * y)) / 4.0
    return u, v, p


def exact(kind, xy, t, Re, bc_param=(1.0, 0.0, 0.0, 0.0)):
    """Closed-form (u (n,2), p (n,)) or None when the problem has none."""
    x, y = xy[:, 0], xy[:, 1]
    if kind == BC_TG:
        u, v, p = _tg_shape(x, y)
        e = np.exp(-8 * np.pi ** 2 * t / Re)
        return np.stack([u * e, v * e], 1), p * e * e
    if kind == BC_TG_PERIODIC:
        u, v, p = _tg_shape(x, y)
        g = np.cos(2 * np.pi * t)
        return np.stack([u * g, v * g], 1), p * g * g
    return None


def dirichlet_value(kind, xy, t, Re, bc_param=(1.0, 0.0, 0.0, 0.0)):
    """Velocity prescribed at the given vertices at time t (n, 2)."""
    x, y = xy[:, 0], xy[:, 1]
    out = np.zeros((xy.shape[0], 2))
    if kind == BC_CAVITY:
        lid = (y == 1.0) & (x > 0.0) & (x < 1.0)
        out[lid, 0] = bc_param[0]
        return out
    if kind == BC_CHANNEL:
        Umax, H = bc_param[0], bc_param[1]
        inl = x == 0.0
        out[inl, 0] = 4.0 * Umax * y[inl] * (H - y[inl]) / (H * H)
        return out
    return exact(kind, xy, t, Re, bc_param)[0]


def body_force(kind, xy, t, Re, bc_param=(1.0, 0.0, 0.0, 0.0)):
    """Nodal values of f at time t (n, 2)."""
    if kind == BC_TG_PERIODIC:
        u, v, _ = _tg_shape(xy[:, 0], xy[:, 1])
        g = np.cos(2 * np.pi * t)
        gp = -2 * np.pi * np.sin(2 * np.pi * t)
        c = gp + 8 * np.pi ** 2 * g / Re
        return np.stack([c * u, c * v], 1)
    return np.zeros((xy.shape[0], 2))


def initial_state(kind, xy, dirichlet, dt, Re, bc_param=(1.0, 0.0, 0.0, 0.0)):
    """(U^0, U^{-1}, P^0) for the BDF2 start."""
    ex0 = exact(kind, xy, 0.0, Re, bc_param)
    if ex0 is not None:
        exm = exact(kind, xy, -dt, Re, bc_param)
        return ex0[0].copy(), exm[0].copy(), ex0[1].copy()
    U0 = np.zeros((xy.shape[0], 2))
    uD = dirichlet_value(kind, xy, 0.0, Re, bc_param)
    U0[dirichlet] = uD[dirichlet]
    return U0, U0.copy(), np.zeros(xy.shape[0])
