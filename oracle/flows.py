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
* BC_JOBELIN_OPEN (5): the vortex of Section 3.2 on [0,1]^2: u = sin x sin(y+t),
  v = cos x cos(y+t), p = cos x sin(y+t), with the body force that makes it a solution of
  Eq. 1; velocity Dirichlet data on x = 1, y = 0, y = 1, the traction of Eq. 4 on the
  y-axis x = 0 (Gamma_N, outward normal (-1, 0)) taken from the closed form (the paper
  calls it homogeneous, but the closed form has -p n + grad u . n / Re = ((1 - 1/Re)
  sin(y+t), 0) there), and the pressure on Gamma_N from the closed form.
* BC_JOBELIN_DISK (6): the vortex of Section 3.3 on the disk x^2 + y^2 < 1/4:
  u = sin(x+t) sin(y+t), v = cos(x+t) cos(y+t), p = cos(x-y+t), velocity Dirichlet data on
  the whole boundary.

The body forces are f = u_t + (u . grad) u - Lap u / Re + grad p written out from the
derivatives of the closed forms (both fields are divergence free and Lap u = -2 u).

Start of BDF2 (Eq. 5 needs u^{n-1}): where a closed form exists u^{-1} is the
exact field at t = -dt, otherwise u^{-1} = u^0.  p^0 is the exact pressure at
t = 0, or 0.
"""

import numpy as np

BC_CAVITY, BC_CHANNEL, BC_TG, BC_TG_PERIODIC = 0, 1, 2, 3
BC_JOBELIN_OPEN, BC_JOBELIN_DISK = 5, 6


def _jobelin(kind, x, y, t):
    """(u, v, p) and the first derivatives the body force and the traction need:
    returns dict with u, v, p, u_t, v_t, u_x, u_y, v_x, v_y, p_x, p_y."""
    if kind == BC_JOBELIN_OPEN:
        a, b = x, y + t
        sa, ca, sb, cb = np.sin(a), np.cos(a), np.sin(b), np.cos(b)
        d = {"u": sa * sb, "v": ca * cb, "p": ca * sb,
             "u_t": sa * cb, "v_t": -ca * sb,
             "p_x": -sa * sb, "p_y": ca * cb}
    else:
        a, b, c = x + t, y + t, x - y + t
        sa, ca, sb, cb = np.sin(a), np.cos(a), np.sin(b), np.cos(b)
        d = {"u": sa * sb, "v": ca * cb, "p": np.cos(c),
             "u_t": ca * sb + sa * cb, "v_t": -sa * cb - ca * sb,
             "p_x": -np.sin(c), "p_y": np.sin(c)}
    d.update({"u_x": ca * sb, "u_y": sa * cb, "v_x": -sa * cb, "v_y": -ca * sb})
    return d


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
    if kind in (BC_JOBELIN_OPEN, BC_JOBELIN_DISK):
        d = _jobelin(kind, x, y, t)
        return np.stack([d["u"], d["v"]], 1), d["p"]
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
    if kind in (BC_JOBELIN_OPEN, BC_JOBELIN_DISK):
        d = _jobelin(kind, xy[:, 0], xy[:, 1], t)
        # Lap u = -2 u, Lap v = -2 v for both vortices
        fx = d["u_t"] + d["u"] * d["u_x"] + d["v"] * d["u_y"] + 2.0 * d["u"] / Re + d["p_x"]
        fy = d["v_t"] + d["u"] * d["v_x"] + d["v"] * d["v_y"] + 2.0 * d["v"] / Re + d["p_y"]
        return np.stack([fx, fy], 1)
    return np.zeros((xy.shape[0], 2))


def traction(kind, xy, t, Re, bc_param=(1.0, 0.0, 0.0, 0.0)):
    """Nodal traction t = -p n + (grad u) n / Re of Eq. 4 on the natural boundary (zero for
    every kind but BC_JOBELIN_OPEN, whose Gamma_N is x = 0 with outward normal (-1, 0))."""
    out = np.zeros((xy.shape[0], 2))
    if kind == BC_JOBELIN_OPEN:
        d = _jobelin(kind, xy[:, 0], xy[:, 1], t)
        out[:, 0] = d["p"] - d["u_x"] / Re
        out[:, 1] = -d["v_x"] / Re
    return out


def natural_normal(kind, xy):
    """Outward unit normal on the natural boundary (the y-axis of the open-boundary vortex)."""
    n = np.zeros((xy.shape[0], 2))
    if kind == BC_JOBELIN_OPEN:
        n[:, 0] = -1.0
    return n


def natural_pressure(kind, xy, t, Re, bc_param=(1.0, 0.0, 0.0, 0.0)):
    """Pressure prescribed on the natural boundary at time t, or None (then it stays 0 there,
    as on the channel's outflow)."""
    if kind == BC_JOBELIN_OPEN:
        return exact(kind, xy, t, Re, bc_param)[1]
    return None


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
