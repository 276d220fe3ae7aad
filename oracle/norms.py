"""Discrete error norms (oracle; test infrastructure only).

The paper tabulates L-infinity and L2 norms of the velocity, pressure and
pressure-gradient errors (Tables 1-3) without defining them.  Reading used
here: L2 is the finite-element norm sqrt(e^T M e) of the nodal error e (exact
for the P1 interpolant of the error), L-infinity is the largest nodal error.
For the pressure, which is fixed only up to a constant on pure-Dirichlet
velocity domains, the M-weighted mean of both fields is removed first.
"""

import numpy as np


def l2(M, e):
    e = np.asarray(e, dtype=np.float64)
    if e.ndim == 2:
        return float(np.sqrt(sum(e[:, d] @ (M @ e[:, d]) for d in range(e.shape[1]))))
    return float(np.sqrt(e @ (M @ e)))


def linf(e):
    e = np.asarray(e, dtype=np.float64)
    if e.ndim == 2:
        return float(np.sqrt((e ** 2).sum(axis=1)).max())
    return float(np.abs(e).max())


def remove_mean(M, p):
    w = np.asarray(M.sum(axis=1)).ravel()
    return p - (w @ p) / w.sum()


def pressure_errors(M, p, p_exact):
    e = remove_mean(M, p) - remove_mean(M, p_exact)
    return l2(M, e), linf(e)
