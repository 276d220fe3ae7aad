"""Seeded synthetic inputs shared by the CUDA path's callers and by the oracle.

This package only *generates problem inputs*: base triangle meshes (coordinates,
connectivity, boundary flags) and the parameter sets of the benchmark workloads.
It holds none of the method's arithmetic (no refinement, no assembly, no
solver, no transfer operator), so neither side of a parity test can borrow the
other's implementation through it.

Boundary flags (one byte per vertex, combined with bitwise OR):

* ``VEL_DIR`` (1): the velocity is prescribed there (Dirichlet part of the
  boundary, Eqs. 3 and 10 of the paper).
* ``PHI_ZERO`` (2): the pressure increment vanishes there (phi = 0 on the
  natural/traction part of the boundary, Eq. 14).

A vertex with neither flag is interior (or lies on a part of the boundary where
only the homogeneous Neumann condition for phi of Eq. 13 applies).
"""

from .meshes import (VEL_DIR, PHI_ZERO, square_mesh, crisscross_mesh,
                     channel_cylinder_mesh, open_square_mesh, disk_mesh, BaseMesh)
from .configs import WORKLOADS, Workload, batch_instances

__all__ = ["VEL_DIR", "PHI_ZERO", "square_mesh", "crisscross_mesh",
           "channel_cylinder_mesh", "open_square_mesh", "disk_mesh", "BaseMesh", "WORKLOADS", "Workload",
           "batch_instances"]
