"""Parameter sets of the benchmark workloads (inputs only).

Each :class:`Workload` names a base mesh, how many uniform refinements build the
velocity (fine) level, how many coarsening levels the pressure increment uses,
and the physical/numerical parameters of the incremental pressure-correction
step (Reynolds number, time step, standard chi=0 or rotational chi=1 form).
"""

from dataclasses import dataclass, field

import numpy as np

from .meshes import square_mesh, channel_cylinder_mesh, VEL_DIR

# boundary-condition kinds understood by both sides (problem statements, not method)
BC_CAVITY = 0        # lid-driven cavity on [0,1]^2: u=(1,0) on y=1, 0<x<1; no slip elsewhere
BC_CHANNEL = 1       # channel with cylinder: parabolic inflow at x=0, traction-free outflow
BC_TG = 2            # decaying Taylor-Green vortex (paper Eqs. 28-30), exact Dirichlet data
BC_TG_PERIODIC = 3   # Taylor-Green with g(t)=cos(2 pi t) amplitude and matching body force


@dataclass
class Workload:
    name: str
    base: str                 # "square", "channel"
    base_n: int               # squares per side (square) or seed (channel)
    n_levels: int             # uniform refinements of the base mesh
    k: int                    # coarsening levels of the pressure-increment mesh
    Re: float
    dt: float
    steps: int
    chi: int
    bc: int
    tol_poisson: float
    tol_mom: float
    bc_param: tuple = (1.0, 0.0, 0.0, 0.0)
    extra: dict = field(default_factory=dict)

    def base_mesh(self):
        if self.base == "square":
            return square_mesh(self.base_n, boundary_flags=VEL_DIR)
        if self.base == "channel":
            return channel_cylinder_mesh(seed=self.base_n, h=self.extra.get("h", 0.0084))
        raise ValueError(self.base)


WORKLOADS = {
    # 64x64 cavity (8192 triangles), pressure on 32x32 (k=1), Re=100, standard form
    "cavity64_k1": Workload("cavity64_k1", "square", 32, 1, 1, 100.0, 0.01, 50, 0,
                            BC_CAVITY, 1e-10, 1e-10),
    # 512x512 cavity (524,288 triangles), rotational form, pressure 1-3 levels coarser
    "cavity512_k1": Workload("cavity512_k1", "square", 64, 3, 1, 400.0, 0.002, 200, 1,
                             BC_CAVITY, 1e-8, 1e-8),
    "cavity512_k2": Workload("cavity512_k2", "square", 64, 3, 2, 400.0, 0.002, 200, 1,
                             BC_CAVITY, 1e-8, 1e-8),
    "cavity512_k3": Workload("cavity512_k3", "square", 64, 3, 3, 400.0, 0.002, 200, 1,
                             BC_CAVITY, 1e-8, 1e-8),
    # manufactured periodic-forced Taylor-Green, Re=100, same 512x512 hierarchy
    "tgp512_k2": Workload("tgp512_k2", "square", 64, 3, 2, 100.0, 0.002, 200, 1,
                          BC_TG_PERIODIC, 1e-8, 1e-8),
    # channel with cylinder: ~16k-triangle Delaunay base, 3 refinements (~1.05M
    # triangles), pressure 2 levels coarser; nu = 1e-3 (Re=20 on the mean inflow
    # speed 0.2 and the diameter 0.1); Umax = 0.3
    "channel1m_k2": Workload("channel1m_k2", "channel", 0, 3, 2, 1000.0, 0.002, 100, 1,
                             BC_CHANNEL, 1e-8, 1e-8, bc_param=(0.3, 0.41, 0.0, 0.0)),
}


def batch_instances(n=256, seed=20181203):
    """Seeded list of uneven cavity instances (fine sizes 32^2..256^2 x 2 triangles).

    Each entry: fine squares per side, coarsening levels k (1..3), Reynolds number.
    The base mesh of an instance is the pressure mesh (fine side >> k squares),
    refined k times.
    """
    rng = np.random.default_rng(seed)
    sides = rng.choice(np.array([32, 64, 128, 256]), size=n)
    Re = rng.uniform(10.0, 400.0, size=n)
    k = rng.integers(1, 4, size=n)
    return [{"n_fine": int(s), "k": int(kk), "Re": float(r)} for s, kk, r in zip(sides, k, Re)]
