"""Solver parameter sets of the named forms, and training of the learned guess on a workload.

A *form* is one way of running the same CGP step: ``fp64`` (every solve in FP64),
``mixed`` (FP32-inner / FP64-outer refinement, previous increment as the coarse guess),
``mixed_zero`` (the same from a zero guess), ``mixed_jacobi`` (Jacobi alone in the on-chip
coarse solve), ``mixed_proj`` / ``fp64_proj`` (the coarse guess projected onto the last
increments), ``mixed_learned`` / ``learned`` (that projection refined by the learned
network, mixed or FP64).
The benchmark and the full-size parity tests build their solvers here, so both run the
same configuration.  Argument marshalling only: nothing here computes the method.
"""

import time

from . import binding as cg

FORMS = ("fp64", "mixed", "learned", "mixed_learned", "mixed_zero", "mixed_jacobi", "mixed_proj", "fp64_proj")


def workload_params(w, form, use_graph=1, tol_inner=0.0, mass_mode=0, chi=None, tol=None):
    """cgp_params of workload ``w`` (workloads.Workload) in ``form``; ``tol`` = (momentum,
    Poisson, mass) tolerances in place of the workload's."""
    if form not in FORMS:
        raise ValueError(form)
    mixed = form.startswith("mixed")
    if form in ("learned", "mixed_learned"):
        guess = cg.CGP_GUESS_LEARNED
    elif form.endswith("_proj"):
        guess = cg.CGP_GUESS_PROJ
    elif form == "mixed_zero":
        guess = cg.CGP_GUESS_ZERO
    else:
        guess = cg.CGP_GUESS_PREV
    tm, tp, tms = (w.tol_mom, w.tol_poisson, 1e-10) if tol is None else tol
    return cg.make_params(w.Re, w.dt, chi=w.chi if chi is None else chi, k=w.k, tol_mom=tm,
                          tol_poisson=tp, tol_mass=tms, max_it_mom=1000, max_it_poisson=50000,
                          max_it_mass=1000, precision=cg.CGP_MIXED if mixed else cg.CGP_FP64,
                          guess=guess, bc_kind=w.bc, bc_param=w.bc_param, use_graph=use_graph,
                          tol_inner=tol_inner,
                          precond=cg.CGP_PRECOND_JACOBI if form == "mixed_jacobi" else cg.CGP_PRECOND_AUTO,
                          mass_mode=mass_mode)


def train_guess(w, pairs=150, iters=400, seed_offset=1, lr=2e-3, batch=8):
    """Train the learned-guess network on (rhs, projection guess, increment) triples that the
    library's solver (mixed form, projection guess) records on another seed of the same
    workload (the timed runs use seed ``w.base_n``).  Returns (FP32 parameter vector, info
    dict)."""
    import torch
    from .learned import PairStore, train, init_params
    from workloads import channel_cylinder_mesh
    t0 = time.time()
    if w.base == "channel":
        base = channel_cylinder_mesh(seed=w.base_n + seed_offset, h=w.extra.get("h", 0.0084))
    else:
        base = w.base_mesh()
    mesh = cg.Mesh(base.xy, base.tri, base.tag, w.n_levels)
    rec = cg.Solver(mesh, workload_params(w, "mixed_proj"))
    store = PairStore(rec.nc, pairs)
    store.record(rec, pairs)
    rec.close()
    torch.cuda.synchronize()
    t_rec = time.time() - t0
    net = cg.cgp_mlp_create(mesh.handle, w.n_levels - w.k, batch)
    cg.cgp_mlp_set_params(net, init_params(0))
    t1 = time.time()
    hist = train(net, store, iters, batch=batch, lr=lr, log_every=max(1, iters // 4))
    torch.cuda.synchronize()
    t_train = time.time() - t1
    p = cg.cgp_mlp_get_params(net)
    cg.cgp_mlp_destroy(net)
    del store
    mesh.close()
    return p, {"pairs": pairs, "iters": iters, "record_s": round(t_rec, 2), "train_s": round(t_train, 2),
               "loss": [(int(i), round(float(l), 5)) for i, l in hist],
               "train_mesh_seed": w.base_n + seed_offset if w.base == "channel" else w.base_n}
