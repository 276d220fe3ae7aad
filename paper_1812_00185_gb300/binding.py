"""Thin ctypes binding of ``include/cgp.h`` (argument marshalling only).

The functions below carry the C names and call straight into ``libcgp.so``; every
step of the method runs in the library's CUDA kernels.  PyTorch is used only for
device memory (the solver workspace) and for the current CUDA stream.  If the
library has not been built, :func:`load` raises: there is no fallback path.
"""

import ctypes
import os
from ctypes import POINTER, byref, c_double, c_int32, c_int64, c_size_t, c_uint8, c_void_p

import numpy as np

from . import build as _build

CGP_OK, CGP_EINVAL, CGP_ENOTCONV, CGP_EBREAKDOWN, CGP_ENONFINITE, CGP_ETIMEOUT, CGP_ECUDA, CGP_ENOMEM = \
    0, -1, -2, -3, -4, -5, -6, -7
CGP_VEL_DIR, CGP_PHI_ZERO = 1, 2
CGP_BC_CAVITY, CGP_BC_CHANNEL, CGP_BC_TG, CGP_BC_TG_PERIODIC, CGP_BC_USER = 0, 1, 2, 3, 4
CGP_BC_JOBELIN_OPEN, CGP_BC_JOBELIN_DISK = 5, 6
CGP_BATCH_AUTO, CGP_BATCH_WHOLE_STEP, CGP_BATCH_BRANCHES = 0, 1, 2
CGP_RESTRICT_INJECT, CGP_RESTRICT_PT = 0, 1
CGP_PRECOND_AUTO, CGP_PRECOND_JACOBI, CGP_PRECOND_COARSE = 0, 1, 2
CGP_FP64, CGP_MIXED = 0, 1
CGP_GUESS_ZERO, CGP_GUESS_PREV, CGP_GUESS_LEARNED, CGP_GUESS_PROJ = 0, 1, 2, 3
CGP_MASS_CONSISTENT, CGP_MASS_LUMPED = 0, 1
(CGP_COARSE_AUTO, CGP_COARSE_KERNELS, CGP_COARSE_CLUSTER, CGP_COARSE_PERSISTENT, CGP_COARSE_PERSISTENT_MEM,
 CGP_COARSE_ONCHIP) = 0, 1, 2, 3, 4, 5
CGP_HOST, CGP_DEVICE = 0, 1
(CGP_VEC_U, CGP_VEC_UPREV, CGP_VEC_P, CGP_VEC_UTILDE, CGP_VEC_RHS_C, CGP_VEC_PHI_C,
 CGP_VEC_PHI_F) = range(7)
(CGP_MAT_M, CGP_MAT_K, CGP_MAT_CX, CGP_MAT_CY, CGP_MAT_KC, CGP_MAT_CXC, CGP_MAT_CYC,
 CGP_MAT_A) = range(8)

_ERRNAMES = {0: "CGP_OK", -1: "CGP_EINVAL", -2: "CGP_ENOTCONV", -3: "CGP_EBREAKDOWN",
             -4: "CGP_ENONFINITE", -5: "CGP_ETIMEOUT", -6: "CGP_ECUDA", -7: "CGP_ENOMEM"}


class CgpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_ERRNAMES.get(code, "?"), code, msg))
        self.code = code


class MeshDesc(ctypes.Structure):
    _fields_ = [("n_vert", c_int32), ("n_tri", c_int32), ("xy", POINTER(c_double)),
                ("tri", POINTER(c_int32)), ("vert_tag", POINTER(c_uint8)), ("n_levels", c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("Re", c_double), ("dt", c_double), ("chi", c_int32), ("k", c_int32),
                ("tol_mom", c_double), ("tol_poisson", c_double), ("tol_mass", c_double),
                ("max_it_mom", c_int32), ("max_it_poisson", c_int32), ("max_it_mass", c_int32),
                ("precision", c_int32), ("guess", c_int32), ("mass_mode", c_int32), ("bc_kind", c_int32),
                ("bc_param", c_double * 4), ("use_graph", c_int32), ("tol_inner", c_double),
                ("coarse_mode", c_int32), ("cluster_size", c_int32),
                ("restrict_mode", c_int32), ("precond", c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("steps", c_int64), ("t", c_double), ("it_mom", c_int32), ("it_poisson", c_int32),
                ("it_corr", c_int32), ("it_mass", c_int32), ("sum_it_mom", c_int64),
                ("sum_it_poisson", c_int64), ("sum_it_corr", c_int64), ("sum_it_mass", c_int64),
                ("res_mom", c_double), ("res_poisson", c_double), ("status", c_int32), ("launches", c_int64),
                ("guess_used", c_int64), ("sum_outer_poisson", c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_SIGS = {
    "cgp_last_error": (ctypes.c_char_p, []),
    "cgp_mesh_create": (c_int32, [POINTER(MeshDesc), c_void_p, POINTER(c_void_p)]),
    "cgp_mesh_level_info": (c_int32, [c_void_p, c_int32, POINTER(c_int32), POINTER(c_int32), POINTER(c_int64)]),
    "cgp_mesh_get_level": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                     c_void_p]),
    "cgp_mesh_destroy": (None, [c_void_p]),
    "cgp_workspace_size": (c_int32, [c_void_p, POINTER(Params), POINTER(c_size_t)]),
    "cgp_assemble": (c_int32, [c_void_p, POINTER(Params), c_void_p, c_size_t, c_void_p, POINTER(c_void_p)]),
    "cgp_set_fields": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_double, c_int32, c_void_p]),
    "cgp_step": (c_int32, [c_void_p, c_int32, c_void_p]),
    "cgp_get_fields": (c_int32, [c_void_p, c_void_p, c_void_p, POINTER(c_double), POINTER(Stats), c_int32,
                                 c_void_p]),
    "cgp_get_vector": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p]),
    "cgp_set_vector": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p]),
    "cgp_get_matrix": (c_int32, [c_void_p, c_int32, c_void_p, c_int32, c_void_p]),
    "cgp_solver_info": (c_int32, [c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int64),
                                  POINTER(c_int64)]),
    "cgp_set_dirichlet": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p]),
    "cgp_set_forcing": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p]),
    "cgp_record_pairs": (c_int32, [c_void_p, c_int32, c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    "cgp_coarse_info": (c_int32, [c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32)]),
    "cgp_coarse_subdomains": (c_int32, [c_void_p, POINTER(c_int32)]),
    "cgp_set_wait_test": (c_int32, [c_void_p, c_int32]),
    "cgp_exact_fields": (c_int32, [c_void_p, c_double, c_void_p, c_void_p, c_int32, c_void_p]),
    "cgp_mlp_copy_state": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "cgp_poisson_solve": (c_int32, [c_void_p, c_void_p, c_void_p, POINTER(c_int32), c_int32, c_void_p]),
    "cgp_prolong": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p]),
    "cgp_profile_step": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "cgp_solver_destroy": (None, [c_void_p]),
    "cgp_mlp_param_count": (c_int32, []),
    "cgp_mlp_create": (c_int32, [c_void_p, c_int32, c_int32, POINTER(c_void_p)]),
    "cgp_mlp_set_params": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p]),
    "cgp_mlp_get_params": (c_int32, [c_void_p, c_void_p, c_int32, c_void_p]),
    "cgp_mlp_forward": (c_int32, [c_void_p, c_void_p, c_void_p, c_int32, c_void_p, c_void_p]),
    "cgp_mlp_grad": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, c_void_p, POINTER(ctypes.c_float),
                               c_void_p]),
    "cgp_mlp_train_step": (c_int32, [c_void_p, c_void_p, c_void_p, c_void_p, c_int32, ctypes.c_float,
                                     POINTER(ctypes.c_float), c_void_p]),
    "cgp_guess_set": (c_int32, [c_void_p, c_void_p, c_void_p]),
    "cgp_mlp_destroy": (None, [c_void_p]),
    "cgp_batch_create": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_void_p, POINTER(c_void_p)]),
    "cgp_batch_create_mode": (c_int32, [c_void_p, c_int32, c_int32, c_int32, c_int32, c_void_p, POINTER(c_void_p)]),
    "cgp_batch_mode": (c_int32, [c_void_p, POINTER(c_int32)]),
    "cgp_batch_step": (c_int32, [c_void_p, c_int32, c_void_p]),
    "cgp_batch_info": (c_int32, [c_void_p, POINTER(c_int32), POINTER(c_int32), POINTER(c_int32), c_void_p,
                                 c_int32]),
    "cgp_batch_destroy": (None, [c_void_p]),
    "cgp_pcg_sell_noalloc": (c_int32, [c_int32, c_int32, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p,
                                       c_double, c_int32, c_void_p, c_void_p]),
}

BATCH_CANDIDATES = [(c, t) for c in (1, 2, 4, 8) for t in (256, 512, 1024)]

PROF_NAMES = ["mom_prep", "mom_assemble", "mom_setup", "mom_init", "bicg_p", "bicg_v", "bicg_s", "bicg_t",
              "bicg_x", "coarse_rhs", "pois_setup", "pois_init", "pois_spmv", "pois_update", "phi_mean",
              "phi_sub", "prolong", "corr_rhs", "corr_setup", "corr_init", "corr_spmv", "corr_update", "div",
              "mass_setup", "mass_init", "mass_spmv", "mass_update", "finish", "pois_onelaunch", "mlp_forward",
              "ir_resid", "ir_update", "to_f32", "f32_init", "f32_bicg_p", "f32_bicg_v", "f32_bicg_s", "f32_bicg_t",
              "f32_bicg_x",
              "pois_pupd", "corr_pupd", "mass_pupd", "cheb_mass", "cheb_corr", "proj"]

_LIB = None


def load(build_if_missing=True):
    """Load libcgp.so (building it first if asked); raises if it cannot be had."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise RuntimeError("libcgp.so is not built (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIB = lib
    return lib


def exported_symbols():
    return list(_SIGS)


def _check(rc, allow=()):
    if rc != CGP_OK and rc not in allow:
        raise CgpError(rc, load().cgp_last_error().decode())
    return rc


def _ptr(a):
    """Device or host address of a torch tensor / numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return c_void_p(a.data_ptr())
    return a.ctypes.data_as(c_void_p)


def _stream(stream):
    if stream is None:
        import torch
        return c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return c_void_p(stream.cuda_stream)
    return c_void_p(stream)


# ---------------------------------------------------------------- C-named wrappers
def cgp_last_error():
    return load().cgp_last_error().decode()


def cgp_mesh_create(xy, tri, tag, n_levels, stream=None):
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    tag = np.ascontiguousarray(tag, dtype=np.uint8)
    d = MeshDesc(int(xy.shape[0]), int(tri.shape[0]), xy.ctypes.data_as(POINTER(c_double)),
                 tri.ctypes.data_as(POINTER(c_int32)), tag.ctypes.data_as(POINTER(c_uint8)), int(n_levels))
    out = c_void_p()
    _check(load().cgp_mesh_create(byref(d), _stream(stream), byref(out)))
    return out


def cgp_mesh_level_info(mesh, level):
    nv, nt, nnz = c_int32(), c_int32(), c_int64()
    _check(load().cgp_mesh_level_info(mesh, level, byref(nv), byref(nt), byref(nnz)))
    return nv.value, nt.value, nnz.value


def cgp_mesh_get_level(mesh, level):
    nv, nt, nnz = cgp_mesh_level_info(mesh, level)
    nv_prev = cgp_mesh_level_info(mesh, level - 1)[0] if level > 0 else nv
    xy = np.empty((nv, 2)); tri = np.empty((nt, 3), np.int32); tag = np.empty(nv, np.uint8)
    rp = np.empty(nv + 1, np.int32); col = np.empty(nnz, np.int32)
    par = np.empty((max(nv - nv_prev, 0), 2), np.int32)
    _check(load().cgp_mesh_get_level(mesh, level, _ptr(xy), _ptr(tri), _ptr(tag), _ptr(rp), _ptr(col),
                                     _ptr(par) if level > 0 else None))
    return {"xy": xy, "tri": tri, "tag": tag, "rowptr": rp, "col": col, "parents": par}


def cgp_mesh_destroy(mesh):
    load().cgp_mesh_destroy(mesh)


def make_params(Re, dt, chi=0, k=1, tol_mom=1e-10, tol_poisson=1e-10, tol_mass=1e-12, max_it_mom=500,
                max_it_poisson=20000, max_it_mass=500, precision=CGP_FP64, guess=CGP_GUESS_PREV,
                mass_mode=CGP_MASS_CONSISTENT, bc_kind=CGP_BC_CAVITY, bc_param=(1.0, 0.0, 0.0, 0.0),
                use_graph=1, tol_inner=0.0, coarse_mode=0, cluster_size=0, restrict_mode=0, precond=0):
    p = Params()
    p.Re, p.dt, p.chi, p.k = Re, dt, chi, k
    p.tol_mom, p.tol_poisson, p.tol_mass = tol_mom, tol_poisson, tol_mass
    p.max_it_mom, p.max_it_poisson, p.max_it_mass = max_it_mom, max_it_poisson, max_it_mass
    p.precision, p.guess, p.mass_mode, p.bc_kind = precision, guess, mass_mode, bc_kind
    for i in range(4):
        p.bc_param[i] = bc_param[i] if i < len(bc_param) else 0.0
    p.use_graph = use_graph
    p.tol_inner, p.coarse_mode, p.cluster_size = tol_inner, coarse_mode, cluster_size
    p.restrict_mode = restrict_mode
    p.precond = precond
    return p


def cgp_workspace_size(mesh, params):
    n = c_size_t()
    _check(load().cgp_workspace_size(mesh, byref(params), byref(n)))
    return n.value


def cgp_assemble(mesh, params, workspace, stream=None):
    out = c_void_p()
    nbytes = workspace.numel() * workspace.element_size()
    _check(load().cgp_assemble(mesh, byref(params), _ptr(workspace), nbytes, _stream(stream), byref(out)))
    return out


def cgp_set_fields(solver, U, Uprev, P, t, where=CGP_HOST, stream=None):
    if where == CGP_HOST:
        U = np.ascontiguousarray(U, dtype=np.float64)
        Uprev = None if Uprev is None else np.ascontiguousarray(Uprev, dtype=np.float64)
        P = np.ascontiguousarray(P, dtype=np.float64)
    _check(load().cgp_set_fields(solver, _ptr(U), _ptr(Uprev), _ptr(P), float(t), where, _stream(stream)))


def cgp_step(solver, n_steps, stream=None):
    _check(load().cgp_step(solver, int(n_steps), _stream(stream)))


def cgp_get_fields(solver, U=None, P=None, where=CGP_HOST, stream=None, allow=(CGP_ENOTCONV,)):
    """Returns (U, P, t, stats, status).  With where=CGP_HOST new numpy arrays are made."""
    nf = cgp_solver_info(solver)[0]
    if where == CGP_HOST:
        U = np.empty((nf, 2)) if U is None else U
        P = np.empty(nf) if P is None else P
    t = c_double()
    st = Stats()
    rc = load().cgp_get_fields(solver, _ptr(U), _ptr(P), byref(t), byref(st), where, _stream(stream))
    if rc == CGP_ECUDA or rc == CGP_EINVAL:
        _check(rc)
    _check(rc, allow=allow)
    return U, P, t.value, st.as_dict(), rc


def cgp_set_dirichlet(solver, uD, stream=None):
    uD = np.ascontiguousarray(uD, dtype=np.float64)
    _check(load().cgp_set_dirichlet(solver, _ptr(uD), CGP_HOST, _stream(stream)))


def cgp_set_forcing(solver, F, stream=None):
    F = np.ascontiguousarray(F, dtype=np.float64)
    _check(load().cgp_set_forcing(solver, _ptr(F), CGP_HOST, _stream(stream)))


def cgp_record_pairs(solver, n_steps, rhs, prev, target, where=None, stream=None):
    """Advance n_steps steps, storing (rhs, previous increment, increment) per step into the
    given arrays (n_steps x N_c; torch CUDA tensors, or numpy arrays for the host form)."""
    if where is None:
        where = CGP_DEVICE if hasattr(rhs, "is_cuda") and rhs.is_cuda else CGP_HOST
    _check(load().cgp_record_pairs(solver, int(n_steps), _ptr(rhs), _ptr(prev), _ptr(target), where,
                                   _stream(stream)))


def cgp_coarse_info(solver):
    """(kind, ctas, cluster) of the coarse Poisson solver that runs."""
    k, n, c = c_int32(), c_int32(), c_int32()
    _check(load().cgp_coarse_info(solver, byref(k), byref(n), byref(c)))
    return k.value, n.value, c.value


def cgp_exact_fields(solver, t, stream=None):
    """Closed-form (U (N_f, 2), P (N_f,)) of a manufactured problem kind at time t (host)."""
    nf = cgp_solver_info(solver)[0]
    U = np.empty((nf, 2))
    P = np.empty(nf)
    _check(load().cgp_exact_fields(solver, float(t), _ptr(U), _ptr(P), CGP_HOST, _stream(stream)))
    return U, P


def cgp_set_wait_test(solver, on):
    """Test hook: bounded device waits of the coarse solves wait for a signal nothing sends
    (short limit), so the next solve returns CGP_ETIMEOUT; on = 0 restores them."""
    _check(load().cgp_set_wait_test(solver, int(on)))


def cgp_coarse_subdomains(solver):
    """Subdomains of the coarse solve's coarse correction (0: Jacobi alone)."""
    m = c_int32()
    _check(load().cgp_coarse_subdomains(solver, byref(m)))
    return m.value


def cgp_solver_info(solver):
    nf, nc, zf, zc = c_int32(), c_int32(), c_int64(), c_int64()
    _check(load().cgp_solver_info(solver, byref(nf), byref(nc), byref(zf), byref(zc)))
    return nf.value, nc.value, zf.value, zc.value


def cgp_get_vector(solver, which, stream=None):
    nf, nc, _, _ = cgp_solver_info(solver)
    n = {CGP_VEC_U: 2 * nf, CGP_VEC_UPREV: 2 * nf, CGP_VEC_P: nf, CGP_VEC_UTILDE: 2 * nf,
         CGP_VEC_RHS_C: nc, CGP_VEC_PHI_C: nc, CGP_VEC_PHI_F: nf}[which]
    out = np.empty(n)
    _check(load().cgp_get_vector(solver, which, _ptr(out), CGP_HOST, _stream(stream)))
    return out.reshape(-1, 2) if n == 2 * nf and which in (CGP_VEC_U, CGP_VEC_UPREV, CGP_VEC_UTILDE) else out


def cgp_get_vector_device(solver, which, out, stream=None):
    """Device-to-device copy of a solver vector into a torch tensor (no synchronisation)."""
    _check(load().cgp_get_vector(solver, which, _ptr(out), CGP_DEVICE, _stream(stream)))


def cgp_set_vector(solver, which, data, stream=None):
    data = np.ascontiguousarray(data, dtype=np.float64)
    _check(load().cgp_set_vector(solver, which, _ptr(data), CGP_HOST, _stream(stream)))


def cgp_get_matrix(solver, which, stream=None):
    nf, nc, zf, zc = cgp_solver_info(solver)
    out = np.empty(zc if which in (CGP_MAT_KC, CGP_MAT_CXC, CGP_MAT_CYC) else zf)
    _check(load().cgp_get_matrix(solver, which, _ptr(out), CGP_HOST, _stream(stream)))
    return out


def cgp_poisson_solve(solver, rhs, phi0=None, stream=None, allow=(CGP_ENOTCONV,)):
    nc = cgp_solver_info(solver)[1]
    rhs = np.ascontiguousarray(rhs, dtype=np.float64)
    phi = np.zeros(nc) if phi0 is None else np.array(phi0, dtype=np.float64)
    it = c_int32()
    rc = load().cgp_poisson_solve(solver, _ptr(rhs), _ptr(phi), byref(it), CGP_HOST, _stream(stream))
    _check(rc, allow=allow)
    return phi, it.value, rc


def cgp_prolong(solver, phi_c, stream=None):
    nf, nc, _, _ = cgp_solver_info(solver)
    phi_c = np.ascontiguousarray(phi_c, dtype=np.float64)
    out = np.empty(nf)
    _check(load().cgp_prolong(solver, _ptr(phi_c), _ptr(out), CGP_HOST, _stream(stream)))
    return out


def cgp_profile_step(solver, stream=None):
    """Advance one step with per-launch event timing: {kernel: (launches, total ms)}."""
    n = len(PROF_NAMES)
    counts = np.zeros(n, np.int32)
    ms = np.zeros(n)
    _check(load().cgp_profile_step(solver, _stream(stream), n, _ptr(counts), _ptr(ms)))
    return {PROF_NAMES[i]: (int(counts[i]), float(ms[i])) for i in range(n) if counts[i]}


def cgp_solver_destroy(solver):
    load().cgp_solver_destroy(solver)


# ---------------------------------------------------------------- allocation-free solve
def cgp_pcg_sell_noalloc(n, nslices, sell_ptr, sell_col, val, dinv, b, x, tol, maxit, info, stream=None):
    """All array arguments are device tensors; see include/cgp.h.  Asynchronous."""
    _check(load().cgp_pcg_sell_noalloc(int(n), int(nslices), _ptr(sell_ptr), _ptr(sell_col), _ptr(val), _ptr(dinv),
                                       _ptr(b), _ptr(x), float(tol), int(maxit), _ptr(info), _stream(stream)))


# ---------------------------------------------------------------- batches
def cgp_batch_create(solvers, cluster_size=0, threads=0, stream=None, mode=None):
    """mode: None = the library's default (CGP_BATCH_AUTO), else CGP_BATCH_WHOLE_STEP or
    CGP_BATCH_BRANCHES."""
    arr = (c_void_p * len(solvers))(*[s.handle if hasattr(s, "handle") else s for s in solvers])
    out = c_void_p()
    if mode is None:
        _check(load().cgp_batch_create(arr, len(solvers), int(cluster_size), int(threads), _stream(stream),
                                       byref(out)))
    else:
        _check(load().cgp_batch_create_mode(arr, len(solvers), int(cluster_size), int(threads), int(mode),
                                            _stream(stream), byref(out)))
    return out


def cgp_batch_mode(batch):
    m = c_int32()
    _check(load().cgp_batch_mode(batch, byref(m)))
    return m.value


def cgp_batch_step(batch, n_steps, stream=None):
    _check(load().cgp_batch_step(batch, int(n_steps), _stream(stream)))


def cgp_batch_info(batch):
    cs, th, ncl = c_int32(), c_int32(), c_int32()
    trials = np.zeros(len(BATCH_CANDIDATES), np.float32)
    _check(load().cgp_batch_info(batch, byref(cs), byref(th), byref(ncl), _ptr(trials), len(BATCH_CANDIDATES)))
    return {"cluster_size": cs.value, "threads": th.value, "clusters": ncl.value,
            "trials_ms": {"%dx%d" % ct: round(float(v), 4) for ct, v in zip(BATCH_CANDIDATES, trials) if v >= 0}}


def cgp_batch_destroy(batch):
    load().cgp_batch_destroy(batch)


# ---------------------------------------------------------------- learned guess
def cgp_mlp_param_count():
    return int(load().cgp_mlp_param_count())


def cgp_mlp_create(mesh, level, max_batch):
    out = c_void_p()
    _check(load().cgp_mlp_create(mesh, int(level), int(max_batch), byref(out)))
    return out


def cgp_mlp_set_params(m, params, stream=None):
    params = np.ascontiguousarray(params, dtype=np.float32)
    assert params.size == cgp_mlp_param_count()
    _check(load().cgp_mlp_set_params(m, _ptr(params), CGP_HOST, _stream(stream)))


def cgp_mlp_get_params(m, stream=None):
    out = np.empty(cgp_mlp_param_count(), np.float32)
    _check(load().cgp_mlp_get_params(m, _ptr(out), CGP_HOST, _stream(stream)))
    return out


def cgp_mlp_forward(m, r, q, batch, pred, stream=None):
    """r, q, pred: device tensors of batch * N doubles."""
    _check(load().cgp_mlp_forward(m, _ptr(r), _ptr(q), int(batch), _ptr(pred), _stream(stream)))


def cgp_mlp_grad(m, r, q, target, batch, stream=None):
    g = np.empty(cgp_mlp_param_count(), np.float32)
    loss = ctypes.c_float()
    _check(load().cgp_mlp_grad(m, _ptr(r), _ptr(q), _ptr(target), int(batch), _ptr(g), byref(loss),
                               _stream(stream)))
    return float(loss.value), g


def cgp_mlp_train_step(m, r, q, target, batch, lr, want_loss=True, stream=None):
    loss = ctypes.c_float()
    _check(load().cgp_mlp_train_step(m, _ptr(r), _ptr(q), _ptr(target), int(batch), float(lr),
                                     byref(loss) if want_loss else None, _stream(stream)))
    return float(loss.value) if want_loss else None


def cgp_guess_set(solver, m, stream=None):
    _check(load().cgp_guess_set(solver, m, _stream(stream)))


def cgp_mlp_copy_state(dst, src, stream=None):
    """Weights and Adam state of src into dst (device to device, asynchronous)."""
    _check(load().cgp_mlp_copy_state(dst, src, _stream(stream)))


def cgp_mlp_destroy(m):
    load().cgp_mlp_destroy(m)


# ---------------------------------------------------------------- convenience objects
class Mesh:
    """Owns a cgp_mesh built from a base mesh (xy, tri, tag) with n_levels refinements."""

    def __init__(self, xy, tri, tag, n_levels, stream=None):
        self.handle = cgp_mesh_create(xy, tri, tag, n_levels, stream)
        self.n_levels = n_levels

    def level(self, l):
        return cgp_mesh_get_level(self.handle, l)

    def info(self, l):
        return cgp_mesh_level_info(self.handle, l)

    def close(self):
        if self.handle:
            cgp_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Owns a cgp_solver and its torch-allocated device workspace."""

    def __init__(self, mesh, params, stream=None):
        import torch
        self.mesh = mesh
        self.params = params
        nbytes = cgp_workspace_size(mesh.handle, params)
        self.workspace = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        self.handle = cgp_assemble(mesh.handle, params, self.workspace, stream)
        self.nf, self.nc, self.nnzf, self.nnzc = cgp_solver_info(self.handle)

    def step(self, n=1, stream=None):
        cgp_step(self.handle, n, stream)

    def fields(self, stream=None):
        return cgp_get_fields(self.handle, stream=stream)

    def vector(self, which):
        return cgp_get_vector(self.handle, which)

    def coarse_info(self):
        return cgp_coarse_info(self.handle)

    def coarse_subdomains(self):
        return cgp_coarse_subdomains(self.handle)

    def matrix(self, which):
        return cgp_get_matrix(self.handle, which)

    def set_fields(self, U, Uprev, P, t):
        cgp_set_fields(self.handle, U, Uprev, P, t)

    def set_vector(self, which, data):
        cgp_set_vector(self.handle, which, data)

    def close(self):
        if self.handle:
            cgp_solver_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
