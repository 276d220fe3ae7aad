"""The allocation-free solve entry point (cgp_pcg_sell_noalloc) through the C ABI, against
the solver's own coarse Poisson solve (cgp_poisson_solve) and the oracle's direct solve.

Callers that cannot allocate device memory hand this entry point only the operator, the
right-hand side and the output buffers; its scratch is a fixed array inside the library.
The test builds the coarse operator of Eq. 23 (with its phi = 0 rows eliminated) in the
SELL-32 layout on the host, calls the entry point twice in a row on the same scratch (two
right-hand sides), and compares each result with the existing entry point's and with the
oracle's; then a warm start (fewer iterations, the same solution) and an iteration cap
(CGP_ENOTCONV with a finite iterate).  This file is collected last, so a run that stops at
the first failure has run every other test first.
"""

import numpy as np
import pytest

from workloads import channel_cylinder_mesh
from oracle.cgp import CGPOracle
from oracle import flows

pytestmark = pytest.mark.gpu


def _sell(rowptr, col, val):
    n = rowptr.size - 1
    ns = (n + 31) // 32
    ptr = np.zeros(ns + 1, np.int32)
    widths = []
    for s in range(ns):
        w = max(rowptr[r + 1] - rowptr[r] for r in range(32 * s, min(32 * s + 32, n)))
        widths.append(w)
        ptr[s + 1] = ptr[s] + 32 * w
    scol = np.zeros(ptr[-1], np.int32)
    sval = np.zeros(ptr[-1])
    for s in range(ns):
        for lane in range(32):
            r = 32 * s + lane
            ln = rowptr[r + 1] - rowptr[r] if r < n else 0
            for k in range(widths[s]):
                e = ptr[s] + 32 * k + lane
                if k < ln:
                    scol[e] = col[rowptr[r] + k]
                    sval[e] = val[rowptr[r] + k]
                else:
                    scol[e] = 32 * s
    return ns, ptr, scol, sval


def test_noalloc_solve_matches_poisson_entry_point(lib):
    import torch
    from paper_1812_00185_gb300 import binding as cg
    base = channel_cylinder_mesh(seed=9, h=0.05)
    mesh = cg.Mesh(base.xy, base.tri, base.tag, 2)
    s = cg.Solver(mesh, cg.make_params(20.0, 0.01, k=1, bc_kind=cg.CGP_BC_CHANNEL, bc_param=(0.3, 0.41),
                                       guess=cg.CGP_GUESS_ZERO, tol_poisson=1e-11, max_it_poisson=20000))
    lev = mesh.level(1)
    rp, col, tag = lev["rowptr"].astype(np.int64), lev["col"], lev["tag"]
    n = rp.size - 1
    K = s.matrix(cg.CGP_MAT_KC)
    # phi = 0 rows and columns replaced by the identity, as the solver does for Eq. 23
    z = (tag & cg.CGP_PHI_ZERO) != 0
    rows = np.repeat(np.arange(n), np.diff(rp))
    K0 = np.where(z[rows] | z[col], (rows == col).astype(float), K)
    dinv = 1.0 / K0[rows == col]
    ns, sptr, scol, sval = _sell(rp, col, K0)
    dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), device="cuda")
    d_ptr, d_col, d_val, d_dinv = dev(sptr), dev(scol), dev(sval), dev(dinv)
    info = torch.zeros(2, dtype=torch.int32, device="cuda")
    o = CGPOracle(base, 2, 1, 20.0, 0.01, 0, flows.BC_CHANNEL, bc_param=(0.3, 0.41, 0, 0))
    rng = np.random.default_rng(3)
    b = None
    for call in range(2):                      # two calls in a row share the scratch array
        b = rng.standard_normal(n)
        b[z] = 0.0
        ref, it_ref, rc = cg.cgp_poisson_solve(s.handle, b)
        assert rc == 0
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        cg.cgp_pcg_sell_noalloc(n, ns, d_ptr, d_col, d_val, d_dinv, dev(b), x, 1e-11, 20000, info)
        torch.cuda.synchronize()
        it, status = info.cpu().tolist()
        got = x.cpu().numpy()
        assert status == 0 and 0 < it < 20000, (call, it, status)
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-8, call
        exact = o.poisson(b)
        assert np.linalg.norm(got - exact) / np.linalg.norm(exact) < 1e-8, call
    # warm start: x on entry is the initial guess (the solution slightly perturbed)
    x0 = exact + 1e-6 * np.linalg.norm(exact) / np.sqrt(n) * rng.standard_normal(n)
    x0[z] = 0.0
    x = dev(x0)
    cg.cgp_pcg_sell_noalloc(n, ns, d_ptr, d_col, d_val, d_dinv, dev(b), x, 1e-11, 20000, info)
    torch.cuda.synchronize()
    it_warm, status = info.cpu().tolist()
    assert status == 0 and it_warm < it, (it_warm, it)
    assert np.linalg.norm(x.cpu().numpy() - exact) / np.linalg.norm(exact) < 1e-8
    # iteration cap: the solve stops with CGP_ENOTCONV and a finite iterate
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    cg.cgp_pcg_sell_noalloc(n, ns, d_ptr, d_col, d_val, d_dinv, dev(b), x, 1e-11, 5, info)
    torch.cuda.synchronize()
    it_cap, status = info.cpu().tolist()
    assert status == cg.CGP_ENOTCONV and it_cap <= 5 and torch.isfinite(x).all()
    s.close()
    mesh.close()


def test_noalloc_rejects_sizes_beyond_its_scratch(lib):
    import torch
    from paper_1812_00185_gb300 import binding as cg
    n = 65537
    t = torch.zeros(8, device="cuda")
    with pytest.raises(cg.CgpError) as e:
        cg.cgp_pcg_sell_noalloc(n, (n + 31) // 32, t, t, t, t, t, t, 1e-8, 10, t)
    assert e.value.code == cg.CGP_EINVAL
