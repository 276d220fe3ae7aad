"""Host logic of the on-chip coarse solve: the plan that distributes the coarse system over a
thread-block cluster (which warp of which CTA owns which rows, where each matrix entry finds
its column's value, which values go to which halo) and the subdomain coarse space of its
preconditioner (E = Z^T A Z and its pseudo-inverse).  A small C++ driver, built with nvcc,
runs the library's planner on coarse Poisson systems of oracle mesh levels and checks every
invariant the kernel's gathers rely on, and E^+ against the pseudo-inverse identities.  No
GPU needed."""

import os
import shutil
import subprocess

import numpy as np
import pytest

from workloads import square_mesh, channel_cylinder_mesh, WORKLOADS
from oracle.mesh import build_hierarchy
from oracle import fem
from oracle.cgp import _symmetric_eliminate, PHI_ZERO

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
LIMIT = 232448 - 2048      # opt-in shared memory per CTA of the target GPU, less static use


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    if not os.path.exists(NVCC):
        pytest.skip("nvcc not available")
    out = str(tmp_path_factory.mktemp("plan") / "onchip_plan_check")
    subprocess.check_call([NVCC, "-O2", "-std=c++17", "-x", "cu", "-o", out,
                           os.path.join(ROOT, "tests", "onchip_plan_check.cu"),
                           os.path.join(ROOT, "paper_1812_00185_gb300", "csrc", "onchip_plan.cu")])
    return out


def coarse_system(lev):
    """The coarse Poisson matrix (stiffness with phi = 0 rows and columns eliminated) of a
    level, as SELL-32 in the library's layout: slice width = longest row, column-major,
    padding column = the slice's first row with value 0."""
    n = lev.rowptr.shape[0] - 1
    K = fem.static_operators(lev.xy, lev.tri)["K"]
    mask = (lev.tag & PHI_ZERO) != 0
    A = _symmetric_eliminate(K, mask).tocsr()
    S = (n + 31) // 32
    deg = np.diff(lev.rowptr)
    w = np.array([deg[32 * s:32 * s + 32].max() for s in range(S)])
    ptr = np.concatenate([[0], np.cumsum(32 * w)]).astype(np.int32)
    col = np.repeat((32 * np.arange(S)).astype(np.int32), 32 * w)
    val = np.zeros(ptr[-1])
    row = np.repeat(np.arange(n), deg)
    k = np.arange(len(row)) - lev.rowptr[row]
    e = ptr[row // 32] + 32 * k + row % 32
    col[e] = lev.col
    val[e] = np.asarray(A[row, lev.col]).ravel()   # pattern entries whose value is zero included
    return n, S, np.asarray(lev.rowptr, np.int32), ptr, col, val, (~mask).astype(np.uint8)


def run_check(driver, path, lev, ncl, spc, limit=LIMIT):
    n, S, rp, ptr, col, val, ins = coarse_system(lev)
    with open(path, "wb") as f:
        np.array([n, S], np.int64).tofile(f)
        rp.tofile(f)
        ptr.tofile(f)
        col.tofile(f)
        val.tofile(f)
        ins.tofile(f)
        np.ascontiguousarray(lev.xy, np.float64).tofile(f)
    return subprocess.run([driver, path, str(ncl), str(spc), str(limit)], capture_output=True, text=True)


@pytest.mark.parametrize("mesh,levels,lv,ncl,spc", [
    ("square", 2, 2, 16, 4),     # 33x33 structured level, pure Neumann (E singular)
    ("square", 2, 2, 16, 0),     # Jacobi alone
    ("channel", 1, 1, 16, 4),    # unstructured, with phi = 0 rows and a hole
    ("channel", 1, 1, 16, 8),
    ("channel", 1, 1, 8, 2),
    ("square", 1, 1, 8, 1),      # 17x17 level: fewer rows than a slice per warp
])
def test_plan_invariants(driver, tmp_path, mesh, levels, lv, ncl, spc):
    if mesh == "square":
        base = square_mesh(8)
    else:
        base = channel_cylinder_mesh(seed=4, h=0.03)
    lev = build_hierarchy(base.xy, base.tri, base.tag, levels)[lv]
    r = run_check(driver, str(tmp_path / "system.bin"), lev, ncl, spc)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr


def test_channel_coarse_system_fits_on_chip(driver, tmp_path):
    """The 32,489-row coarse system of the 1M-triangle channel (k = 2) fits one 16-CTA
    cluster with 4 and with 8 subdomains per CTA."""
    w = WORKLOADS["channel1m_k2"]
    base = w.base_mesh()
    lev = build_hierarchy(base.xy, base.tri, base.tag, w.n_levels - w.k)[w.n_levels - w.k]
    for spc in (4, 8):
        r = run_check(driver, str(tmp_path / "system.bin"), lev, 16, spc)
        assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
