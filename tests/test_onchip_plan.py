"""Host logic of the on-chip coarse solve: the plan that distributes the coarse system over a
thread-block cluster (which CTA owns which SELL-32 slices, where each matrix entry finds its
column's value, which values go to which halo).  A small C++ driver, built with nvcc, runs
the library's planner on SELL-32 patterns of oracle mesh levels and checks every invariant
the kernel's gathers rely on.  No GPU needed."""

import os
import shutil
import subprocess
import tempfile

import numpy as np
import pytest

from workloads import square_mesh, channel_cylinder_mesh
from oracle.mesh import build_hierarchy

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


def sell_pattern(lev):
    """SELL-32 of a level's CSR: slice width = longest row, column-major, padding column =
    the slice's first row (the library's layout)."""
    n = lev.rowptr.shape[0] - 1
    S = (n + 31) // 32
    deg = np.diff(lev.rowptr)
    w = np.array([deg[32 * s:32 * s + 32].max() for s in range(S)])
    ptr = np.concatenate([[0], np.cumsum(32 * w)]).astype(np.int32)
    col = np.zeros(ptr[-1], np.int32)
    for s in range(S):
        for l in range(32):
            i = 32 * s + l
            for k in range(w[s]):
                e = ptr[s] + 32 * k + l
                col[e] = lev.col[lev.rowptr[i] + k] if i < n and k < deg[i] else 32 * s
    return n, S, ptr, col


@pytest.mark.parametrize("mesh,levels,lv,ncl", [
    ("square", 2, 2, 16),        # 33x33 structured level
    ("channel", 1, 1, 16),       # unstructured, with phi = 0 rows and a hole
    ("channel", 1, 1, 8),
    ("square", 1, 1, 8),         # 17x17 level: one or two slices per CTA
])
def test_plan_invariants(driver, tmp_path, mesh, levels, lv, ncl):
    if mesh == "square":
        base = square_mesh(8)
    else:
        base = channel_cylinder_mesh(seed=4, h=0.03)
    lev = build_hierarchy(base.xy, base.tri, base.tag, levels)[lv]
    n, S, ptr, col = sell_pattern(lev)
    if S < ncl:
        pytest.skip("fewer slices than CTAs")
    path = str(tmp_path / "pattern.bin")
    with open(path, "wb") as f:
        np.array([n, S], np.int64).tofile(f)
        ptr.tofile(f)
        col.tofile(f)
        np.ascontiguousarray(lev.xy, np.float64).tofile(f)
    r = subprocess.run([driver, path, str(ncl), str(LIMIT)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.startswith("OK"), r.stdout + r.stderr
