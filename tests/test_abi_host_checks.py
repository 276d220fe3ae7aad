"""Argument checks of the C ABI that return before any CUDA call, so they run without a GPU:
malformed mesh descriptors, NULL handles and out-of-range levels give CGP_EINVAL and a
message in cgp_last_error, and leave the output handle NULL."""

import ctypes

import numpy as np
import pytest

from paper_1812_00185_gb300 import binding as cg


def _desc(nv=3, nt=1, n_levels=1, null=None):
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]] * max(1, nv), np.float64)[:max(nv, 1)]
    tri = np.zeros((max(nt, 1), 3), np.int32)
    tri[0] = (0, 1, 2)
    tag = np.zeros(max(nv, 1), np.uint8)
    keep = (xy, tri, tag)
    d = cg.MeshDesc(nv, nt,
                    None if null == "xy" else xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                    None if null == "tri" else tri.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                    None if null == "tag" else tag.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                    n_levels)
    return d, keep


@pytest.mark.parametrize("case", ["two_vertices", "no_triangles", "levels_negative", "levels_above_4",
                                  "null_xy", "null_tri", "null_tag", "index_range"])
def test_mesh_descriptor_rejected(case):
    kw = {"two_vertices": dict(nv=2), "no_triangles": dict(nt=0), "levels_negative": dict(n_levels=-1),
          "levels_above_4": dict(n_levels=5), "null_xy": dict(null="xy"), "null_tri": dict(null="tri"),
          "null_tag": dict(null="tag")}.get(case, {})
    if case == "index_range":
        # 2^27 base triangles refined 4 times: more than 2^31 / 3 triangles on the finest level
        d, keep = _desc(nt=1, n_levels=4)
        d.n_tri = 1 << 27
    else:
        d, keep = _desc(**kw)
    lib = cg.load()
    out = ctypes.c_void_p(12345)
    rc = lib.cgp_mesh_create(ctypes.byref(d), ctypes.c_void_p(0), ctypes.byref(out))
    assert rc == cg.CGP_EINVAL
    assert out.value is None
    msg = cg.cgp_last_error()
    assert msg.startswith("cgp_mesh_create:"), msg


def test_null_arguments_rejected():
    lib = cg.load()
    d, keep = _desc()
    assert lib.cgp_mesh_create(ctypes.byref(d), ctypes.c_void_p(0), None) == cg.CGP_EINVAL
    assert lib.cgp_mesh_create(None, ctypes.c_void_p(0), ctypes.byref(ctypes.c_void_p())) == cg.CGP_EINVAL
    nv, nt, nnz = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    assert lib.cgp_mesh_level_info(None, 0, ctypes.byref(nv), ctypes.byref(nt), ctypes.byref(nnz)) == cg.CGP_EINVAL
    assert "bad mesh or level" in cg.cgp_last_error()
    p = cg.make_params(100.0, 0.01)
    n = ctypes.c_size_t()
    assert lib.cgp_workspace_size(None, ctypes.byref(p), ctypes.byref(n)) == cg.CGP_EINVAL
    assert "null mesh or params" in cg.cgp_last_error()
    out = ctypes.c_void_p(12345)
    assert lib.cgp_assemble(None, ctypes.byref(p), None, 0, ctypes.c_void_p(0), ctypes.byref(out)) == cg.CGP_EINVAL
    assert out.value is None


def test_error_string_is_cleared_by_the_next_call():
    lib = cg.load()
    d, keep = _desc(nv=2)
    assert lib.cgp_mesh_create(ctypes.byref(d), ctypes.c_void_p(0), ctypes.byref(ctypes.c_void_p())) == cg.CGP_EINVAL
    assert cg.cgp_last_error() != ""
    d, keep = _desc(n_levels=9)
    assert lib.cgp_mesh_create(ctypes.byref(d), ctypes.c_void_p(0), ctypes.byref(ctypes.c_void_p())) == cg.CGP_EINVAL
    assert "invalid descriptor" in cg.cgp_last_error()
