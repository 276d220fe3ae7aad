"""Host-side checks of cgp_workspace_size / cgp_assemble on a real mesh: every out-of-range
field of cgp_params gives CGP_EINVAL, a workspace that is too small or not 256-byte
aligned gives CGP_ENOMEM, and none of them leaves state behind (a valid solver assembled
afterwards steps normally).  No kernel runs on the rejected inputs."""

import numpy as np
import pytest

from workloads import square_mesh

pytestmark = pytest.mark.gpu

BAD = [("Re", 0.0), ("Re", float("nan")), ("dt", -1.0), ("chi", 2), ("k", -1), ("k", 3),
       ("tol_mom", 0.0), ("tol_poisson", 0.0), ("tol_mass", 0.0), ("max_it_mom", 0),
       ("max_it_poisson", 0), ("max_it_mass", 0), ("bc_kind", 99), ("restrict_mode", 2),
       ("precond", 3), ("precision", 7), ("guess", 4), ("mass_mode", 9), ("coarse_mode", 99),
       ("cluster_size", 17), ("tol_inner", 1.0)]


@pytest.fixture(scope="module")
def mesh(lib):
    from paper_1812_00185_gb300 import binding as cg
    base = square_mesh(4)
    m = cg.Mesh(base.xy, base.tri, base.tag, 2)
    yield m
    m.close()


@pytest.mark.parametrize("field,value", BAD)
def test_out_of_range_params(mesh, field, value):
    from paper_1812_00185_gb300 import binding as cg
    p = cg.make_params(100.0, 0.01, k=1)
    setattr(p, field, value)
    with pytest.raises(cg.CgpError) as e:
        cg.cgp_workspace_size(mesh.handle, p)
    assert e.value.code == cg.CGP_EINVAL
    assert "invalid cgp_params" in str(e.value)


def test_workspace_size_and_alignment(mesh):
    import torch
    from paper_1812_00185_gb300 import binding as cg
    p = cg.make_params(100.0, 0.01, k=1)
    need = cg.cgp_workspace_size(mesh.handle, p)
    assert need > 0
    small = torch.empty(need - 256, dtype=torch.uint8, device="cuda")
    with pytest.raises(cg.CgpError) as e:
        cg.cgp_assemble(mesh.handle, p, small)
    assert e.value.code == cg.CGP_ENOMEM
    buf = torch.empty(need + 512, dtype=torch.uint8, device="cuda")
    base = (-buf.data_ptr()) % 256            # first 256-byte boundary inside buf
    shifted = buf[base + 8:base + 8 + need]   # 8 bytes past it
    with pytest.raises(cg.CgpError) as e:
        cg.cgp_assemble(mesh.handle, p, shifted)
    assert e.value.code == cg.CGP_ENOMEM
    # nothing left behind: a valid solver on the same mesh assembles and steps
    s = cg.Solver(mesh, p)
    s.step(2)
    U, P, t, stats, rc = s.fields()
    assert rc == cg.CGP_OK and t == pytest.approx(0.02)
    assert np.isfinite(U).all() and np.isfinite(P).all() and np.abs(U).max() > 0
    s.close()
