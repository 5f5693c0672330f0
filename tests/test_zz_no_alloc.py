"""The allocation-free deflation projection (dtr_deflate_project_static).

It exists for callers that cannot let the library allocate device memory or
pass it a workspace, such as applications whose device memory is entirely
owned by their own pool allocator.  Its scratch is a fixed device array inside
the library, so this test checks, through the C ABI, that two calls in a row
(the second sees the first call's leftovers in that array) give the same
results as the workspace-based dtr_deflate_project, and that sizes above the
array's limits are refused.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1603_05988_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-12)])
def test_static_scratch_projection_matches_workspace_entry_point(prec, tol):
    import torch
    assert torch.cuda.is_available()
    from paper_1603_05988_gb300 import dtr
    dims = (4, 4, 4, 8)
    lat = dtr.make_lattice(dims)
    V = synth.random_orthonormal(lat.N, 100, 3)
    lam = np.linspace(0.8, 1.9, 100) * np.where(np.arange(100) % 3 == 0, -1.0, 1.0)
    D = dtr.defl_create(lat, V, lam, prec=prec)
    for call, nrhs in enumerate((16, 5)):
        z = dtr.gen_noise(lat, 77, call, 16, False, 0, nrhs)
        d_ref, C_ref, _ = dtr.deflate_project(D, z, want_coeff=True)
        d_st, C_st = dtr.deflate_project_static(D, z, want_coeff=True)
        torch.cuda.synchronize()
        d_ref, d_st = d_ref.cpu().numpy(), d_st.cpu().numpy()
        assert np.abs(d_st - d_ref).max() <= tol * np.abs(d_ref).max()
        C_ref, C_st = C_ref.cpu().numpy(), C_st.cpu().numpy()
        assert np.abs(C_st - C_ref).max() <= tol * np.abs(C_ref).max()


def test_static_scratch_projection_rejects_oversize():
    from paper_1603_05988_gb300 import dtr
    lat = dtr.make_lattice((4, 4, 4, 4))
    z = dtr.gen_noise(lat, 1, 0, 1, False, 0, 17)
    D = dtr.defl_create(lat, synth.random_orthonormal(lat.N, 8, 1), np.linspace(1.0, 2.0, 8))
    with pytest.raises(dtr.DtrError):
        dtr.deflate_project_static(D, z)                     # nrhs 17 > 16
    Dbig = dtr.defl_create(lat, synth.random_orthonormal(lat.N, 129, 2), np.linspace(1.0, 2.0, 129))
    with pytest.raises(dtr.DtrError):
        dtr.deflate_project_static(Dbig, z[:4].contiguous())  # k 129 > 128
