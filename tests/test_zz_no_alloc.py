"""The allocation-free deflation projection (dtr_deflate_project_static).

It exists for callers that cannot let the library allocate device memory or
pass it a workspace, such as applications whose device memory is entirely
owned by their own pool allocator.  Its scratch is a fixed device array inside
the library, so this test checks, through the C ABI, that two calls in a row
(the second sees the first call's leftovers in that array) give the same
results as the workspace-based dtr_deflate_project and as the oracle's
deflation term on the stored (rounded) V, that a call leaves the device's free
memory unchanged, and that sizes above the array's limits and a
Galerkin-corrected space are refused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from paper_1603_05988_gb300 import synth

pytestmark = pytest.mark.gpu


def _setup(prec, k=100, dims=(4, 4, 4, 8)):
    from paper_1603_05988_gb300 import dtr
    lat = dtr.make_lattice(dims)
    V = synth.random_orthonormal(lat.N, k, 3)
    lam = np.linspace(0.8, 1.9, k) * np.where(np.arange(k) % 3 == 0, -1.0, 1.0)
    return lat, V, lam, dtr.defl_create(lat, V, lam, prec=prec)


# Both entry points accumulate in FP64 from the same stored V (BF16 and FP32
# values widen exactly), so they agree to FP64 rounding; the oracle evaluates
# z^H V diag(1/lambda) V^H g5 z on the same rounded V in FP64.
@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-12), ("bf16", 1e-12)])
def test_static_scratch_projection_matches_workspace_entry_point(prec, tol):
    import torch
    assert torch.cuda.is_available()
    from oracle import deflation, wilson
    from paper_1603_05988_gb300 import dtr
    lat, V, lam, D = _setup(prec)
    Vs = {"f64": V, "f32": V.astype(np.complex64).astype(np.complex128),
          "bf16": deflation.bf16_round(V)}[prec]
    for call, nrhs in enumerate((16, 5)):
        z = dtr.gen_noise(lat, 77, call, 16, False, 0, nrhs)
        d_ref, C_ref, _ = dtr.deflate_project(D, z, want_coeff=True)
        d_st, C_st = dtr.deflate_project_static(D, z, want_coeff=True)
        torch.cuda.synchronize()
        d_ref, d_st = d_ref.cpu().numpy(), d_st.cpu().numpy()
        assert np.abs(d_st - d_ref).max() <= tol * np.abs(d_ref).max()
        C_ref, C_st = C_ref.cpu().numpy(), C_st.cpu().numpy()
        assert np.abs(C_st - C_ref).max() <= tol * np.abs(C_ref).max()
        Zh = z.cpu().numpy().T
        d_or = deflation.quadrature_gamma5(Vs, lam, Zh)
        assert np.abs(d_st - d_or).max() <= 1e-12 * np.abs(d_or).max()
        # C = V^H [Z, g5 Z] of the oracle, column by column
        C_or = np.concatenate([Vs.conj().T @ Zh, Vs.conj().T @ wilson.gamma5_vec(Zh)], axis=1).T
        assert np.abs(C_st - C_or).max() <= 1e-12 * np.abs(C_or).max()


def test_static_scratch_projection_allocates_nothing():
    """A warmed-up call through the raw C entry point, with caller-allocated
    outputs, leaves the device's free memory exactly as it was."""
    import torch
    from paper_1603_05988_gb300 import dtr
    lat, V, lam, D = _setup("bf16", k=64)
    z = dtr.gen_noise(lat, 5, 0, 16, False, 0, 16)
    d = torch.empty(16, dtype=torch.complex128, device="cuda")
    C = torch.empty((32, 64), dtype=torch.complex128, device="cuda")
    lib = dtr._lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def call():
        rc = lib.dtr_deflate_project_static(D._h, ctypes.c_void_p(z.data_ptr()), 16, ctypes.c_void_p(d.data_ptr()),
                                            ctypes.c_void_p(C.data_ptr()), stream)
        assert rc == 0, lib.dtr_last_error().decode()

    call()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(3):
        call()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_static_scratch_projection_rejects_oversize_and_galerkin():
    from paper_1603_05988_gb300 import dtr
    lat = dtr.make_lattice((4, 4, 4, 4))
    z = dtr.gen_noise(lat, 1, 0, 1, False, 0, 17)
    D = dtr.defl_create(lat, synth.random_orthonormal(lat.N, 8, 1), np.linspace(1.0, 2.0, 8))
    with pytest.raises(dtr.DtrError):
        dtr.deflate_project_static(D, z)                     # nrhs 17 > 16
    Dbig = dtr.defl_create(lat, synth.random_orthonormal(lat.N, 129, 2), np.linspace(1.0, 2.0, 129))
    with pytest.raises(dtr.DtrError):
        dtr.deflate_project_static(Dbig, z[:4].contiguous())  # k 129 > 128
    # a Galerkin-corrected space is refused (only the eigenvalue form is supported)
    U = synth.random_su3_links((4, 4, 4, 4), 0.5, 1000)
    g = dtr.gauge_from_host(lat, U)
    D.gram(g, -0.4)
    with pytest.raises(dtr.DtrError):
        dtr.deflate_project_static(D, z[:4].contiguous())
