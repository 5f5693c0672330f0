"""Estimator calls that cover part of a run, the per-run reuse of the
hierarchical-probing projection sums, its compensated FP32 accumulation for
FP32/BF16 deflation spaces, and the concurrent lanes of the 8^4 benchmark shape.
"""
import numpy as np
import pytest

from oracle import deflation, noise
from paper_1603_05988_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dtr():
    from paper_1603_05988_gb300 import dtr as d
    return d


@pytest.fixture(scope="module")
def c8(dtr):
    w = synth.WORKLOADS["wilson8x8x8x8_hp16x256_k100"]
    lat = dtr.make_lattice(w.dims)
    g = dtr.gauge_from_host(lat, synth.random_su3_links(w.dims, w.eps, w.gauge_seed))
    return dict(w=w, lat=lat, g=g)


@pytest.mark.parametrize("prec", ["f64", "bf16"])
def test_run_split_over_calls_equals_one_call(dtr, c8, prec):
    """A 16-vector run in blocks of 4 (W computed once, reused by the next
    three blocks) equals the same run split over four calls of four vectors
    (vec_first = 0, 4, 8, 12): identical samples."""
    w, lat, g = c8["w"], c8["lat"], c8["g"]
    V = synth.disjoint_orthonormal(lat.N, 40, 6)
    lam = np.linspace(0.9, 1.6, 40) * np.where(np.arange(40) % 2 == 0, 1.0, -1.0)
    D = dtr.defl_create(lat, V, lam, prec=prec)
    sp = dtr.solve_params(tol=1e-10, solver="mixed_f32")
    one = dtr.trace_estimate(g, w.m0, D, dtr.trace_params(seed=4, z0_first=2, n_z0=1, ncolors=16, nvec=16, block=4,
                                                          solve=sp))
    parts = []
    for v0 in range(0, 16, 4):
        o = dtr.trace_estimate(g, w.m0, D, dtr.trace_params(seed=4, z0_first=2, n_z0=1, ncolors=16, nvec=4, block=4,
                                                            solve=sp, vec_first=v0))
        parts.append(o["samples"][0])
    assert np.array_equal(np.concatenate(parts), one["samples"][0])
    with pytest.raises(dtr.DtrError):
        dtr.trace_estimate(g, w.m0, D, dtr.trace_params(seed=4, n_z0=1, ncolors=16, nvec=4, block=4, solve=sp,
                                                        vec_first=13))


def test_hp_projection_bf16_k1000_compensated(dtr, c8):
    """BF16 V with k = 1000 on hierarchical-probing blocks: the per-vector
    deflation terms (compensated FP32 tile sums, FP64 across tiles) equal the
    oracle's FP64 gamma5 form on the rounded V to 1e-12."""
    w, lat, g = c8["w"], c8["lat"], c8["g"]
    k = 1000
    rng = np.random.default_rng(8)
    V = (rng.standard_normal((lat.N, k)) + 1j * rng.standard_normal((lat.N, k))) / np.sqrt(2 * lat.N)
    lam = np.linspace(0.8, 2.0, k) * np.where(np.arange(k) % 3 == 0, -1.0, 1.0)
    D = dtr.defl_create(lat, V, lam, prec="bf16")
    p = dtr.trace_params(seed=12, z0_first=5, n_z0=1, ncolors=16, nvec=16, block=8,
                         solve=dtr.solve_params(tol=1e-10, solver="mixed_f32"))
    out = dtr.trace_estimate(g, w.m0, D, p, want_replay=True)
    d_gpu = out["replay"][0].sum(axis=1)
    Z = noise.noise_vectors(w.dims, 12, 5, 16, False, 0, 16)
    d_ref = deflation.quadrature_gamma5(deflation.bf16_round(V), lam, Z)
    assert np.abs(d_gpu - d_ref).max() <= 1e-12 * np.abs(d_ref).max()


def test_eight_lanes_at_benchmark_shape_never_time_out(dtr, c8):
    """The 8^4 benchmark shape (16-vector HP runs, 16-RHS blocks, k = 100 FP64)
    on 8 concurrent lanes, graph-driven mixed solves: each lane's cooperative
    grid is co-resident by construction (a cooperative launch starts only when
    all its CTAs fit), so no bounded barrier wait gives up (that would return
    DTR_ETIMEOUT) over several waves, and all solves converge."""
    w, lat, g = c8["w"], c8["lat"], c8["g"]
    V = synth.disjoint_orthonormal(lat.N, w.k, 2)
    D = dtr.defl_create(lat, V, np.linspace(0.9, 1.4, w.k))
    p = dtr.trace_params(seed=0, z0_first=1000, n_z0=24, ncolors=16, nvec=16, block=16, lanes=8,
                         solve=dtr.solve_params(tol=1e-10, solver="mixed_f32"))
    ws = dtr.TraceWorkspace(g, D, p)
    for rep in range(3):
        p.z0_first = 1000 + 24 * rep
        out = dtr.trace_estimate(g, w.m0, D, p, workspace=ws)
        assert out["status"] == 0 and out["all_converged"] and out["max_true_residual"] <= 1e-10
