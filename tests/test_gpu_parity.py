"""GPU parity: the CUDA library (through its C ABI) against the FP64 oracle.

Tolerances:
  noise / colouring          bit-exact (integer work)
  dslash FP64                1e-13 relative (max-norm), FP32 arithmetic 2e-6
  solves                     true residual <= tol, recomputed by the oracle in FP64
  per-vector z^H A^-1 z      1e-8 relative after solves to 1e-10
  trace                      1e-10 relative for identical noise (solves to 1e-12)
  deflation terms / T_D      1e-12 relative (FP64 V), 1e-5 (FP32 V)
"""
import numpy as np
import pytest

from oracle import deflation, estimator, exact, noise, solve, wilson
from paper_1603_05988_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dtr():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1603_05988_gb300 import dtr as _dtr
    return _dtr


def _cpu(t):
    return t.detach().cpu().numpy()


def _setup(dtr, dims, eps, m0, seed):
    U = synth.random_su3_links(dims, eps, seed)
    lat = dtr.make_lattice(dims)
    g = dtr.gauge_from_host(lat, U)
    return U, lat, g


@pytest.mark.parametrize("dims,seed,run,ncolors,dil,q0,nrhs", [
    ((4, 4, 4, 4), 0, 0, 1, False, 0, 1),
    ((4, 4, 4, 4), 7, 3, 16, False, 0, 16),
    ((8, 8, 8, 8), 123, 5, 32, False, 3, 29),        # ragged column range
    ((8, 8, 8, 8), 2**63 + 5, 17, 512, False, 500, 12),
    ((4, 4, 4, 4), 9, 1, 256, True, 100, 64),         # dilution
    ((2, 4, 6, 8), 3, 2, 2, False, 0, 2),
])
def test_noise_bit_exact(dtr, dims, seed, run, ncolors, dil, q0, nrhs):
    lat = dtr.make_lattice(dims)
    z = _cpu(dtr.gen_noise(lat, seed, run, ncolors, dil, q0, nrhs))
    ref = noise.noise_vectors(dims, seed, run, ncolors, dil, q0, nrhs)
    assert np.array_equal(z.T, ref)


def test_noise_rejects_bad_colouring(dtr):
    lat = dtr.make_lattice((4, 4, 4, 6))
    with pytest.raises(dtr.DtrError):
        dtr.gen_noise(lat, 0, 0, 32, False, 0, 1)      # period 4 does not divide 6
    with pytest.raises(dtr.DtrError):
        dtr.gen_noise(lat, 0, 0, 3, False, 0, 1)


@pytest.mark.parametrize("dims,nrhs", [((2, 2, 2, 2), 1), ((4, 4, 4, 4), 5), ((6, 4, 2, 4), 16),
                                       ((4, 4, 4, 8), 64), ((8, 8, 8, 8), 16)])
@pytest.mark.parametrize("dagger", [False, True])
def test_dslash_fp64(dtr, dims, nrhs, dagger):
    import torch
    U, lat, g = _setup(dtr, dims, 0.8, -0.6, 11)
    rng = np.random.default_rng(1)
    X = rng.standard_normal((nrhs, lat.N)) + 1j * rng.standard_normal((nrhs, lat.N))
    out = _cpu(dtr.dslash(g, -0.6, torch.from_numpy(X).cuda(), dagger=dagger))
    A = wilson.explicit_dagger(U, dims, -0.6) if dagger else wilson.explicit(U, dims, -0.6)
    ref = (A @ X.T).T
    assert np.abs(out - ref).max() <= 1e-13 * np.abs(ref).max()


def test_dslash_fp32(dtr):
    import torch
    dims = (4, 4, 4, 8)
    U, lat, g = _setup(dtr, dims, 0.8, -0.75, 12)
    rng = np.random.default_rng(2)
    X = rng.standard_normal((8, lat.N)) + 1j * rng.standard_normal((8, lat.N))
    out = _cpu(dtr.dslash(g, -0.75, torch.from_numpy(X).cuda(), prec="f32"))
    ref = (wilson.explicit(U, dims, -0.75) @ X.T).T
    assert np.abs(out - ref).max() <= 2e-6 * np.abs(ref).max()


@pytest.mark.parametrize("prec,tol", [("bf16", 3e-2), ("f16", 4e-3)])
@pytest.mark.parametrize("dims,nrhs", [((4, 4, 4, 4), 1), ((4, 4, 4, 8), 3), ((8, 4, 4, 8), 8)])
def test_dslash_half_storage(dtr, prec, tol, dims, nrhs):
    """BF16/FP16 storage of fields and two-row links, FP32 math: max-norm error
    relative to the largest output entry within the storage precision."""
    import torch
    U, lat, g = _setup(dtr, dims, 0.8, -0.75, 13)
    rng = np.random.default_rng(3)
    X = rng.standard_normal((nrhs, lat.N)) + 1j * rng.standard_normal((nrhs, lat.N))
    out = _cpu(dtr.dslash(g, -0.75, torch.from_numpy(X).cuda(), prec=prec))
    ref = (wilson.explicit(U, dims, -0.75) @ X.T).T
    err = np.abs(out - ref).max() / np.abs(ref).max()
    assert err <= tol, err
    with pytest.raises(dtr.DtrError):
        dtr.dslash(g, -0.75, torch.from_numpy(X).cuda(), prec=prec, dagger=True)


def test_gauge_roundtrip(dtr):
    U, lat, g = _setup(dtr, (4, 4, 2, 2), 0.5, -0.4, 3)
    assert np.array_equal(g.to_host(), U)


@pytest.mark.parametrize("engine", ["persistent", "kernels"])
@pytest.mark.parametrize("solver", ["f64", "mixed_f32"])
@pytest.mark.parametrize("dims,nrhs", [((4, 4, 4, 4), 8), ((4, 4, 4, 8), 13), ((8, 8, 8, 8), 64)])
def test_solve_true_residual(dtr, solver, dims, nrhs, engine):
    import torch
    U, lat, g = _setup(dtr, dims, 0.5, -0.4, 1000)
    Z = noise.noise_vectors(dims, 5, 0, 16 if nrhs <= 16 else 512, False, 0, nrhs)
    p = dtr.solve_params(tol=1e-10, solver=solver, engine=engine)
    y, stats = dtr.solve_batch(g, -0.4, torch.from_numpy(np.ascontiguousarray(Z.T)).cuda(), params=p)
    Y = _cpu(y).T
    A = wilson.explicit(U, dims, -0.4)
    res = np.linalg.norm(Z - A @ Y, axis=0) / np.linalg.norm(Z, axis=0)
    assert np.all(res <= 1e-10), res
    assert all(s["converged"] for s in stats)
    assert np.allclose([s["true_residual"] for s in stats], res, rtol=1e-3, atol=1e-14)


def test_solve_initial_guess_and_zero_rhs(dtr):
    import torch
    dims = (4, 4, 4, 4)
    U, lat, g = _setup(dtr, dims, 0.5, -0.4, 1000)
    Z = noise.noise_vectors(dims, 1, 0, 2, False, 0, 2)
    Z[:, 1] = 0.0                                    # zero right-hand side
    A = wilson.explicit(U, dims, -0.4)
    Y0 = solve.dense_solve(A.toarray(), Z)
    y, st = dtr.solve_batch(g, -0.4, torch.from_numpy(np.ascontiguousarray(Z.T)).cuda(),
                            y0=torch.from_numpy(np.ascontiguousarray(Y0.T)).cuda())
    assert st[0]["converged"] and st[1]["converged"]
    assert np.abs(_cpu(y)[1]).max() == 0.0
    assert st[0]["iterations"] == 0              # exact guess: nothing to do


@pytest.mark.parametrize("dims,nrhs", [((4, 4, 4, 4), 8), ((8, 8, 8, 8), 16)])
def test_mixed_graph_matches_host_loop(dtr, dims, nrhs):
    """The CUDA-graph solve (device-driven WHILE loop over defect-correction
    cycles) runs the same kernels in the same order as the host-driven loop:
    bit-identical solutions and iteration counts."""
    import torch
    U, lat, g = _setup(dtr, dims, 0.5, -0.4, 1000)
    Z = noise.noise_vectors(dims, 7, 1, 16, False, 0, nrhs)
    z = torch.from_numpy(np.ascontiguousarray(Z.T)).cuda()
    outs = []
    for graph in (False, True):
        p = dtr.solve_params(tol=1e-10, solver="mixed_f32", graph=graph)
        y, st = dtr.solve_batch(g, -0.4, z, params=p)
        outs.append((_cpu(y), [s["iterations"] for s in st], [s["restarts"] for s in st]))
    assert np.array_equal(outs[0][0], outs[1][0])
    assert outs[0][1] == outs[1][1] and outs[0][2] == outs[1][2]
    A = wilson.explicit(U, dims, -0.4)
    res = np.linalg.norm(Z - A @ outs[1][0].T, axis=0) / np.linalg.norm(Z, axis=0)
    assert np.all(res <= 1e-10), res


def test_mixed_graph_not_converged_reports(dtr):
    """An iteration cap ends the graph's loop: DTR_ENOTCONV with the statistics written."""
    import torch
    dims = (4, 4, 4, 4)
    U, lat, g = _setup(dtr, dims, 0.5, -0.4, 1000)
    Z = noise.noise_vectors(dims, 1, 0, 2, False, 0, 2)
    p = dtr.solve_params(tol=1e-12, maxiter=3, solver="mixed_f32")
    y, st = dtr.solve_batch(g, -0.4, torch.from_numpy(np.ascontiguousarray(Z.T)).cuda(), params=p,
                            allow_notconv=True)
    assert not st[0]["converged"] and st[0]["iterations"] <= 8


def test_barrier_timeout_is_reported(dtr):
    """A barrier whose peer never arrives gives up within its budget and raises
    the error word (the solver maps it to DTR_ETIMEOUT); the context stays usable."""
    timed_out, err = dtr.selftest_barrier(2_000_000)      # ~1 ms at 2 GHz
    assert timed_out == 1 and err == 1
    lat = dtr.make_lattice((4, 4, 4, 4))
    z = dtr.gen_noise(lat, 1, 0, 1, False, 0, 1)           # GPU still answers
    assert z.abs().max().item() == 1.0


def test_solve_not_converged_reports(dtr):
    import torch
    dims = (4, 4, 4, 4)
    U, lat, g = _setup(dtr, dims, 0.5, -0.4, 1000)
    Z = noise.noise_vectors(dims, 1, 0, 2, False, 0, 2)
    p = dtr.solve_params(tol=1e-12, maxiter=3, check_every=1)
    with pytest.raises(dtr.DtrError) as e:
        dtr.solve_batch(g, -0.4, torch.from_numpy(np.ascontiguousarray(Z.T)).cuda(), params=p)
    assert e.value.code == dtr.DTR_ENOTCONV
    y, st = dtr.solve_batch(g, -0.4, torch.from_numpy(np.ascontiguousarray(Z.T)).cuda(), params=p,
                            allow_notconv=True)
    assert not st[0]["converged"] and st[0]["iterations"] <= 4


@pytest.fixture(scope="module")
def cfg1(dtr):
    """4^4, eps 0.5, m0 -0.4, k = 32 smallest triplets by dense eig (oracle)."""
    dims, m0 = (4, 4, 4, 4), -0.4
    U = synth.random_su3_links(dims, 0.5, 1000)
    A = wilson.explicit(U, dims, m0)
    AH = wilson.explicit_dagger(U, dims, m0)
    Ad = A.toarray()
    tr, Ainv = exact.trace_inverse_lu(Ad)
    V, lam, sig = deflation.smallest_triplets(Ad, 32)
    lat = dtr.make_lattice(dims)
    g = dtr.gauge_from_host(lat, U)
    return dict(dims=dims, m0=m0, U=U, A=A, AH=AH, Ad=Ad, tr=tr, Ainv=Ainv, V=V, lam=lam, sig=sig, lat=lat, g=g)


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 2e-5)])
def test_deflate_project(dtr, cfg1, prec, tol):
    import torch
    c = cfg1
    D = dtr.defl_create(c["lat"], c["V"], c["lam"], prec=prec)
    Z = noise.noise_vectors(c["dims"], 3, 4, 16, False, 0, 11)
    d, C, x0 = dtr.deflate_project(D, torch.from_numpy(np.ascontiguousarray(Z.T)).cuda(), True, True)
    d_ref = deflation.quadrature(c["AH"], c["V"], c["sig"], Z)      # paper's literal A^H form
    assert np.abs(_cpu(d) - d_ref).max() <= tol * np.abs(d_ref).max()
    assert abs(D.T_D() - deflation.T_D(c["AH"], c["V"], c["sig"])) <= tol * abs(D.T_D())
    C = _cpu(C)
    Cz = c["V"].conj().T @ Z
    Cg = c["V"].conj().T @ wilson.gamma5_vec(Z)
    assert np.abs(C[:11].T - Cz).max() <= tol * np.abs(Cz).max() * 10
    assert np.abs(C[11:].T - Cg).max() <= tol * np.abs(Cg).max() * 10
    x0_ref = c["V"] @ ((c["V"].conj().T @ wilson.gamma5_vec(Z)) / c["lam"][:, None])
    assert np.abs(_cpu(x0).T - x0_ref).max() <= tol * np.abs(x0_ref).max() * 10


def test_trace_parity_4x4x4x4_mc64_k32(dtr, cfg1):
    """The 4^4 workload: 64 Z4 vectors, k = 32; identical noise on both sides."""
    c = cfg1
    D = dtr.defl_create(c["lat"], c["V"], c["lam"])
    p = dtr.trace_params(seed=0, n_z0=64, ncolors=1, nvec=1, block=64,
                         solve=dtr.solve_params(tol=1e-12))
    out = dtr.trace_estimate(c["g"], c["m0"], D, p, want_replay=True)
    N = c["Ad"].shape[0]
    Z = np.stack([noise.z0_vector(0, r, N) for r in range(64)], axis=1)
    ref = estimator.deflated_hp(c["AH"], lambda Z: c["Ainv"] @ Z, Z, c["V"], c["sig"])
    t_gpu = out["samples"][:, 0]
    assert np.abs(t_gpu - ref["t"]).max() <= 1e-8 * np.abs(ref["t"]).max()
    assert abs(out["T_D"] - ref["T_D"]) <= 1e-12 * abs(ref["T_D"])
    assert abs(out["trace"] - ref["trace"][-1]) <= 1e-10 * abs(ref["trace"][-1])
    # replay record: per-m terms sum to the deflation quadrature of each sample
    d_ref = ref["defl"]
    assert np.abs(out["replay"][:, 0, :].sum(axis=1) - d_ref).max() <= 1e-11 * np.abs(d_ref).max()
    assert out["all_converged"] and out["max_true_residual"] <= 1e-12
    # statistics against the oracle's definitions on the same samples
    assert abs(out["var_samples"] - estimator.sample_variance(ref["t"])) <= 1e-9 * out["var_samples"]


def test_trace_mixed_matches_fp64(dtr, cfg1):
    c = cfg1
    D = dtr.defl_create(c["lat"], c["V"], c["lam"])
    outs = []
    for solver in ("f64", "mixed_f32"):
        p = dtr.trace_params(seed=4, n_z0=4, ncolors=16, nvec=16, block=16,
                             solve=dtr.solve_params(tol=1e-12, solver=solver))
        outs.append(dtr.trace_estimate(c["g"], c["m0"], D, p))
    assert np.abs(outs[0]["samples"] - outs[1]["samples"]).max() <= 1e-8 * np.abs(outs[0]["samples"]).max()
    assert abs(outs[0]["trace"] - outs[1]["trace"]) <= 1e-10 * abs(outs[0]["trace"])


def test_trace_graph_captured_once_and_reused(dtr, cfg1):
    """Repeated trace runs on one workspace reuse one captured graph; the
    kernels of its device-driven loop are counted on the device."""
    c = cfg1
    D = dtr.defl_create(c["lat"], c["V"], c["lam"])
    p = dtr.trace_params(seed=9, n_z0=1, ncolors=16, nvec=16, block=16,
                         solve=dtr.solve_params(tol=1e-10, solver="mixed_f32"))
    ws = dtr.TraceWorkspace(c["g"], D, p)
    dtr.trace_estimate(c["g"], c["m0"], D, p, workspace=ws)
    c0, l0 = dtr.graph_stats()
    k0 = dtr.kernel_launches()
    for r in range(1, 4):
        p.z0_first = r
        out = dtr.trace_estimate(c["g"], c["m0"], D, p, workspace=ws)
        assert out["all_converged"]
    c1, l1 = dtr.graph_stats()
    assert c1 == c0 and l1 - l0 == 3
    # per run: pre-part (3) + at least one cycle body (init, scal init, persistent, accumulate,
    # residual, loop condition), plus the estimator's own kernels
    assert dtr.kernel_launches() - k0 >= 3 * (3 + 6)


@pytest.mark.parametrize("solver", ["mixed_f32", "f64"])
def test_trace_lanes_bit_identical(dtr, cfg1, solver):
    """Blocks solved concurrently on several lanes (own streams, workspace
    slices and SM shares) give the same per-sample records as one lane."""
    c = cfg1
    D = dtr.defl_create(c["lat"], c["V"], c["lam"])
    outs = {}
    for lanes, grid in ((1, 32), (4, 32), (4, 0)):
        p = dtr.trace_params(seed=11, n_z0=6, ncolors=16, nvec=16, block=8, lanes=lanes,
                             solve=dtr.solve_params(tol=1e-10, solver=solver, grid=grid))
        outs[lanes, grid] = dtr.trace_estimate(c["g"], c["m0"], D, p, want_replay=True)
    a, b = outs[1, 32], outs[4, 32]        # same grid: same reduction order, bit-identical
    assert np.array_equal(a["samples"], b["samples"])
    assert np.array_equal(a["replay"], b["replay"])
    assert a["iterations"] == b["iterations"]
    assert a["trace"] == b["trace"] and a["jk_err"] == b["jk_err"]
    # the default grid of a lane is its share of the SMs: another summation order
    d = outs[4, 0]
    assert np.abs(d["samples"] - a["samples"]).max() <= 1e-9 * np.abs(a["samples"]).max()


def test_trace_autotune_picks_fastest_measured_candidate(dtr, cfg1):
    """The autotuner times every lane count on real trace waves, returns the
    fastest and caches the choice for the problem shape."""
    c = cfg1
    D = dtr.defl_create(c["lat"], c["V"], c["lam"])
    p = dtr.trace_params(seed=3, n_z0=1, ncolors=16, nvec=16, block=16,
                         solve=dtr.solve_params(tol=1e-10, solver="mixed_f32"))
    t = dtr.trace_autotune(c["g"], c["m0"], D, p, reps=2, force=True)
    assert [e["lanes"] for e in t["table"]] == [1, 2, 4, 8]
    assert all(e["block"] == 16 and e["rhs_per_s"] > 0 for e in t["table"])
    assert t["rhs_per_s"] == max(e["rhs_per_s"] for e in t["table"])
    assert t["lanes"] in (1, 2, 4, 8) and not t["cached"]
    t2 = dtr.trace_autotune(c["g"], c["m0"], D, p)
    assert t2["cached"] and t2["lanes"] == t["lanes"]
    # the chosen shape runs and matches the one-lane records on the same grid
    p1 = dtr.trace_params(seed=3, n_z0=t["lanes"], ncolors=16, nvec=16, block=16, lanes=1,
                          solve=dtr.solve_params(tol=1e-10, solver="mixed_f32", grid=16))
    pl = dtr.trace_params(seed=3, n_z0=t["lanes"], ncolors=16, nvec=16, block=16, lanes=t["lanes"],
                          solve=dtr.solve_params(tol=1e-10, solver="mixed_f32", grid=16))
    a, b = dtr.trace_estimate(c["g"], c["m0"], D, p1), dtr.trace_estimate(c["g"], c["m0"], D, pl)
    assert np.array_equal(a["samples"], b["samples"])


def test_sharded_trace_one_process_matches_library(dtr, cfg1):
    """The sharded driver (records gathered over a process group, statistics
    formed on the host) reproduces the library's own statistics."""
    import socket
    import torch.distributed as dist
    from paper_1603_05988_gb300 import shard
    c = cfg1
    D = dtr.defl_create(c["lat"], c["V"], c["lam"])
    mk = lambda z0, n: dtr.trace_params(seed=2, z0_first=z0, n_z0=n, ncolors=16, nvec=16, block=16,
                                         solve=dtr.solve_params(tol=1e-10, solver="mixed_f32"))
    ref = dtr.trace_estimate(c["g"], c["m0"], D, mk(0, 5))
    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=0, world_size=1)
    try:
        st = shard.sharded_trace_estimate(c["g"], c["m0"], D, 5, mk)
    finally:
        dist.destroy_process_group()
    assert np.array_equal(st["samples"], ref["samples"])
    assert abs(st["trace"] - ref["trace"]) <= 1e-14 * abs(ref["trace"])
    assert abs(st["jk_err"] - ref["jk_err"]) <= 1e-12 * ref["jk_err"]
    assert abs(st["var_runs"] - ref["var_runs"]) <= 1e-12 * ref["var_runs"]


def test_trace_hp_projection_matches_generic(dtr, cfg1):
    """The HP-structured deflation projection (per-colour sums of V^H z0) and
    the generic contraction V^H [Z, g5 Z] give the same per-m terms."""
    c = cfg1
    D = dtr.defl_create(c["lat"], c["V"], c["lam"])
    outs = []
    for use_x0 in (False, True):     # use_x0 forces the generic projection
        p = dtr.trace_params(seed=8, n_z0=2, ncolors=32, nvec=32, block=16, use_x0=use_x0,
                             solve=dtr.solve_params(tol=1e-12))
        outs.append(dtr.trace_estimate(c["g"], c["m0"], D, p, want_replay=True))
    a, b = outs[0]["replay"], outs[1]["replay"]
    assert np.abs(a - b).max() <= 1e-12 * np.abs(b).max()
    assert np.abs(outs[0]["samples"] - outs[1]["samples"]).max() <= 1e-8 * np.abs(outs[1]["samples"]).max()


def test_trace_deflated_blocks_spanning_runs(dtr, cfg1):
    """Blocks that straddle two z0 runs take the generic projection."""
    c = cfg1
    D = dtr.defl_create(c["lat"], c["V"], c["lam"])
    p = dtr.trace_params(seed=3, z0_first=2, n_z0=3, ncolors=32, nvec=20, block=8,
                         solve=dtr.solve_params(tol=1e-12, solver="mixed_f32"))
    out = dtr.trace_estimate(c["g"], c["m0"], D, p)
    for r in range(3):
        Z = noise.noise_vectors(c["dims"], 3, 2 + r, 32, False, 0, 20)
        ref = estimator.deflated_hp(c["AH"], lambda Z: c["Ainv"] @ Z, Z, c["V"], c["sig"])
        assert np.abs(out["samples"][r] - ref["t"]).max() <= 1e-8 * np.abs(ref["t"]).max()
        assert abs(out["trace_runs"][r] - ref["trace"][-1]) <= 1e-10 * abs(ref["trace"][-1])


def test_trace_complete_probing_exact(dtr, cfg1):
    """256 colours x 12-fold dilution at 4^4 probe every entry of A^-1:
    the estimate equals Tr(A^-1) (dense LU) for any z0 and any deflation."""
    c = cfg1
    D = dtr.defl_create(c["lat"], c["V"], c["lam"])
    p = dtr.trace_params(seed=11, n_z0=1, ncolors=256, nvec=256, dilute12=True, block=64,
                         solve=dtr.solve_params(tol=1e-12, solver="mixed_f32"))
    out = dtr.trace_estimate(c["g"], c["m0"], D, p)
    assert abs(out["trace"] - c["tr"]) <= 1e-9 * abs(c["tr"])


def test_trace_no_deflation_hp_matches_oracle(dtr, cfg1):
    c = cfg1
    p = dtr.trace_params(seed=2, z0_first=5, n_z0=3, ncolors=32, nvec=20, block=8,   # ragged last block
                         solve=dtr.solve_params(tol=1e-12))
    out = dtr.trace_estimate(c["g"], c["m0"], None, p)
    for r in range(3):
        Z = noise.noise_vectors(c["dims"], 2, 5 + r, 32, False, 0, 20)
        ref = estimator.deflated_hp(c["AH"], lambda Z: c["Ainv"] @ Z, Z)
        assert np.abs(out["samples"][r] - ref["t"]).max() <= 1e-8 * np.abs(ref["t"]).max()
        assert abs(out["trace_runs"][r] - ref["trace"][-1]) <= 1e-10 * abs(ref["trace"][-1])
    m, v = estimator.jackknife_mean(out["trace_runs"])
    assert abs(np.sqrt(v) - out["jk_err"]) <= 1e-9 * max(out["jk_err"], 1e-30)


@pytest.mark.parametrize("solver", ["f64", "mixed_f32"])
def test_trace_8x8x8x8_hp16_sampled(dtr, solver):
    """The 8^4 workload's launch shape (16-colour HP, blocks of 16, k = 100 FP64
    deflation vectors): sampled t_j recomputed one by one by the oracle (CGNR
    to 1e-13), the deflation term by the oracle's gamma5 form for the same V."""
    import torch
    dims, m0 = (8, 8, 8, 8), -0.6
    U = synth.random_su3_links(dims, 0.7, 1001)
    lat = dtr.make_lattice(dims)
    g = dtr.gauge_from_host(lat, U)
    V = synth.random_orthonormal(lat.N, 100, 5)
    lam = np.where(np.arange(100) % 2 == 0, 1.0, -1.0) * np.linspace(0.9, 1.4, 100)
    D = dtr.defl_create(lat, V, lam)
    p = dtr.trace_params(seed=0, n_z0=2, ncolors=16, nvec=16, block=16,
                         solve=dtr.solve_params(tol=1e-10, solver=solver))
    out = dtr.trace_estimate(g, m0, D, p)
    assert out["all_converged"] and out["max_true_residual"] <= 1e-10
    assert abs(out["T_D"] - deflation.T_D_gamma5(V, lam)) <= 1e-12 * abs(out["T_D"])
    A = wilson.explicit(U, dims, m0)
    for r, j in [(0, 0), (0, 7), (1, 15)]:
        z = noise.noise_vectors(dims, 0, r, 16, False, j, 1)
        y, it, res = solve.cgnr(A, z, tol=1e-13)
        t_ref = np.vdot(z[:, 0], y[:, 0]) - deflation.quadrature_gamma5(V, lam, z)[0]
        assert abs(out["samples"][r, j] - t_ref) <= 1e-8 * abs(t_ref)
