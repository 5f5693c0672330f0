"""Kernel micro-benchmarks of libdtr (CUDA-event timing through the C ABI).

    python -m paper_1603_05988_gb300.kbench dslash --lattice 32,32,32,64 --prec bf16 --nrhs 1 --reps 20
    python -m paper_1603_05988_gb300.kbench solve --lattice 8,8,8,8 --nrhs 16 --reps 3 [--no-graph]
        [--solver f64,mixed_f32,mixed_f16,mixed_bf16] [--inner-tol T] [--eps E --gauge-seed S --m0 M]
    python -m paper_1603_05988_gb300.kbench trace --lattice 16,16,16,32 --eps 0.8 --m0 -0.75 --gauge-seed 1002 \
        --k 200 --prec f32 --ncolors 512 --nvec 512 --block 32 --solver f64,mixed_f32,mixed_f16,mixed_bf16
    python -m paper_1603_05988_gb300.kbench learned --lattice 16,16,16,32 --eval-lattice 24,24,24,48 \
        --eps 0.8 --m0 -0.75 --gauge-seed 1002 --nrhs 8 [--steps 200 --batch 8 --pool 16 | --stream-pairs 20000]
    python -m paper_1603_05988_gb300.kbench deflate --lattice 16,16,16,32 --k 256[,1000] --prec bf16 --nrhs 16 --reps 20
    python -m paper_1603_05988_gb300.kbench net --lattice 16,16,16,32 --nrhs 8 --reps 5
    python -m paper_1603_05988_gb300.kbench eig --lattice 16,16,16,32 --eps 0.8 --m0 -0.75 --gauge-seed 1002 \
        --k 200 --prec f32 [--degree 16 --iters 60 --tol 1e-2 --time-limit 0 --device-gauge]

Large lattices take their links from the seeded 16^3x32 field repeated
periodically (exact SU(3) matrices; the stencil's cost does not depend on
their values), so set-up does not spend a minute drawing 8 M random links.
Prints one JSON line per measurement: average launch time, algorithmic bytes
and flops per launch, achieved GB/s and TFLOP/s.
"""
import argparse
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

# algorithmic bytes per site and right-hand side (in + out) and per site for the four 3x3 links, by
# storage precision (each array touched once); the half-precision stencil moves 96 B of links per site
# instead of 144 when it stores two rows and rebuilds the third (dtr.half_link_rows() == 2)
SPINOR_BYTES = {"f64": 2 * 192, "f32": 2 * 96, "bf16": 2 * 48, "f16": 2 * 48}
LINK_BYTES = {"f64": 576, "f32": 288, "bf16": 144, "f16": 144}


def link_stored_bytes(prec):
    from . import dtr
    if prec in ("bf16", "f16"):
        return 48 * dtr.half_link_rows()
    return LINK_BYTES[prec]
FLOPS_PER_SITE = 1368.0   # 1320 hopping (8 directions x (12 + 2 x 66 + 24) - 24) + 48 diagonal


def tiled_links(dims, eps=0.8, seed=1002, base=(16, 16, 16, 32)):
    """Seeded links on min(dims, base), repeated periodically to fill dims."""
    from . import synth
    b = tuple(min(d, bb) for d, bb in zip(dims, base))
    if any(d % s for d, s in zip(dims, b)):
        raise ValueError("lattice extents must be multiples of the tile %r" % (b,))
    small = synth.random_su3_links(b, eps, seed)
    if b == tuple(dims):
        return small
    s7 = small.reshape(b[3], b[2], b[1], b[0], 4, 3, 3)          # (t, z, y, x, mu, a, b)
    reps = (dims[3] // b[3], dims[2] // b[2], dims[1] // b[1], dims[0] // b[0], 1, 1, 1)
    return np.ascontiguousarray(np.tile(s7, reps).reshape(-1, 4, 3, 3))


def dslash_case(gauge, dims, prec, nrhs, reps, m0=-0.75):
    from . import dtr
    ms = dtr.time_dslash(gauge, m0, nrhs, prec=prec, reps=reps)
    V = int(np.prod(dims))
    b = nrhs if prec in ("bf16", "f16") else dtr_pad(nrhs)
    alg_bytes = V * nrhs * SPINOR_BYTES[prec] + V * LINK_BYTES[prec]
    moved = V * nrhs * SPINOR_BYTES[prec] + V * link_stored_bytes(prec)
    flops = V * nrhs * FLOPS_PER_SITE
    return {"kernel": "dslash", "lattice": list(dims), "prec": prec, "nrhs": nrhs, "padded_width": b,
            "link_rows": dtr.half_link_rows() if prec in ("bf16", "f16") else 3,
            "avg_launch_ms": ms, "alg_bytes_per_launch": alg_bytes, "stored_bytes_per_launch": moved,
            "flops_per_launch": flops, "moved_gbs": moved / (ms * 1e-3) / 1e9,
            "achieved_gbs": alg_bytes / (ms * 1e-3) / 1e9, "achieved_tflops": flops / (ms * 1e-3) / 1e12}


def solve_case(gauge, dims, nrhs, reps, m0, graph=True, grid=0, solver="mixed_f32", inner_tol=1e-5,
               engine="persistent"):
    """Solves of nrhs Z4 right-hand sides to 1e-10 (persistent engine), with the
    persistent launches timed on the device.  solver: f64, mixed_f32 (FP32 inner
    vectors), mixed_f16 / mixed_bf16 (half-storage inner vectors)."""
    import time
    import torch
    from . import dtr
    lat = gauge.lat
    z = dtr.gen_noise(lat, 0, 1, 16 if nrhs <= 16 else 512, False, 0, nrhs)
    p = dtr.solve_params(tol=1e-10, solver=solver, graph=graph, grid=grid, inner_tol=inner_tol, engine=engine)
    dtr.solve_batch(gauge, m0, z, params=p)
    dtr.profile_persistent(1)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        y, st = dtr.solve_batch(gauge, m0, z, params=p)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / reps
    prof = dtr.profile_persistent(0)
    its = float(np.mean([s["iterations"] for s in st]))
    return {"kernel": "solve", "solver": solver, "engine": engine, "inner_tol": inner_tol, "lattice": list(dims),
            "nrhs": nrhs,
            "graph": graph, "ms_per_solve": dt * 1e3, "rhs_per_s": nrhs / dt,
            "iterations_per_rhs": its, "cycles_max": int(max(s["restarts"] for s in st)),
            "max_true_residual": float(max(s["true_residual"] for s in st)),
            "all_converged": bool(all(s["converged"] for s in st)),
            "persistent_launches": prof["launches"],
            "persistent_ms_per_launch": prof["ms"] / max(prof["launches"], 1),
            "site_rhs_iterations_per_solve": prof["site_rhs_iterations"] / reps}


def trace_case(dims, eps, m0, seed, k, defl_prec, ncolors, nvec, block, solvers):
    """The whole estimator (noise + HP mask, deflation projection, batched solves
    to 1e-10, reductions) for one z0 run of nvec probing vectors in blocks of
    `block` columns, with a k-vector deflation space stored in defl_prec (columns
    with disjoint supports: the projection's cost does not depend on the values);
    wall-clock RHS/s per solver after one warm-up run."""
    import time
    import torch
    from . import dtr, synth
    lat = dtr.make_lattice(dims)
    g = dtr.gauge_from_host(lat, synth.random_su3_links(dims, eps, seed))
    if k * 256 <= lat.N and lat.N * k <= (1 << 29):
        V = synth.disjoint_orthonormal(lat.N, k, 4)
        lam = np.where(np.arange(k) % 2 == 0, 1.0, -1.0) * np.linspace(0.8, 1.5, k)
        D = dtr.defl_create(lat, V, lam, prec=defl_prec)
        del V
    else:  # too large to build on the host: one filter iteration of the device eigensolver
        D, _, _ = dtr.eig_deflation(g, m0, dtr.eig_params(k, store=defl_prec, degree=4, max_iter=1, tol=1e-2))
    rows = []
    for solver in solvers:
        sp = dtr.solve_params(tol=1e-10, solver=solver)
        warm = dtr.trace_params(seed=0, z0_first=100, n_z0=1, ncolors=ncolors, nvec=nvec, block=block, solve=sp)
        dtr.trace_estimate(g, m0, D, warm)
        p = dtr.trace_params(seed=0, z0_first=0, n_z0=1, ncolors=ncolors, nvec=nvec, block=block, solve=sp)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        out = dtr.trace_estimate(g, m0, D, p)
        dt = time.perf_counter() - t0
        rows.append({"kernel": "trace estimate", "lattice": list(dims), "k": k, "defl_prec": defl_prec,
                     "ncolors": ncolors, "nvec": nvec, "block": block, "solver": solver, "s": dt,
                     "rhs_per_s": nvec / dt, "iterations_per_rhs": out["iterations"] / max(out["n_solves"], 1),
                     "all_converged": bool(out["all_converged"]), "max_true_residual": out["max_true_residual"],
                     "trace": [out["trace"].real, out["trace"].imag]})
    return rows


def learned_case(train_dims, eval_dims, eps, m0, seed, steps, batch, pool, nrhs, gmres_m=16, stream_pairs=0,
                 precision="bf16"):
    """The learned preconditioner at the sizes of its workload: the network is
    trained at train_dims on pool x batch (residual, error) pairs from the
    library's own solves (residual loss, Adam, all on the GPU), then FGMRES(m)
    with the trained network, FGMRES(m) without it and the mixed FP32 BiCGStab
    solve held-out Z4 right-hand sides to 1e-10 at train_dims and at eval_dims
    (the same weights: the network is a translation-invariant stencil).  Training
    uses the network's `precision` kernels; the evaluation runs FGMRES with both
    kernel sets and times one network application (4 layers x 93,312 flop per site
    and RHS) with each."""
    import time
    import torch
    from . import dtr, learned, synth

    def gauge_at(dims, gseed):
        lat = dtr.make_lattice(dims)
        return dtr.gauge_from_host(lat, synth.random_su3_links(dims, eps, gseed))

    g = gauge_at(train_dims, seed)
    net = dtr.Net(g.lat, act=0, init_scale=1.0 / (4.0 + m0), noise=1e-3, seed=1, precision=precision)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if stream_pairs:
        hist, ts, tt = learned.train_stream(net, g, m0, pairs=stream_pairs, batch=batch, lr=3e-4)
        npairs, nsteps = stream_pairs, len(hist)
    else:
        hist = learned.train(net, g, m0, steps=steps, batch=batch, lr=3e-4, pool=pool)
        npairs, nsteps, ts, tt = pool * batch, steps, None, None
    torch.cuda.synchronize()
    out = {"kernel": "learned preconditioner", "train_lattice": list(train_dims), "eps": eps, "m0": m0,
           "train_precision": precision,
           "pairs": npairs, "steps": nsteps, "train_s": time.perf_counter() - t0, "solve_s": ts, "step_s": tt,
           "loss_first": float(np.mean(hist[:5])), "loss_last": float(np.mean(hist[-10:])),
           "loss_curve": [float(np.mean(hist[i:i + max(1, len(hist) // 10)]))
                          for i in range(0, len(hist), max(1, len(hist) // 10))], "eval": []}
    W = net.weights()
    for dims in (train_dims, eval_dims):
        if tuple(dims) == tuple(train_dims):
            gg, nn = g, net
        else:
            gg = gauge_at(dims, seed + 1)
            nn = dtr.Net(gg.lat, act=0, weights=W)
        z = torch.cat([dtr.gen_noise(gg.lat, 4242, k, 1, False, 0, 1) for k in range(nrhs)])
        row = {"lattice": list(dims), "apply": {}}
        for prec in ("bf16", "f32"):
            nn.set_precision(prec)
            nn.apply(z)
            torch.cuda.synchronize()
            reps = 5
            t1 = time.perf_counter()
            for _ in range(reps):
                nn.apply(z)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t1) * 1e3 / reps
            row["apply"][prec] = {"ms": ms, "tflops": 4 * 93312.0 * gg.lat.N / 12 * nrhs / (ms * 1e-3) / 1e12}
        runs = [("fgmres_plain", "bf16", dtr.solve_params(tol=1e-10, solver="fgmres_net", net=None, gmres_m=gmres_m))]
        for prec in ("bf16", "f32"):
            runs.append(("fgmres_learned_" + prec, prec,
                         dtr.solve_params(tol=1e-10, solver="fgmres_net", net=nn, gmres_m=gmres_m)))
        runs.append(("bicgstab_mixed_f32", "bf16", dtr.solve_params(tol=1e-10, solver="mixed_f32")))
        for name, prec, p in runs:
            nn.set_precision(prec)
            dtr.solve_batch(gg, m0, z, params=p, allow_notconv=True)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            y, st = dtr.solve_batch(gg, m0, z, params=p, allow_notconv=True)
            torch.cuda.synchronize()
            row[name] = {"ms": (time.perf_counter() - t1) * 1e3,
                         "iterations_per_rhs": float(np.mean([s["iterations"] for s in st])),
                         "converged": bool(all(s["converged"] for s in st)),
                         "max_true_residual": float(max(s["true_residual"] for s in st))}
        out["eval"].append(row)
    return out


def net_case(dims, nrhs, reps, act=1, seed=3):
    """One application of the learned preconditioner's network (4 layers) to nrhs fields,
    with the tensor-core kernels (BF16 layer inputs) and the FP32 CUDA-core kernels; CUDA
    events around `reps` applications.  Useful work: 4 x 93,312 flop per site and RHS."""
    import torch
    from . import dtr
    lat = dtr.make_lattice(dims)
    net = dtr.Net(lat, act=act, init_scale=0.5, noise=0.05, seed=seed)
    x = torch.cat([dtr.gen_noise(lat, 4242, k, 1, False, 0, 1) for k in range(nrhs)])
    out = {"kernel": "network apply", "lattice": list(dims), "nrhs": nrhs, "act": act}
    for prec in ("bf16", "f32"):
        net.set_precision(prec)
        net.apply(x)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(reps):
            net.apply(x)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        out[prec] = {"ms": ms, "useful_tflops": 4 * 93312.0 * lat.V * nrhs / (ms * 1e-3) / 1e12}
    return out


def deflate_case(dims, k, nrhs, reps, prec="bf16"):
    """The deflation contraction C = V^H [Z, g5 Z] of an nrhs-column Z4 block with k
    vectors stored in `prec` (tensor cores for BF16).  Algorithmic work: V read once
    (N k x 4 B in BF16) plus the block (N x nrhs x 16 B); 8 N k (2 nrhs) real flops."""
    from . import dtr, synth
    lat = dtr.make_lattice(dims)
    V = synth.disjoint_orthonormal(lat.N, k, 3, support=max(1, min(256, lat.N // k)))
    lam = np.linspace(0.5, 1.5, k)
    D = dtr.defl_create(lat, V, lam, prec=prec)
    del V
    ms = dtr.time_deflate(D, nrhs, reps)
    vb = {"bf16": 4, "f32": 8, "f64": 16}[prec]
    alg_bytes = lat.N * k * vb + lat.N * nrhs * 16
    flops = 8.0 * lat.N * k * 2 * nrhs
    return {"kernel": "deflation contraction", "lattice": list(dims), "k": k, "nrhs": nrhs, "prec": prec,
            "avg_launch_ms": ms, "alg_bytes_per_launch": alg_bytes, "flops_per_launch": flops,
            "achieved_gbs": alg_bytes / (ms * 1e-3) / 1e9, "achieved_tflops": flops / (ms * 1e-3) / 1e12}


def eig_case(dims, eps, m0, seed, k, store, degree, iters, tol, time_limit, device_gauge, first_degree=0):
    """The setup eigensolver: the k smallest-|lambda| eigenpairs of g5 A to a relative residual tol
    (or until iters / time_limit), with its wall time, iterations and memory."""
    import torch
    from . import dtr, synth
    lat = dtr.make_lattice(dims)
    g = dtr.make_gauge(lat, eps, seed) if device_gauge else dtr.gauge_from_host(lat, synth.random_su3_links(dims, eps, seed))
    p = dtr.eig_params(k, store=store, tol=tol, degree=degree, first_degree=first_degree, max_iter=iters,
                       time_limit_s=time_limit)
    torch.cuda.synchronize()
    D, res, st = dtr.eig_deflation(g, m0, p)
    _, lam = D.to_host() if lat.N * k <= 50_000_000 else (None, None)
    out = {"kernel": "setup eigensolver", "lattice": list(dims), "eps": eps, "m0": m0, "k": k, "store": store,
           "degree": degree, "tol": tol, "gauge": "device" if device_gauge else "host"}
    out.update(st)
    out["median_residual"] = float(np.median(res))
    out["T_D"] = [D.T_D().real, D.T_D().imag]
    if lam is not None:
        out["abs_lambda_range"] = [float(np.abs(lam).min()), float(np.abs(lam).max())]
    out["peak_device_gb"] = torch.cuda.max_memory_allocated() / 1e9
    return out


def dtr_pad(n):
    b = 1
    while b < n:
        b <<= 1
    return b


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["dslash", "solve", "deflate", "learned", "trace", "eig", "net"])
    ap.add_argument("--k", default="256", help="deflation vectors (comma list for deflate)")
    ap.add_argument("--lattice", default="32,32,32,64")
    ap.add_argument("--prec", default="bf16")
    ap.add_argument("--nrhs", default="1")
    ap.add_argument("--reps", type=int, default=20)
    ap.add_argument("--m0", type=float, default=-0.6)
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--solver", default="mixed_f32", help="solve: comma list of f64, mixed_f32, mixed_f16, mixed_bf16")
    ap.add_argument("--inner-tol", type=float, default=1e-5)
    ap.add_argument("--engine", default="persistent", choices=["persistent", "kernels"],
                    help="solve: one persistent launch per (inner) solve, or one kernel per BiCGStab step")
    ap.add_argument("--eps", type=float, default=0.7)
    ap.add_argument("--gauge-seed", type=int, default=1001)
    ap.add_argument("--eval-lattice", default="24,24,24,48", help="learned: evaluation lattice")
    ap.add_argument("--ncolors", type=int, default=512, help="trace: probing colours")
    ap.add_argument("--nvec", type=int, default=512, help="trace: probing vectors of the z0 run")
    ap.add_argument("--block", type=int, default=32, help="trace: right-hand sides per block")
    ap.add_argument("--steps", type=int, default=200, help="learned: Adam steps")
    ap.add_argument("--batch", type=int, default=8, help="learned: pairs per step")
    ap.add_argument("--pool", type=int, default=16, help="learned: batches of independent pairs")
    ap.add_argument("--net-precision", default="bf16", choices=["bf16", "f32"],
                    help="learned: kernels used for training (bf16: tensor cores)")
    ap.add_argument("--stream-pairs", type=int, default=0,
                    help="learned: train on this many distinct pairs, a fresh batch from new solves every step")
    ap.add_argument("--degree", type=int, default=16, help="eig: Chebyshev degree")
    ap.add_argument("--iters", type=int, default=60, help="eig: iterations at most")
    ap.add_argument("--tol", type=float, default=1e-2, help="eig: relative residual target")
    ap.add_argument("--time-limit", type=float, default=0.0, help="eig: stop after this many seconds")
    ap.add_argument("--device-gauge", action="store_true", help="eig, solve: generate the gauge field on the device")
    a = ap.parse_args(argv)
    import torch
    torch.cuda.set_device(0)
    from . import build as _b
    if not os.path.exists(_b.LIB):
        _b.build()
    from . import dtr
    dims = tuple(int(x) for x in a.lattice.split(","))
    if a.what == "trace":
        for row in trace_case(dims, a.eps, a.m0, a.gauge_seed, int(a.k), a.prec, a.ncolors, a.nvec, a.block,
                              a.solver.split(",")):
            print(json.dumps(row), flush=True)
        return
    if a.what == "learned":
        ev = tuple(int(v) for v in a.eval_lattice.split(","))
        print(json.dumps(learned_case(dims, ev, a.eps, a.m0, a.gauge_seed, a.steps, a.batch, a.pool,
                                      int(a.nrhs.split(",")[0]), stream_pairs=a.stream_pairs,
                                      precision=a.net_precision)), flush=True)
        return
    if a.what == "eig":
        for prec in a.prec.split(","):
            print(json.dumps(eig_case(dims, a.eps, a.m0, a.gauge_seed, int(a.k), prec, a.degree, a.iters, a.tol,
                                      a.time_limit, a.device_gauge)), flush=True)
        return
    if a.what == "deflate":
        for prec in a.prec.split(","):
            for kk in a.k.split(","):
                for n in a.nrhs.split(","):
                    print(json.dumps(deflate_case(dims, int(kk), int(n), a.reps, prec)), flush=True)
        return
    if a.what == "net":
        for n in a.nrhs.split(","):
            print(json.dumps(net_case(dims, int(n), a.reps)), flush=True)
        return
    lat = dtr.make_lattice(dims)
    if a.what == "solve":
        from . import synth
        g = dtr.make_gauge(lat, a.eps, a.gauge_seed) if a.device_gauge else \
            dtr.gauge_from_host(lat, synth.random_su3_links(dims, a.eps, a.gauge_seed))
        for solver in a.solver.split(","):
            for n in a.nrhs.split(","):
                print(json.dumps(solve_case(g, dims, int(n), a.reps, a.m0, graph=not a.no_graph, solver=solver,
                                            inner_tol=a.inner_tol, engine=a.engine)), flush=True)
        return
    g = dtr.gauge_from_host(lat, tiled_links(dims))
    for prec in a.prec.split(","):
        for n in a.nrhs.split(","):
            print(json.dumps(dslash_case(g, dims, prec, int(n), a.reps)), flush=True)


if __name__ == "__main__":
    main()
