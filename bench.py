#!/usr/bin/env python3
"""Benchmark of the deflated hierarchical-probing trace estimator (Algorithm 1).

Headline workload (the largest that fits one GB300), wilson32x32x32x64_hp512x8_k1000:
32^3x64 lattice (N = 25,165,824), eps 0.8, m0 -0.78, gauge seed 1003 (links
generated on the device), k = 1000 deflation vectors stored in BF16 and built on
the device by the setup eigensolver, 512 hierarchical-probing vectors per z0 run,
mixed-precision batched solves (FP32 inner BiCGStab in FP64 defect correction,
CUDA-graph captured) to a true relative residual of 1e-10, launch shape (RHS
block 8-64 and concurrent lanes) chosen by the library's autotuner.

One step = one wave of the whole path over W = lanes x block probing vectors of
one z0 run (noise + HP mask, deflation projection, batched solves, FP64 z^H y
reductions): 512 / W consecutive steps make one run of Algorithm 1.  Metric:
right-hand sides solved per second, plus variance x time to a 1e-3 relative
trace error for this path and for the plain FP64 GPU path on the same seeds.
The 8^4 workload (wilson8x8x8x8_hp16x256_k100) is measured the same way and
reported under "extra".

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the program the CUDA path is checked
against) on bounded samples of the same workload.  Under torchrun (N > 1) every
rank runs its own z0 runs (weak scaling, no data-path collective); rank 0 prints.
"""
import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "wilson32x32x32x64_hp512x8_k1000"
SMALL = "wilson8x8x8x8_hp16x256_k100"
METRIC = "RHS solves/s (deflated HP Tr(A^-1) estimator, true residual 1e-10)"
UNIT = "RHS/s"
L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--eig-time", type=float, default=45.0,
                    help="wall-time cap (s) of the 32^3x64 setup eigensolver (untimed setup)")
    ap.add_argument("--eig-iters", type=int, default=40, help="iteration cap of the setup eigensolvers")
    ap.add_argument("--eig-degree", type=int, default=48, help="Chebyshev degree of the setup eigensolvers")
    ap.add_argument("--f64-steps", type=int, default=2, help="steps of the plain FP64 path timed for comparison")
    ap.add_argument("--var-runs", type=int, default=2, help="complete z0 runs of 512 vectors for Var_T")
    ap.add_argument("--small-steps", type=int, default=48, help="timed steps of the 8^4 workload (extra)")
    ap.add_argument("--skip-small", action="store_true", help="skip the 8^4 workload")
    ap.add_argument("--skip-learned", action="store_true", help="skip the learned-preconditioner line (16^3x32)")
    ap.add_argument("--learned-pairs", type=int, default=20000,
                    help="distinct (residual, error) pairs the network trains on in the bench (streamed: a fresh "
                         "batch of 16 from new solves every Adam step)")
    ap.add_argument("--skip-kernels", action="store_true", help="skip the standalone kernel roofline lines")
    ap.add_argument("--skip-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-autotune", action="store_true", help="use --block/--lanes instead of the autotuner")
    ap.add_argument("--solver", default="auto", choices=["auto", "mixed_f32", "mixed_f16"],
                    help="inner-solve storage of the mixed solver (auto: the faster on one timed wave)")
    ap.add_argument("--block", type=int, default=32)
    ap.add_argument("--lanes", type=int, default=1)
    ap.add_argument("--cpu-procs", type=int, default=0, help="CPU oracle processes (0: cores, memory permitting)")
    ap.add_argument("--ref-lattice", default="", help="reference arm: lattice of the oracle samples (default: the "
                                                       "workload's 32^3x64)")
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven solver cycles instead of the CUDA graph (same kernels and results; lets a "
                         "profiler list the kernels of the solver loop)")
    return ap.parse_args()


def measured_peaks():
    """HBM copy bandwidth (GB/s) measured on the GB300s, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "hbm_gbs of MEASURED_PEAKS.json (of measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "6.8 TB/s fallback (MEASURED_PEAKS.json absent; of fallback)"


def log(what, **kw):
    """Progress record on stderr (the result line goes to stdout at the end)."""
    sys.stderr.write(json.dumps(dict(stage=what, **kw)) + "\n")
    sys.stderr.flush()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms in a thread."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------- CPU oracle
# The oracle as it stands, on the host cores, on bounded samples of the 32^3x64
# workload: its operator (oracle.wilson.apply_at, the per-site coding) applied at
# every 16th site of a 32^3x64 field in each process, extrapolated to the whole
# field; the right-hand side's cost is (2 x iterations + 2) applications in its
# CGNR, with the iteration count from its CGNR to 1e-10 at 8^4 (same eps, m0).
SAMPLE_STRIDE = 16
_CPU_STATE = {}


def _links_chunk(args):
    path, eps, seed, s0, s1 = args
    sys.path.insert(0, ROOT)
    from oracle import gauge
    out = np.load(path, mmap_mode="r+")
    sites = np.repeat(np.arange(s0, s1), 4)
    mu = np.tile(np.arange(4), s1 - s0)
    out[s0:s1] = gauge.links_at(seed, eps, sites, mu).reshape(s1 - s0, 4, 3, 3)
    out.flush()
    return s1 - s0


def _cpu_links_file(dims, eps, seed, pool):
    """The device generator's field drawn by the oracle (counter-based), shared by the workers."""
    path = os.path.join(tempfile.gettempdir(), "dtr_links_%s_%g_%d.npy" % ("x".join(map(str, dims)), eps, seed))
    if not os.path.exists(path):
        V = int(np.prod(dims))
        tmp = path + ".%d.tmp.npy" % os.getpid()
        np.lib.format.open_memmap(tmp, mode="w+", dtype=np.complex128, shape=(V, 4, 3, 3)).flush()
        step = max(1, V // 64)
        pool.map(_links_chunk, [(tmp, eps, seed, s0, min(V, s0 + step)) for s0 in range(0, V, step)])
        os.replace(tmp, path)
    return path


def _cpu_sample(args):
    """Time the oracle's operator at every SAMPLE_STRIDE-th site of the field (one process)."""
    links_path, dims, m0, q = args
    os.environ["OMP_NUM_THREADS"] = "1"
    sys.path.insert(0, ROOT)
    from oracle import wilson
    if _CPU_STATE.get("key") != (links_path, q):
        N = 12 * int(np.prod(dims))
        rng = np.random.default_rng(q)
        _CPU_STATE.update(key=(links_path, q), U=np.load(links_path, mmap_mode="r"),
                          psi=rng.standard_normal(N) + 1j * rng.standard_normal(N))
    V = int(np.prod(dims))
    sites = np.arange(q % SAMPLE_STRIDE, V, SAMPLE_STRIDE)
    t0 = time.perf_counter()
    wilson.apply_at(_CPU_STATE["U"], dims, m0, _CPU_STATE["psi"], sites)
    return (time.perf_counter() - t0) * V / len(sites)   # one whole-field application


def _cgnr_iterations_8x8(eps, m0, seed):
    """CGNR iterations to 1e-10 for the same (eps, m0) at 8^4 (explicit matrix), with the time per RHS."""
    from oracle import gauge, noise, solve, wilson
    dims = (8, 8, 8, 8)
    U = gauge.random_su3_links(dims, eps, seed)
    A = wilson.explicit(U, dims, m0)
    z = noise.noise_vectors(dims, 0, 0, 16, False, 0, 1)[:, 0]
    t0 = time.perf_counter()
    _, it, res = solve.cgnr(A, z, tol=1e-10)
    return it, time.perf_counter() - t0


def cpu_procs(requested):
    n = os.cpu_count() or 1
    try:
        with open("/proc/meminfo") as f:
            avail = [int(l.split()[1]) for l in f if l.startswith("MemAvailable")][0] * 1024
    except (OSError, IndexError):
        avail = 16 << 30
    by_mem = max(1, int(avail * 0.25 // (2 << 30)))    # ~1 GB per worker at 32^3x64; a quarter of free memory
    p = min(n, by_mem, 32)
    if requested > 0:
        p = min(p, requested)
    return max(1, p)


def _cpu_model():
    try:
        with open("/proc/cpuinfo") as f:
            for l in f:
                if l.lower().startswith(("model name", "cpu part")):
                    return l.split(":", 1)[1].strip()
    except OSError:
        pass
    return None


class CpuOracle:
    """A pool of spawned oracle processes on the 32^3x64 workload (or `dims`)."""

    def __init__(self, nprocs, dims=None):
        w = _workload(WORKLOAD)
        self.dims = tuple(dims) if dims else w.dims
        self.m0, self.n = w.m0, nprocs
        self.pool = mp.get_context("spawn").Pool(nprocs)
        self.path = _cpu_links_file(self.dims, w.eps, w.gauge_seed, self.pool)
        self.iters, self.t8 = _cgnr_iterations_8x8(w.eps, w.m0, w.gauge_seed)

    def step(self):
        """All processes at once; returns (wall seconds, mean whole-field application seconds)."""
        t0 = time.perf_counter()
        ts = self.pool.map(_cpu_sample, [(self.path, self.dims, self.m0, q) for q in range(self.n)])
        return time.perf_counter() - t0, float(np.mean(ts))

    def rhs_per_s(self, t_apply):
        return self.n / (t_apply * (2 * self.iters + 2))

    def sample_note(self, t_apply):
        return ("extrapolated per RHS: %d processes, each the FP64 oracle's operator (per-site coding) at every %dth "
                "site of a %s field, scaled to one whole-field application (%.2f s); RHS cost = (2 x %d + 2) "
                "applications, %d = the oracle's CGNR iterations to 1e-10 at 8^4 with the same eps and m0"
                % (self.n, SAMPLE_STRIDE, "x".join(map(str, self.dims)), t_apply, self.iters, self.iters))

    def close(self):
        self.pool.close()
        self.pool.join()


def cpu_oracle_baseline(nprocs, reps=3, dims=None):
    o = CpuOracle(nprocs, dims)
    try:
        t_apply = min(o.step()[1] for _ in range(reps))
        return {"value": o.rhs_per_s(t_apply), "cores": nprocs, "t_apply_s": t_apply, "cgnr_iterations": o.iters,
                "nproc": os.cpu_count(), "cpu_model": _cpu_model(), "sample": o.sample_note(t_apply)}
    finally:
        o.close()


def _workload(name):
    from paper_1603_05988_gb300 import synth
    return synth.WORKLOADS[name]


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    n = cpu_procs(args.cpu_procs)
    dims = tuple(int(x) for x in args.ref_lattice.split(",")) if args.ref_lattice else None
    o = CpuOracle(n, dims)
    try:
        walls, applies = [], []
        for s in range(args.warmup + args.steps):
            wt, ta = o.step()
            if s >= args.warmup:
                walls.append(wt)
                applies.append(ta)
        t_apply = float(np.mean(applies))
        value = o.rhs_per_s(t_apply)
        note = o.sample_note(t_apply)
    finally:
        o.close()
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(walls) / len(walls),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "lattice": list(o.dims),
                   "step": "%d oracle processes, one sampled operator application each" % n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": n, "kind": "oracle", "sample": note,
                         "nproc": os.cpu_count(), "cpu_model": _cpu_model()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU path
def persistent_roofline(prof, sms, lanes, wall_ms, block, hbm_peak, hbm_note, workload, vec_bytes=96):
    """Roofline of the persistent BiCGStab kernel from its device-timed launches.
    Algorithmic bytes per site, RHS and iteration: the fused minimum of one BiCGStab
    iteration, two stencils (a vector in + a vector out + 288 / b B of FP32 links each)
    and six vector passes, a vector being 96 B per site and RHS in FP32 storage and 48 B
    in FP16; flops 2 x 1368 + 12 x 104."""
    bytes_unit = 2 * (2 * vec_bytes + 288.0 / block) + 6 * vec_bytes
    flop_unit = 2 * 1368.0 + 12 * 104.0
    n = max(prof["launches"], 1)
    pms = prof["ms"] / n
    units = prof["site_rhs_iterations"] / n
    gbs = units * bytes_unit / (pms / 1e3) / 1e9 if pms > 0 else 0.0
    tfl = units * flop_unit / (pms / 1e3) / 1e12 if pms > 0 else 0.0
    grid = sms // lanes if lanes > 1 else sms
    share = grid / sms
    fp32_peak = sms * 128 * 2 * 2.07e9 / 1e12
    # DRAM bytes per site, RHS and iteration of the same kernel under ncu (16^3x32, 16 RHS, FP16
    # storage: profiles/persistent_bicgstab_f16_16x16x16x32_b16.md), scaled to this launch's units;
    # the FP32-storage counters predate the current kernel, so none is given for it
    traffic, traffic_note = None, "no capture of the current FP32-storage kernel"
    if vec_bytes == 48 and block == 16:
        traffic = 848.0 * units
        traffic_note = ("848 B per site, RHS and iteration (ncu DRAM read + write at 16^3x32, 16 RHS, FP16 storage) "
                        "x this launch's site-RHS-iterations")
    return {"bound": "hbm", "achieved": gbs, "peak": hbm_peak * share, "unit": "GB/s", "frac": gbs / (hbm_peak * share),
            "traffic": traffic, "traffic_note": traffic_note,
            "kernel": "k_bicgstab_persistent (%s-stored inner BiCGStab, %d RHS, %s)"
                                       % ("FP32" if vec_bytes == 96 else "FP16", block, workload),
            "avg_launch_ms": pms, "launches": prof["launches"], "alg_bytes_per_launch": units * bytes_unit,
            "alg_bytes_note": "%.0f B per site, RHS and iteration (two stencils 2 x (%d + %d + 288/%d) + six "
                              "%d B vector passes: the fused minimum) x site-RHS-iterations of the launch"
                              % (bytes_unit, vec_bytes, vec_bytes, block, vec_bytes),
            "peak_note": hbm_note + "; times the launch's SM share %d/%d" % (grid, sms),
            "fp32": {"achieved_tflops": tfl, "peak_tflops": fp32_peak * share, "frac": tfl / (fp32_peak * share),
                     "note": "3984 flop per site, RHS and iteration; FP32 peak = SMs x 128 x 2 x 2.07 GHz (nominal)"},
            "aggregate_gbs": prof["site_rhs_iterations"] * bytes_unit / (wall_ms / 1e3) / 1e9 if wall_ms else None,
            "ctas_per_launch": grid, "concurrent_launches": lanes}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1603_05988_gb300 import build as _build
    if not os.path.exists(_build.LIB):
        _build.build()
    from paper_1603_05988_gb300 import dtr, synth

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(x):
        if world == 1:
            return x
        t = torch.tensor([x], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        return float(t.item())

    hbm_peak, hbm_note = measured_peaks()
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    w = synth.WORKLOADS[WORKLOAD]
    ncol = w.ncolors                                   # 512 probing vectors per run

    # ---------------------------------------------------------------- setup
    lat = dtr.make_lattice(w.dims)
    t0 = time.perf_counter()
    gauge = dtr.make_gauge(lat, w.eps, w.gauge_seed)
    t_gauge = time.perf_counter() - t0
    ep = dtr.eig_params(w.k, store=w.defl_prec, tol=1e-2, degree=args.eig_degree, max_iter=args.eig_iters,
                        time_limit_s=args.eig_time, seed=rank)
    defl, eres, est = dtr.eig_deflation(gauge, w.m0, ep)
    torch.cuda.empty_cache()
    log("32^3x64 setup", **{k_: est[k_] for k_ in ("iterations", "converged", "seconds", "max_residual", "t_filter",
                                                   "t_gram", "t_host", "t_rotate")})
    bound = (abs(4.0 + w.m0) + 4.0)
    lam = defl.lambdas()
    rn = eres * np.abs(lam) / bound                    # the same residuals relative to the bound on ||A||
    setup = {"gauge_s": t_gauge, "eigensolver": {k_: est[k_] for k_ in ("iterations", "converged", "basis", "seconds",
                                                                         "max_residual")},
             "residual_median": float(np.median(eres)),
             "residual_vs_norm": {"max": float(rn.max()), "median": float(np.median(rn)),
                                  "below_1e-2": int(np.sum(rn <= 1e-2))},
             "abs_lambda_range": [float(np.abs(lam).min()), float(np.abs(lam).max())],
             "residual_note": "||Q v - lambda v|| / (|lambda| ||v||), and relative to the bound |4 + m0| + 4 = %.2f "
                              "on ||A|| (the scale of a tolerance stated against the matrix norm)" % bound,
             "eigensolver_workspace_gb": est["workspace_bytes"] / 1e9, "T_D": [defl.T_D().real, defl.T_D().imag]}

    def params(solver, lanes, block, run, vec0, nvec, graph=True):
        return dtr.trace_params(seed=w.noise_seed, z0_first=run, n_z0=1, ncolors=ncol, nvec=nvec, vec_first=vec0,
                                block=block, lanes=lanes,
                                solve=dtr.solve_params(tol=w.tol, solver=solver, graph=graph and not args.no_graph))

    # launch shape: lanes x block, every candidate that fits beside the deflation space
    free, _ = torch.cuda.mem_get_info()
    if args.no_autotune:
        tune = {"lanes": args.lanes, "block": args.block, "table": [], "forced": True}
    else:
        tp = dtr.trace_params(seed=w.noise_seed, z0_first=0, n_z0=1, ncolors=ncol, nvec=ncol, block=0,
                              solve=dtr.solve_params(tol=w.tol, solver="mixed_f32", graph=not args.no_graph))
        tune = dtr.trace_autotune(gauge, w.m0, defl, tp, reps=1, max_workspace_bytes=free - (6 << 30))
        torch.cuda.empty_cache()
    L, B = tune["lanes"], tune["block"]
    log("32^3x64 autotune", lanes=L, block=B, table=tune.get("table"))
    W = L * B                                          # probing vectors per step
    steps_per_run = ncol // W
    wsh = {"ws": dtr.TraceWorkspace(gauge, defl, params("mixed_f32", L, B, 0, 0, W))}   # current workspace
    base = 1 + rank * 100003

    def step(solver, i, g=None):
        run = base + i // steps_per_run
        v0 = (i % steps_per_run) * W
        return dtr.trace_estimate(g or gauge, w.m0, defl, params(solver, L, B, run, v0, W, GRAPH),
                                  workspace=wsh["ws"])

    # inner-solve storage (FP32 or FP16 Krylov vectors) and cycle driver (one CUDA graph per solve
    # with device-side loop control, or host-driven launches of the same kernels): the fastest on a
    # timed wave at this shape (the second of two, the first capturing the graph)
    cands = ["mixed_f32", "mixed_f16"] if args.solver == "auto" else [args.solver]
    graphs = [False] if args.no_graph else [True, False]
    solver_t = {}
    if len(cands) * len(graphs) > 1:
        for c_ in cands:
            for g_ in graphs:
                for rep in range(2):
                    torch.cuda.synchronize()
                    t0 = time.perf_counter()
                    dtr.trace_estimate(gauge, w.m0, defl, params(c_, L, B, 400000 + rep, 0, W, g_),
                                       workspace=wsh["ws"])
                    torch.cuda.synchronize()
                    solver_t["%s/%s" % (c_, "graph" if g_ else "host")] = W / (time.perf_counter() - t0)
        best = max(solver_t, key=solver_t.get)
        SOLVER, GRAPH = best.split("/")[0], best.endswith("graph")
    else:
        SOLVER, GRAPH = cands[0], graphs[0]
    log("32^3x64 solver", choice=SOLVER, graph=GRAPH, rhs_per_s=solver_t)
    # warm-up on runs of their own
    for i in range(args.warmup):
        dtr.trace_estimate(gauge, w.m0, defl, params(SOLVER, L, B, 500000 + i, 0, W, GRAPH), workspace=wsh["ws"])
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = dtr.kernel_launches()
    dtr.profile_persistent(1)
    torch.cuda.nvtx.range_push("timed")               # the timed region, for profilers' launch lists
    samples = {}
    ms = []
    iters = 0
    maxres = 0.0
    for i in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        out = step(SOLVER, i)
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
        samples[i] = out["samples"][0]
        iters += out["iterations"]
        maxres = max(maxres, out["max_true_residual"])
        if not out["all_converged"] or out["max_true_residual"] > w.tol:
            raise RuntimeError("step did not converge: %r" % (out["max_true_residual"],))
    torch.cuda.nvtx.range_pop()
    prof = dtr.profile_persistent(0)
    launches = dtr.kernel_launches() - launches0
    barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(ms))
    value = W * args.steps * world / (total_ms / 1e3)

    # complete z0 runs (untimed steps beyond the timed ones) for the run-to-run variance
    nvar = max(args.var_runs, 1) * steps_per_run
    for i in range(args.steps, nvar):
        samples[i] = step(SOLVER, i)["samples"][0]
    td = defl.T_D()
    traces = []
    for r in range(max(args.var_runs, 1)):
        t_r = np.concatenate([samples[r * steps_per_run + j] for j in range(steps_per_run)])
        traces.append(td + t_r.mean())
    tr_mean = complex(np.mean(traces))
    var_T = float(np.sum(np.abs(np.array(traces) - tr_mean) ** 2) / max(len(traces) - 1, 1))

    log("32^3x64 mixed", solver=SOLVER, value=value, ms_per_step=total_ms / args.steps, lanes=L, block=B,
        iterations_per_rhs=iters / (args.steps * W), var_T=var_T, trace=[tr_mean.real, tr_mean.imag])
    # plain FP64 path on the same seeds (the first steps of the timed sequence), in its own workspace
    wsh["ws"] = None
    torch.cuda.empty_cache()
    wsh["ws"] = dtr.TraceWorkspace(gauge, defl, params("f64", L, B, 0, 0, W))
    ms64, diff = [], 0.0
    step("f64", 0)                                     # warm-up
    for i in range(args.f64_steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        o64 = step("f64", i)
        e1.record()
        torch.cuda.synchronize()
        ms64.append(e0.elapsed_time(e1))
        diff = max(diff, float(np.abs(o64["samples"][0] - samples[i]).max() / np.abs(samples[i]).max()))
    value64 = W * args.f64_steps / (sum(ms64) / 1e3)
    log("32^3x64 fp64", value=value64, max_rel_sample_diff=diff)
    wsh["ws"] = None
    torch.cuda.empty_cache()
    wsh["ws"] = dtr.TraceWorkspace(gauge, defl, params("mixed_f32", L, B, 0, 0, W))
    t_run = ncol / value * world
    t_run64 = ncol / value64
    ttr = t_run * var_T / (1e-3 * abs(tr_mean)) ** 2
    ttr64 = t_run64 * var_T / (1e-3 * abs(tr_mean)) ** 2

    # end to end through the public API: the gauge links uploaded from pinned host memory,
    # then the same steps, each reading its samples and run traces back to the host
    U_host = gauge.to_host()
    U_pin = torch.empty((lat.V, 4, 3, 3, 2), dtype=torch.float64, pin_memory=True)
    U_pin.numpy()[:] = U_host.view(np.float64).reshape(lat.V, 4, 3, 3, 2)
    del U_host
    U_np = U_pin.numpy().view(np.complex128).reshape(lat.V, 4, 3, 3)
    barrier()
    t0 = time.perf_counter()
    gauge_e = dtr.gauge_from_host(lat, U_np)
    for i in range(args.steps):
        o = step(SOLVER, i, g=gauge_e)
        _ = o["samples"].sum()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = W * args.steps * world / e2e_s
    log("32^3x64 e2e", value=e2e_value)
    up_bytes = U_np.nbytes
    del gauge_e, U_pin, U_np

    roof = persistent_roofline(prof, sms, L, total_ms, B, hbm_peak, hbm_note, "32^3x64",
                               vec_bytes=48 if SOLVER == "mixed_f16" else 96)
    head = {
        "value": value, "ms_per_step": total_ms / args.steps, "rhs_per_step": W, "lanes": L, "block": B,
        "iterations_per_rhs": iters / (args.steps * W), "max_true_residual": maxres, "launches": launches,
        "clocks": clk, "roofline": roof, "setup": setup,
        "autotune": {"lanes": L, "block": B, "table": [(c["lanes"], c["block"], round(c["rhs_per_s"], 1))
                                                       for c in tune.get("table", [])]},
        "fp64_path": {"value": value64, "unit": UNIT, "steps": args.f64_steps, "ms_per_step": sum(ms64) / len(ms64),
                      "max_rel_sample_diff_vs_mixed": diff},
        "variance_x_time": {"trace": [tr_mean.real, tr_mean.imag], "var_T": var_T, "runs": len(traces),
                            "time_to_1e-3_s": ttr, "time_to_1e-3_s_fp64_path": ttr64,
                            "speedup_vs_fp64_path": ttr64 / ttr if ttr > 0 else t_run64 / t_run,
                            "note": "Var_T over %d complete runs of 512 vectors (complex form); both paths give the "
                                    "same samples (max relative difference above), so they share Var_T" % len(traces)},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": up_bytes / args.steps,
                "d2h_bytes_per_step": W * 16 + 16,
                "note": "host wall clock: dtr_gauge_from_host of the links from pinned host memory (%d B; "
                        "h2d_bytes_per_step = that / steps), then %d dtr_trace_estimate calls reading samples and "
                        "run traces back to the host; the noise is drawn on the device from (seed, run); the "
                        "deflation space (setup output, %.1f GB) stays resident" % (up_bytes, args.steps,
                                                                                    lat.N * w.k * 4 / 1e9)},
    }
    wsh["ws"] = None
    torch.cuda.empty_cache()

    # ------------------------------------------------------ the 8^4 workload
    small = None
    if not args.skip_small:
        del defl, gauge
        torch.cuda.empty_cache()
        small = measure_small(args, dtr, synth, torch, barrier, max_over_ranks, sms, hbm_peak, hbm_note, rank, world)
        log("8^4", value=small["value"], speedup_vs_fp64_path=small["speedup_vs_fp64_path"],
            setup=small["setup"])

    learned_line = None
    if not args.skip_learned:
        torch.cuda.empty_cache()
        learned_line = measure_learned(args, dtr, synth, torch)
        log("learned", **{k_: v for k_, v in learned_line.items() if k_ in ("rhs_per_s", "speedup_vs_fp64_path")})

    # ------------------------------------------- standalone kernel rooflines
    kern = {} if args.skip_kernels else kernel_rooflines(dtr, hbm_peak, hbm_note)
    log("kernels", **{k_: round(v["frac"], 4) for k_, v in kern.items()})

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        c = cpu_oracle_baseline(cpu_procs(args.cpu_procs))
        cpu = dict(c, unit=UNIT, kind="oracle")

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": ("f16" if SOLVER == "mixed_f16" else "f32") + "+f64 (%s-stored inner BiCGStab with FP32 "
                     "arithmetic, FP64 defect correction; BF16 deflation space with FP64 accumulation; FP64 "
                     "reductions)" % ("FP16" if SOLVER == "mixed_f16" else "FP32"),
            "data": "synthetic (random SU(3) links generated on the device, seeded)",
            "config": {"workload": WORKLOAD, "lattice": list(w.dims), "eps": w.eps, "m0": w.m0, "k": w.k,
                       "defl_prec": w.defl_prec, "ncolors": ncol, "rhs_per_step": W, "block": B, "lanes": L,
                       "tol": w.tol, "solver": SOLVER, "solver_wave_rhs_per_s": solver_t,
                       "graph": GRAPH,
                       "l2": "inputs far larger than L2 (V 100.7 GB, one 32-RHS FP64 field 12.9 GB)",
                       "step": "one wave of %d probing vectors of a z0 run (%d steps per run of 512)"
                               % (W, steps_per_run)},
            "clocks": clk,
            "e2e": head["e2e"],
            "gpu_launches": launches,
            "roofline": roof,
            "cpu_baseline": cpu,
            "setup": setup,
            "autotune": head["autotune"],
            "iterations_per_rhs": head["iterations_per_rhs"],
            "fp64_path": head["fp64_path"],
            "variance_x_time": head["variance_x_time"],
            "speedup_vs_fp64_path": value / value64,
            "extra": {"wilson8x8x8x8_hp16x256_k100": small, "learned_16x16x16x32": learned_line, **kern},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def measure_small(args, dtr, synth, torch, barrier, max_over_ranks, sms, hbm_peak, hbm_note, rank, world):
    """The 8^4 workload: 16-colour HP runs in 16-RHS blocks, k = 100 FP64 deflation
    vectors from the GPU eigensolver, L z0 runs in flight per step (autotuned)."""
    w = synth.WORKLOADS[SMALL]
    lat = dtr.make_lattice(w.dims)
    gauge = dtr.gauge_from_host(lat, synth.random_su3_links(w.dims, w.eps, w.gauge_seed))
    ep = dtr.eig_params(w.k, store="f64", tol=1e-2, degree=48, max_iter=max(args.eig_iters, 60), seed=rank)
    defl, eres, est = dtr.eig_deflation(gauge, w.m0, ep)

    def params(solver, z0, lanes):
        return dtr.trace_params(seed=w.noise_seed, z0_first=z0, n_z0=lanes, ncolors=w.ncolors, nvec=w.ncolors,
                                block=w.block, solve=dtr.solve_params(tol=w.tol, solver=solver,
                                                                      graph=not args.no_graph), lanes=lanes)
    lanes = {}
    tables = {}
    for s_ in ("mixed_f32", "f64"):
        t = dtr.trace_autotune(gauge, w.m0, defl, params(s_, 0, 1), reps=3 if s_ == "mixed_f32" else 1)
        lanes[s_] = t["lanes"]
        tables[s_] = [(c["lanes"], round(c["rhs_per_s"])) for c in t["table"]]
    wss = {s_: dtr.TraceWorkspace(gauge, defl, params(s_, 0, lanes[s_])) for s_ in lanes}
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    base = rank * 1000003

    def run_steps(solver, nsteps, first):
        L = lanes[solver]
        ms, traces, iters = [], [], 0
        for i in range(nsteps):
            flush.fill_(i & 0xFF)                       # evict L2 between timed steps
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            out = dtr.trace_estimate(gauge, w.m0, defl, params(solver, first + i * L, L), workspace=wss[solver])
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
            traces.extend(out["trace_runs"])
            iters += out["iterations"]
            if not out["all_converged"] or out["max_true_residual"] > w.tol:
                raise RuntimeError("8^4 step did not converge")
        return ms, traces, iters

    L = lanes["mixed_f32"]
    run_steps("mixed_f32", args.warmup, base + 900000)
    barrier()
    dtr.profile_persistent(1)
    ms, traces, iters = run_steps("mixed_f32", args.small_steps, base)
    prof = dtr.profile_persistent(0)
    total_ms = max_over_ranks(sum(ms))
    value = w.ncolors * L * args.small_steps * world / (total_ms / 1e3)
    L64 = lanes["f64"]
    nf = max(1, min(6, (args.small_steps * L) // L64))
    run_steps("f64", 1, base + 900000)
    ms64, traces64, _ = run_steps("f64", nf, base)
    value64 = w.ncolors * L64 * nf / (sum(ms64) / 1e3)
    ncmp = min(len(traces), len(traces64))
    tdiff = max(abs(a - b) / abs(b) for a, b in zip(traces[:ncmp], traces64[:ncmp]))
    tr_mean = complex(np.mean(traces))
    var_T = float(np.sum(np.abs(np.array(traces) - tr_mean) ** 2) / (len(traces) - 1))
    t_run = (total_ms / (args.small_steps * L)) / 1e3
    t_run64 = (sum(ms64) / (nf * L64)) / 1e3
    # roofline: at 8^4 the persistent kernel is L2-resident and latency-bound; against its SM share of FP32
    fp32_peak = sms * 128 * 2 * 2.07e9 / 1e12
    flop_unit = 2 * 1368.0 + 12 * 104.0
    n = max(prof["launches"], 1)
    pms = prof["ms"] / n
    achieved = prof["site_rhs_iterations"] * flop_unit / n / (pms / 1e3) / 1e12 if pms > 0 else 0.0
    grid = sms // L if L > 1 else sms
    return {"value": value, "unit": UNIT, "steps": args.small_steps, "ms_per_step": total_ms / args.small_steps,
            "rhs_per_step": w.ncolors * L, "lanes": L, "block": w.block, "autotune": tables,
            "iterations_per_rhs": iters / (args.small_steps * w.ncolors * L),
            "setup": {"eigensolver": {k_: est[k_] for k_ in ("iterations", "converged", "seconds", "max_residual")},
                      "tol": 1e-2},
            "fp64_path": {"value": value64, "lanes": L64, "steps": nf, "max_rel_trace_diff_vs_mixed": tdiff},
            "speedup_vs_fp64_path": value / value64,
            "variance_x_time": {"var_T": var_T, "runs": len(traces),
                                "time_to_1e-3_s": t_run * var_T / (1e-3 * abs(tr_mean)) ** 2,
                                "time_to_1e-3_s_fp64_path": t_run64 * var_T / (1e-3 * abs(tr_mean)) ** 2,
                                "speedup_vs_fp64_path": t_run64 / t_run},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak * grid / sms, "unit": "TFLOP/s",
                         "frac": achieved / (fp32_peak * grid / sms),
                         "kernel": "k_bicgstab_persistent (FP32 inner solve, 16 RHS, 8^4, L2-resident)",
                         "avg_launch_ms": pms, "launches": prof["launches"], "ctas_per_launch": grid},
            "l2": "flushed (256 MiB write) before every timed step"}


def measure_learned(args, dtr, synth, torch):
    """The learned preconditioner on the 16^3x32 workload (eps 0.8, m0 -0.75, k = 200 FP32
    deflation vectors from the setup eigensolver, 512-colour HP runs, 32-RHS blocks): the
    network is trained on the GPU on `learned_pairs` distinct (residual, error) pairs drawn from
    the library's own solves, then one run's first blocks are solved by FGMRES(16) with the
    network, FGMRES(16) without it, the mixed FP32 BiCGStab and the plain FP64 BiCGStab on the
    same seeds.  All four give the same samples, so variance x time compares as time per RHS."""
    from paper_1603_05988_gb300 import learned
    w = synth.WORKLOADS["wilson16x16x16x32_hp512x4_k200"]
    lat = dtr.make_lattice(w.dims)
    g = dtr.gauge_from_host(lat, synth.random_su3_links(w.dims, w.eps, w.gauge_seed))
    defl, _, est = dtr.eig_deflation(g, w.m0, dtr.eig_params(w.k, store=w.defl_prec, tol=1e-2, degree=48,
                                                             max_iter=60))
    net = dtr.Net(lat, act=0, init_scale=1.0 / (4.0 + w.m0), noise=1e-3, seed=1)
    hist, t_solve, t_train = learned.train_stream(net, g, w.m0, pairs=args.learned_pairs, batch=16)
    # one network application to 16 right-hand sides with each kernel set (CUDA events)
    xa = torch.cat([dtr.gen_noise(lat, 4242, k, 1, False, 0, 1) for k in range(16)])
    napply = {}
    for prec in ("bf16", "f32"):
        net.set_precision(prec)
        net.apply(xa)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(5):
            net.apply(xa)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        napply[prec] = {"ms": ms, "useful_tflops": 4 * 93312.0 * lat.V * 16 / (ms * 1e-3) / 1e12}
    net.set_precision("bf16")
    napply["note"] = ("4 layers x 93,312 flop per site and RHS (81 offsets x 24 x 24 x 2); bf16 = tensor-core "
                      "convolutions with BF16 layer inputs (M = 128 sites, N = 32 of which 24 real, five K = 16 MMAs "
                      "per 3 offsets: 1.48x the useful flops issued), f32 = CUDA-core FP32")
    solvers = {"fgmres_learned": dtr.solve_params(tol=w.tol, solver="fgmres_net", net=net, gmres_m=16),
               "fgmres_plain": dtr.solve_params(tol=w.tol, solver="fgmres_net", net=None, gmres_m=16),
               "mixed_f32": dtr.solve_params(tol=w.tol, solver="mixed_f32"),
               "f64": dtr.solve_params(tol=w.tol, solver="f64")}
    B = w.block
    out = {"workload": w.name, "pairs": args.learned_pairs, "train_steps": len(hist), "train_solve_s": t_solve,
           "train_step_s": t_train, "loss_first": float(np.mean(hist[:4])), "loss_last": float(np.mean(hist[-4:])),
           "eigensolver": {k_: est[k_] for k_ in ("iterations", "converged", "max_residual", "seconds")},
           "network_apply_16rhs": napply,
           "rhs_per_s": {}, "iterations_per_rhs": {}, "steps": 2}
    samples = {}
    for name, sp in solvers.items():
        p = dtr.trace_params(seed=w.noise_seed, z0_first=1, n_z0=1, ncolors=w.ncolors, nvec=B, block=B, solve=sp)
        ws = dtr.TraceWorkspace(g, defl, p)
        dtr.trace_estimate(g, w.m0, defl, p, workspace=ws, allow_notconv=True)          # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        its, smp = 0, []
        for i in range(2):
            p.vec_first = i * B
            o = dtr.trace_estimate(g, w.m0, defl, p, workspace=ws)
            its += o["iterations"]
            smp.append(o["samples"][0])
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out["rhs_per_s"][name] = 2 * B / dt
        out["iterations_per_rhs"][name] = its / (2 * B)
        samples[name] = np.concatenate(smp)
        del ws
    ref = samples["f64"]
    out["max_rel_sample_diff_vs_fp64"] = {n: float(np.abs(v - ref).max() / np.abs(ref).max())
                                           for n, v in samples.items() if n != "f64"}
    out["variance_x_time_speedup_vs_fp64_path"] = {n: out["rhs_per_s"][n] / out["rhs_per_s"]["f64"]
                                                   for n in solvers if n != "f64"}
    out["note"] = ("variance x time ratio = RHS/s ratio (identical samples); the network sees no links, so at this "
                   "disorder it learns little (the weak-disorder gains kbench learned measures do not carry over)")
    return out


def kernel_rooflines(dtr, hbm_peak, hbm_note):
    """Standalone kernels: the BF16-storage stencil (HBM) and the FP64 stencil (FP64 pipe) at
    32^3x64, and the tensor-core deflation contraction (HBM) at 16^3x32."""
    from paper_1603_05988_gb300 import kbench
    out = {}
    dims = (32, 32, 32, 64)
    lat = dtr.make_lattice(dims)
    g = dtr.make_gauge(lat, 0.8, 1003)
    hb = kbench.dslash_case(g, dims, "bf16", 1, 30)
    out["roofline_stencil_bf16_hbm"] = {
        "bound": "hbm", "achieved": hb["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
        "frac": hb["achieved_gbs"] / hbm_peak, "traffic": 4.946e8 if hb["link_rows"] == 3 else None,
        "traffic_note": "DRAM read + write of one launch under ncu (407.4 + 87.2 MB): "
                        "profiles/dslash_half_bf16_32x32x32x64.md",
        "kernel": "dslash BF16 storage, FP32 math, 1 RHS, 32^3x64", "avg_launch_ms": hb["avg_launch_ms"],
        "alg_bytes_per_launch": hb["alg_bytes_per_launch"],
        "alg_bytes_note": "240 B per site (48 + 48 B spinors, 144 B for four 3x3 BF16 links)", "peak_note": hbm_note}
    f64 = kbench.dslash_case(g, dims, "f64", 16, 5)
    fp64_peak = 1.25
    out["roofline_stencil_fp64_pipe"] = {
        "bound": "alu", "achieved": f64["achieved_tflops"], "peak": fp64_peak, "unit": "TFLOP/s",
        "frac": f64["achieved_tflops"] / fp64_peak, "traffic": None,
        "kernel": "dslash FP64 (the plain FP64 path's stencil), 16 RHS, 32^3x64",
        "avg_launch_ms": f64["avg_launch_ms"], "achieved_gbs": f64["achieved_gbs"],
        "peak_note": "nominal GB300 FP64 rate 1.25 TFLOP/s (no measured FP64 peak on this pool); 1368 flop per "
                     "site and RHS; at 6.7 TB/s the same stencil would need ~9.5 TFLOP/s of FP64"}
    del g, lat
    dc = kbench.deflate_case((16, 16, 16, 32), 256, 16, 20, "bf16")
    vbytes = dc["alg_bytes_per_launch"] - 1572864 * 16 * 16
    out["roofline_deflation_tc_hbm"] = {
        "bound": "hbm", "achieved": vbytes / (dc["avg_launch_ms"] * 1e-3) / 1e9, "peak": hbm_peak, "unit": "GB/s",
        "frac": vbytes / (dc["avg_launch_ms"] * 1e-3) / 1e9 / hbm_peak, "traffic": 1.6427e9,
        "traffic_note": "DRAM read + write of one launch under ncu (1639.6 + 3.1 MB, 1.02x the V bytes): "
                        "profiles/defl_tc_bf16_16x16x16x32_k256_b16.md",
        "kernel": "k_defl_tc (tcgen05 BF16 x Z4 contraction, FP32 accumulation in TMEM), 16^3x32, k=256, 16 RHS",
        "avg_launch_ms": dc["avg_launch_ms"], "alg_bytes_per_launch": vbytes,
        "alg_bytes_note": "V only (N k 4 B): the contraction's algorithmic bytes with Z regenerated from the seed; "
                          "the kernel reads Z as one-byte codes (N b B, 1.6% of V here)",
        "achieved_tflops": dc["achieved_tflops"], "peak_note": hbm_note}
    return out


if __name__ == "__main__":
    sys.exit(main())
