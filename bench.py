#!/usr/bin/env python3
"""Benchmark of the deflated hierarchical-probing trace estimator (Algorithm 1)
on the 8^4 Wilson-Dirac workload: eps 0.7, m0 -0.6, 16-colour hierarchical
probing per Z4 vector z0, blocks of 16 right-hand sides per launch, k = 100
FP64 deflation vectors, solves to a true relative residual of 1e-10.

One step = one wave of L z0 runs of the whole path (noise + HP mask,
deflation projection, 16 batched solves per run, FP64 z^H y reductions and run
statistics) = 16 L right-hand sides, where L (runs in flight at once, each on
its own stream and SM share; every solve is still one 16-RHS block) is chosen
by the library's autotuner before the timed region.  Metric: right-hand sides
solved per second (whole job), plus the variance x time figure of merit (time
to a 1e-3 relative trace error) for the mixed-precision path and for the plain
FP64 path (autotuned the same way) on the same seeds.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the program the CUDA path is
checked against) on a bounded sample of the same workload.  Under torchrun
(N > 1) every rank runs its own z0 runs (weak scaling, no data-path
collective); rank 0 prints the line.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "wilson8x8x8x8_hp16x256_k100"
METRIC = "RHS solves/s (deflated HP Tr(A^-1) estimator, true residual 1e-10)"
UNIT = "RHS/s"
L2_FLUSH_BYTES = 256 << 20   # > 129 MB L2


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=128)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--solver", default="mixed_f32", choices=["mixed_f32", "f64"])
    ap.add_argument("--f64-steps", type=int, default=6, help="steps of the plain FP64 path timed for comparison")
    ap.add_argument("--eig-iters", type=int, default=150,
                    help="cap on setup eigensolver iterations (deflation-space quality; untimed)")
    ap.add_argument("--skip-hbm", action="store_true", help="skip the 32^3x64 half-precision stencil measurement")
    ap.add_argument("--cpu-sample-rhs", type=int, default=16,
                    help="RHS in the CPU-oracle baseline sample (16: about 13 s of one Grace core)")
    ap.add_argument("--lanes", type=int, default=0, help="z0 runs in flight per step (0 = autotune)")
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven solver cycles instead of the CUDA graph (same kernels and results; lets a "
                         "profiler list the kernels of the solver loop)")
    return ap.parse_args()


def measured_hbm_peak():
    """HBM copy bandwidth (GB/s) measured on the GB300s, else the recipe's fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "hbm_gbs of MEASURED_PEAKS.json (of measured)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "6.8 TB/s fallback (MEASURED_PEAKS.json absent; of fallback)"


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
CPU_SAMPLE_CODE = r"""
import json, sys, time
import numpy as np
sys.path.insert(0, sys.argv[1])
from paper_1603_05988_gb300 import synth
from oracle import noise, solve, wilson, deflation
w = synth.WORKLOADS[sys.argv[2]]
nrhs, reps = int(sys.argv[3]), int(sys.argv[4])
U = synth.random_su3_links(w.dims, w.eps, w.gauge_seed)
A = wilson.explicit(U, w.dims, w.m0)
AH = wilson.explicit_dagger(U, w.dims, w.m0)
V = synth.random_orthonormal(w.N, w.k, 0)
sig = np.linspace(0.9, 1.4, w.k)
times = []
for r in range(reps):
    t0 = time.perf_counter()
    Z = noise.noise_vectors(w.dims, w.noise_seed, 100000 + r, w.ncolors, False, 0, nrhs)
    Y, it, res = solve.cgnr(A, Z, tol=w.tol)
    t = np.einsum("ij,ij->j", np.conj(Z), Y) - deflation.quadrature(AH, V, sig, Z)
    times.append(time.perf_counter() - t0)
print(json.dumps({"times": times, "iters": int(it), "res": float(np.max(res))}))
"""


def cpu_oracle_sample(nrhs, reps):
    """Run the FP64 oracle (one thread) on `reps` samples of `nrhs` RHS each."""
    env = dict(os.environ)
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        env[v] = "1"
    out = subprocess.run([sys.executable, "-c", CPU_SAMPLE_CODE, ROOT, WORKLOAD, str(nrhs), str(reps)],
                         capture_output=True, text=True, env=env, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError("CPU oracle sample failed: " + out.stderr[-2000:])
    return json.loads(out.stdout.strip().splitlines()[-1])


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    steps, warm = args.steps, args.warmup
    # one RHS per step: the oracle's Algorithm 1 quadrature on one probing vector
    r = cpu_oracle_sample(1, steps + warm)
    ts = r["times"][warm:]
    value = len(ts) / sum(ts)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1e3 * sum(ts) / len(ts), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "step": "1 RHS (CPU oracle sample)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d steps x 1 RHS at 8^4, CGNR to 1e-10 + deflation quadrature (paper A^H form)"
                                   % steps},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU path
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
    from paper_1603_05988_gb300 import dtr, eigensolver, synth

    w = synth.WORKLOADS[WORKLOAD]
    U = synth.random_su3_links(w.dims, w.eps, w.gauge_seed)
    lat = dtr.make_lattice(w.dims)
    gauge = dtr.gauge_from_host(lat, U)
    t0 = time.perf_counter()
    V, lam, eres, eit = eigensolver.smallest_gamma5_eigpairs(gauge, w.m0, w.k, iters=args.eig_iters, tol=1e-2,
                                                                     seed=rank)
    t_setup = time.perf_counter() - t0
    defl = dtr.defl_create(lat, V, lam, prec=w.defl_prec)

    def params(solver, z0, lanes):
        return dtr.trace_params(seed=w.noise_seed, z0_first=z0, n_z0=lanes, ncolors=w.ncolors, nvec=w.ncolors,
                                block=w.block, solve=dtr.solve_params(tol=w.tol, solver=solver, graph=not args.no_graph),
                                lanes=lanes)

    # launch shape: the library's autotuner times 1, 2, 4, 8 lanes (untimed setup)
    tune = {}
    for s_ in (args.solver, "f64"):
        if s_ in tune:
            continue
        if args.lanes > 0:
            tune[s_] = {"lanes": args.lanes, "block": w.block, "rhs_per_s": None, "table": [], "forced": True}
        else:
            tune[s_] = dtr.trace_autotune(gauge, w.m0, defl, params(s_, 0, 1), reps=3 if s_ == args.solver else 1)
    lanes = {s_: t["lanes"] for s_, t in tune.items()}
    wss = {s_: dtr.TraceWorkspace(gauge, defl, params(s_, 0, lanes[s_])) for s_ in lanes}
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    base = rank * 1000003

    def run_steps(solver, nsteps, first, timed):
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
                raise RuntimeError("step did not converge: %r" % (out["max_true_residual"],))
        return ms, traces, iters

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

    L = lanes[args.solver]
    # warm-up
    run_steps(args.solver, args.warmup, base + 900000, False)
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = dtr.kernel_launches()
    dtr.profile_persistent(1)                          # device-timed persistent solver launches
    torch.cuda.nvtx.range_push("timed")
    ms, traces, iters = run_steps(args.solver, args.steps, base, True)
    torch.cuda.nvtx.range_pop()
    prof = dtr.profile_persistent(0)
    launches = dtr.kernel_launches() - launches0
    barrier()
    clk = clocks.stop()
    total_ms = max_over_ranks(sum(ms))
    rhs_per_step = w.ncolors * L
    value = rhs_per_step * args.steps * world / (total_ms / 1e3)

    # end-to-end through the public calls from host-resident inputs (host wall
    # clock): upload of the gauge field and of the deflation space from host
    # memory, then the steps, each reading its samples and traces back to the host
    V_host, lam_host = np.asarray(V), np.asarray(lam)         # the eigensolver returns host arrays
    barrier()
    t0 = time.perf_counter()
    gauge_e = dtr.gauge_from_host(lat, U)
    defl_e = dtr.defl_create(lat, V_host, lam_host, prec=w.defl_prec)
    t_up = time.perf_counter() - t0
    for i in range(args.steps):
        out = dtr.trace_estimate(gauge_e, w.m0, defl_e, params(args.solver, base + i * L, L),
                                 workspace=wss[args.solver])
        _ = out["samples"].sum()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = rhs_per_step * args.steps * world / e2e_s
    up_bytes = U.size * 16 + V_host.size * 16 + lam_host.size * 8
    del gauge_e, defl_e
    # the same steps with the inputs already resident (per-step public call only)
    barrier()
    t0 = time.perf_counter()
    for i in range(args.steps):
        out = dtr.trace_estimate(gauge, w.m0, defl, params(args.solver, base + i * L, L), workspace=wss[args.solver])
        _ = out["samples"].sum()
    torch.cuda.synchronize()
    e2e_res_value = rhs_per_step * args.steps * world / max_over_ranks(time.perf_counter() - t0)

    # plain FP64 path on the same seeds (reference GPU path of the metric)
    L64 = lanes["f64"]
    nf = max(1, min(args.f64_steps, (args.steps * L) // L64))
    run_steps("f64", 1, base + 900000, False)
    ms64, traces64, iters64 = run_steps("f64", nf, base, True)
    value64 = w.ncolors * L64 * nf / (sum(ms64) / 1e3)
    ncmp = min(len(traces), len(traces64))
    trace_diff = max(abs(a - b) / abs(b) for a, b in zip(traces[:ncmp], traces64[:ncmp]))

    # variance x time: Var_T over the timed runs, t_run the mean time per run
    tr_mean = complex(np.mean(traces))
    var_T = float(np.sum(np.abs(np.array(traces) - tr_mean) ** 2) / (len(traces) - 1))
    t_run = (total_ms / (args.steps * L)) / 1e3
    t_run64 = (sum(ms64) / (nf * L64)) / 1e3
    ttr = t_run * var_T / (1e-3 * abs(tr_mean)) ** 2
    ttr64 = t_run64 * var_T / (1e-3 * abs(tr_mean)) ** 2

    # roofline of the dominant kernel: the persistent BiCGStab kernel (one
    # cooperative launch per inner solve), timed inside the timed region by
    # device global-timer stamps (first block entry to last block exit; the
    # launches sit in CUDA-graph loop bodies, where events cannot be recorded);
    # algorithmic FP32 flops per site, RHS and iteration: two stencils
    # (2 x 1368) plus the fused vector work (12 complex x 104 flops)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    fp32_peak = sms * 128 * 2 * 2.07e9 / 1e12          # TFLOP/s: SMs x FP32 lanes x FMA x max clock
    flop_per_unit = 2 * 1368.0 + 12 * 104.0
    pms = prof["ms"] / max(prof["launches"], 1)
    pflops = prof["site_rhs_iterations"] * flop_per_unit / max(prof["launches"], 1)
    achieved = pflops / (pms / 1e3) / 1e12 if pms > 0 else 0.0
    grid = sms // L if L > 1 else sms                   # CTAs (one per SM) of one launch
    share = grid / sms
    agg = prof["site_rhs_iterations"] * flop_per_unit / (total_ms / 1e3) / 1e12
    roof = {"bound": "alu", "achieved": achieved, "peak": fp32_peak * share, "unit": "TFLOP/s",
            "frac": achieved / (fp32_peak * share), "traffic": 2.978e7,
            "traffic_note": "DRAM read + write of one launch under ncu (26.47 + 3.32 MB), same kernel and problem "
                            "(8^4, 16 RHS) on 152 CTAs: profiles/persistent_bicgstab_f32_8x8x8x8_b16.md",
            "kernel": "k_bicgstab_persistent<float,512,0,float2> (FP32 inner solve, 16 RHS, 8^4, L2-resident)",
            "avg_launch_ms": pms, "launches": prof["launches"], "flops_per_launch": pflops,
            "ctas_per_launch": grid, "concurrent_launches": L,
            "peak_note": "FP32 peak = %d SMs x 128 lanes x 2 flop x 2.07 GHz (of nominal clocks) = %.1f TFLOP/s, "
                         "times the launch's SM share %d/%d" % (sms, fp32_peak, grid, sms),
            "aggregate": {"achieved": agg, "peak": fp32_peak, "frac": agg / fp32_peak,
                          "note": "all persistent-kernel flops in the timed region / timed wall time"},
            "share_note": "share of GPU time in the timed region: profiles/launches_wilson8x8x8x8_hp16x256_k100.md"}

    # the stencil core alone at the bench's shape, and the half-precision stencil
    # on a lattice far larger than L2 (HBM roofline)
    from paper_1603_05988_gb300 import kbench
    st8 = kbench.dslash_case(gauge, w.dims, "f32", w.block, 200)
    roof_stencil = {"bound": "alu", "achieved": st8["achieved_tflops"], "peak": fp32_peak, "unit": "TFLOP/s",
                    "frac": st8["achieved_tflops"] / fp32_peak, "traffic": None,
                    "kernel": "dslash FP32, 16 RHS, 8^4", "avg_launch_ms": st8["avg_launch_ms"]}
    hbm_peak, hbm_note = measured_hbm_peak()
    roof_hbm = roof_tc = None
    if not args.skip_hbm:
        dims_big = (32, 32, 32, 64)
        lat_big = dtr.make_lattice(dims_big)
        g_big = dtr.gauge_from_host(lat_big, kbench.tiled_links(dims_big))
        hb = kbench.dslash_case(g_big, dims_big, "bf16", 1, 30)
        roof_hbm = {"bound": "hbm", "achieved": hb["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
                    "frac": hb["achieved_gbs"] / hbm_peak,
                    "traffic": 4.946e8 if hb["link_rows"] == 3 else None,
                    "traffic_note": "DRAM read + write of one launch under ncu (407.4 + 87.2 MB): "
                                    "profiles/dslash_half_bf16_32x32x32x64.md",
                    "kernel": "dslash BF16 storage, FP32 math, 1 RHS, 32^3x64",
                    "avg_launch_ms": hb["avg_launch_ms"], "alg_bytes_per_launch": hb["alg_bytes_per_launch"],
                    "alg_bytes_note": "240 B per site (48 + 48 B spinors, 144 B for four 3x3 BF16 links); the "
                                      "kernel stores %d rows per link and moves %d B per launch (%.0f GB/s)"
                                      % (hb["link_rows"], hb["stored_bytes_per_launch"], hb["moved_gbs"]),
                    "peak_note": hbm_note}
        del g_big, lat_big
        # the tensor-core (tcgen05) deflation contraction: BF16 V, one 16-column Z4 block
        dc = kbench.deflate_case((16, 16, 16, 32), 256, 16, 20, "bf16")
        roof_tc = {"bound": "hbm", "achieved": dc["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
                   "frac": dc["achieved_gbs"] / hbm_peak, "traffic": 2.0169e9,
                   "kernel": "k_defl_tc (tcgen05 BF16 x Z4 contraction, FP32 accumulation in TMEM), "
                             "16^3x32, k=256, 16 RHS",
                   "avg_launch_ms": dc["avg_launch_ms"], "alg_bytes_per_launch": dc["alg_bytes_per_launch"],
                   "achieved_tflops": dc["achieved_tflops"],
                   "alg_bytes_note": "N k 4 B (V) + N b 16 B (Z) per launch; traffic = DRAM read + write of "
                                     "one launch under ncu (profiles/defl_tc_bf16_16x16x16x32_k256_b16.md)",
                   "tensor_pipe_active_pct": 14.3, "peak_note": hbm_note}

    # CPU oracle baseline on a bounded sample (rank 0, N = 1 only)
    cpu = None
    if rank == 0 and world == 1:
        r = cpu_oracle_sample(args.cpu_sample_rhs, 1)
        tcpu = r["times"][-1]
        cpu = {"value": args.cpu_sample_rhs / tcpu, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": "%d RHS of the 8^4 workload: CGNR to 1e-10 (%d iters) + deflation quadrature, "
                         "%.1f s" % (args.cpu_sample_rhs, r["iters"], tcpu)}

    scal_bytes = 7440
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (FP32 inner BiCGStab, FP64 defect correction, "
                                                            "FP64 deflation and reductions)"
            if args.solver == "mixed_f32" else "f64",
            "data": "synthetic (random SU(3) links, seeded)",
            "config": {"workload": WORKLOAD, "lattice": list(w.dims), "eps": w.eps, "m0": w.m0,
                       "rhs_per_step": rhs_per_step, "block": w.block, "ncolors": w.ncolors, "k": w.k,
                       "lanes": L, "z0_runs_per_step": L,
                       "autotune": {s_: {"lanes": t["lanes"], "table": [(c["lanes"], round(c["rhs_per_s"]))
                                                                        for c in t["table"]]}
                                    for s_, t in tune.items()},
                       "defl_prec": w.defl_prec, "tol": w.tol, "solver": args.solver,
                       "l2": "flushed (256 MiB write) before every timed step",
                       "deflation_space": "subspace iteration on (g5 A)^-1: %d its, max rel residual %.2e, "
                                          "setup %.1f s (untimed)" % (eit, float(np.max(eres)), t_setup)},
            "clocks": clk,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": up_bytes / args.steps,
                    "d2h_bytes_per_step": rhs_per_step * 16 + scal_bytes * L,
                    "upload_s": t_up,
                    "note": "host wall clock: dtr_make_gauge + dtr_defl_create from host arrays (links %d B, "
                            "V + lambda %d B; h2d_bytes_per_step = that / steps), then %d dtr_trace_estimate "
                            "calls reading samples and traces back to the host; the noise is drawn on the device "
                            "from (seed, run)" % (U.size * 16, V_host.size * 16 + lam_host.size * 8, args.steps),
                    "resident_inputs": {"value": e2e_res_value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "note": "same steps, gauge and V already on the device"}},
            "gpu_launches": launches,
            "roofline": roof,
            "roofline_stencil_fp32": roof_stencil,
            "roofline_stencil_bf16_hbm": roof_hbm,
            "roofline_deflation_tc_hbm": roof_tc,
            "cpu_baseline": cpu,
            "fp64_path": {"value": value64, "unit": UNIT, "steps": nf, "ms_per_step": sum(ms64) / nf,
                          "lanes": L64, "iterations_per_rhs": iters64 / (nf * w.ncolors * L64),
                          "max_rel_trace_diff_vs_mixed": trace_diff},
            "iterations_per_rhs": iters / (args.steps * rhs_per_step),
            "variance_x_time": {"trace": [tr_mean.real, tr_mean.imag], "var_T": var_T, "runs": len(traces),
                                "time_to_1e-3_s": ttr, "time_to_1e-3_s_fp64_path": ttr64,
                                "speedup_vs_fp64_path": ttr64 / ttr},
            "speedup_vs_fp64_path": value / value64,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
