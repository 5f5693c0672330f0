"""The estimator over several processes, one GPU each (Algorithm 1 over z0 runs).

The z0 runs of Algorithm 1 are independent, so the work shards by runs with no
exchange on the data path: rank q of W takes the contiguous runs
[R q / W, R (q+1) / W) and runs them through `dtr.trace_estimate` on its own
GPU.  The only communication is one gather of the per-sample records (R x s
complex numbers) in rank order, which is run order; every rank then forms the
run statistics from the whole record with the same arithmetic, in the same
order, as the library's single-process host code, so the merged result does
not depend on the number of processes.
"""
import numpy as np


def runs_for_rank(n_runs, rank, world):
    """Contiguous [lo, hi) share of n_runs z0 runs for `rank` of `world` (ragged-safe)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    return (n_runs * rank) // world, (n_runs * (rank + 1)) // world


def run_statistics(samples, T_D=0j):
    """Run statistics of a (R, s) record of samples t_j (run order), as the
    library forms them: Trace_r = T_D + mean_j t_j; mean over runs; variance over
    runs (complex form, 1/(R-1)); delete-1 jackknife error of the mean; variance of
    the individual samples.  Operation order follows the library's host code."""
    S = np.asarray(samples, dtype=np.complex128)
    R, s = S.shape
    td, td_im = float(np.real(T_D)), float(np.imag(T_D))
    tr = []
    mx = my = 0.0
    for r in range(R):
        sx = sy = 0.0
        for j in range(s):
            sx += float(S[r, j].real)
            sy += float(S[r, j].imag)
        t = (td + sx / s, td_im + sy / s)
        tr.append(t)
        mx += t[0]
        my += t[1]
    inv = 1.0 / R
    mx, my = mx * inv, my * inv
    var_runs = jk = 0.0
    if R > 1:
        for t in tr:
            dx, dy = t[0] - mx, t[1] - my
            var_runs += dx * dx + dy * dy
        var_runs /= (R - 1)
        totx, toty = mx * R, my * R
        f = 1.0 / (R - 1)
        loo = [((totx - t[0]) * f, (toty - t[1]) * f) for t in tr]
        lx = ly = 0.0
        for v in loo:
            lx += v[0]
            ly += v[1]
        lx, ly = lx * inv, ly * inv
        for v in loo:
            dx, dy = v[0] - lx, v[1] - ly
            jk += dx * dx + dy * dy
        jk = float(np.sqrt(jk * (R - 1) / R))
    var_s = 0.0
    ns = R * s
    if ns > 1:
        sx = sy = 0.0
        for r in range(R):
            for j in range(s):
                sx += float(S[r, j].real)
                sy += float(S[r, j].imag)
        g = 1.0 / ns
        sx, sy = sx * g, sy * g
        for r in range(R):
            for j in range(s):
                dx, dy = float(S[r, j].real) - sx, float(S[r, j].imag) - sy
                var_s += dx * dx + dy * dy
        var_s /= (ns - 1)
    return {"trace": complex(mx, my), "trace_runs": np.array([complex(*t) for t in tr]), "var_runs": var_runs,
            "jk_err": jk, "var_samples": var_s}


def gather_records(local, group=None):
    """All-gather per-rank (runs_r, s) complex records; returns the (R, s) record in run order."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, np.asarray(local, dtype=np.complex128), group=group)
    parts = [p for p in parts if p is not None and p.size]
    return np.concatenate(parts, axis=0) if parts else np.zeros((0, 0), dtype=np.complex128)


def sharded_trace_estimate(gauge, m0, defl, n_runs, make_params, group=None):
    """Algorithm 1 over n_runs z0 runs shared by the processes of `group`.

    make_params(z0_first, n_z0) -> dtr.trace_params for this rank's runs.  Each
    rank solves its share on its own GPU; the sample records are gathered and
    every rank returns the statistics of all runs (plus its own solve counts)."""
    import torch.distributed as dist
    from . import dtr
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    lo, hi = runs_for_rank(n_runs, rank, world)
    local = np.zeros((0, 0), dtype=np.complex128)
    own = {"n_solves": 0, "iterations": 0, "all_converged": True}
    if hi > lo:
        out = dtr.trace_estimate(gauge, m0, defl, make_params(lo, hi - lo))
        local = out["samples"]
        own = {"n_solves": out["n_solves"], "iterations": out["iterations"], "all_converged": out["all_converged"]}
    record = gather_records(local, group)
    stats = run_statistics(record, defl.T_D() if defl is not None else 0j)
    stats.update(own)
    stats["samples"] = record
    return stats
