"""Multi-process (gloo, world size 2, CPU) checks of the estimator's sharding by
z0 runs: the run partition covers every run once (ragged splits included), the
gathered record is in run order, and the merged run statistics are identical
to those of one process over all runs.  The per-run samples come from the
oracle's Algorithm 1 on a tiny lattice (no GPU involved)."""
import os
import socket

import numpy as np
import pytest

from oracle import estimator, exact, noise, wilson
from paper_1603_05988_gb300 import shard, synth

DIMS, M0, SEED, R = (2, 2, 2, 4), -0.4, 21, 5


def _records(runs):
    U = synth.random_su3_links(DIMS, 0.5, 77)
    A = wilson.explicit(U, DIMS, M0)
    AH = wilson.explicit_dagger(U, DIMS, M0)
    _, Ainv = exact.trace_inverse_lu(A.toarray())
    rows = []
    for r in runs:
        Z = noise.noise_vectors(DIMS, SEED, r, 1, False, 0, 4)
        rows.append(estimator.deflated_hp(AH, lambda Z: Ainv @ Z, Z)["t"])
    return np.array(rows).reshape(len(rows), -1)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = shard.runs_for_rank(R, rank, world)
        local = _records(range(lo, hi))
        record = shard.gather_records(local)
        stats = shard.run_statistics(record)
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank), record=record, lo=lo, hi=hi,
                 stats=np.array([stats["trace"].real, stats["trace"].imag, stats["var_runs"], stats["jk_err"],
                                 stats["var_samples"]]))
    finally:
        dist.destroy_process_group()


def test_runs_for_rank_partition():
    for n in (0, 1, 5, 7, 64):
        for world in (1, 2, 3, 8):
            parts = [shard.runs_for_rank(n, q, world) for q in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(world - 1))
            assert max(h - l for l, h in parts) - min(h - l for l, h in parts) <= 1


def test_run_statistics_against_definitions():
    S = _records(range(R))
    st = shard.run_statistics(S, 3.0 + 0.5j)
    tr = 3.0 + 0.5j + S.mean(axis=1)
    assert np.allclose(st["trace_runs"], tr, rtol=1e-14, atol=0)
    assert abs(st["trace"] - tr.mean()) <= 1e-13 * abs(tr.mean())
    assert abs(st["var_runs"] - estimator.sample_variance(tr)) <= 1e-12 * st["var_runs"]
    m, v = estimator.jackknife_mean(tr)
    assert abs(st["jk_err"] - np.sqrt(v)) <= 1e-12 * st["jk_err"]
    assert abs(st["var_samples"] - estimator.sample_variance(S.ravel())) <= 1e-12 * st["var_samples"]


def test_two_ranks_gloo_merge_is_identical_to_one_process(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    full = _records(range(R))
    ref = shard.run_statistics(full)
    refv = np.array([ref["trace"].real, ref["trace"].imag, ref["var_runs"], ref["jk_err"], ref["var_samples"]])
    for q in range(world):
        d = np.load(tmp_path / ("rank%d.npz" % q))
        assert (int(d["lo"]), int(d["hi"])) == shard.runs_for_rank(R, q, world)
        assert np.array_equal(d["record"], full)               # gathered in run order
        assert np.array_equal(d["stats"], refv)                # bit-identical statistics
