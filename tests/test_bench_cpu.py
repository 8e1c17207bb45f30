"""bench.py host-side contract on the CPU: the reference arm (the oracle timed
on host cores) prints one JSON line with the required keys, alone and under a
two-rank gloo launch (rank 0 prints, the other rank exits without work)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
REQUIRED = {"impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
            "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"}


def _json_lines(out):
    return [json.loads(ln) for ln in out.splitlines() if ln.startswith("{")]


@pytest.mark.slow
def test_reference_arm_prints_one_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert REQUIRED <= set(d), REQUIRED - set(d)
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "applies/s"
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0


@pytest.mark.slow
def test_reference_arm_two_ranks_gloo():
    env = dict(os.environ, MASTER_ADDR="127.0.0.1")
    r = subprocess.run([sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
                        "--master-addr", "127.0.0.1", "--master-port", "29631", os.path.join(ROOT, "bench.py"),
                        "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"],
                       capture_output=True, text=True, timeout=900, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-3000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["n_gpus"] == 2


def _reduce_rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r: 10 (r + 1) ms, 100 (r + 1) applies, r + 1 solves
        q.put((rank, bench.reduce_over_ranks(10.0 * (rank + 1), (100 * (rank + 1), rank + 1), dist, "cpu")))
    finally:
        dist.destroy_process_group()


def test_rank_reduction_two_ranks_gloo():
    """The whole-job figures of an N-rank bench run: the time is the slowest
    rank's, the applies and solves the sum over ranks (two gloo ranks on the
    CPU; the GPU run does the same over NCCL)."""
    import multiprocessing as mp

    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(3.0, (5, 1), None, "cpu") == (3.0, [5.0, 1.0])
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_reduce_rank, args=(r, 2, 29637, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert out[0] == out[1] == (20.0, [300.0, 3.0])


def test_oracle_per_solve_check_of_saved_solutions(tmp_path):
    """The CPU leg's per-solve check: a saved solution is identified by its
    distribution (seed), index and count; the oracle recomputes b, the true
    residual and (small N_s) the distance from its exact solution.  The
    oracle's own exact solution passes with residual and error at rounding
    level; a perturbed copy shows the perturbation."""
    import numpy as np

    sys.path.insert(0, ROOT)
    import bench
    import rt_workloads as W
    from oracle.transfer import Transfer

    at = W.batch_instances(512)[379]
    assert at.Ns <= 120
    xs = Transfer(at).exact_I()
    path = str(tmp_path / "s.npz")
    np.savez(path, **{f"batched__{W.BATCH_SEED}__379__512": xs,
                      f"served200__{W.BATCH_SEED}__379__512": xs * (1 + 1e-6)})
    out = bench.oracle_errors(path)
    assert "error" not in out, out
    assert out["batched"]["true_resid_max"] < 1e-12 and out["batched"]["err_vs_lu_max"] < 1e-12
    assert 5e-7 < out["served200"]["err_vs_lu_max"] < 2e-6
