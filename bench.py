#!/usr/bin/env python3
"""Benchmark of the GB300 transfer-operator path.

One step = one pass of the whole hot path over one atmosphere: the
right-hand side (formal solve with boundaries), the Jacobi diagonal, and a
Jacobi-preconditioned GMRES(30) solve to ||r||/||b|| < 1e-8, each iteration
being one matrix-free apply (quadrature T, formal solver Lambda) plus the
Arnoldi orthogonalisation.  Workload: N_s=300, N_mu=32, N_nu=101
(1,939,200 unknowns), tau 1e-4..1e8, x in [-8,8], eps=1e-4, a=1e-3, W2=1,
DELO-linear, FP64.

Reported value: operator applies per second over the timed solves (whole job
over all ranks).  Extra keys: solves/s, the standalone apply rate and its
algorithmic HBM bandwidth, the roofline object (against the FP64 rate
measured by a DFMA probe kernel), the small (slab70) and large (slab300,
three methods x two formal solvers x two precisions) workloads, the
30-case size sweep, the batched and served streams, and the oracle: timed
on one core and on all cores, and evaluating the per-solve error of the
batched and served mixed-precision solutions (its true residual, and the
distance from its exact LU solution where that is affordable).

Multi-GPU: independent replicas (one atmosphere per rank, no collective on
the data path; weak scaling), timed between barriers, max over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "operator applies/s & HBM GB/s; batched solves/s at resid 1e-8; p50/p99 latency"
FP64_NOMINAL_TFLOPS = 1.25   # 2 FLOP x 2 FP64 lanes/clk/SM x 152 SMs x 2.06 GHz (context only)
# DRAM bytes (read + write) of one block-MGS step at j = 15 on slab300: the
# sum over its six launches in one ncu capture of `bench.py --probe bmgs
# --probe-ns 300` (k_bdot 78.7 MB, 3 x k_bmgs<4,4> 146.7-147.0 MB,
# k_bmgs<4,0> 78.7 MB, k_bscale 15.6 MB); retaken whenever these kernels change
MGS_STEP_DRAM_BYTES = 613.3e6
# GMRES restart length of the batched and served solves (local-Lambda, FP32
# operator inside FP64 refinement).  The Arnoldi step's FP64 work grows with
# the cycle length, the step count falls with it; on the 512-atmosphere batch
# restart 6-12 gave 274-294 solves/s against 214 at 30 (5: 224, 15: 267,
# 20: 248), so the served cycles are 10 steps long.  The single-instance
# FP64 comparison runs at the same restart.
BATCH_RESTART = 10
WORKLOAD = "slab300: Ns=300 Nmu=32 Nnu=101 (1,939,200 unknowns), line-centre tau 1e-4..1e8, x in [-8,8], " \
           "eps=1e-4 a=1e-3 W2=1, DELO-linear; Jacobi-GMRES(30) to 1e-8"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precond", default="jacobi", choices=["jacobi", "local_lambda", "none"])
    ap.add_argument("--apply-reps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-deep", action="store_true")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-small", action="store_true")
    ap.add_argument("--no-matrix", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--probe", choices=["apply32", "apply64", "gmres32", "gmres64", "bmgs", "batch"],
                    help="run only a short sequence of one operation (the target of ncu captures) and exit")
    ap.add_argument("--probe-ns", type=int, default=1000, help="N_s of the sweep atmosphere (300: slab300)")
    ap.add_argument("--probe-reps", type=int, default=4)
    ap.add_argument("--probe-budget-gb", type=int, default=160,
                    help="device-memory budget of the batch probe's server (its arena is allocated at once; "
                         "keep it to a few GB for multi-pass ncu captures)")
    return ap.parse_args()


def probe_main(args):
    """A few operations on one atmosphere, for profilers: FP32 / FP64 applies
    (apply32, apply64), one Jacobi-GMRES(30) solve (gmres32: FP32 operator
    with FP64 refinement, gmres64: FP64), 60 iterations at most, the
    block-MGS Arnoldi step at j = 15 (bmgs: the bench's roofline object, on a
    random 17-vector basis, w restored before each step), or one batch of
    --batch-count uneven atmospheres through the server (batch)."""
    import torch

    import rt_workloads as W
    from paper_2110_11873_gb300 import Problem
    from paper_2110_11873_gb300 import build as B

    B.build()
    if args.probe == "batch":
        from paper_2110_11873_gb300 import Server
        ats = W.batch_instances(args.batch_count)
        srv = Server(mem_budget_bytes=args.probe_budget_gb << 30, max_slots=len(ats), restart=BATCH_RESTART,
                     precond="local_lambda", precision="fp32_refine")
        tickets = [srv.submit(a) for a in ats]
        res = _drain(srv, tickets)
        st = srv.stats()
        srv.close()
        print(json.dumps({"probe": "batch", "instances": len(ats), "ok": sum(r[0][0] == 0 for r in res.values()),
                          "cycles": st["cycles"]}))
        return
    at = W.slab300() if args.probe_ns == 300 else W.sweep(args.probe_ns)
    P = Problem(at)
    if args.probe == "bmgs":
        jm = 15
        g = torch.Generator("cuda").manual_seed(1)
        V = torch.randn((jm + 2) * P.N, dtype=torch.float64, device="cuda", generator=g)
        w0 = torch.randn(P.N, dtype=torch.float64, device="cuda", generator=g)
        w = torch.empty_like(w0)
        gram = torch.zeros((jm + 2) * 4, dtype=torch.float64, device="cuda")
        h = torch.empty(jm + 2, dtype=torch.float64, device="cuda")
        for _ in range(args.probe_reps):
            w.copy_(w0)
            P.arnoldi_bmgs(V, jm, w, gram, h)
    elif args.probe.startswith("apply"):
        dt = torch.float32 if args.probe == "apply32" else torch.float64
        x = torch.rand(P.N, dtype=dt, device="cuda", generator=torch.Generator("cuda").manual_seed(1))
        y = torch.empty_like(x)
        for _ in range(args.probe_reps):
            (P.apply_f32 if args.probe == "apply32" else P.apply)(x, out=y)
    else:
        b = P.rhs()
        for _ in range(args.probe_reps):
            P.solve(b, "gmres", restart=30, precond="jacobi", rtol=1e-8, maxit=60,
                    precision="fp32_refine" if args.probe == "gmres32" else "fp64")
    torch.cuda.synchronize()
    P.check()
    print(json.dumps({"probe": args.probe, "ns": args.probe_ns, "reps": args.probe_reps, "N": P.N,
                      "staged": P.staged_formal}))
    P.close()


# ----------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# -------------------------------------------------------------- CPU oracle
def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(precond: str, cycles: int = 5, budget_s: float = 20.0, threads: int = 1):
    """The oracle as it stands on a bounded sample of the same workload:
    `cycles` GMRES(30) restart cycles (30 applies + MGS each), in a child
    process with `threads` BLAS / OpenMP threads (1, or all the cores of this
    process's affinity mask).  The oracle's formal solver is vectorised numpy
    over the rays with a Python loop over heights, so extra cores help only
    its BLAS and einsum parts."""
    code = f"""
import json, os, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
import rt_workloads as W
from oracle.transfer import Transfer
from oracle import krylov as K
at = W.slab300()
tr = Transfer(at)
b = tr.rhs_I()
d = tr.jacobi_I()
Minv = {{"jacobi": lambda v: v / d, "local_lambda": tr.local_lambda_I_inverse, "none": None}}[{precond!r}]
t0 = time.perf_counter()
x, info = K.gmres(tr.apply_I, b, M_inv=Minv, restart=30, maxit={30 * cycles}, tol=1e-30)
dt = time.perf_counter() - t0
print(json.dumps({{"applies": info.applies, "seconds": dt}}))
"""
    n = str(threads)
    env = dict(os.environ, OMP_NUM_THREADS=n, OPENBLAS_NUM_THREADS=n, MKL_NUM_THREADS=n)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env,
                       timeout=max(120.0, 10 * budget_s))
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return {"value": d["applies"] / d["seconds"], "unit": "applies/s", "cores": threads, "kind": "oracle",
            "seconds": d["seconds"],
            "sample": f"{cycles} GMRES(30) restart cycle(s) of the slab300 {precond} solve ({d['applies']} applies, "
                      f"{d['seconds']:.1f} s), numpy FP64, {threads} BLAS/OpenMP thread(s)"}


def oracle_errors(npz_path: str, budget_s: float = 120.0):
    """Per-solve error of saved GPU solutions against the oracle (run by the
    CPU-baseline leg, in a child process): for each solution x of an
    atmosphere of the batch or stream distribution, the oracle's FP64 true
    residual ||b - A x|| / ||b||, and, for N_s <= 120 (where assembling the
    sigma-form matrix is cheap), ||x - x*|| / ||x*|| with x* the oracle's
    exact (LU-lifted) solution."""
    code = f"""
import json, sys, time
sys.path.insert(0, {ROOT!r})
import numpy as np
import rt_workloads as W
from oracle.transfer import Transfer
z = np.load({npz_path!r})
out = {{}}
t0 = time.perf_counter()
for key in sorted(z.files):
    kind, seed, idx, count = key.split("__")
    ats = W.batch_instances(int(count), seed=int(seed))
    at = ats[int(idx)]
    tr = Transfer(at)
    x = z[key]
    b = tr.rhs_I()
    res = float(np.linalg.norm(b - tr.apply_I(x)) / np.linalg.norm(b))
    err = None
    if at.Ns <= 120:
        xs = tr.exact_I()
        err = float(np.linalg.norm(x - xs) / np.linalg.norm(xs))
    out.setdefault(kind, []).append({{"index": int(idx), "Ns": at.Ns, "Nmu": at.Nmu, "Nnu": at.Nnu,
                                     "true_resid": res, "err_vs_lu": err}})
    if time.perf_counter() - t0 > {budget_s}:
        break
print(json.dumps(out))
"""
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=10 * budget_s)
    if r.returncode != 0:
        return {"error": r.stderr[-400:]}
    raw = json.loads(r.stdout.strip().splitlines()[-1])
    summary = {}
    for kind, rows in raw.items():
        errs = [row["err_vs_lu"] for row in rows if row["err_vs_lu"] is not None]
        summary[kind] = {"solves_checked": len(rows), "true_resid_max": max(row["true_resid"] for row in rows),
                         "err_vs_lu_checked": len(errs), "err_vs_lu_max": max(errs) if errs else None,
                         "err_vs_lu_mean": (sum(errs) / len(errs)) if errs else None, "per_solve": rows}
    return summary


def reference_main(args, rank, world):
    """--impl reference: the oracle timed on the host cores on the same workload."""
    if rank != 0:
        return
    for _ in range(args.warmup):
        cpu_baseline(args.precond, cycles=1)
    vals, secs = [], []
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(args.precond, cycles=1)
        if "value" in cb:
            vals.append(cb["value"])
            secs.append(cb["seconds"])
    if not vals:
        print(json.dumps({"impl": "reference", "unavailable": cb.get("error", "oracle failed")}))
        return
    v = statistics.median(vals)
    cb["value"] = v
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": "applies/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.median(secs),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": bench_config(args.precond, world),
           "cpu_baseline": cb,
           "e2e": {"value": v, "unit": "applies/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ------------------------------------------------------- batching / serving
def _drain(srv, tickets, timeout_s=600.0, want_x=()):
    import time as _t
    out = {}
    t0 = _t.perf_counter()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t, want_x=t in want_x)
                if r is not None:
                    out[t] = (r, _t.perf_counter())
        if _t.perf_counter() - t0 > timeout_s:
            raise RuntimeError("server did not finish")
        _t.sleep(0.0005)
    return out


def batch_bench(W, Server, Problem, torch, count, keep=24):
    import numpy as np
    """512 seeded uneven atmospheres submitted at once to one server: FP32
    operator inside FP64 refinement, local-Lambda preconditioner, resident
    together (one launch per phase for all of them).  Compared with the plain
    FP64 single-instance path on the first 16 of the same atmospheres; the
    first `keep` solutions are returned for the oracle's per-solve check."""
    import time as _t
    ats = W.batch_instances(count)
    n1 = min(16, count)
    keep = min(keep, count)
    srv = Server(mem_budget_bytes=160 << 30, max_slots=count, restart=BATCH_RESTART, precond="local_lambda",
                 precision="fp32_refine")
    t0 = _t.perf_counter()
    tickets = [srv.submit(a) for a in ats]
    res = _drain(srv, tickets, want_x=set(tickets[:max(n1, keep)]))
    wall = _t.perf_counter() - t0
    ok = [r for (r, _) in res.values() if r[0] == 0]
    rel = [r[1].rel_resid for r in ok]
    its = [r[1].iters for r in ok]
    stats = srv.stats()
    srv.close()
    # plain FP64 single-instance path, same atmospheres, same final residual
    torch.cuda.synchronize()
    t1 = _t.perf_counter()
    xref = []
    for a in ats[:n1]:
        P = Problem(a)
        b = P.rhs()
        xs, info = P.solve(b, "gmres", restart=BATCH_RESTART, precond="local_lambda", rtol=1e-8)
        xref.append(xs.cpu().numpy())
        P.close()
    torch.cuda.synchronize()
    single = n1 / (_t.perf_counter() - t1)
    errs = []
    for t, xr in zip(tickets[:n1], xref):
        xb = res[t][0][2]
        errs.append(float(np.linalg.norm(xb - xr) / np.linalg.norm(xr)))
    kept = {i: res[t][0][2] for i, t in enumerate(tickets[:keep]) if res[t][0][0] == 0}
    out = {"workload": f"{count} uneven atmospheres (splitmix64 seed 0x2110118730000001): Ns~U[50,400], "
                       "Nnu~U{21..101} odd, Nmu in {8,16,32}, eps log-U[1e-6,1e-2], a log-U[1e-4,1e-2], "
                       "B=1+c log10(1+tau)",
           "precision": "FP32 operator, FP64 Arnoldi and FP64 restart residual (refinement)",
           "restart": BATCH_RESTART, "solves": len(ok), "failed": count - len(ok), "wall_s": wall, "solves_per_s": len(ok) / wall,
           "iters_mean": sum(its) / max(len(its), 1), "rel_resid_max": max(rel) if rel else None,
           "cycles": stats["cycles"],
           "grids_ctas": {"quadrature": stats["grid_quad"], "formal": stats["grid_formal"],
                          "vector": stats["grid_vec"], "autotuned": bool(stats["tuned"])},
           "fp64_single_instance_solves_per_s": single, "fp64_single_instance_sample": n1,
           "rel_err_vs_fp64_gpu_max": max(errs), "rel_err_vs_fp64_gpu_mean": sum(errs) / len(errs)}
    return out, kept


def serve_bench(W, Server, rates, nreq, keep=8):
    """Served stream: Poisson arrivals of requests drawn like the uneven batch,
    admitted by a 64 GB device-memory budget; per-request latency from
    submission to completion.  The first `keep` solutions of every rate are
    returned for the oracle's per-solve check."""
    import time as _t
    ats = W.batch_instances(nreq, seed=W.STREAM_SEED)
    out, kept = {}, {}
    for rate in rates:
        arr = W.poisson_arrivals(rate, nreq)
        srv = Server(mem_budget_bytes=64 << 30, max_slots=512, restart=BATCH_RESTART, precond="local_lambda",
                     precision="fp32_refine")
        pending, lat, done_t = {}, [], []
        kept[rate] = {}
        t0 = _t.perf_counter()
        i = 0
        while i < nreq or pending:
            now = _t.perf_counter() - t0
            while i < nreq and arr[i] <= now:
                pending[srv.submit(ats[i])] = i
                i += 1
            for t in list(pending):
                k = pending[t]
                r = srv.poll(t, want_x=k < keep)
                if r is not None:
                    del pending[t]
                    lat.append(r[1].t_total_ms)
                    done_t.append(_t.perf_counter() - t0)
                    if k < keep and r[0] == 0:
                        kept[rate][k] = r[2]
            if now > 600:
                raise RuntimeError("served stream did not finish")
            _t.sleep(0.0002)
        srv.close()
        lat.sort()
        span = max(done_t) - float(arr[0])
        out[str(rate)] = {"offered_req_per_s": rate, "requests": nreq, "restart": BATCH_RESTART,
                          "achieved_solves_per_s": nreq / span,
                          "p50_ms": lat[len(lat) // 2], "p99_ms": lat[min(len(lat) - 1, int(0.99 * len(lat)))]}
    return out, kept


def solve_alg_bytes(info, N: int, m: int = 30) -> float:
    """Algorithmic bytes of one GMRES(m) solve with info.iters Arnoldi steps in
    info.restarts cycles: (2j+6)*N*8 for step j of a cycle, 2*N*8 more per
    cycle for the restart residual's apply."""
    steps, total = info.iters, 0.0
    for c in range(max(info.restarts, 1)):
        k = min(m, steps - c * m)
        if k <= 0:
            break
        total += sum((2 * j + 6) for j in range(k)) * N * 8 + 2 * N * 8
    return total


def reduce_over_ranks(seconds: float, counts, dist, device: str):
    """Whole-job timing over the ranks: (the slowest rank's time, the sum of
    each count over all ranks).  dist None: this process alone.  NCCL takes
    device tensors, gloo host ones."""
    import torch
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    c = torch.tensor([float(v) for v in counts], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), [float(v) for v in c.tolist()]


def bench_config(precond: str, world: int) -> dict:
    """The `config` object of both arms' JSON lines."""
    return {"workload": WORKLOAD, "precond": precond, "restart": 30, "rtol": 1e-8,
            "parallelism": f"replicas x{world}",
            "l2": "Krylov basis 31 x 15.5 MB = 480 MB > 129 MB L2; standalone slab300 applies flush L2 with a "
                  "256 MB write before each launch; N_s >= 1000 applies (x and y 103-206 MB each, > L2) run back to "
                  "back"}


def timed_solve(P, torch, b, method, reps=1, **kw):
    """(solve result, mean wall ms) of `reps` solves after one untimed solve
    (which captures the solver's graphs)."""
    P.solve(b, method, **kw)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        _, r = P.solve(b, method, raise_on_error=False, **kw)
    torch.cuda.synchronize()
    return r, (time.perf_counter() - t0) * 1000 / reps


def fp64_peak(lib, torch, stream, iters=10000, reps=5):
    """The FP64 rate of this GPU: the library's DFMA probe kernel (only fused
    multiply-adds, 8 independent chains per thread, 4 CTAs per SM) timed
    with CUDA events on `stream`; the best of `reps` launches, TFLOP/s."""
    import ctypes
    sink = torch.zeros(1, dtype=torch.float64, device="cuda")
    h = ctypes.c_void_p(stream.cuda_stream)
    ptr = ctypes.c_void_p(sink.data_ptr())
    for _ in range(2):
        lib.rt_probe_fp64_fma(iters, ptr, h)
    best, flop = 0.0, 0
    for _ in range(reps):
        a = torch.cuda.Event(enable_timing=True)
        b_ = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        flop = lib.rt_probe_fp64_fma(iters, ptr, h)
        b_.record(stream)
        torch.cuda.synchronize()
        if flop <= 0:
            return None
        best = max(best, flop / (a.elapsed_time(b_) * 1e-3) / 1e12)
    sm = None
    try:
        q = subprocess.run(["nvidia-smi", "-i", str(torch.cuda.current_device()), "--query-gpu=clocks.sm",
                            "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=10)
        sm = float(q.stdout.strip().splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        pass
    return {"tflops": best, "flop_per_launch": flop, "sm_mhz_after": sm,
            "how": "rt_probe_fp64_fma: FP64 fused multiply-adds only, 8 independent chains per thread, "
                   "4 x 256-thread CTAs per SM; best of 5 launches timed with CUDA events"}


# ------------------------------------------------------------------- main
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist = dist_mod
    if args.probe:
        probe_main(args)
        return
    if args.impl == "reference":
        if dist is not None:
            import torch
            dist.init_process_group("gloo")
        reference_main(args, rank, world)
        if dist is not None:
            dist.destroy_process_group()
        return

    import numpy as np
    import torch

    import rt_workloads as W
    from paper_2110_11873_gb300 import Problem, _native
    from paper_2110_11873_gb300 import build as B

    torch.cuda.set_device(local)
    if dist is not None:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    B.build()
    lib = _native.load()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    at = W.slab300()
    P = Problem(at)
    N = P.N
    stream = torch.cuda.current_stream()
    b = torch.empty(N, dtype=torch.float64, device="cuda")
    d = torch.empty(N, dtype=torch.float64, device="cuda")
    x = torch.empty(N, dtype=torch.float64, device="cuda")

    def step():
        P.rhs(out=b)
        P.jacobi_diag(out=d)
        _, info = P.solve(b, "gmres", x=x, restart=30, precond=args.precond, rtol=1e-8)
        return info

    for _ in range(max(args.warmup, 3)):
        info = step()
    assert info.ok, info
    barrier()
    applies = 0
    solves = 0
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        barrier()
        launches0 = lib.rt_launch_count()
        e0.record(stream)
        for _ in range(args.steps):
            info = step()
            applies += info.applies
            solves += 1
        e1.record(stream)
        barrier()
        launches1 = lib.rt_launch_count()
    ms_max, (applies_all, solves_all) = reduce_over_ranks(e0.elapsed_time(e1), (applies, solves), dist, "cuda")
    value = applies_all / (ms_max / 1000.0)

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def timed(fn, reps, flush_l2):
        """Mean ms per call.  flush_l2: each call timed alone after a 256 MB
        write that evicts the 129 MB L2 (the flush also keeps the GPU busy
        while the host enqueues the call).  Otherwise (inputs larger than L2)
        the calls run back to back between one pair of events, so the host's
        enqueue time does not count as GPU time."""
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        if not flush_l2:
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            for _ in range(reps):
                fn()
            a1.record(stream)
            torch.cuda.synchronize()
            return a0.elapsed_time(a1) / reps
        evs = []
        for _ in range(reps):
            flush.zero_()   # 256 MB write: evicts the 129 MB L2 before the launch
            a0 = torch.cuda.Event(enable_timing=True)
            a1 = torch.cuda.Event(enable_timing=True)
            a0.record(stream)
            fn()
            a1.record(stream)
            evs.append((a0, a1))
        torch.cuda.synchronize()
        return statistics.mean(a.elapsed_time(b_) for a, b_ in evs)

    # ---- the FP64 rate that bounds the Arnoldi step (measured, not nominal)
    peak64 = fp64_peak(lib, torch, stream)
    fp64_tflops = peak64["tflops"] if peak64 else FP64_NOMINAL_TFLOPS

    # ---- dominant kernels of the step: the block-MGS Arnoldi orthogonalisation
    # (k_bdot + 4 x k_bmgs + k_bscale of rt_arnoldi_bmgs), at the
    # mean Arnoldi index j = 15 of a GMRES(30) cycle; the 17-vector basis
    # (264 MB) is larger than L2.  FP64-pipe bound on this GPU: algorithmic
    # work per step = the MGS loop's 2(j+1) FMA + 1 FMA (norm) + 1 multiply
    # per element, 2 FLOP per FMA.
    jm = 15
    V = torch.randn((jm + 2) * N, dtype=torch.float64, device="cuda")
    w = torch.randn(N, dtype=torch.float64, device="cuda")
    gram = torch.zeros((jm + 2) * 4, dtype=torch.float64, device="cuda")
    hbuf = torch.empty(jm + 2, dtype=torch.float64, device="cuda")
    mgs_ms = timed(lambda: P.arnoldi_bmgs(V, jm, w, gram, hbuf), 20, False)
    mgs_flop = (2 * (2 * (jm + 1) + 1) + 1) * N
    mgs_tflops = mgs_flop / (mgs_ms * 1e-3) / 1e12
    nblk = (jm + 1 + 3) // 4
    # each basis vector read twice (dots, then update); w read by the first
    # kernel, read and written by each block pass, read once more to write v_{j+1}
    mgs_bytes = (2 * (jm + 1) + 2 * nblk + 3) * N * 8
    mgs_gbs = mgs_bytes / (mgs_ms * 1e-3) / 1e9
    del V

    # ---- the operator apply y = x - Lambda T J x, FP64 and FP32, L2 flushed
    xin = torch.randn(N, dtype=torch.float64, device="cuda")
    yout = torch.empty_like(xin)
    apply_ms = timed(lambda: P.apply(xin, out=yout), args.apply_reps, True)
    x32 = xin.float()
    y32 = torch.empty_like(x32)
    apply32_ms = timed(lambda: P.apply_f32(x32, out=y32), args.apply_reps, True)
    apply_gbs = 2 * N * 8 / (apply_ms * 1e-3) / 1e9
    apply32_gbs = 2 * N * 4 / (apply32_ms * 1e-3) / 1e9
    apply64_flop = 11 * (N // 2)   # about 11 FP64 operations per (height, ray) and both Stokes parameters
    # the deep atmosphere (N_s=2000, N_mu=64, N_nu=201: 51.5M unknowns, 206 MB
    # per FP32 vector), the HBM-bound case of the FP32 operator
    deep = None
    if not args.no_deep:
        Pd = Problem(W.sweep(2000))
        xd = torch.randn(Pd.N, dtype=torch.float32, device="cuda")
        yd = torch.empty_like(xd)
        deep_ms = timed(lambda: Pd.apply_f32(xd, out=yd), 20, False)   # x and y: 206 MB each, > L2
        deep = {"workload": "sweep: Ns=2000 Nmu=64 Nnu=201 (51,456,000 unknowns), FP32 operator",
                "kernels": "k_quad (quadrature, multipolar components) + k_staged (TMA-staged formal solver)"
                if Pd.staged_formal else "k_moments + k_formal (register-ring FP32 kernels)",
                "ms": deep_ms, "alg_gbs": 2 * Pd.N * 4 / (deep_ms * 1e-3) / 1e9,
                "two_pass_gbs": 3 * Pd.N * 4 / (deep_ms * 1e-3) / 1e9, "peak_gbs": hbm_peak, "peak_source": hbm_src,
                "note": "alg_gbs counts x read + y written (2*N*4 B); two_pass_gbs adds the quadrature's read of x "
                        "(3*N*4 B), the traffic of the two-kernel design (x does not fit in L2)"}
        deep["frac_of_hbm"] = deep["alg_gbs"] / hbm_peak
        deep["two_pass_frac_of_hbm"] = deep["two_pass_gbs"] / hbm_peak
        del xd, yd
        Pd.close()

    # ---- end to end through the public API with host buffers
    b_host = torch.empty(N, dtype=torch.float64).pin_memory()
    x_host = torch.empty(N, dtype=torch.float64).pin_memory()
    P.rhs(out=b)
    b_host.copy_(b)
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    e2e_applies = 0
    for _ in range(args.steps):
        b.copy_(b_host, non_blocking=True)
        _, info = P.solve(b, "gmres", x=x, restart=30, precond=args.precond, rtol=1e-8)
        x_host.copy_(x, non_blocking=True)
        torch.cuda.synchronize()
        e2e_applies += info.applies
    e2e_max, (e2e_all,) = reduce_over_ranks(time.perf_counter() - t0, (e2e_applies,), dist, "cuda")
    e2e_value = e2e_all / e2e_max

    # ---- the small atmosphere: slab70, FP64 Jacobi-GMRES(30)
    small = None
    if not args.no_small:
        Ps = Problem(W.slab70())
        bs = Ps.rhs()
        r1, ms1 = timed_solve(Ps, torch, bs, "gmres", reps=10, restart=30, precond="jacobi", rtol=1e-8)
        small = {"workload": "slab70: Ns=70 Nmu=16 (8 GL per hemisphere) Nnu=21 (47,040 unknowns), line-centre "
                             "tau 1e-4..1e6, x in [-6,6], eps=1e-4 a=1e-3 W2=1, DELO-linear; FP64 Jacobi-GMRES(30) "
                             "to 1e-8",
                 "iters": r1.iters, "applies": r1.applies, "status": r1.status, "rel_resid": r1.rel_resid,
                 "solve_ms": ms1, "solves_per_s": 1000.0 / ms1, "applies_per_s": r1.applies * 1000.0 / ms1}
        Ps.close()

    # ---- the large atmosphere: three methods x two formal solvers x two
    # precisions, with the literal I-form Jacobi diagonal and with the
    # paper's (sigma-form) Jacobi carried to the I-form (local Lambda).  The
    # FP32 inner solves of BiCGSTAB and CGS do not converge with the literal
    # diagonal on this system; those rows are capped at 2000 iterations.
    large = None
    if not args.no_matrix:
        large = []
        for fs_name, fs in (("delo_linear", W.FS_DELO_LINEAR), ("implicit_euler", W.FS_IMPLICIT_EULER)):
            Pm = P if fs == W.FS_DELO_LINEAR else Problem(W.slab300(formal_solver=fs))
            bm = Pm.rhs()
            for pc in ("jacobi", "local_lambda"):
                for method in ("gmres", "bicgstab", "cgs"):
                    for precision in ("fp64", "fp32_refine"):
                        # capped where the method does not converge on this system (CGS with local Lambda
                        # diverges even in FP64; FP32 inner solves of BiCGSTAB/CGS with the literal diagonal)
                        cap = 2000 if (method == "cgs" and pc == "local_lambda") or (
                            pc == "jacobi" and method != "gmres" and precision == "fp32_refine") else 20000
                        kw = dict(precond=pc, rtol=1e-8, maxit=cap, precision=precision)
                        if method == "gmres":
                            kw["restart"] = 30
                        r, msm = timed_solve(Pm, torch, bm, method, **kw)
                        large.append({"formal_solver": fs_name, "method": method, "precision": precision,
                                      "precond": pc, "maxit": cap, "iters": r.iters, "applies": r.applies,
                                      "refine_steps": r.refine_steps, "status": r.status,
                                      "rel_resid": r.rel_resid, "solve_ms": msm, "solves_per_s": 1000.0 / msm})
            if Pm is not P:
                Pm.close()

    # ---- local-Lambda solve rate, for context
    _, li = P.solve(b, "gmres", x=x, restart=30, precond="local_lambda", rtol=1e-8)
    torch.cuda.synchronize()
    tl0 = time.perf_counter()
    nl = 3
    for _ in range(nl):
        _, li = P.solve(b, "gmres", x=x, restart=30, precond="local_lambda", rtol=1e-8)
    torch.cuda.synchronize()
    ll_solve_ms = (time.perf_counter() - tl0) * 1000 / nl

    # ---- size sweep: 5 heights x 3 eps x 2 Planck profiles, GMRES(30) to
    # 1e-8 with the FP32 operator, FP64 Arnoldi and refinement; the FP32
    # apply timed per N_s.  Preconditioner: the paper's Jacobi (on the
    # sigma-form) carried to the I-form, i.e. local Lambda, for all 30 cases;
    # the literal I-form diagonal for eps >= 1e-4 (at eps = 1e-6 restarted
    # GMRES with it stagnates for tens of thousands of steps), capped at 3000.
    sweep = None
    if not args.no_sweep:
        sweep = {"workload": "sweep: Nmu=64 Nnu=201, tau 1e-4..1e8, x in [-8,8], a=1e-3, W2=1, DELO-linear; "
                             "GMRES(30) to 1e-8, FP32 operator with FP64 Arnoldi and refinement",
                 "apply": {}, "cases": []}
        for ns in W.SWEEP_NS:
            for Bc in (0.0, 0.5):
                for eps in W.SWEEP_EPS:
                    Pw = Problem(W.sweep(ns, eps=eps, Bc=Bc))
                    if Bc == 0.0 and eps == 1e-4:
                        xs = torch.randn(Pw.N, dtype=torch.float32, device="cuda")
                        ys = torch.empty_like(xs)
                        # vectors of N_s >= 1000 exceed L2; smaller ones are flushed
                        ams = timed(lambda: Pw.apply_f32(xs, out=ys), 10, Pw.N * 4 < 256 << 20 and ns < 1000)
                        sweep["apply"][str(ns)] = {"N": Pw.N, "apply_fp32_ms": ams,
                                                   "alg_gbs": 2 * Pw.N * 4 / (ams * 1e-3) / 1e9,
                                                   "frac_of_hbm": 2 * Pw.N * 4 / (ams * 1e-3) / 1e9 / hbm_peak}
                        del xs, ys
                    bw = Pw.rhs()
                    for pc, cap in (("local_lambda", 20000), ("jacobi", 3000)):
                        if pc == "jacobi" and eps < 1e-4:
                            continue
                        torch.cuda.synchronize()
                        t0s = time.perf_counter()
                        _, si = Pw.solve(bw, "gmres", restart=30, precond=pc, rtol=1e-8, precision="fp32_refine",
                                         maxit=cap, raise_on_error=False)
                        torch.cuda.synchronize()
                        sweep["cases"].append({"Ns": ns, "eps": eps, "B": "1" if Bc == 0.0 else "1+0.5 log10(1+tau)",
                                               "N": Pw.N, "precond": pc, "maxit": cap, "iters": si.iters,
                                               "refine_steps": si.refine_steps, "rel_resid": si.rel_resid,
                                               "status": si.status, "solve_ms": (time.perf_counter() - t0s) * 1000})
                    del bw
                    Pw.close()

    # ---- FP32 operator inside FP64 refinement on the same atmosphere
    refine = {}
    for pc in ("jacobi", "local_lambda"):
        r, msr = timed_solve(P, torch, b, "gmres", restart=30, precond=pc, rtol=1e-8, precision="fp32_refine")
        refine[pc] = {"iters": r.iters, "refine_steps": r.refine_steps, "rel_resid": r.rel_resid, "ms": msr}

    batch, served, saved = None, None, {}
    if not args.no_batch:
        from paper_2110_11873_gb300 import Server
        batch, kept = batch_bench(W, Server, Problem, torch, args.batch_count)
        for i, xk in kept.items():
            saved[f"batched__{W.BATCH_SEED}__{i}__{args.batch_count}"] = xk
    if not args.no_serve:
        from paper_2110_11873_gb300 import Server
        served, kept = serve_bench(W, Server, (200, 1000, 5000), args.serve_requests)
        for rate, d_ in kept.items():
            for i, xk in d_.items():
                saved[f"served{rate}__{W.STREAM_SEED}__{i}__{args.serve_requests}"] = xk

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": "applies/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": bench_config(args.precond, world),
            "solves_per_s": solves_all / (ms_max / 1000.0),
            "solve_alg_gbs": solve_alg_bytes(info, N) * solves_all / (ms_max * 1e-3) / 1e9,
            "solve_alg_gbs_note": "algorithmic bytes of a solve over its time: per Arnoldi step j of a cycle "
                                  "(2j+6)*N*8 (the apply's x and y, each basis vector read twice by the "
                                  "orthogonalisation, w written and read), per cycle one more apply",
            "iters_per_solve": info.iters, "applies_per_solve": info.applies,
            "apply_fp64": {"ms": apply_ms, "applies_per_s": 1000.0 / apply_ms, "alg_gbs": apply_gbs,
                           "tflops": apply64_flop / (apply_ms * 1e-3) / 1e12,
                           "frac_of_fp64": apply64_flop / (apply_ms * 1e-3) / 1e12 / fp64_tflops},
            "apply_fp32": {"ms": apply32_ms, "applies_per_s": 1000.0 / apply32_ms, "alg_gbs": apply32_gbs},
            "apply_fp32_deep": deep,
            "small_fp64": small,
            "large_matrix": large,
            "local_lambda_solve": {"iters": li.iters, "ms": ll_solve_ms, "solves_per_s": 1000.0 / ll_solve_ms},
            "fp32_refine_solve": refine,
            "size_sweep": sweep,
            "batched": batch,
            "served": served,
            "fp64_peak": peak64,
            "roofline": {"kernel": "block-MGS Arnoldi step (k_bdot + 4 x k_bmgs + k_bscale, j=15)",
                         "bound": "alu", "achieved": mgs_tflops, "peak": fp64_tflops, "unit": "TFLOP/s",
                         "frac": mgs_tflops / fp64_tflops, "traffic": MGS_STEP_DRAM_BYTES,
                         "peak_source": "measured: rt_probe_fp64_fma (FP64 FMA-only kernel, CUDA events)"
                         if peak64 else "nominal 1.25 TFLOP/s (probe failed)",
                         "hbm_gbs": mgs_gbs, "hbm_frac": mgs_gbs / hbm_peak,
                         "note": "FP64-pipe bound; algorithmic FLOP per step (2(2(j+1)+1)+1)*N of the MGS loop; "
                                 "hbm_gbs counts (2(j+1)+2*ceil((j+1)/4)+3)*N*8 bytes against the measured copy "
                                 "bandwidth"},
            "clocks": clk.summary(),
            "e2e": {"value": e2e_value, "unit": "applies/s", "h2d_bytes_per_step": N * 8,
                    "d2h_bytes_per_step": N * 8},
            "gpu_launches": launches1 - launches0,
        }
        if not args.no_cpu_baseline and world == 1:
            out["cpu_baseline"] = cpu_baseline(args.precond)
            out["cpu_baseline_all_cores"] = cpu_baseline(args.precond, cycles=5, threads=host_cores())
            if saved:
                import tempfile
                with tempfile.TemporaryDirectory() as td:
                    path = os.path.join(td, "solutions.npz")
                    np.savez(path, **saved)
                    errs = oracle_errors(path)
                for kind, rows in (errs.items() if isinstance(errs, dict) else []):
                    if kind == "batched" and batch is not None:
                        batch["vs_oracle"] = rows
                    elif kind.startswith("served") and served is not None:
                        served.setdefault("vs_oracle", {})[kind[len("served"):]] = rows
                if "error" in errs:
                    out["oracle_errors_failed"] = errs["error"]
        print(json.dumps(out))
    P.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
