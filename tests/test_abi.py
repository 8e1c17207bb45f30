"""The C-ABI library builds, loads and exports every entry point declared in
include/rt_krylov.h; the ctypes structures match the C layout; argument
validation runs on the host (CPU, no device work)."""
import ctypes as C
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2110_11873_gb300 import _native as N
from paper_2110_11873_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "rt_krylov.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return N.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rt_[a-z0-9_]+)\s*\(", text)))


def test_every_declared_function_is_exported_and_bound(lib):
    names = declared_functions()
    assert len(names) >= 14
    out = subprocess.run(["nm", "-D", "--defined-only", N.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\sT\s(rt_\w+)", out))
    bound = {n for n, _, _ in N.SIGNATURES}
    for n in names:
        assert n in exported, n
        assert n in bound, n
        assert getattr(lib, n) is not None


_LAYOUT_C = r"""
#include <stdio.h>
#include <stddef.h>
#include "rt_krylov.h"
#define F(T, f) printf("%s.%s %zu\n", #T, #f, offsetof(T, f))
int main(void) {
  printf("rt_problem_desc %zu\nrt_solver_opts %zu\nrt_solve_info %zu\nrt_server_opts %zu\nrt_server_stats %zu\n",
         sizeof(rt_problem_desc), sizeof(rt_solver_opts), sizeof(rt_solve_info), sizeof(rt_server_opts),
         sizeof(rt_server_stats));
  F(rt_server_opts, precision); F(rt_server_opts, autotune); F(rt_server_opts, graphs);
  F(rt_server_stats, completed); F(rt_server_stats, grid_quad); F(rt_server_stats, tuned);
  F(rt_problem_desc, tau); F(rt_problem_desc, phi_center); F(rt_problem_desc, W2);
  F(rt_problem_desc, freq_norm); F(rt_problem_desc, form);
  F(rt_solver_opts, rtol); F(rt_solver_opts, resid_hist); F(rt_solver_opts, hist_cap);
  F(rt_solver_opts, omega); F(rt_solver_opts, deadline_ms);
  F(rt_solve_info, rel_resid); F(rt_solve_info, err_est); F(rt_solve_info, t_total_ms);
  printf("rt_allocator %zu\n", sizeof(rt_allocator));
  F(rt_allocator, ctx); F(rt_allocator, alloc); F(rt_allocator, release);
  return 0;
}
"""


def test_struct_layouts_match_the_header(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(_LAYOUT_C)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                               check=True).stdout.split("\n") if line)
    structs = {"rt_problem_desc": N.ProblemDesc, "rt_solver_opts": N.SolverOpts, "rt_solve_info": N.SolveInfo,
               "rt_server_opts": N.ServerOpts, "rt_server_stats": N.ServerStats, "rt_allocator": N.Allocator}
    for name, cls in structs.items():
        assert int(got[name]) == C.sizeof(cls), name
    for key, val in got.items():
        if "." in key:
            sname, field = key.split(".")
            assert getattr(structs[sname], field).offset == int(val), key


def test_header_constants_match_the_python_side(tmp_path):
    """The descriptor enums of the header against the constants the Python
    side writes into rt_problem_desc (rt_workloads) and the binding."""
    import rt_workloads as W
    names = {"RT_TAU_LINE_CENTER": W.TAU_LINE_CENTER, "RT_TAU_FREQ_INTEGRATED": W.TAU_FREQ_INTEGRATED,
             "RT_MU_GL_HALF": W.MU_GL_HALF, "RT_MU_GL_FULL": W.MU_GL_FULL,
             "RT_FS_DELO_LINEAR": W.FS_DELO_LINEAR, "RT_FS_IMPLICIT_EULER": W.FS_IMPLICIT_EULER,
             "RT_FS_TRAPEZOIDAL": W.FS_TRAPEZOIDAL, "RT_FS_DELO_PARABOLIC": W.FS_DELO_PARABOLIC,
             "RT_FS_DELOPAR": W.FS_DELOPAR}
    src = tmp_path / "consts.c"
    src.write_text('#include <stdio.h>\n#include "rt_krylov.h"\nint main(void) {\n' +
                   "".join(f'  printf("{n} %d\\n", (int){n});\n' for n in names) + "  return 0;\n}\n")
    exe = tmp_path / "consts"
    subprocess.run(["gcc", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)], check=True)
    got = dict(line.split() for line in subprocess.run([str(exe)], capture_output=True, text=True,
                                                        check=True).stdout.splitlines())
    assert {k: int(v) for k, v in got.items()} == names
    assert (N.RT_FS_DELO_LINEAR, N.RT_FS_IMPLICIT_EULER, N.RT_FS_TRAPEZOIDAL) == tuple(
        int(got[n]) for n in ("RT_FS_DELO_LINEAR", "RT_FS_IMPLICIT_EULER", "RT_FS_TRAPEZOIDAL"))
    assert W.FS_DELOPAR == W.FS_DELO_PARABOLIC


def _desc(**kw):
    tau = np.logspace(-4, 6, 10)
    keep = [tau]
    d = N.ProblemDesc()
    d.Ns, d.Nmu, d.Nnu = 10, 4, 5
    d.tau = tau.ctypes.data_as(C.POINTER(C.c_double))
    d.x_min, d.x_max, d.a, d.eps, d.W2 = -4.0, 4.0, 1e-3, 1e-4, 1.0
    for k, v in kw.items():
        if k == "tau":
            arr = np.asarray(v, dtype=np.float64)
            keep.append(arr)
            d.tau = arr.ctypes.data_as(C.POINTER(C.c_double))
        else:
            setattr(d, k, v)
    return d, keep


@pytest.mark.parametrize("bad", [
    dict(Ns=1), dict(Nmu=3), dict(Nmu=0), dict(Nnu=1), dict(eps=0.0), dict(eps=1.5), dict(a=0.0),
    dict(a=0.5), dict(x_min=4.0), dict(tau_kind=7), dict(mu_quad=5), dict(formal_solver=9), dict(form=2),
    dict(tau=np.r_[np.logspace(-4, 6, 9), 1.0]),
])
def test_invalid_descriptors_are_rejected_on_the_host(lib, bad):
    d, keep = _desc(**bad)
    h = C.c_void_p()
    st = lib.rt_problem_create(C.byref(d), None, C.byref(h))
    assert st == N.RT_EINVAL
    assert not h.value
    assert N.last_error()


def test_null_arguments_are_rejected(lib):
    assert lib.rt_apply(None, None, None, None) == N.RT_EINVAL
    assert lib.rt_problem_size(None) == -1
    assert lib.rt_problem_destroy(None) == N.RT_OK
    o = N.SolverOpts()
    lib.rt_solver_opts_default(C.byref(o))
    assert (o.restart, o.maxit, o.precond, o.rtol, o.omega) == (30, 10000, N.RT_PREC_JACOBI, 1e-8, 1.0)
    # the documented rest: x0 = 0, MGS, FP64, inner_rtol 0 (per solver), max_refine 20, no history, no deadline
    assert (o.x0_kind, o.ortho, o.precision, o.inner_rtol, o.max_refine) == (N.RT_X0_ZERO, N.RT_ORTHO_MGS,
                                                                            N.RT_PRECISION_FP64, 0.0, 20)
    assert not o.resid_hist and o.hist_cap == 0 and o.deadline_ms == 0.0
    info = N.SolveInfo()
    assert lib.rt_solve_gmres(None, C.byref(o), None, None, C.byref(info), None) == N.RT_EINVAL
    so = N.ServerOpts()
    lib.rt_server_opts_default(C.byref(so))
    assert so.max_slots == 64 and so.restart == 30
    assert (so.mem_budget_bytes, so.precond, so.precision, so.autotune, so.graphs) == (
        8 << 30, N.RT_PREC_LOCAL_LAMBDA, N.RT_PRECISION_FP64, 1, 1)
    so.max_slots = 0
    h = C.c_void_p()
    assert lib.rt_server_create(C.byref(so), C.byref(h)) == N.RT_EINVAL and not h.value
    assert lib.rt_poll(None, 1, None, None) == N.RT_EINVAL
    assert lib.rt_precond_stationary(None, N.RT_PREC_SOR, 1.0, None, None, None) == N.RT_EINVAL
    assert lib.rt_precond_local_lambda(None, None, None, None) == N.RT_EINVAL
    assert lib.rt_server_destroy(None) == N.RT_OK


def test_allocator_hook_probe_and_injection_arguments_are_checked_on_the_host(lib):
    """rt_problem_create_with_allocator and rt_server_create_with_allocator
    refuse a hook without alloc or release before touching a device; the
    FP64 probe refuses iters < 1 or a NULL sink; the wait-timeout injection
    refuses a NULL problem or a negative count."""
    d, keep = _desc()
    half = N.Allocator()
    half.alloc = N.ALLOC_FN(lambda ctx, n, st: None)   # release left NULL
    h = C.c_void_p()
    assert lib.rt_problem_create_with_allocator(C.byref(d), C.byref(half), None, C.byref(h)) == N.RT_EINVAL
    assert not h.value and "alloc and release" in N.last_error()
    so = N.ServerOpts()
    lib.rt_server_opts_default(C.byref(so))
    assert lib.rt_server_create_with_allocator(C.byref(so), C.byref(half), C.byref(h)) == N.RT_EINVAL
    bad, keep2 = _desc(Ns=1)
    assert lib.rt_problem_create_with_allocator(C.byref(bad), None, None, C.byref(h)) == N.RT_EINVAL
    assert lib.rt_probe_fp64_fma(0, C.c_void_p(16), None) == -1
    assert lib.rt_probe_fp64_fma(10, None, None) == -1
    assert lib.rt_problem_inject_wait_timeout(None, 1) == N.RT_EINVAL
    assert lib.rt_batch_cancel(None, 1) == N.RT_EINVAL
