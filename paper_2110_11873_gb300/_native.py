"""ctypes binding of include/rt_krylov.h (argument marshalling only).

The library is built in-tree by ``paper_2110_11873_gb300.build``; if it is
missing, loading raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librtkrylov.so")

(RT_OK, RT_EINVAL, RT_ENOMEM, RT_ECUDA, RT_ENOTCONV, RT_EBREAKDOWN, RT_ENUMERIC, RT_EPENDING, RT_ETIMEOUT,
 RT_ECANCELED) = range(10)
STATUS_NAMES = {0: "RT_OK", 1: "RT_EINVAL", 2: "RT_ENOMEM", 3: "RT_ECUDA", 4: "RT_ENOTCONV",
                5: "RT_EBREAKDOWN", 6: "RT_ENUMERIC", 7: "RT_EPENDING", 8: "RT_ETIMEOUT", 9: "RT_ECANCELED"}

RT_TAU_LINE_CENTER, RT_TAU_FREQ_INTEGRATED = 0, 1
RT_MU_GL_HALF, RT_MU_GL_FULL = 0, 1
RT_FS_DELO_LINEAR, RT_FS_IMPLICIT_EULER, RT_FS_TRAPEZOIDAL = 0, 1, 2
RT_PREC_NONE, RT_PREC_JACOBI, RT_PREC_LOCAL_LAMBDA, RT_PREC_JACOBI_LEFT = 0, 1, 2, 3
RT_PREC_SOR, RT_PREC_SSOR, RT_PREC_SOR_LEFT, RT_PREC_SSOR_LEFT = 4, 5, 6, 7
RT_FORM_I, RT_FORM_SIGMA = 0, 1
RT_X0_ZERO, RT_X0_USER, RT_X0_PAPER = 0, 1, 2
RT_ORTHO_MGS, RT_ORTHO_CGS2 = 0, 1
RT_PRECISION_FP64, RT_PRECISION_FP32_REFINE = 0, 1


class ProblemDesc(C.Structure):
    _fields_ = [
        ("Ns", C.c_int32), ("Nmu", C.c_int32), ("Nnu", C.c_int32),
        ("tau", C.POINTER(C.c_double)), ("B", C.POINTER(C.c_double)), ("phi", C.POINTER(C.c_double)),
        ("phi_center", C.c_double), ("x_min", C.c_double), ("x_max", C.c_double),
        ("a", C.c_double), ("eps", C.c_double), ("W2", C.c_double),
        ("tau_kind", C.c_int32), ("mu_quad", C.c_int32), ("formal_solver", C.c_int32),
        ("freq_norm", C.c_int32), ("form", C.c_int32),
    ]


class SolverOpts(C.Structure):
    _fields_ = [
        ("restart", C.c_int32), ("maxit", C.c_int32), ("precond", C.c_int32), ("x0_kind", C.c_int32),
        ("ortho", C.c_int32), ("precision", C.c_int32), ("rtol", C.c_double), ("inner_rtol", C.c_double),
        ("max_refine", C.c_int32), ("resid_hist", C.POINTER(C.c_double)), ("hist_cap", C.c_int32),
        ("omega", C.c_double), ("deadline_ms", C.c_double),
    ]


class SolveInfo(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("iters", C.c_int32), ("restarts", C.c_int32), ("applies", C.c_int32),
        ("refine_steps", C.c_int32), ("hist_len", C.c_int32), ("rel_resid", C.c_double),
        ("err_est", C.c_double), ("t_total_ms", C.c_double),
    ]


class ServerOpts(C.Structure):
    _fields_ = [
        ("mem_budget_bytes", C.c_int64), ("max_slots", C.c_int32), ("restart", C.c_int32),
        ("precond", C.c_int32), ("precision", C.c_int32), ("autotune", C.c_int32), ("graphs", C.c_int32),
    ]


class ServerStats(C.Structure):
    _fields_ = [
        ("resident", C.c_int32), ("queued", C.c_int32), ("arena_in_use", C.c_int64),
        ("arena_largest_free", C.c_int64), ("cycles", C.c_int64), ("completed", C.c_int64),
        ("grid_quad", C.c_int32), ("grid_formal", C.c_int32), ("grid_vec", C.c_int32), ("tuned", C.c_int32),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_size_t, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("ctx", C.c_void_p), ("alloc", ALLOC_FN), ("release", RELEASE_FN)]


# (name, restype, argtypes) for every entry point of include/rt_krylov.h
_P = C.c_void_p
SIGNATURES = [
    ("rt_problem_create", C.c_int, [C.POINTER(ProblemDesc), _P, C.POINTER(_P)]),
    ("rt_problem_create_with_allocator", C.c_int, [C.POINTER(ProblemDesc), C.POINTER(Allocator), _P,
                                                    C.POINTER(_P)]),
    ("rt_problem_destroy", C.c_int, [_P]),
    ("rt_problem_size", C.c_int64, [_P]),
    ("rt_problem_grids", C.c_int, [_P] + [C.POINTER(C.c_double)] * 6),
    ("rt_apply", C.c_int, [_P, _P, _P, _P]),
    ("rt_apply_f32", C.c_int, [_P, _P, _P, _P]),
    ("rt_problem_check", C.c_int, [_P, _P]),
    ("rt_problem_formal_kernel", C.c_int, [_P]),
    ("rt_problem_inject_wait_timeout", C.c_int, [_P, C.c_int32]),
    ("rt_rhs", C.c_int, [_P, _P, _P]),
    ("rt_jacobi_diag", C.c_int, [_P, _P, _P]),
    ("rt_precond_local_lambda", C.c_int, [_P, _P, _P, _P]),
    ("rt_precond_stationary", C.c_int, [_P, C.c_int32, C.c_double, _P, _P, _P]),
    ("rt_arnoldi_mgs", C.c_int, [_P, _P, C.c_int32, _P, _P, _P]),
    ("rt_arnoldi_bmgs", C.c_int, [_P, _P, C.c_int32, _P, _P, _P, _P]),
    ("rt_arnoldi_mgs_static", C.c_int, [_P, C.c_int64, C.c_int32, _P, _P, _P]),
    ("rt_solver_opts_default", None, [C.POINTER(SolverOpts)]),
    ("rt_solve_gmres", C.c_int, [_P, C.POINTER(SolverOpts), _P, _P, C.POINTER(SolveInfo), _P]),
    ("rt_solve_bicgstab", C.c_int, [_P, C.POINTER(SolverOpts), _P, _P, C.POINTER(SolveInfo), _P]),
    ("rt_solve_cgs", C.c_int, [_P, C.POINTER(SolverOpts), _P, _P, C.POINTER(SolveInfo), _P]),
    ("rt_solve_richardson", C.c_int, [_P, C.POINTER(SolverOpts), _P, _P, C.POINTER(SolveInfo), _P]),
    ("rt_server_opts_default", None, [C.POINTER(ServerOpts)]),
    ("rt_server_create", C.c_int, [C.POINTER(ServerOpts), C.POINTER(_P)]),
    ("rt_server_create_with_allocator", C.c_int, [C.POINTER(ServerOpts), C.POINTER(Allocator), C.POINTER(_P)]),
    ("rt_batch_submit", C.c_int, [_P, C.POINTER(ProblemDesc), C.POINTER(SolverOpts), C.POINTER(C.c_uint64)]),
    ("rt_poll", C.c_int, [_P, C.c_uint64, C.POINTER(SolveInfo), C.POINTER(C.c_double)]),
    ("rt_batch_cancel", C.c_int, [_P, C.c_uint64]),
    ("rt_server_stats_get", C.c_int, [_P, C.POINTER(ServerStats)]),
    ("rt_server_destroy", C.c_int, [_P]),
    ("rt_last_error", C.c_char_p, []),
    ("rt_launch_count", C.c_int64, []),
    ("rt_probe_fp64_fma", C.c_int64, [C.c_int32, _P, _P]),
]

_lib = None


def load(path: str = LIB_PATH):
    """Load librtkrylov.so and declare its signatures (raises if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2110_11873_gb300.build.build() "
                          "(there is no fallback implementation)")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def last_error() -> str:
    return (load().rt_last_error() or b"").decode()


class RTError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {last_error()}")


def check(status: int, where: str):
    if status != RT_OK:
        raise RTError(status, where)
