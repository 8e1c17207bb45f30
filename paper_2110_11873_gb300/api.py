"""Thin Python layer over the C ABI: PyTorch supplies device memory and the
stream; every step of the computation runs in the library's kernels."""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import Optional

import numpy as np
import torch

from . import _native as N

_DESC_FIELDS = ("Ns", "Nmu", "Nnu", "tau", "B", "x_min", "x_max", "a", "eps", "W2", "tau_kind",
                "mu_quad", "formal_solver", "freq_norm")


def _dptr(arr: np.ndarray):
    return arr.ctypes.data_as(C.POINTER(C.c_double))


def _stream_handle(stream: Optional[torch.cuda.Stream]):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


@dataclasses.dataclass
class SolveResult:
    status: int
    iters: int
    restarts: int
    applies: int
    refine_steps: int
    rel_resid: float
    err_est: float
    t_total_ms: float
    history: np.ndarray

    @property
    def ok(self) -> bool:
        return self.status == N.RT_OK

    @property
    def status_name(self) -> str:
        return N.STATUS_NAMES.get(self.status, str(self.status))


def _desc_of(atm, keep: list, phi=None, phi_center=0.0) -> "N.ProblemDesc":
    f = {k: getattr(atm, k) for k in _DESC_FIELDS}
    tau = np.ascontiguousarray(f["tau"], dtype=np.float64)
    B = np.ascontiguousarray(f["B"], dtype=np.float64)
    keep += [tau, B]
    d = N.ProblemDesc()
    d.Ns, d.Nmu, d.Nnu = int(f["Ns"]), int(f["Nmu"]), int(f["Nnu"])
    d.tau = _dptr(tau)
    d.B = _dptr(B)
    if phi is not None:
        ph = np.ascontiguousarray(phi, dtype=np.float64)
        keep.append(ph)
        d.phi = _dptr(ph)
    d.phi_center = float(phi_center)
    d.x_min, d.x_max = float(f["x_min"]), float(f["x_max"])
    d.a, d.eps, d.W2 = float(f["a"]), float(f["eps"]), float(f["W2"])
    d.tau_kind, d.mu_quad = int(f["tau_kind"]), int(f["mu_quad"])
    d.formal_solver, d.freq_norm = int(f["formal_solver"]), int(f["freq_norm"])
    return d


class TorchAllocator:
    """An rt_allocator backed by PyTorch's caching allocator: the library's
    device workspaces are then PyTorch allocations (counted by
    torch.cuda.memory_allocated, reused from its cache).  Keeps counts of the
    blocks it handed out and took back.  ``fail_after``: refuse every request
    after that many (to exercise the library's out-of-memory path)."""

    def __init__(self, device=None, fail_after: Optional[int] = None):
        self.device = torch.cuda.current_device() if device is None else int(device)
        self.fail_after = fail_after
        self.allocs = 0
        self.releases = 0
        self.live = {}

        def _alloc(ctx, nbytes, stream):
            if self.fail_after is not None and self.allocs >= self.fail_after:
                return None
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device, stream=int(stream or 0))
            except Exception:   # out of memory: the library reports RT_ENOMEM
                return None
            self.allocs += 1
            self.live[int(p)] = int(nbytes)
            return p

        def _release(ctx, ptr, nbytes, stream):
            self.releases += 1
            self.live.pop(int(ptr), None)
            torch.cuda.caching_allocator_delete(int(ptr))

        self._fa = N.ALLOC_FN(_alloc)
        self._fr = N.RELEASE_FN(_release)
        self.struct = N.Allocator(None, self._fa, self._fr)


class Server:
    """Batched / served solves (rt_server_*): submit atmospheres, poll results.
    ``allocator``: a TorchAllocator (or any object with an rt_allocator
    ``struct``) from which the server takes its device memory."""

    def __init__(self, mem_budget_bytes: int = 8 << 30, max_slots: int = 64, restart: int = 30,
                 precond: str = "local_lambda", precision: str = "fp64", autotune: bool = True, graphs: bool = True,
                 allocator=None):
        self.lib = N.load()
        self.allocator = allocator
        o = N.ServerOpts()
        self.lib.rt_server_opts_default(C.byref(o))
        o.mem_budget_bytes, o.max_slots, o.restart = int(mem_budget_bytes), int(max_slots), int(restart)
        o.precond = {"none": N.RT_PREC_NONE, "jacobi": N.RT_PREC_JACOBI,
                     "local_lambda": N.RT_PREC_LOCAL_LAMBDA}[precond]
        o.precision = {"fp64": N.RT_PRECISION_FP64, "fp32_refine": N.RT_PRECISION_FP32_REFINE}[precision]
        o.autotune = 1 if autotune else 0
        o.graphs = 1 if graphs else 0
        h = C.c_void_p()
        if allocator is None:
            N.check(self.lib.rt_server_create(C.byref(o), C.byref(h)), "rt_server_create")
        else:
            N.check(self.lib.rt_server_create_with_allocator(C.byref(o), C.byref(allocator.struct), C.byref(h)),
                    "rt_server_create_with_allocator")
        self.handle = h
        self.sizes = {}

    def submit(self, atm, rtol: float = 1e-8, maxit: int = 10000, deadline_ms: float = 0.0) -> int:
        """Queue one solve; deadline_ms > 0 cancels it if unfinished that long after submission."""
        keep = []
        d = _desc_of(atm, keep)
        o = N.SolverOpts()
        self.lib.rt_solver_opts_default(C.byref(o))
        o.rtol, o.maxit, o.deadline_ms = rtol, maxit, deadline_ms
        t = C.c_uint64()
        N.check(self.lib.rt_batch_submit(self.handle, C.byref(d), C.byref(o), C.byref(t)), "rt_batch_submit")
        self.sizes[t.value] = 2 * d.Ns * d.Nmu * d.Nnu
        return t.value

    def cancel(self, ticket: int) -> None:
        """Cancel a request: a queued one ends at once, a resident one after the
        restart cycle in progress; its poll then reports RT_ECANCELED."""
        N.check(self.lib.rt_batch_cancel(self.handle, C.c_uint64(ticket)), "rt_batch_cancel")

    def poll(self, ticket: int, want_x: bool = True):
        """None while pending; else (status, SolveResult, x or None)."""
        info = N.SolveInfo()
        x = np.empty(self.sizes[ticket]) if want_x else None
        st = self.lib.rt_poll(self.handle, C.c_uint64(ticket), C.byref(info),
                              _dptr(x) if x is not None else None)
        if st == N.RT_EPENDING:
            return None
        self.sizes.pop(ticket, None)
        res = SolveResult(info.status, info.iters, info.restarts, info.applies, info.refine_steps,
                          info.rel_resid, info.err_est, info.t_total_ms, np.zeros(0))
        return st, res, x

    def stats(self) -> dict:
        st = N.ServerStats()
        N.check(self.lib.rt_server_stats_get(self.handle, C.byref(st)), "rt_server_stats_get")
        return {f: getattr(st, f) for f, _ in N.ServerStats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.rt_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Problem:
    """One atmosphere on the current CUDA device.

    ``atm`` is any object with the descriptor fields of rt_problem_desc
    (Ns, Nmu, Nnu, tau, B, x_min, x_max, a, eps, W2, tau_kind, mu_quad,
    formal_solver, freq_norm); ``phi`` optionally overrides the internal
    Voigt profile (with ``phi_center`` for line-centre tau).  ``form``
    selects the linear system: "I" (Eq. 19, N = 2*Ns*Nmu*Nnu) or "sigma"
    (Eq. 18, N = 2*Ns); apply, rhs, jacobi_diag, precond_local_lambda and
    solve then work on that system.  ``allocator``: a TorchAllocator (or any
    object with an rt_allocator ``struct``) that supplies the problem's
    device workspaces instead of cudaMalloc.
    """

    def __init__(self, atm, phi: Optional[np.ndarray] = None, phi_center: float = 0.0,
                 stream: Optional[torch.cuda.Stream] = None, form: str = "I", allocator=None):
        self.lib = N.load()
        self.allocator = allocator
        f = {k: getattr(atm, k) for k in _DESC_FIELDS}
        self._tau = np.ascontiguousarray(f["tau"], dtype=np.float64)
        self._B = np.ascontiguousarray(f["B"], dtype=np.float64)
        self._phi = None if phi is None else np.ascontiguousarray(phi, dtype=np.float64)
        d = N.ProblemDesc()
        d.Ns, d.Nmu, d.Nnu = int(f["Ns"]), int(f["Nmu"]), int(f["Nnu"])
        d.tau = _dptr(self._tau)
        d.B = _dptr(self._B)
        d.phi = _dptr(self._phi) if self._phi is not None else None
        d.phi_center = float(phi_center)
        d.x_min, d.x_max = float(f["x_min"]), float(f["x_max"])
        d.a, d.eps, d.W2 = float(f["a"]), float(f["eps"]), float(f["W2"])
        d.tau_kind, d.mu_quad = int(f["tau_kind"]), int(f["mu_quad"])
        d.formal_solver, d.freq_norm = int(f["formal_solver"]), int(f["freq_norm"])
        d.form = {"I": N.RT_FORM_I, "sigma": N.RT_FORM_SIGMA}[form]
        self.form = form
        self.desc = d
        self.Ns, self.Nmu, self.Nnu = d.Ns, d.Nmu, d.Nnu
        self.device = torch.device("cuda", torch.cuda.current_device())
        h = C.c_void_p()
        if allocator is None:
            N.check(self.lib.rt_problem_create(C.byref(d), _stream_handle(stream), C.byref(h)), "rt_problem_create")
        else:
            N.check(self.lib.rt_problem_create_with_allocator(C.byref(d), C.byref(allocator.struct),
                                                              _stream_handle(stream), C.byref(h)),
                    "rt_problem_create_with_allocator")
        self.handle = h
        self.N = int(self.lib.rt_problem_size(h))

    def close(self):
        if getattr(self, "handle", None):
            torch.cuda.synchronize(self.device)
            self.lib.rt_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # ---------------------------------------------------------------- grids
    def grids(self):
        out = {k: np.zeros(self.Nmu) for k in ("mu", "w_mu")}
        out.update({k: np.zeros(self.Nnu) for k in ("x", "phi", "w_nu", "phi_hat")})
        N.check(self.lib.rt_problem_grids(self.handle, *(_dptr(out[k]) for k in
                                                         ("mu", "w_mu", "x", "phi", "w_nu", "phi_hat"))),
                "rt_problem_grids")
        return out

    # ------------------------------------------------------------- operator
    def _vec(self, x: Optional[torch.Tensor], dtype=torch.float64) -> torch.Tensor:
        if x is None:
            return torch.empty(self.N, dtype=dtype, device=self.device)
        if x.dtype != dtype or x.device != self.device or not x.is_contiguous() or x.numel() != self.N:
            raise ValueError(f"expected a contiguous {dtype} vector of {self.N} on {self.device}")
        return x

    def apply(self, x: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """y = x - Lambda(T(J x)) in FP64."""
        x = self._vec(x)
        y = self._vec(out)
        N.check(self.lib.rt_apply(self.handle, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                  _stream_handle(stream)), "rt_apply")
        return y

    def apply_f32(self, x: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        x = self._vec(x, torch.float32)
        y = self._vec(out, torch.float32)
        N.check(self.lib.rt_apply_f32(self.handle, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                      _stream_handle(stream)), "rt_apply_f32")
        return y

    @property
    def staged_formal(self) -> bool:
        """True when FP32 applies use the shared-memory tensor-copy kernel."""
        return self.lib.rt_problem_formal_kernel(self.handle) == 1

    def inject_wait_timeout(self, count: int = 1) -> None:
        """Arm the next `count` tensor-copy FP32 applies to give up one wait
        (failure injection; the following check() raises RT_ETIMEOUT)."""
        N.check(self.lib.rt_problem_inject_wait_timeout(self.handle, int(count)), "rt_problem_inject_wait_timeout")

    def check(self, stream=None) -> None:
        """Raise RTError(RT_ETIMEOUT) when a bounded device wait of this
        problem's kernels gave up since the last check (synchronises)."""
        N.check(self.lib.rt_problem_check(self.handle, _stream_handle(stream)), "rt_problem_check")

    def rhs(self, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        b = self._vec(out)
        N.check(self.lib.rt_rhs(self.handle, C.c_void_p(b.data_ptr()), _stream_handle(stream)), "rt_rhs")
        return b

    def jacobi_diag(self, out: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        d = self._vec(out)
        N.check(self.lib.rt_jacobi_diag(self.handle, C.c_void_p(d.data_ptr()), _stream_handle(stream)),
                "rt_jacobi_diag")
        return d

    def precond_local_lambda(self, v: torch.Tensor, out: Optional[torch.Tensor] = None, stream=None):
        v = self._vec(v)
        z = self._vec(out)
        N.check(self.lib.rt_precond_local_lambda(self.handle, C.c_void_p(v.data_ptr()),
                                                 C.c_void_p(z.data_ptr()), _stream_handle(stream)),
                "rt_precond_local_lambda")
        return z

    def precond_stationary(self, v: torch.Tensor, kind: str = "ssor", omega: float = 1.0,
                           out: Optional[torch.Tensor] = None, stream=None):
        """z = P^-1 v for the sigma-form SOR ("sor") or SSOR ("ssor") preconditioner."""
        v = self._vec(v)
        z = self._vec(out)
        k = {"sor": N.RT_PREC_SOR, "ssor": N.RT_PREC_SSOR}[kind]
        N.check(self.lib.rt_precond_stationary(self.handle, k, float(omega), C.c_void_p(v.data_ptr()),
                                               C.c_void_p(z.data_ptr()), _stream_handle(stream)),
                "rt_precond_stationary")
        return z

    def arnoldi_mgs(self, V: torch.Tensor, j: int, w: torch.Tensor, h: Optional[torch.Tensor] = None,
                    stream=None) -> torch.Tensor:
        """One MGS Arnoldi step: orthogonalise w against V[0..j], write
        V[j+1] = w/||w||; returns h (j+2 values)."""
        if V.dtype != torch.float64 or not V.is_contiguous() or V.numel() < (j + 2) * self.N:
            raise ValueError("V must be a contiguous float64 tensor of at least (j+2)*N values")
        w = self._vec(w)
        h = torch.empty(j + 2, dtype=torch.float64, device=self.device) if h is None else h
        N.check(self.lib.rt_arnoldi_mgs(self.handle, C.c_void_p(V.data_ptr()), int(j), C.c_void_p(w.data_ptr()),
                                        C.c_void_p(h.data_ptr()), _stream_handle(stream)), "rt_arnoldi_mgs")
        return h

    def arnoldi_bmgs(self, V: torch.Tensor, j: int, w: torch.Tensor, gram: torch.Tensor,
                     h: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
        """One block-MGS Arnoldi step (the GMRES orthogonalisation): as
        arnoldi_mgs, with gram ((j+2) x 4 doubles, rows 1..j read, row j+1
        written) holding <v_i, v_{i-d}>, d = 1..3."""
        if V.dtype != torch.float64 or not V.is_contiguous() or V.numel() < (j + 2) * self.N:
            raise ValueError("V must be a contiguous float64 tensor of at least (j+2)*N values")
        if gram.dtype != torch.float64 or not gram.is_contiguous() or gram.numel() < (j + 2) * 4:
            raise ValueError("gram must be a contiguous float64 tensor of at least (j+2)*4 values")
        w = self._vec(w)
        h = torch.empty(j + 2, dtype=torch.float64, device=self.device) if h is None else h
        N.check(self.lib.rt_arnoldi_bmgs(self.handle, C.c_void_p(V.data_ptr()), int(j), C.c_void_p(w.data_ptr()),
                                         C.c_void_p(gram.data_ptr()), C.c_void_p(h.data_ptr()),
                                         _stream_handle(stream)), "rt_arnoldi_bmgs")
        return h

    # --------------------------------------------------------------- solvers
    def solve(self, b: torch.Tensor, method: str = "gmres", x: Optional[torch.Tensor] = None, *,
              restart: int = 30, maxit: int = 10000, precond: str = "jacobi", rtol: float = 1e-8,
              x0=False, precision: str = "fp64", inner_rtol: float = 0.0, max_refine: int = 20,
              hist_cap: int = 0, omega: float = 1.0, raise_on_error: bool = True, stream=None):
        """Solve A x = b; returns (x, SolveResult).  ``x0=True`` uses ``x`` as initial guess,
        ``x0="paper"`` the paper's (sigma = [1, 0, 1, 0, ...], lifted to the I-form).
        ``precond``: "none", "jacobi", "local_lambda", "jacobi_left" (GMRES), and for the
        sigma-form "sor", "ssor", "sor_left", "ssor_left" (GMRES) with relaxation ``omega``.
        ``inner_rtol`` (precision "fp32_refine"): 0 takes the library's default, rtol for
        GMRES and 1e-4 for BiCGSTAB/CGS."""
        b = self._vec(b)
        x = self._vec(x) if x is not None else torch.zeros(self.N, dtype=torch.float64, device=self.device)
        o = N.SolverOpts()
        self.lib.rt_solver_opts_default(C.byref(o))
        o.restart, o.maxit, o.rtol = restart, maxit, rtol
        o.precond = {"none": N.RT_PREC_NONE, "jacobi": N.RT_PREC_JACOBI,
                     "local_lambda": N.RT_PREC_LOCAL_LAMBDA, "jacobi_left": N.RT_PREC_JACOBI_LEFT,
                     "sor": N.RT_PREC_SOR, "ssor": N.RT_PREC_SSOR, "sor_left": N.RT_PREC_SOR_LEFT,
                     "ssor_left": N.RT_PREC_SSOR_LEFT}[precond]
        o.omega = omega
        o.x0_kind = N.RT_X0_PAPER if x0 == "paper" else (N.RT_X0_USER if x0 else N.RT_X0_ZERO)
        o.precision = {"fp64": N.RT_PRECISION_FP64, "fp32_refine": N.RT_PRECISION_FP32_REFINE}[precision]
        o.inner_rtol, o.max_refine = inner_rtol, max_refine
        hist = np.zeros(max(hist_cap, 1))
        if hist_cap:
            o.resid_hist, o.hist_cap = _dptr(hist), hist_cap
        info = N.SolveInfo()
        fn = {"gmres": self.lib.rt_solve_gmres, "bicgstab": self.lib.rt_solve_bicgstab,
              "cgs": self.lib.rt_solve_cgs, "richardson": self.lib.rt_solve_richardson}[method]
        st = fn(self.handle, C.byref(o), C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), C.byref(info),
                _stream_handle(stream))
        res = SolveResult(info.status, info.iters, info.restarts, info.applies, info.refine_steps,
                          info.rel_resid, info.err_est, info.t_total_ms, hist[: info.hist_len].copy())
        if raise_on_error and st not in (N.RT_OK, N.RT_ENOTCONV, N.RT_EBREAKDOWN):
            raise N.RTError(st, f"rt_solve_{method}")
        return x, res
