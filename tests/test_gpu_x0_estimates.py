"""The paper's initial guess (RT_X0_PAPER) and the solvers' own residual
estimates (rt_solve_info.err_est), on the GPU.

* sigma-form: the initial guess is sigma = [1, 0, 1, 0, ...] exactly
  (Sect. 4.2); the paper's iteration counts (Tables 2 and 3) run through it
  in test_gpu_sigma.py;
* I-form: the initial guess is Lambda(T sigma) + t for that sigma (Eq. 16),
  against the oracle's lift at 1e-12 per Stokes block; GMRES from it after a
  forced equal number of steps gives the iterate of the oracle's textbook
  GMRES from the same x0 (the GPU's, read back) to 1e-7 per block -- the
  initial residual b - A x0 nearly cancels, which lifts the operators'
  rounding difference -- with residual norms equal to 1e-6, and with the
  local-Lambda preconditioner the oracle's count within one; converged solves from it
  reach the oracle's LU solution; BiCGSTAB, CGS and Richardson accept it;
* err_est: GMRES reports |g_{j+1}| / ||b|| of its last Arnoldi step -- the
  last entry of its residual history, bit for bit -- below rtol when it
  converged; BiCGSTAB and CGS their recursively updated residual, below
  rtol; Richardson the FP64 residual it formed (= rel_resid); with an FP32
  operator inside FP64 refinement a positive finite estimate; a solve that
  takes no step reports rel_resid.
"""
import numpy as np
import pytest
import torch

import rt_workloads as W
from oracle import krylov as K
from oracle.transfer import Transfer
from paper_2110_11873_gb300 import _native as N

from gpu_util import assert_close_scaled, problem, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slab70():
    at = W.slab70()
    tr = Transfer(at)
    return at, problem(at), tr, tr.rhs_I()


def _paper_x0_I(at, tr):
    return tr.lift(np.tile([1.0, 0.0], at.Ns))


def test_sigma_form_initial_guess_is_one_zero():
    at = W.paper(40, freq_norm=0)
    P = problem(at, form="sigma")
    b = P.rhs()
    x, info = P.solve(b, "gmres", x0="paper", rtol=1e30)   # the initial residual already meets rtol
    assert info.status == 0 and info.iters == 0
    np.testing.assert_array_equal(to_host(x), np.tile([1.0, 0.0], at.Ns))


@pytest.mark.parametrize("name,at", [("slab70", W.slab70()),
                                     ("ragged-B", W.slab(37, 6, 33, 1e-4, 1e6, 6.0, Bc=0.3, eps=1e-3)),
                                     ("euler", W.tiny().with_(formal_solver=W.FS_IMPLICIT_EULER))])
def test_I_form_initial_guess_is_the_lifted_sigma(name, at):
    tr = Transfer(at)
    P = problem(at)
    x, info = P.solve(P.rhs(), "gmres", x0="paper", rtol=1e30)
    assert info.status == 0 and info.iters == 0
    assert_close_scaled(to_host(x), _paper_x0_I(at, tr), 1e-12, f"paper x0 {name}")


@pytest.mark.parametrize("prec,iters", [("local_lambda", 12), ("jacobi", 40)])
def test_gmres_from_the_paper_guess_matches_the_oracle(slab70, prec, iters):
    at, P, tr, b = slab70
    # the oracle starts from the GPU's own initial guess (pinned to the
    # oracle's lift above), so only the solvers are compared
    x0g, i0 = P.solve(to_dev(b), "gmres", x0="paper", rtol=1e30)
    assert i0.iters == 0
    x0 = to_host(x0g)
    assert_close_scaled(x0, _paper_x0_I(at, tr), 1e-12, "paper x0")
    xg, info = P.solve(to_dev(b), "gmres", x0="paper", restart=30, precond=prec, rtol=1e-30, maxit=iters)
    assert info.status == N.RT_ENOTCONV and info.iters == iters
    d = tr.jacobi_I()
    M = {"jacobi": lambda v: v / d, "local_lambda": tr.local_lambda_I_inverse}[prec]
    xo, io = K.gmres(tr.apply_I, b, M_inv=M, x0=x0, restart=30, tol=1e-30, maxit=iters)
    assert io.iters == iters
    # r0 = b - A x0 nearly cancels when x0 is this close to the solution, so
    # the two operators' rounding difference in A x0 reaches the iterate far
    # above rounding (2.6e-10 in I and 3.5e-9 in Q, relative, after 12
    # local-Lambda steps on slab70); a wrong or ignored x0 moves it at O(1).
    # The residual norm that GMRES minimises agrees closely.
    xgh = to_host(xg)
    assert_close_scaled(xgh, xo, 1e-7, f"gmres {prec} from the paper's x0 after {iters}")
    rg, ro = (np.linalg.norm(b - tr.apply_I(v)) for v in (xgh, xo))
    assert abs(rg - ro) <= 1e-6 * ro, (rg, ro)
    if prec == "local_lambda":   # a stable count: converged from the same x0, the same count within one
        _, ic = P.solve(to_dev(b), "gmres", x0="paper", restart=30, precond=prec, rtol=1e-8)
        _, oc = K.gmres(tr.apply_I, b, M_inv=M, x0=x0, restart=30, tol=1e-8)
        assert ic.status == 0 and abs(ic.iters - oc.iters) <= 1, (ic.iters, oc.iters)


@pytest.fixture(scope="module")
def thin():
    at = W.slab(30, 8, 21, 1e-4, 1e6, 6.0, eps=1e-2)   # Richardson converges in a few dozen sweeps
    tr = Transfer(at)
    return at, problem(at), tr, tr.rhs_I()


@pytest.mark.parametrize("method", ["gmres", "bicgstab", "cgs", "richardson"])
def test_converged_solves_from_the_paper_guess(slab70, thin, method):
    at, P, tr, b = thin if method == "richardson" else slab70
    prec = "jacobi" if method in ("cgs", "richardson") else "local_lambda"
    x, info = P.solve(to_dev(b), method, x0="paper", restart=30, precond=prec, rtol=1e-8, maxit=20000)
    assert info.status == 0, (method, info)
    xh = to_host(x)
    assert np.linalg.norm(b - tr.apply_I(xh)) / np.linalg.norm(b) < 1e-8
    assert info.applies >= info.iters   # the initial residual takes a product with A


def test_gmres_estimate_is_its_last_history_entry(slab70):
    at, P, tr, b = slab70
    for prec in ("local_lambda", "jacobi"):
        x, info = P.solve(to_dev(b), "gmres", restart=30, precond=prec, rtol=1e-8, hist_cap=5000)
        assert info.status == 0 and len(info.history) == info.iters
        assert info.err_est == info.history[-1]
        assert info.err_est < 1e-8
        # the estimate tracks the true residual (FP64 Arnoldi on this operator)
        assert info.rel_resid < 1e-8 and 0.1 < info.err_est / info.rel_resid < 10.0, (prec, info)


@pytest.mark.parametrize("method,prec", [("bicgstab", "local_lambda"), ("cgs", "jacobi")])
def test_bicgstab_cgs_estimate_is_the_recursive_residual(slab70, method, prec):
    at, P, tr, b = slab70
    x, info = P.solve(to_dev(b), method, precond=prec, rtol=1e-8, hist_cap=20000)
    assert info.status == 0
    assert info.err_est < 1e-8
    if method == "cgs":   # (a BiCGSTAB run may stop at a half step, which the history does not record)
        assert info.err_est == info.history[-1]


def test_richardson_estimate_is_its_residual(thin):
    at, P, tr, b = thin
    x, info = P.solve(to_dev(b), "richardson", precond="jacobi", rtol=1e-8, maxit=5000)
    assert info.status == 0 and info.err_est == info.rel_resid


def test_refinement_estimate_and_no_step_cases(slab70):
    at, P, tr, b = slab70
    x, info = P.solve(to_dev(b), "gmres", precond="local_lambda", precision="fp32_refine", rtol=1e-8)
    assert info.status == 0 and np.isfinite(info.err_est) and info.err_est > 0.0
    # converged at the initial guess: no step, the estimate is the residual itself
    x2, info2 = P.solve(to_dev(b), "gmres", x=x, x0=True, precond="local_lambda", rtol=1e-2)
    assert info2.iters == 0 and info2.err_est == info2.rel_resid
