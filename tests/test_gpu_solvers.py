"""GPU Krylov solvers against the oracle (C-ABI path).

* iteration counts within +-1 of the range the oracle's textbook solvers
  (same algorithm, x0, restart length and stopping rule) give for b and for
  b perturbed by 1e-15 relative: where a method amplifies rounding (CGS, and
  BiCGSTAB or restarted GMRES with the literal I-form Jacobi diagonal) that
  range is wide -- on slab70 the oracle's own Jacobi-BiCGSTAB count moves
  between 217 and 284 -- and a fixed +-1 would test the rounding, not the
  method; where the method is stable the range is one count;
* FP64 iterates at a forced equal number of iterations agree element by
  element, per Stokes block (each scaled by its own largest entry), to
  1e-10 relative, or to 20 times the oracle's own change under the 1e-15
  perturbation where that is larger;
* a NaN placed in b or in the initial guess ends every solver with
  RT_ENUMERIC;
* converged FP64 solutions satisfy ||b - A x||/||b|| < rtol with the
  oracle's FP64 operator, and mixed-precision solutions reach the same
  residual after refinement and lie within 1e-6 of the exact (LU) solution.
"""
import numpy as np
import pytest
import torch

import rt_workloads as W
from oracle import krylov as K
from oracle.transfer import Transfer
from paper_2110_11873_gb300 import _native as N

from gpu_util import assert_close_scaled, assert_iterate as _assert_iterate, perturbed as _perturbed, problem, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def slab70():
    at = W.slab70()
    tr = Transfer(at)
    return at, problem(at), tr, tr.rhs_I(), tr.exact_I()


def _oracle_solve(tr, b, method, prec, **kw):
    d = tr.jacobi_I()
    Minv = {"none": None, "jacobi": lambda v: v / d, "local_lambda": tr.local_lambda_I_inverse}[prec]
    fn = {"gmres": K.gmres, "bicgstab": K.bicgstab, "cgs": K.cgs}[method]
    return fn(tr.apply_I, b, M_inv=Minv, **kw)


def _oracle_count_range(tr, b, method, prec, copies=2, **kw):
    """Iteration counts of the oracle for b and for `copies` rounding-level
    perturbations of b: (min, max, info for b, x for b)."""
    xo, io = _oracle_solve(tr, b, method, prec, **kw)
    counts = [io.iters]
    for sd in range(1, copies + 1):
        counts.append(_oracle_solve(tr, _perturbed(b, sd), method, prec, **kw)[1].iters)
    return min(counts), max(counts), io, xo


def _assert_count(got, lo, hi):
    """A stable method (lo == hi) must match within +-1; for a method whose
    count the oracle's own rounding moves, the band is the sampled range
    widened on each side by its width (a new sample falls outside the range
    of k samples with probability 2/(k+1))."""
    pad = 1 + (hi - lo)
    assert lo - pad <= got <= hi + pad, (got, lo, hi)


def _true_rel(tr, b, x):
    return np.linalg.norm(b - tr.apply_I(x)) / np.linalg.norm(b)


@pytest.mark.parametrize("prec", ["local_lambda", "jacobi", "none"])
def test_gmres_slab70(slab70, prec):
    at, P, tr, b, xs = slab70
    xg, info = P.solve(to_dev(b), "gmres", restart=30, precond=prec, rtol=1e-8)
    assert info.ok, info
    lo, hi, io, xo = _oracle_count_range(tr, b, "gmres", prec, restart=30, tol=1e-8)
    _assert_count(info.iters, lo, hi)
    x = to_host(xg)
    assert _true_rel(tr, b, x) < 1e-8
    assert abs(info.rel_resid - _true_rel(tr, b, x)) < 1e-10
    # same accuracy class as the oracle against the exact LU solution
    eo = np.linalg.norm(xo - xs) / np.linalg.norm(xs)
    eg = np.linalg.norm(x - xs) / np.linalg.norm(xs)
    assert eg < 5 * eo + 1e-12, (eg, eo)


@pytest.mark.parametrize("prec,iters", [("local_lambda", 12), ("jacobi", 75)])
def test_gmres_iterates_at_equal_iteration_count(slab70, prec, iters):
    at, P, tr, b, xs = slab70
    xg, info = P.solve(to_dev(b), "gmres", restart=30, precond=prec, rtol=1e-30, maxit=iters)
    assert info.status == N.RT_ENOTCONV and info.iters == iters
    xo, io = _oracle_solve(tr, b, "gmres", prec, restart=30, tol=1e-30, maxit=iters)
    assert io.iters == iters
    xp, _ = _oracle_solve(tr, _perturbed(b, 1), "gmres", prec, restart=30, tol=1e-30, maxit=iters)
    _assert_iterate(to_host(xg), xo, xp, f"gmres {prec} after {iters}")


@pytest.mark.parametrize("method,prec", [("bicgstab", "local_lambda"), ("bicgstab", "jacobi"), ("cgs", "jacobi")])
def test_bicgstab_cgs_slab70(slab70, method, prec):
    """(CGS with the local-Lambda preconditioner is left out: on slab70 the
    oracle's own CGS diverges for some 1e-15 perturbations of b; its iterates
    are compared at equal counts below.)"""
    at, P, tr, b, xs = slab70
    xg, info = P.solve(to_dev(b), method, precond=prec, rtol=1e-8, maxit=4000)
    lo, hi, io, xo = _oracle_count_range(tr, b, method, prec, copies=3, tol=1e-8, maxit=4000)
    assert io.status == K.OK
    assert info.ok, info
    _assert_count(info.iters, lo, hi)
    assert _true_rel(tr, b, to_host(xg)) < 2e-8


@pytest.mark.parametrize("method", ["bicgstab", "cgs"])
def test_bicgstab_cgs_iterates_at_equal_iteration_count(slab70, method):
    at, P, tr, b, xs = slab70
    xg, info = P.solve(to_dev(b), method, precond="local_lambda", rtol=1e-30, maxit=6)
    xo, io = _oracle_solve(tr, b, method, "local_lambda", tol=1e-30, maxit=6)
    assert info.iters == io.iters == 6
    # the method's own amplification of rounding: the oracle against itself
    xp, _ = _oracle_solve(tr, _perturbed(b, 1), method, "local_lambda", tol=1e-30, maxit=6)
    _assert_iterate(to_host(xg), xo, xp, method)


def test_mixed_precision_refinement_slab70(slab70):
    at, P, tr, b, xs = slab70
    xg, info = P.solve(to_dev(b), "gmres", precond="local_lambda", rtol=1e-8, precision="fp32_refine",
                       inner_rtol=1e-4)
    assert info.ok and info.refine_steps >= 2, info
    x = to_host(xg)
    assert _true_rel(tr, b, x) < 1e-8
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-6


@pytest.mark.parametrize("prec", ["jacobi", "local_lambda"])
def test_fp32_refine_default_refines_at_every_restart(slab70, prec):
    """The default inner tolerance of FP32-refine GMRES is the outer one:
    every restart cycle of the inner solve starts from its FP64 residual, so
    the one inner solve is the refinement.  It meets the stopping rule with
    the oracle's FP64 operator, in one outer step, with an Arnoldi step count
    close to the FP64 solver's; and a smaller explicit inner tolerance stops
    where the outer one is met instead of over-solving."""
    at, P, tr, b, xs = slab70
    _, i64 = P.solve(to_dev(b), "gmres", precond=prec, rtol=1e-8)
    xg, info = P.solve(to_dev(b), "gmres", precond=prec, rtol=1e-8, precision="fp32_refine")
    assert info.ok and info.refine_steps == 1, info
    assert info.iters <= 1.3 * i64.iters + 10, (info.iters, i64.iters)
    x = to_host(xg)
    assert _true_rel(tr, b, x) < 1e-8
    if prec == "local_lambda":   # well conditioned: the residual bounds the error
        assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-6
    _, i6 = P.solve(to_dev(b), "gmres", precond=prec, rtol=1e-8, precision="fp32_refine", inner_rtol=1e-6)
    # a second step asks only for what the outer tolerance still needs (about
    # 1e-2), not 1e-6 again (which took the residual to about 1e-12)
    assert i6.ok and i6.refine_steps <= 2 and i6.rel_resid > 1e-11, i6


def test_user_initial_guess_and_zero_rhs(slab70):
    at, P, tr, b, xs = slab70
    # the exact solution as initial guess: converged before any iteration
    xg, info = P.solve(to_dev(b), "gmres", x=to_dev(xs), x0=True, precond="local_lambda")
    assert info.ok and info.iters == 0 and info.applies == 1
    # b = 0: x = 0
    z = torch.zeros(tr.N, dtype=torch.float64, device="cuda")
    for m in ("gmres", "bicgstab", "cgs"):
        xg, info = P.solve(z, m, x=to_dev(xs), precond="jacobi")
        assert info.ok and info.iters == 0 and float(xg.abs().max()) == 0.0


def test_maxit_reached_reports_not_converged(slab70):
    at, P, tr, b, xs = slab70
    xg, info = P.solve(to_dev(b), "gmres", precond="jacobi", maxit=7)
    assert info.status == N.RT_ENOTCONV and info.iters == 7
    xg, info = P.solve(to_dev(b), "bicgstab", precond="jacobi", maxit=3)
    assert info.status == N.RT_ENOTCONV and info.iters == 3


def test_residual_history_is_recorded(slab70):
    at, P, tr, b, xs = slab70
    xg, info = P.solve(to_dev(b), "gmres", precond="local_lambda", hist_cap=200)
    xo, io = _oracle_solve(tr, b, "gmres", "local_lambda", restart=30, tol=1e-8)
    n = min(len(info.history), len(io.history))
    assert n >= info.iters - 1
    np.testing.assert_allclose(info.history[:n], io.history[:n], rtol=1e-6, atol=1e-11)


@pytest.mark.slow
@pytest.mark.parametrize("fs", [W.FS_DELO_LINEAR, W.FS_IMPLICIT_EULER])
def test_slab300_gmres_fp64_and_mixed(fs):
    """The benchmark workload: 1,939,200 unknowns."""
    at = W.slab300(formal_solver=fs)
    P, tr = problem(at), Transfer(at)
    b = tr.rhs_I()
    xs = tr.exact_I()
    lo, hi, io, xo = _oracle_count_range(tr, b, "gmres", "local_lambda", copies=1, restart=30, tol=1e-8)
    xg, info = P.solve(to_dev(b), "gmres", precond="local_lambda", rtol=1e-8)
    assert info.ok
    _assert_count(info.iters, lo, hi)
    assert _true_rel(tr, b, to_host(xg)) < 1e-8
    xm, im = P.solve(to_dev(b), "gmres", precond="local_lambda", rtol=1e-8, precision="fp32_refine")
    assert im.ok
    x = to_host(xm)
    assert _true_rel(tr, b, x) < 1e-8
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-6


@pytest.mark.parametrize("precond", ["jacobi", "local_lambda"])
def test_richardson_matches_the_oracle(precond):
    """Preconditioned Richardson (Eq. 20) on an I-form atmosphere with
    eps = 1e-2 (a few dozen sweeps): the same count as the oracle's loop
    within 1, and the true residual below the tolerance."""
    at = W.slab(30, 8, 21, 1e-4, 1e6, 6.0, eps=1e-2)
    tr = Transfer(at)
    P = problem(at)
    b = tr.rhs_I()
    M_inv = (lambda v: v / tr.jacobi_I()) if precond == "jacobi" else tr.local_lambda_I_inverse
    _, oi = K.richardson(tr.apply_I, b, M_inv=M_inv, tol=1e-8, maxit=5000)
    xg, info = P.solve(to_dev(b), "richardson", precond=precond, rtol=1e-8, maxit=5000, hist_cap=5000)
    assert info.status == 0, info
    assert abs(info.iters - oi.iters) <= 1, (info.iters, oi.iters)
    x = to_host(xg)
    assert np.linalg.norm(b - tr.apply_I(x)) / np.linalg.norm(b) < 1e-8
    assert len(info.history) == info.iters and info.history[-1] < 1e-8 <= info.history[-2]


@pytest.mark.slow
def test_slab300_jacobi_gmres_iterates_and_count():
    """The benchmarked solve itself: Jacobi-GMRES(30) on slab300 (FP64).
    After a forced 60 Arnoldi steps (two restarts) the GPU iterate equals the
    oracle's element by element per Stokes block; the converged count lies
    in the band the oracle's own counts span for b and a 1e-15 perturbation
    of b, and the converged solution meets the stopping rule with the
    oracle's operator."""
    at = W.slab300()
    P, tr = problem(at), Transfer(at)
    b = tr.rhs_I()
    xg, info = P.solve(to_dev(b), "gmres", restart=30, precond="jacobi", rtol=1e-30, maxit=60)
    assert info.status == N.RT_ENOTCONV and info.iters == 60 and info.restarts == 2, info
    xo, io = _oracle_solve(tr, b, "gmres", "jacobi", restart=30, tol=1e-30, maxit=60)
    xp, _ = _oracle_solve(tr, _perturbed(b, 1), "gmres", "jacobi", restart=30, tol=1e-30, maxit=60)
    assert io.iters == 60
    _assert_iterate(to_host(xg), xo, xp, "slab300 jacobi gmres after 60")
    xc, ic = P.solve(to_dev(b), "gmres", restart=30, precond="jacobi", rtol=1e-8)
    assert ic.ok, ic
    lo, hi, _, _ = _oracle_count_range(tr, b, "gmres", "jacobi", copies=1, restart=30, tol=1e-8)
    _assert_count(ic.iters, lo, hi)
    assert _true_rel(tr, b, to_host(xc)) < 1e-8


@pytest.mark.parametrize("method,precision", [("gmres", "fp64"), ("gmres", "fp32_refine"), ("bicgstab", "fp64"),
                                              ("cgs", "fp64"), ("richardson", "fp64")])
def test_nan_in_the_right_hand_side_reports_numeric(slab70, method, precision):
    """A NaN placed in b on the host: every solver stops with RT_ENUMERIC
    instead of iterating on NaN, and the problem stays usable."""
    at, P, tr, b, xs = slab70
    bn = b.copy()
    bn[bn.size // 3] = np.nan
    _, info = P.solve(to_dev(bn), method, precond="jacobi", rtol=1e-8, maxit=200, precision=precision,
                      raise_on_error=False)
    assert info.status == N.RT_ENUMERIC, info
    xg, info = P.solve(to_dev(b), "gmres", precond="local_lambda", rtol=1e-8)
    assert info.ok and _true_rel(tr, b, to_host(xg)) < 1e-8


def test_nan_in_the_initial_guess_reports_numeric(slab70):
    at, P, tr, b, xs = slab70
    x0 = xs.copy()
    x0[7] = np.nan
    for method in ("gmres", "bicgstab", "cgs"):
        _, info = P.solve(to_dev(b), method, x=to_dev(x0), x0=True, precond="jacobi", rtol=1e-8, maxit=50,
                          raise_on_error=False)
        assert info.status == N.RT_ENUMERIC, (method, info)


@pytest.mark.parametrize("method", ["bicgstab", "cgs"])
@pytest.mark.parametrize("prec", ["local_lambda", "jacobi"])
def test_bicgstab_cgs_with_fp32_operator_and_refinement(slab70, method, prec):
    """BiCGSTAB and CGS with the FP32 operator inside FP64 iterative
    refinement, on an atmosphere where their FP64 counts are stable under
    perturbations of the FP32 size (eps = 1e-2; the oracle's CGS counts move
    by less than one iteration under 1e-7 perturbations of b): the stopping
    rule with the oracle's FP64 operator and the exact (LU) solution within
    1e-6.  On slab70 with the literal Jacobi diagonal the FP32 inner solves
    do not converge (the FP64 counts there already move by 30% under 1e-15
    perturbations); the refinement then rejects their corrections, so the
    returned iterate's residual is never worse than the initial guess's, and
    the reported residual is the true one."""
    at = W.slab(40, 8, 21, 1e-4, 1e6, 6.0, eps=1e-2)
    tr = Transfer(at)
    P = problem(at)
    b = tr.rhs_I()
    xs = tr.exact_I()
    xg, info = P.solve(to_dev(b), method, precond=prec, rtol=1e-8, precision="fp32_refine", inner_rtol=1e-4,
                       maxit=4000)
    assert info.ok and info.refine_steps >= 2, info
    x = to_host(xg)
    assert _true_rel(tr, b, x) < 1e-8
    assert np.linalg.norm(x - xs) / np.linalg.norm(xs) < 1e-6
    at70, P70, tr70, b70, xs70 = slab70
    xj, ij = P70.solve(to_dev(b70), method, precond="jacobi", rtol=1e-8, precision="fp32_refine", maxit=600,
                       raise_on_error=False)
    assert ij.status in (N.RT_OK, N.RT_ENOTCONV), ij
    rj = _true_rel(tr70, b70, to_host(xj))
    assert rj <= 1.0 + 1e-12
    assert abs(ij.rel_resid - rj) < 1e-6
