"""Pins of the oracle's operators (Eq. 7-19, Algorithm 1) against closed forms,
invariants and brute force on tiny grids (CPU)."""
import math

import numpy as np
import pytest

import rt_workloads as W
from oracle.formal import FS_DELO_LINEAR, FS_IMPLICIT_EULER, FS_TRAPEZOIDAL
from oracle.transfer import Transfer

SOLVERS = [FS_DELO_LINEAR, FS_IMPLICIT_EULER, FS_TRAPEZOIDAL]


def _tiny(fs=FS_DELO_LINEAR, **kw):
    at = W.tiny(6, 4, 5, formal_solver=fs)
    at = at.with_(B=W.planck_profile(at.tau, 1.0, 0.4), eps=3e-2)
    return Transfer(at.with_(**kw) if kw else at)


def test_radiation_moments_closed_forms():
    tr = Transfer(W.slab70())
    g = tr.g
    ones = np.ones((g.Ns, g.Nmu, g.Nnu))
    zeros = np.zeros_like(ones)
    J00, J20 = tr.radiation_moments(ones, zeros)
    np.testing.assert_allclose(J00, 1.0, atol=1e-15)
    np.testing.assert_allclose(J20, 0.0, atol=1e-15)
    mu2 = np.broadcast_to((g.mu ** 2)[None, :, None], ones.shape)
    J00, J20 = tr.radiation_moments(mu2, zeros)
    np.testing.assert_allclose(J00, 1.0 / 3.0, atol=1e-15)
    np.testing.assert_allclose(J20, math.sqrt(2) / 15.0, atol=1e-15)
    J00, J20 = tr.radiation_moments(zeros, ones)
    np.testing.assert_allclose(J00, 0.0, atol=0)
    np.testing.assert_allclose(J20, -math.sqrt(2) / 2.0, atol=1e-15)


def test_source_functions():
    tr = Transfer(W.slab70())
    g = tr.g
    SI, SQ = tr.T_apply(np.ones(g.Ns), np.zeros(g.Ns))
    assert np.all(SI == 1.0) and np.all(SQ == 0.0)
    SI, SQ = tr.T_apply(np.zeros(g.Ns), np.ones(g.Ns))
    np.testing.assert_allclose(SI, np.broadcast_to(math.sqrt(2) * (3 * g.mu ** 2 - 1) / 4, SI.shape))
    np.testing.assert_allclose(SQ, np.broadcast_to(math.sqrt(2) * (3 * g.mu ** 2 - 3) / 4, SQ.shape))


def test_eps_one_gives_identity_and_planck_source():
    """eps = 1: xi = 0, so A = Id and sigma00 = B, sigma20 = 0 exactly."""
    tr = _tiny(eps=1.0)
    x = W.random_vector(tr.N, 3)
    assert np.array_equal(tr.apply_I(x), x)
    sig = tr.exact_sigma().reshape(-1, 2)
    np.testing.assert_allclose(sig[:, 0], tr.g.B, rtol=1e-15)
    assert np.all(sig[:, 1] == 0.0)


@pytest.mark.parametrize("fs", SOLVERS)
def test_unpolarizable_line_has_no_Q(fs):
    """W2 = 0: sigma20 = 0 and Q = 0 everywhere."""
    tr = _tiny(fs, W2=0.0)
    sig = tr.exact_sigma().reshape(-1, 2)
    assert np.all(sig[:, 1] == 0.0)
    I = tr.exact_I().reshape(tr.shape)
    assert np.all(I[1] == 0.0)


@pytest.mark.parametrize("fs", SOLVERS)
def test_jacobi_diagonals_match_assembled_matrices(fs):
    tr = _tiny(fs)
    AI = tr.assemble_I()
    np.testing.assert_allclose(tr.jacobi_I(), np.diag(AI), rtol=0, atol=1e-15)
    As = tr.assemble_sigma()
    np.testing.assert_allclose(tr.jacobi_sigma(), np.diag(As), rtol=0, atol=1e-15)
    M = tr.local_blocks_sigma()
    for k in range(tr.g.Ns):
        np.testing.assert_allclose(M[k], As[2 * k:2 * k + 2, 2 * k:2 * k + 2], rtol=0, atol=1e-15)


@pytest.mark.parametrize("fs", SOLVERS)
def test_sigma_and_I_forms_have_the_same_solution(fs):
    """If sigma* solves Eq. (18), Lambda T sigma* + t solves Eq. (19): compare
    the lifted 2N_s LU solution with an LU solve of the assembled I-form."""
    tr = _tiny(fs)
    I_lift = tr.exact_I()
    I_direct = np.linalg.solve(tr.assemble_I(), tr.rhs_I())
    np.testing.assert_allclose(I_lift, I_direct, rtol=1e-12, atol=1e-14)
    # and sigma* = J I* + c
    s00, s20 = tr.J_apply(I_direct)
    c00, _ = tr.c_vector()
    np.testing.assert_allclose(np.stack([s00 + c00, s20], 1).reshape(-1), tr.exact_sigma(),
                               rtol=1e-12, atol=1e-14)


def test_spectra_of_the_two_forms():
    """The nonzero spectrum of Lambda T J equals that of J Lambda T: eig(A_I)
    is eig(A_sigma) plus N - 2N_s unit eigenvalues."""
    tr = _tiny()
    ls = np.linalg.eigvals(tr.assemble_sigma())
    lI = np.linalg.eigvals(tr.assemble_I())
    for lam in ls:
        assert np.min(np.abs(lI - lam)) < 1e-8
    far = np.abs(lI - 1.0) > 1e-6
    assert far.sum() <= ls.size


@pytest.mark.parametrize("fs", [FS_DELO_LINEAR, FS_IMPLICIT_EULER])
def test_coefficient_matrix_is_positive_definite(fs):
    """A = Id - J Lambda T is nonsymmetric and positive definite (Sect. 3.2,
    Fig. 1), for the paper's formal solvers (the trapezoidal rule is not one of
    them, and on optically thick steps its symmetric part is indefinite)."""
    tr = _tiny(fs, eps=1e-4)
    A = tr.assemble_sigma()
    assert np.abs(A - A.T).max() > 1e-3
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0
    assert np.all(np.linalg.eigvals(A).real > 0)


def test_local_lambda_preconditioner_is_an_exact_inverse():
    tr = _tiny()
    v = W.random_vector(tr.N, 5)
    np.testing.assert_allclose(tr.local_lambda_I_inverse(tr.local_lambda_I(v)), v, rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(tr.local_lambda_I(tr.local_lambda_I_inverse(v)), v, rtol=1e-13, atol=1e-14)


def test_local_lambda_preconditioned_spectrum_is_block_jacobi_sigma_form():
    """spec(A_I P^{-1}) = spec(M^{-1} A_sigma) plus unit eigenvalues, with M the
    2x2-per-height block diagonal of A_sigma."""
    tr = _tiny(eps=1e-3)
    AI = tr.assemble_I()
    Pinv = tr.assemble(tr.local_lambda_I_inverse, tr.N)
    lI = np.linalg.eigvals(AI @ Pinv)
    As = tr.assemble_sigma()
    M = np.zeros_like(As)
    for k, blk in enumerate(tr.local_blocks_sigma()):
        M[2 * k:2 * k + 2, 2 * k:2 * k + 2] = blk
    ls = np.linalg.eigvals(np.linalg.solve(M, As))
    for lam in ls:
        assert np.min(np.abs(lI - lam)) < 1e-8


def test_rhs_of_the_two_forms():
    """b_I = Lambda T c + t and b_sigma = J t + c from the same pieces."""
    tr = _tiny()
    t = tr.transmitted()
    c00, c20 = tr.c_vector()
    SI, SQ = tr.T_apply(c00, c20)
    np.testing.assert_allclose(tr.rhs_I(), tr.Lambda_apply(SI, SQ) + t, rtol=1e-14, atol=1e-15)
    s00, s20 = tr.J_apply(t)
    np.testing.assert_allclose(tr.rhs_sigma(), np.stack([s00 + c00, s20], 1).reshape(-1), rtol=1e-15)
    # transmitted radiation: zero for mu<0 rays (no light enters at the top), and
    # the bottom value B(tau_Ns) at the bottom for mu>0 rays
    T = t.reshape(tr.shape)
    dn = tr.g.mu < 0
    assert np.all(T[:, :, dn, :] == 0.0)
    assert np.all(T[0, -1, ~dn, :] == tr.g.B[-1])
    assert np.all(T[1] == 0.0)


@pytest.mark.slow
def test_sqrt_eps_surface_law_under_refinement():
    """Semi-infinite isothermal slab, CRD: S(0) = sqrt(eps) B.  On the discrete
    grid the ratio approaches 1 as the depth grid is refined."""
    ratios = []
    for Ns in (70, 140, 280):
        at = W.slab(Ns, 16, 21, 1e-4, 1e8, 6.0, eps=1e-2, W2=0.0)
        tr = Transfer(at)
        ratios.append(tr.exact_sigma()[0] / math.sqrt(at.eps))
    assert ratios[0] < ratios[1] < ratios[2] <= 1.0
    assert abs(ratios[2] - 1.0) < 0.02, ratios
