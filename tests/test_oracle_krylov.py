"""Pins of the oracle's Krylov solvers (Sect. 2) and of the whole oracle against
the iteration counts printed in the paper (Tables 1-3)."""
import json
import os

import numpy as np
import pytest

import rt_workloads as W
from oracle import krylov as K
from oracle.transfer import Transfer

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_iterations.json")


def _random_system(n, seed, shift=3.0):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) / np.sqrt(n) + shift * np.eye(n)
    b = rng.standard_normal(n)
    return A, b


@pytest.mark.parametrize("k", [1, 2, 3, 5, 8])
def test_gmres_iterate_minimises_the_residual_over_the_krylov_space(k):
    """x_k = argmin_{z in K_k(A,b)} ||b - A z||_2 (Sect. 2.1), checked by a
    least-squares solve on an orthonormalised Krylov matrix."""
    A, b = _random_system(40, k, shift=1.0)
    x, info = K.gmres(lambda v: A @ v, b, restart=k, maxit=k, tol=1e-30)
    assert info.iters == k
    Kmat = np.empty((40, k))
    v = b.copy()
    for j in range(k):
        Kmat[:, j] = v
        v = A @ v
    Qk, _ = np.linalg.qr(Kmat)
    c, *_ = np.linalg.lstsq(A @ Qk, b, rcond=None)
    np.testing.assert_allclose(x, Qk @ c, rtol=1e-10, atol=1e-12)


@pytest.mark.parametrize("ortho", ["mgs", "cgs2"])
def test_gmres_terminates_within_n_steps(ortho):
    """Without restarts GMRES ends after at most N steps (Sect. 2)."""
    A, b = _random_system(30, 7)
    x, info = K.gmres(lambda v: A @ v, b, restart=30, tol=1e-13, ortho=ortho)
    assert info.status == K.OK and info.iters <= 30
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-11)


def test_gmres_restarts_and_right_preconditioning():
    A, b = _random_system(60, 11, shift=2.5)
    d = np.abs(np.diag(A)) + 0.5
    x, info = K.gmres(lambda v: A @ v, b, M_inv=lambda v: v / d, restart=3, tol=1e-10)
    assert info.status == K.OK and info.restarts > 1
    true = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert true == pytest.approx(info.rel_resid, rel=1e-12) and true < 1e-10


@pytest.fixture(scope="module")
def tiny_problem():
    tr = Transfer(W.tiny(6, 4, 5, eps=1e-2))
    return tr, tr.rhs_I(), np.linalg.solve(tr.assemble_I(), tr.rhs_I())


@pytest.mark.parametrize("method", ["gmres", "gmres-cgs2", "bicgstab", "cgs", "richardson"])
@pytest.mark.parametrize("prec", ["none", "jacobi", "local-lambda"])
def test_solvers_reach_the_direct_solution(tiny_problem, method, prec):
    tr, b, xs = tiny_problem
    d = tr.jacobi_I()
    Minv = {"none": None, "jacobi": lambda v: v / d, "local-lambda": tr.local_lambda_I_inverse}[prec]
    if method == "richardson" and prec != "local-lambda":
        pytest.skip("Richardson only converges with a good preconditioner")
    kw = dict(M_inv=Minv, tol=1e-11, maxit=5000)
    if method.startswith("gmres"):
        x, info = K.gmres(tr.apply_I, b, restart=10,
                          ortho="cgs2" if method.endswith("cgs2") else "mgs", **kw)
    else:
        x, info = getattr(K, method)(tr.apply_I, b, **kw)
    assert info.status == K.OK
    assert np.linalg.norm(b - tr.apply_I(x)) / np.linalg.norm(b) < 1e-11
    np.testing.assert_allclose(x, xs, rtol=1e-8, atol=1e-10)


def test_mgs_and_cgs2_give_the_same_iterates(tiny_problem):
    tr, b, _ = tiny_problem
    x1, i1 = K.gmres(tr.apply_I, b, restart=7, maxit=21, tol=1e-30, ortho="mgs")
    x2, i2 = K.gmres(tr.apply_I, b, restart=7, maxit=21, tol=1e-30, ortho="cgs2")
    assert i1.iters == i2.iters == 21
    np.testing.assert_allclose(x1, x2, rtol=1e-10, atol=1e-13)


# --------------------------------------------------------------- paper mode
def _paper_system(Ns, Nmu=20, Nnu=20):
    """The paper's sigma-form problem, with its plain trapezoidal rule
    (no renormalisation of the spectral weights)."""
    tr = Transfer(W.paper(Ns, Nmu=Nmu, Nnu=Nnu, freq_norm=0))
    return tr, tr.rhs_sigma(), tr.jacobi_sigma(), np.tile([1.0, 0.0], Ns)


def _paper_counts(tr, b, d, x0, prec):
    """Preconditioning as in MATLAB's built-ins: gmres preconditions from the
    left (D^{-1} A x = D^{-1} b, stopping on the preconditioned residual),
    bicgstab and cgs from the right (stopping on the true residual)."""
    tol = 1e-6
    if not prec:
        return {"GMRES": K.gmres(tr.apply_sigma, b, x0=x0, restart=b.size, tol=tol)[1].iters}
    Minv = lambda v: v / d
    return {
        "GMRES": K.gmres(lambda v: tr.apply_sigma(v) / d, b / d, x0=x0, restart=b.size, tol=tol)[1].iters,
        "BICGSTAB": K.bicgstab(tr.apply_sigma, b, M_inv=Minv, x0=x0, tol=tol)[1].iters,
        "CGS": K.cgs(tr.apply_sigma, b, M_inv=Minv, x0=x0, tol=tol)[1].iters,
        "Richardson": K.richardson(tr.apply_sigma, b, M_inv=Minv, x0=x0, tol=tol, maxit=3000)[1].iters,
    }


@pytest.mark.slow
def test_paper_tables_2_and_3():
    gold = json.load(open(GOLDEN))
    t2, t3 = gold["table2_no_prec"], gold["table3_jacobi"]
    for i, Ns in enumerate(gold["Ns"]):
        sysm = _paper_system(Ns)
        c0 = _paper_counts(*sysm, prec=False)
        c1 = _paper_counts(*sysm, prec=True)
        assert c0["GMRES"] == t2["GMRES"][i], (Ns, c0)
        assert c1["GMRES"] == t3["GMRES"][i], (Ns, c1)
        assert c1["CGS"] == t3["CGS"][i], (Ns, c1)
        assert abs(c1["BICGSTAB"] - t3["BICGSTAB"][i]) <= 1, (Ns, c1)
        # the paper counts one more Richardson sweep than the updates made here
        assert c1["Richardson"] + 1 == t3["Richardson"][i], (Ns, c1)


@pytest.mark.slow
def test_paper_table_1_gmres_independent_of_angular_and_spectral_grids():
    gold = json.load(open(GOLDEN))["table1_nmu_nnu"]
    for n, ref in zip(gold["Nmu_Nnu"][:4], gold["GMRES"][:4]):
        tr, b, d, x0 = _paper_system(40, n, n)
        assert K.gmres(tr.apply_sigma, b, x0=x0, restart=80, tol=1e-6)[1].iters == ref
