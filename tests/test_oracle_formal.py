"""Pins of the oracle's formal solvers (Eq. 9-10) against closed forms (CPU)."""
import math

import mpmath
import numpy as np
import pytest

import rt_workloads as W
from oracle import formal as F
from oracle.grids import Grids


def _atm(tau, Nmu=4, Nnu=5, fs=F.FS_DELO_LINEAR, x_max=3.0):
    tau = np.asarray(tau, dtype=np.float64)
    return W.Atmosphere(Ns=tau.size, Nmu=Nmu, Nnu=Nnu, tau=tau, B=np.ones(tau.size),
                        x_min=-x_max, x_max=x_max, a=1e-3, eps=1e-4, W2=1.0,
                        tau_kind=W.TAU_LINE_CENTER, mu_quad=W.MU_GL_HALF, formal_solver=fs)


def _linear_solution(tau, r, s0, s1, I0, down):
    """Exact solution of dI/dt = S - I along a ray for S linear in tau,
    evaluated with 40 significant digits.

    t is the optical path from the entry node; S(t) = S(0) + S' t;
    I(t) = S(t) - S' + (I0 - S(0) + S') e^{-t}.
    """
    mpmath.mp.dps = 40
    r, s0, s1, I0 = (mpmath.mpf(float(v)) for v in (r, s0, s1, I0))
    taus = [mpmath.mpf(float(v)) for v in tau]
    out = []
    for tk in taus:
        if down:
            t = r * (tk - taus[0])
            S0, Sp = s0 + s1 * taus[0], s1 / r
        else:
            t = r * (taus[-1] - tk)
            S0, Sp = s0 + s1 * taus[-1], -s1 / r
        out.append(float(S0 + Sp * t - Sp + (I0 - S0 + Sp) * mpmath.exp(-t)))
    return np.array(out)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_delo_linear_exact_for_linear_source(seed):
    rng = np.random.default_rng(seed)
    tau = np.cumsum(rng.uniform(1e-3, 0.7, 40)) + rng.uniform(0, 1e-2)
    g = Grids(_atm(tau))
    fs = F.FormalSolver(g)
    s0, s1, Itop, Ibot = 0.3, 1.7, 0.25, 2.0
    S = np.repeat((s0 + s1 * tau)[:, None], g.Nmu, axis=1)
    I = fs.solve(S, inflow_top=Itop, inflow_bottom=Ibot)
    for m in range(g.Nmu):
        for p in range(g.Nnu):
            r = g.phi_hat[p] / abs(g.mu[m])
            down = g.mu[m] < 0
            ref = _linear_solution(tau, r, s0, s1, Itop if down else Ibot, down)
            np.testing.assert_allclose(I[:, m, p], ref, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("fs_kind", [F.FS_DELO_LINEAR, F.FS_IMPLICIT_EULER, F.FS_TRAPEZOIDAL])
def test_constant_source_is_preserved(fs_kind):
    tau = W.log_tau(1e-6, 1e7, 50)
    g = Grids(_atm(tau, fs=fs_kind))
    fs = F.FormalSolver(g)
    np.testing.assert_allclose(fs.e + fs.alpha + fs.beta, 1.0, rtol=0, atol=5e-16)
    I = fs.solve(np.ones((g.Ns, g.Nmu)), inflow_top=1.0, inflow_bottom=1.0)
    np.testing.assert_allclose(I, 1.0, rtol=0, atol=1e-14)
    # thick ray, zero inflow: deep inside the slab I -> S for the L-stable
    # schemes; the trapezoidal step factor tends to -1 as Delta grows, so its
    # zero-inflow transient does not die out on optically thick steps
    I0 = fs.solve(np.ones((g.Ns, g.Nmu)))
    down = g.mu < 0
    if fs_kind != F.FS_TRAPEZOIDAL:
        assert np.all(np.abs(I0[-1, down, :] - 1.0) < 1e-12)
    else:
        assert np.all(np.abs(I0[-1, down, :] - 1.0) < 1e-2)


def _sine_solution(t_end, omega, c):
    """int_0^t e^{-(t-s)} sin(c + omega s) ds."""
    f = lambda t: (math.sin(c + omega * t) - omega * math.cos(c + omega * t)) / (1 + omega ** 2)
    return f(t_end) - math.exp(-t_end) * f(0.0)


@pytest.mark.parametrize("fs_kind,order", [(F.FS_IMPLICIT_EULER, 1), (F.FS_TRAPEZOIDAL, 2),
                                           (F.FS_DELO_LINEAR, 2)])
def test_observed_order_of_accuracy(fs_kind, order):
    """Error at the end of a line-centre ray for S = sin(tau), halving the step."""
    errs = []
    for Ns in (21, 41, 81, 161):
        tau = np.linspace(0.0, 3.0, Ns)
        g = Grids(_atm(tau, Nnu=3, fs=fs_kind, x_max=1.0))
        fs = F.FormalSolver(g)
        I = fs.solve(np.repeat(np.sin(tau)[:, None], g.Nmu, axis=1))
        m = 0                                  # the most oblique downward ray
        r = g.phi_hat[1] / abs(g.mu[m])        # p=1 is x=0, phi_hat=1
        ref = _sine_solution(r * 3.0, 1.0 / r, 0.0)
        errs.append(abs(I[-1, m, 1] - ref))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) > order - 0.15 and max(rates) < order + 0.3, rates


def test_delo_coefficients_against_high_precision():
    """alpha, beta, e against 50-digit evaluations of the defining formulas,
    across the small-Delta series and the direct branch."""
    D = np.concatenate([np.logspace(-14, 2.8, 400), [F.DELO_SERIES_BELOW * (1 - 1e-12),
                                                      F.DELO_SERIES_BELOW * (1 + 1e-12)]])
    e, al, be = F.delo_linear(D)
    mpmath.mp.dps = 50
    for i, d in enumerate(D):
        dm = mpmath.mpf(float(d))
        w0 = 1 - mpmath.exp(-dm)
        w1 = dm - w0
        b_ref = w1 / dm
        a_ref = w0 - b_ref
        assert abs(be[i] - float(b_ref)) <= 1e-15 * float(b_ref), d
        assert abs(al[i] - float(a_ref)) <= 1e-15 * float(a_ref), d
        assert abs(e[i] - float(mpmath.exp(-dm))) <= 1e-15 * float(mpmath.exp(-dm)), d


def test_point_source_is_one_sided():
    """Lambda on a point-like source at height j: zero upwind of j, decay by
    the factor e of each step downwind (Sect. 4.4)."""
    tau = W.log_tau(1e-3, 1e3, 30)
    g = Grids(_atm(tau))
    fs = F.FormalSolver(g)
    j = 12
    S = np.zeros((g.Ns, g.Nmu))
    S[j, :] = 1.0
    I = fs.solve(S)
    dn, up = g.mu < 0, g.mu > 0
    assert np.all(I[:j, dn, :] == 0.0)
    assert np.all(I[j + 1:, up, :] == 0.0)
    np.testing.assert_allclose(I[j, dn, :], fs.beta[j - 1, dn, :], rtol=1e-15)
    np.testing.assert_allclose(I[j + 1, dn, :], fs.e[j, dn, :] * I[j, dn, :] + fs.alpha[j, dn, :], rtol=1e-15)
    for k in range(j + 2, g.Ns):
        np.testing.assert_allclose(I[k, dn, :], fs.e[k - 1, dn, :] * I[k - 1, dn, :], rtol=1e-15)
    for k in range(j - 2, -1, -1):
        np.testing.assert_allclose(I[k, up, :], fs.e[k, up, :] * I[k + 1, up, :], rtol=1e-15)


# ------------------------------------------------------------ DELO-parabolic
def _quadratic_solution(tau, r, c, I0, down):
    """Exact solution of dI/dt = S - I along a ray for S quadratic in tau
    (S = c0 + c1 tau + c2 tau^2), 40 digits: with t the path from the entry
    node, I(t) = S - S' + S'' + (I0 - S(0) + S'(0) - S'') e^{-t}."""
    mpmath.mp.dps = 40
    r = mpmath.mpf(float(r))
    c0, c1, c2 = (mpmath.mpf(float(v)) for v in c)
    I0 = mpmath.mpf(float(I0))
    taus = [mpmath.mpf(float(v)) for v in tau]
    t_entry = taus[0] if down else taus[-1]
    sgn = 1 if down else -1

    def S(t):   # S along the path: tau = t_entry + sgn t / r
        x = t_entry + sgn * t / r
        return c0 + c1 * x + c2 * x * x

    def dS(t):
        x = t_entry + sgn * t / r
        return sgn * (c1 + 2 * c2 * x) / r

    d2S = 2 * c2 / (r * r)
    out = []
    for tk in taus:
        t = r * (tk - t_entry) * sgn
        out.append(float(S(t) - dS(t) + d2S + (I0 - S(0) + dS(0) - d2S) * mpmath.exp(-t)))
    return np.array(out)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_delo_parabolic_exact_for_quadratic_source(seed):
    """Exact at every node but the last of a ray (where the step falls back to
    DELO-linear), on non-uniform grids whose steps span the series branch and
    the direct formula."""
    rng = np.random.default_rng(seed)
    tau = np.cumsum(np.exp(rng.uniform(np.log(1e-4), np.log(0.8), 45))) + rng.uniform(0, 1e-2)
    g = Grids(_atm(tau, fs=F.FS_DELO_PARABOLIC))
    fs = F.FormalSolver(g)
    c, Itop, Ibot = (0.3, 1.7, -0.9), 0.25, 2.0
    Sk = c[0] + c[1] * tau + c[2] * tau ** 2
    I = fs.solve(np.repeat(Sk[:, None], g.Nmu, axis=1), inflow_top=Itop, inflow_bottom=Ibot)
    for m in range(g.Nmu):
        for p in range(g.Nnu):
            r = g.phi_hat[p] / abs(g.mu[m])
            down = g.mu[m] < 0
            ref = _quadratic_solution(tau, r, c, Itop if down else Ibot, down)
            keep = slice(0, -1) if down else slice(1, None)
            scale = np.max(np.abs(ref))
            np.testing.assert_allclose(I[keep, m, p], ref[keep], rtol=0, atol=2e-13 * scale)


def test_delo_parabolic_weights_against_high_precision():
    """alpha, beta, gamma against 40-digit quadratures of the Lagrange
    weights of the parabola through the upwind, current and downwind nodes."""
    mpmath.mp.dps = 40
    cases = [(1e-9, 3e-9), (1e-5, 1e-5), (3e-3, 1e-2), (0.2, 0.05), (0.999, 1.3), (1.0, 0.4), (2.5, 2.5),
             (12.0, 30.0), (60.0, 1.0)]
    for d, dn in cases:
        e, al, be, ga = F.delo_parabolic(np.array([d]), np.array([dn]))
        D, Dn = mpmath.mpf(d), mpmath.mpf(dn)
        wts = {
            "up": lambda u: (u - D) * (u - D - Dn) / (D * (D + Dn)),
            "c": lambda u: -u * (u - D - Dn) / (D * Dn),
            "dn": lambda u: u * (u - D) / ((D + Dn) * Dn),
        }
        ref = {k: mpmath.quad(lambda u: mpmath.exp(-(D - u)) * L(u), [0, D]) for k, L in wts.items()}
        for got, key in ((al[0], "up"), (be[0], "c"), (ga[0], "dn")):
            r = float(ref[key])
            assert abs(got - r) <= 1e-14 * max(abs(r), float(1 - mpmath.exp(-D)) * 1e-3), (d, dn, key, got, r)
        assert abs(e[0] - float(mpmath.exp(-D))) <= 1e-15 * float(mpmath.exp(-D))


def test_delo_parabolic_beta_star_is_the_diagonal_of_lambda():
    """beta* against brute force: Lambda applied to a unit source at each
    height, read at that height."""
    tau = W.log_tau(1e-3, 1e3, 14)
    g = Grids(_atm(tau, fs=F.FS_DELO_PARABOLIC))
    fs = F.FormalSolver(g)
    bs = fs.beta_star()
    for k in range(g.Ns):
        S = np.zeros((g.Ns, g.Nmu))
        S[k, :] = 1.0
        np.testing.assert_allclose(fs.solve(S)[k], bs[k], rtol=1e-14, atol=1e-300)


def test_delo_parabolic_constant_source_and_order_three():
    """A constant source is kept (alpha + beta + gamma = 1 - e); for a smooth
    source the error at the end of a ray falls like h^3."""
    tau = W.log_tau(1e-6, 1e7, 50)
    g = Grids(_atm(tau, fs=F.FS_DELO_PARABOLIC))
    fs = F.FormalSolver(g)
    np.testing.assert_allclose(fs.e + fs.alpha + fs.beta + fs.gamma, 1.0, rtol=0, atol=5e-16)
    I = fs.solve(np.ones((g.Ns, g.Nmu)), inflow_top=1.0, inflow_bottom=1.0)
    np.testing.assert_allclose(I, 1.0, rtol=0, atol=1e-14)
    errs = []
    for Ns in (21, 41, 81, 161):
        tau = np.linspace(0.0, 3.0, Ns)
        g = Grids(_atm(tau, Nnu=3, fs=F.FS_DELO_PARABOLIC, x_max=1.0))
        fs = F.FormalSolver(g)
        I = fs.solve(np.repeat(np.sin(tau)[:, None], g.Nmu, axis=1))
        m = g.Nmu - 1                          # an upward ray: its last node is the top, k = 0
        r = g.phi_hat[1] / abs(g.mu[m])
        # the node before the last (k = 1): every step so far was parabolic
        t = r * (3.0 - tau[1])
        ref = _sine_solution(t, -1.0 / r, 3.0)
        errs.append(abs(I[1, m, 1] - ref))
    rates = [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]
    assert min(rates) > 2.7, rates
