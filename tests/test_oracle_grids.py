"""Pins of the oracle's grids against closed forms (CPU)."""
import math

import numpy as np
import pytest
from scipy import integrate

import rt_workloads as W
from oracle import grids as G


@pytest.mark.parametrize("n", [2, 4, 8, 16, 20, 32, 64])
def test_gauss_legendre_full_range_moments(n):
    mu, w = G.mu_grid(n, G.MU_GL_FULL)
    assert np.all(np.diff(mu) > 0)
    np.testing.assert_allclose(mu, -mu[::-1], atol=1e-15)
    # exact for polynomials of degree <= 2n-1: int_{-1}^{1} mu^k = 2/(k+1) (k even), 0 (odd)
    for k in range(0, 2 * n):
        exact = 2.0 / (k + 1) if k % 2 == 0 else 0.0
        assert abs(np.dot(w, mu ** k) - exact) < 1e-14


@pytest.mark.parametrize("n", [8, 16, 32, 64])
def test_gauss_legendre_half_range_moments(n):
    mu, w = G.mu_grid(n, G.MU_GL_HALF)
    pos = mu > 0
    assert pos.sum() == n // 2 and np.all(np.diff(mu) > 0)
    np.testing.assert_allclose(mu[pos], -mu[~pos][::-1], atol=0)
    # each hemisphere: exact for degree <= n-1 on [0,1]: int_0^1 mu^k = 1/(k+1)
    for k in range(0, n):
        assert abs(np.dot(w[pos], mu[pos] ** k) - 1.0 / (k + 1)) < 1e-14


@pytest.mark.parametrize("kind,n", [(G.MU_GL_FULL, 20), (G.MU_GL_HALF, 16), (G.MU_GL_HALF, 8)])
def test_polarization_tensor_quadrature(kind, n):
    """(1/2) int T201 dmu = 0, (1/2) int T201^2 = 1/10, (1/2) int T202^2 = 3/5,
    (1/2) int T202 = -sqrt(2)/2 (closed forms of the after-Eq.-8 polynomials)."""
    mu, w = G.mu_grid(n, kind)
    wh = 0.5 * w
    assert abs(np.dot(wh, G.T201(mu))) < 1e-14
    assert abs(np.dot(wh, G.T201(mu) ** 2) - 0.1) < 1e-14
    assert abs(np.dot(wh, G.T202(mu) ** 2) - 0.6) < 1e-14
    assert abs(np.dot(wh, G.T202(mu)) + math.sqrt(2) / 2) < 1e-14


def test_polarization_tensor_values():
    assert G.T201(1.0) == pytest.approx(math.sqrt(2) / 2, abs=1e-16)
    assert G.T202(1.0) == pytest.approx(0.0, abs=1e-16)
    assert G.T201(0.0) == pytest.approx(-math.sqrt(2) / 4, abs=1e-16)
    assert G.T202(0.0) == pytest.approx(-3 * math.sqrt(2) / 4, abs=1e-16)


def _voigt_integral(a, x):
    """H(a,x) = (1/sqrt(pi)) int_0^inf exp(-a t - t^2/4) cos(x t) dt, by adaptive quadrature."""
    f = lambda t: math.exp(-a * t - 0.25 * t * t) * math.cos(x * t)
    val, err = integrate.quad(f, 0.0, 40.0, limit=400, epsabs=1e-15, epsrel=1e-13)
    return val / math.sqrt(math.pi)


@pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")
@pytest.mark.parametrize("a", [1e-4, 1e-3, 1e-2, 0.5])
@pytest.mark.parametrize("x", [0.0, 0.3, 1.0, 2.5, 4.0])
def test_voigt_against_integral_representation(a, x):
    assert G.voigt_H(a, x) == pytest.approx(_voigt_integral(a, x), rel=1e-10, abs=1e-14)


def test_voigt_limits():
    x = np.linspace(-5, 5, 41)
    # a -> 0: Gaussian core
    np.testing.assert_allclose(G.voigt_H(1e-12, x), np.exp(-x * x), rtol=1e-9, atol=1e-13)
    # far wings: H ~ a/(sqrt(pi) x^2) (1 + 3/(2x^2) + 15/(4x^4))
    a = 1e-3
    for xx in (20.0, 50.0, 200.0):
        asym = a / (math.sqrt(math.pi) * xx * xx) * (1 + 1.5 / xx ** 2 + 3.75 / xx ** 4)
        assert G.voigt_H(a, xx) == pytest.approx(asym, rel=1e-6)
    # unit area of phi = H/sqrt(pi): core by quadrature, tails by the asymptote
    core, _ = integrate.quad(lambda t: G.voigt_H(a, t), -60, 60, limit=800, points=[0.0], epsabs=1e-13)
    tails = 2 * a / (math.sqrt(math.pi) * 60.0)
    assert (core + tails) / math.sqrt(math.pi) == pytest.approx(1.0, abs=1e-7)


def test_spectral_weights():
    at = W.slab70()
    x, phi, w, phat = G.spectral(at)
    assert w.sum() == pytest.approx(1.0, abs=1e-15)
    np.testing.assert_allclose(w, w[::-1], rtol=1e-14)
    assert phat[len(x) // 2] == pytest.approx(1.0, abs=1e-15)     # line-centre scale at x=0
    # plain trapezoid (paper): the truncated line misses ~2a/(pi x_max) of the profile area
    _, _, w0, _ = G.spectral(at.with_(freq_norm=0))
    miss = 2 * at.a / (math.pi * at.x_max)
    assert 1.0 - w0.sum() == pytest.approx(miss, rel=0.05)
    # frequency-integrated convention uses phi itself
    _, phi_p, _, phat_p = G.spectral(W.paper(20))
    np.testing.assert_allclose(phat_p, phi_p)
