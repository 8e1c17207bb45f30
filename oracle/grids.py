"""Discrete grids of the benchmark problem (oracle; test infrastructure only).

Paper anchors
  * angular quadrature: N_mu Gauss-Legendre nodes and weights on [-1,1] (Sect. 4.1);
    the workloads also use a half-range (double-Gauss) variant, N_mu/2 nodes per hemisphere.
  * spectral quadrature: N_nu equally spaced reduced frequencies, trapezoidal rule (Sect. 4.1).
  * absorption profile phi: Voigt profile with damping a (Sect. 3.1, after Eq. 12).
  * the factor phi/2 and the closed integral over mu in Eq. (11)-(12) fix the
    normalisation: the weights below sum to one over (mu, nu).
  * polarization tensor components T^2_{0,1}, T^2_{0,2} (after Eq. 8).
"""
from __future__ import annotations

import math

import numpy as np
from numpy.polynomial import legendre
from scipy.special import wofz

TAU_LINE_CENTER = 0
TAU_FREQ_INTEGRATED = 1
MU_GL_HALF = 0
MU_GL_FULL = 1

SQRT_PI = math.sqrt(math.pi)


def T201(mu):
    """T^2_{0,1}(mu) = sqrt(2) (3 mu^2 - 1) / 4   (after Eq. 8)."""
    return math.sqrt(2.0) * (3.0 * np.asarray(mu) ** 2 - 1.0) / 4.0


def T202(mu):
    """T^2_{0,2}(mu) = sqrt(2) (3 mu^2 - 3) / 4   (after Eq. 8)."""
    return math.sqrt(2.0) * (3.0 * np.asarray(mu) ** 2 - 3.0) / 4.0


def mu_grid(Nmu: int, kind: int):
    """Directions mu_m (ascending) and weights w_m.

    MU_GL_FULL: N_mu Gauss-Legendre nodes on [-1,1] (Sect. 4.1); sum w = 2.
    MU_GL_HALF: N_mu/2 Gauss-Legendre nodes on [0,1] mirrored to [-1,0]; each
    hemisphere's weights sum to 1, so sum w = 2 as well.
    """
    if Nmu < 2 or Nmu % 2:
        raise ValueError("N_mu must be even and >= 2")
    if kind == MU_GL_FULL:
        t, w = legendre.leggauss(Nmu)
        return t.astype(np.float64), w.astype(np.float64)
    if kind == MU_GL_HALF:
        t, w = legendre.leggauss(Nmu // 2)
        mu_pos = 0.5 * (t + 1.0)
        w_pos = 0.5 * w
        mu = np.concatenate([-mu_pos[::-1], mu_pos])
        ww = np.concatenate([w_pos[::-1], w_pos])
        return mu, ww
    raise ValueError("unknown mu quadrature")


def voigt_H(a: float, x):
    """Voigt function H(a,x) = Re w(x + i a), w the Faddeeva function.

    The profile of Sect. 3.1 is phi(x) = H(a,x)/sqrt(pi), normalised to unit
    area over x.  scipy's Faddeeva routine serves as the library primitive.
    """
    return wofz(np.asarray(x, dtype=np.float64) + 1j * a).real


def x_grid(x_min: float, x_max: float, Nnu: int) -> np.ndarray:
    """N_nu equally spaced reduced frequencies in [x_min, x_max] (Sect. 4.1)."""
    return np.linspace(x_min, x_max, Nnu)


def spectral(at):
    """Profile, spectral weights and optical-depth scaling for atmosphere ``at``.

    Returns (x, phi, w_nu, phi_hat):
      phi_p    = H(a, x_p) / sqrt(pi)
      w_nu_p   = trapezoid weight * phi_p, divided by its sum when ``freq_norm``
                 (the trapezoid on a truncated line misses ~2a/(pi x_max) of the
                 profile area, comparable to eps; renormalising keeps the
                 quadrature of a constant exact)
      phi_hat_p converts the vertical optical-depth increment into the one at
                 frequency p: line-centre tau -> H(a,x)/H(a,0); frequency-
                 integrated tau (the paper's choice, Sect. 4.1) -> phi_p.
    """
    x = x_grid(at.x_min, at.x_max, at.Nnu)
    H = voigt_H(at.a, x)
    phi = H / SQRT_PI
    h = (at.x_max - at.x_min) / (at.Nnu - 1)
    c = np.full(at.Nnu, h)
    c[0] *= 0.5
    c[-1] *= 0.5
    w_nu = c * phi
    if at.freq_norm:
        w_nu = w_nu / w_nu.sum()
    if at.tau_kind == TAU_LINE_CENTER:
        phi_hat = H / voigt_H(at.a, 0.0)
    elif at.tau_kind == TAU_FREQ_INTEGRATED:
        phi_hat = phi
    else:
        raise ValueError("unknown tau convention")
    return x, phi, w_nu, phi_hat


class Grids:
    """All per-problem grid quantities of one atmosphere (FP64)."""

    def __init__(self, at):
        self.at = at
        self.Ns, self.Nmu, self.Nnu = at.Ns, at.Nmu, at.Nnu
        self.tau = np.asarray(at.tau, dtype=np.float64)
        if self.tau.shape != (at.Ns,) or np.any(np.diff(self.tau) <= 0):
            raise ValueError("tau must be strictly increasing with N_s entries")
        self.B = np.asarray(at.B, dtype=np.float64)
        self.mu, self.w_mu = mu_grid(at.Nmu, at.mu_quad)
        self.x, self.phi, self.w_nu, self.phi_hat = spectral(at)
        self.eps = float(at.eps)
        self.xi = 1.0 - self.eps
        self.W2 = float(at.W2)
        self.t201 = T201(self.mu)
        self.t202 = T202(self.mu)
        # hat-w_m = w_m / 2 : the 1/2 of Eq. (11)-(12) with the closed mu integral
        self.wm_hat = 0.5 * self.w_mu
