"""Formal solvers of the transfer equations (oracle; test infrastructure only).

Eq. (9)-(10): mu dI/dz = -eta (I - S_I), mu dQ/dz = -eta (Q - S_Q), decoupled.
Along a ray, with t the optical path measured in the propagation direction,
dI/dt = S - I.  Between an upwind node (I_prev, S_prev) and the next node
(I_k, S_k), separated by the optical path Delta, every scheme here is a
one-step map

    I_k = e * I_prev + alpha * S_prev + beta * S_k.

The paper names DELO-linear and implicit Euler (Sect. 4.1) and refers to
earlier papers for their formulas, which are not reproduced in it.  Readings:

* DELO-linear: S is linear in t on each interval, and the RTE is integrated
  exactly (exponential integrator).  With w0 = 1 - e^{-Delta} and
  w1 = Delta - w0:  e = e^{-Delta}, beta = w1/Delta, alpha = w0 - beta,
  evaluated as beta = 1 - w0/Delta and alpha = w0/Delta - e (no cancellation
  for large Delta).  For small Delta both lose their digits to cancellation,
  so the Taylor series of the same expressions is summed instead:
      beta  = sum_{n>=1} (-1)^{n+1} Delta^n / (n+1)!
      alpha = sum_{n>=1} (-1)^{n+1} n Delta^n / (n+1)!
* implicit Euler (backward Euler in t):  I_k = (I_prev + Delta S_k)/(1+Delta).
* trapezoidal (Crank-Nicolson in t):
      I_k = ((1 - Delta/2) I_prev + Delta/2 (S_prev + S_k)) / (1 + Delta/2).
* DELO-parabolic (the paper also names DELOPAR and DELO-parabolic, Sect. 4.1,
  again without formulas): S is interpolated by the parabola through the
  upwind, current and downwind nodes of the ray and the RTE is integrated
  exactly over the interval, so the step map gains a downwind term,
      I_k = e * I_prev + alpha * S_prev + beta * S_k + gamma * S_next.
  With Delta' the downwind optical path and
      q = int_0^Delta e^{-v} v (v - Delta) dv = Delta ((2 - Delta) a - Delta e)
  (a = alpha of DELO-linear; the Taylor series of q/Delta^3 for small Delta)
  the weights are those of DELO-linear plus a correction in q:
      alpha = a + q / (Delta (Delta + Delta')),  beta = b - q / (Delta Delta'),
      gamma = q / (Delta' (Delta + Delta')).
  On the last interval of a ray (no downwind node) the step is DELO-linear.
  The method is exact for S quadratic in t.

Geometry (Sect. 3.1, boundary conditions after Eq. 10; Algorithm 1): heights
are indexed top (k=0, smallest tau) to bottom (k=N_s-1).  Rays with mu<0 enter
at the top and march k=0 -> N_s-1; rays with mu>0 enter at the bottom and
march k=N_s-1 -> 0.  On the interval between k and k+1 the optical path at
frequency p and direction m is
    Delta = (tau_{k+1} - tau_k) * phi_hat_p / |mu_m|.
"""
from __future__ import annotations

import math

import numpy as np

FS_DELO_LINEAR = 0
FS_IMPLICIT_EULER = 1
FS_TRAPEZOIDAL = 2
FS_DELO_PARABOLIC = 3

# below this optical path, DELO-linear coefficients come from their Taylor series
DELO_SERIES_BELOW = 1.0
_SERIES_TERMS = 24   # 1/25! ~ 6e-26: far below FP64 rounding


def delo_linear(D: np.ndarray):
    D = np.asarray(D, dtype=np.float64)
    e = np.exp(-D)
    w0 = -np.expm1(-D)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = w0 / D
    beta = 1.0 - r
    alpha = r - e
    small = D < DELO_SERIES_BELOW
    if np.any(small):
        d = D[small]
        bs = np.zeros_like(d)
        as_ = np.zeros_like(d)
        for n in range(1, _SERIES_TERMS + 1):
            term = (-1.0) ** (n + 1) * d ** n / math.factorial(n + 1)
            bs += term
            as_ += n * term
        beta = beta.copy()
        alpha = alpha.copy()
        beta[small] = bs
        alpha[small] = as_
    return e, alpha, beta


def implicit_euler(D: np.ndarray):
    D = np.asarray(D, dtype=np.float64)
    e = 1.0 / (1.0 + D)
    return e, np.zeros_like(D), D / (1.0 + D)


def trapezoidal(D: np.ndarray):
    D = np.asarray(D, dtype=np.float64)
    h = 0.5 * D
    e = (1.0 - h) / (1.0 + h)
    ab = h / (1.0 + h)
    return e, ab, ab.copy()


def parabolic_q(D: np.ndarray) -> np.ndarray:
    """q = int_0^Delta e^{-v} v (v - Delta) dv, from the DELO-linear alpha for
    Delta >= DELO_SERIES_BELOW and from the Taylor series
    q = -sum_{j>=0} (-1)^j Delta^{j+3} / (j! (j+2) (j+3)) below."""
    D = np.asarray(D, dtype=np.float64)
    e, a, _ = delo_linear(D)
    q = D * ((2.0 - D) * a - D * e)
    small = D < DELO_SERIES_BELOW
    if np.any(small):
        d = D[small]
        acc = np.zeros_like(d)
        for j in range(_SERIES_TERMS + 1):
            acc += (-1.0) ** j * d ** j / (math.factorial(j) * (j + 2) * (j + 3))
        q = q.copy()
        q[small] = -acc * d ** 3
    return q


def delo_parabolic(D: np.ndarray, Dn: np.ndarray):
    """(e, alpha, beta, gamma) of the parabolic step over an interval of optical
    path D whose downwind interval has optical path Dn (Dn = 0: no downwind
    node, the DELO-linear step)."""
    D = np.asarray(D, dtype=np.float64)
    Dn = np.asarray(Dn, dtype=np.float64)
    e, a, b = delo_linear(D)
    q = parabolic_q(D)
    has = Dn > 0.0
    with np.errstate(divide="ignore", invalid="ignore"):
        alpha = np.where(has, a + q / (D * (D + Dn)), a)
        beta = np.where(has, b - q / (D * Dn), b)
        gamma = np.where(has, q / (Dn * (D + Dn)), 0.0)
    return e, alpha, beta, gamma


def step_coefficients(fs: int, D: np.ndarray):
    if fs == FS_DELO_LINEAR:
        return delo_linear(D)
    if fs == FS_IMPLICIT_EULER:
        return implicit_euler(D)
    if fs == FS_TRAPEZOIDAL:
        return trapezoidal(D)
    raise ValueError("unknown formal solver")


def path_depths(g) -> np.ndarray:
    """Delta[i, m, p] on the interval between heights i and i+1, shape (N_s-1, N_mu, N_nu)."""
    dtau = np.diff(g.tau)
    return dtau[:, None, None] * g.phi_hat[None, None, :] / np.abs(g.mu)[None, :, None]


class FormalSolver:
    """Lambda of Eq. (16): maps S(k, m) to I(k, m, p) along every (m, p) ray."""

    def __init__(self, g):
        self.g = g
        self.D = path_depths(g)
        self.down = g.mu < 0.0      # enters at the top
        self.up = g.mu > 0.0        # enters at the bottom
        self.gamma = None
        if g.at.formal_solver == FS_DELO_PARABOLIC:
            # downwind interval of every step: i+1 for mu<0 rays, i-1 for mu>0
            Dn = np.zeros_like(self.D)
            Dn[:-1, self.down, :] = self.D[1:, self.down, :]
            Dn[1:, self.up, :] = self.D[:-1, self.up, :]
            self.e, self.alpha, self.beta, self.gamma = delo_parabolic(self.D, Dn)
        else:
            self.e, self.alpha, self.beta = step_coefficients(g.at.formal_solver, self.D)

    def solve(self, S: np.ndarray, inflow_top=0.0, inflow_bottom=0.0) -> np.ndarray:
        """Formal solution of one Stokes parameter.

        S: (N_s, N_mu) source function.  inflow_top applies to mu<0 rays at
        k=0, inflow_bottom to mu>0 rays at k=N_s-1 (scalars or (N_nu,) arrays).
        Returns I of shape (N_s, N_mu, N_nu).
        """
        g = self.g
        Ns, Nnu = g.Ns, g.Nnu
        I = np.zeros((Ns, g.Nmu, Nnu))
        dn, up = self.down, self.up
        e, al, be = self.e, self.alpha, self.beta
        ga = self.gamma
        # mu < 0: k = 0 -> N_s-1
        I[0, dn, :] = inflow_top
        for k in range(1, Ns):
            i = k - 1
            I[k, dn, :] = (e[i, dn, :] * I[k - 1, dn, :]
                           + al[i, dn, :] * S[k - 1, dn][:, None]
                           + be[i, dn, :] * S[k, dn][:, None])
            if ga is not None and k + 1 < Ns:
                I[k, dn, :] += ga[i, dn, :] * S[k + 1, dn][:, None]
        # mu > 0: k = N_s-1 -> 0
        I[Ns - 1, up, :] = inflow_bottom
        for k in range(Ns - 2, -1, -1):
            i = k
            I[k, up, :] = (e[i, up, :] * I[k + 1, up, :]
                           + al[i, up, :] * S[k + 1, up][:, None]
                           + be[i, up, :] * S[k, up][:, None])
            if ga is not None and k >= 1:
                I[k, up, :] += ga[i, up, :] * S[k - 1, up][:, None]
        return I

    def beta_star(self) -> np.ndarray:
        """Coefficient of S_k in I_k (the diagonal of Lambda), shape (N_s, N_mu, N_nu).

        It is the beta of the step that ends at k; the node where a ray enters
        takes the inflow only, so its entry is 0.  With DELO-parabolic, S_k
        also enters the step before (as its downwind node), and that part of
        I_prev reaches I_k multiplied by e: beta* = beta_k + e_k gamma_{k-1}.
        """
        g = self.g
        bs = np.zeros((g.Ns, g.Nmu, g.Nnu))
        dn, up = self.down, self.up
        bs[1:, dn, :] = self.beta[:, dn, :]
        bs[:-1, up, :] = self.beta[:, up, :]
        if self.gamma is not None:
            e, ga = self.e, self.gamma
            # mu<0: step ending at k uses interval k-1, the one before interval k-2
            bs[2:, dn, :] += e[1:, dn, :] * ga[:-1, dn, :]
            # mu>0: step ending at k uses interval k, the one before interval k+1
            bs[:-2, up, :] += e[:-1, up, :] * ga[1:, up, :]
        return bs
