"""Textbook Krylov solvers (oracle; test infrastructure only).

Sect. 2 of the paper: GMRES (Saad & Schultz 1986) with restarts (Sect. 2.1),
CGS (Sonneveld 1989) and BiCGSTAB (van der Vorst 1992) (Sect. 2.2),
preconditioning (Sect. 2.3, Eq. 6) and the preconditioned Richardson
iteration of Eq. (20).

Conventions shared with the CUDA path (readings; the paper uses MATLAB's
built-ins and does not spell them out):
  * right preconditioning, A P^{-1} u = b, x = P^{-1} u, so every residual
    the methods see is the unpreconditioned one of the stopping rule
    ||b - A x||_2 / ||b||_2 < tol (Sect. 4.2);
  * GMRES: Arnoldi by modified Gram-Schmidt (``ortho="mgs"``) or classical
    Gram-Schmidt applied twice (``"cgs2"``), Givens rotations on the
    Hessenberg matrix; the estimate |g_{j+1}| ends the inner loop, and the
    true residual b - A x computed at the top of every restart cycle decides
    convergence.  ``iters`` counts Arnoldi steps over all cycles;
  * BiCGSTAB / CGS: one iteration = two products with A; the iteration ends
    (and counts) at the first of its two residual checks that passes;
  * x0 = 0 makes the first residual b itself (no product with A).
"""
from __future__ import annotations

import dataclasses
import math
from typing import Callable, List, Optional

import numpy as np

OK = 0
NOT_CONVERGED = 4
BREAKDOWN = 5


@dataclasses.dataclass
class Info:
    status: int = NOT_CONVERGED
    iters: int = 0
    applies: int = 0
    restarts: int = 0
    rel_resid: float = math.inf
    history: List[float] = dataclasses.field(default_factory=list)


def _ident(v):
    return v


def _norm(v):
    return math.sqrt(float(np.dot(v, v)))


def gmres(A: Callable, b: np.ndarray, M_inv: Optional[Callable] = None,
          x0: Optional[np.ndarray] = None, restart: int = 30, tol: float = 1e-8,
          maxit: int = 10000, ortho: str = "mgs"):
    """Restarted, right-preconditioned GMRES(m) (Sect. 2.1)."""
    M_inv = M_inv or _ident
    b = np.asarray(b, dtype=np.float64)
    n = b.size
    m = restart
    info = Info()
    bnorm = _norm(b)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64)
    if bnorm == 0.0:
        info.status, info.rel_resid = OK, 0.0
        return np.zeros(n), info
    first = True
    while True:
        if first and x0 is None:
            r = b.copy()
        else:
            r = b - A(x)
            info.applies += 1
        first = False
        beta = _norm(r)
        info.rel_resid = beta / bnorm
        if info.rel_resid < tol:
            info.status = OK
            return x, info
        if info.iters >= maxit:
            info.status = NOT_CONVERGED
            return x, info
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        breakdown = False
        for j in range(m):
            w = A(M_inv(V[j]))
            info.applies += 1
            if ortho == "mgs":
                for i in range(j + 1):
                    H[i, j] = np.dot(w, V[i])
                    w = w - H[i, j] * V[i]
            elif ortho == "cgs2":
                h1 = V[: j + 1] @ w
                w = w - V[: j + 1].T @ h1
                h2 = V[: j + 1] @ w
                w = w - V[: j + 1].T @ h2
                H[: j + 1, j] = h1 + h2
            else:
                raise ValueError(ortho)
            H[j + 1, j] = _norm(w)
            # earlier rotations on the new column
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            # new rotation zeroing H[j+1, j]
            a_, b_ = H[j, j], H[j + 1, j]
            hn = math.hypot(a_, b_)
            if hn == 0.0:
                breakdown = True
                k = j
                break
            cs[j], sn[j] = a_ / hn, b_ / hn
            wnorm = b_
            H[j, j] = hn
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            info.iters += 1
            k = j + 1
            est = abs(g[j + 1]) / bnorm
            info.history.append(est)
            if wnorm == 0.0:
                break            # lucky breakdown: the solution lies in the current space
            V[j + 1] = w / wnorm
            if est < tol or info.iters >= maxit:
                break
        if k > 0:
            y = np.zeros(k)
            for i in range(k - 1, -1, -1):     # back substitution on the triangle
                y[i] = (g[i] - np.dot(H[i, i + 1:k], y[i + 1:k])) / H[i, i]
            x = x + M_inv(V[:k].T @ y)
        info.restarts += 1
        if breakdown and k == 0:
            info.status = BREAKDOWN
            return x, info


def bicgstab(A: Callable, b: np.ndarray, M_inv: Optional[Callable] = None,
             x0: Optional[np.ndarray] = None, tol: float = 1e-8, maxit: int = 10000):
    """Right-preconditioned BiCGSTAB (van der Vorst 1992; Sect. 2.2)."""
    M_inv = M_inv or _ident
    b = np.asarray(b, dtype=np.float64)
    info = Info()
    bnorm = _norm(b)
    if bnorm == 0.0:
        info.status, info.rel_resid = OK, 0.0
        return np.zeros_like(b), info
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = np.array(x0, dtype=np.float64)
        r = b - A(x)
        info.applies += 1
    info.rel_resid = _norm(r) / bnorm
    if info.rel_resid < tol:
        info.status = OK
        return x, info
    rhat = r.copy()
    rho_old = alpha = omega = 1.0
    v = np.zeros_like(b)
    p = np.zeros_like(b)
    while info.iters < maxit:
        rho = float(np.dot(rhat, r))
        if rho == 0.0:
            info.status = BREAKDOWN
            return x, info
        beta = (rho / rho_old) * (alpha / omega)
        p = r + beta * (p - omega * v)
        phat = M_inv(p)
        v = A(phat)
        info.applies += 1
        rv = float(np.dot(rhat, v))
        if rv == 0.0:
            info.status = BREAKDOWN
            return x, info
        alpha = rho / rv
        s = r - alpha * v
        info.iters += 1
        snorm = _norm(s) / bnorm
        if snorm < tol:
            x = x + alpha * phat
            info.rel_resid = snorm
            info.history.append(snorm)
            info.status = OK
            return x, info
        shat = M_inv(s)
        t = A(shat)
        info.applies += 1
        tt = float(np.dot(t, t))
        if tt == 0.0:
            info.status = BREAKDOWN
            return x, info
        omega = float(np.dot(t, s)) / tt
        x = x + alpha * phat + omega * shat
        r = s - omega * t
        info.rel_resid = _norm(r) / bnorm
        info.history.append(info.rel_resid)
        if info.rel_resid < tol:
            info.status = OK
            return x, info
        if omega == 0.0:
            info.status = BREAKDOWN
            return x, info
        rho_old = rho
    info.status = NOT_CONVERGED
    return x, info


def cgs(A: Callable, b: np.ndarray, M_inv: Optional[Callable] = None,
        x0: Optional[np.ndarray] = None, tol: float = 1e-8, maxit: int = 10000):
    """Right-preconditioned conjugate gradient squared (Sonneveld 1989; Sect. 2.2)."""
    M_inv = M_inv or _ident
    b = np.asarray(b, dtype=np.float64)
    info = Info()
    bnorm = _norm(b)
    if bnorm == 0.0:
        info.status, info.rel_resid = OK, 0.0
        return np.zeros_like(b), info
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = np.array(x0, dtype=np.float64)
        r = b - A(x)
        info.applies += 1
    info.rel_resid = _norm(r) / bnorm
    if info.rel_resid < tol:
        info.status = OK
        return x, info
    rhat = r.copy()
    rho_old = 1.0
    p = np.zeros_like(b)
    q = np.zeros_like(b)
    while info.iters < maxit:
        rho = float(np.dot(rhat, r))
        if rho == 0.0:
            info.status = BREAKDOWN
            return x, info
        if info.iters == 0:
            u = r.copy()
            p = u.copy()
        else:
            beta = rho / rho_old
            u = r + beta * q
            p = u + beta * (q + beta * p)
        phat = M_inv(p)
        vhat = A(phat)
        info.applies += 1
        rv = float(np.dot(rhat, vhat))
        if rv == 0.0:
            info.status = BREAKDOWN
            return x, info
        alpha = rho / rv
        q = u - alpha * vhat
        uhat = M_inv(u + q)
        x = x + alpha * uhat
        qhat = A(uhat)
        info.applies += 1
        r = r - alpha * qhat
        info.iters += 1
        info.rel_resid = _norm(r) / bnorm
        info.history.append(info.rel_resid)
        if info.rel_resid < tol:
            info.status = OK
            return x, info
        rho_old = rho
    info.status = NOT_CONVERGED
    return x, info


def richardson(A: Callable, b: np.ndarray, M_inv: Optional[Callable] = None,
               x0: Optional[np.ndarray] = None, tol: float = 1e-8, maxit: int = 10000):
    """Preconditioned Richardson iteration x <- x + P^{-1}(b - A x) (Eq. 20)."""
    M_inv = M_inv or _ident
    b = np.asarray(b, dtype=np.float64)
    info = Info()
    bnorm = _norm(b)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64)
    r = b.copy() if x0 is None else b - A(x)
    if x0 is not None:
        info.applies += 1
    while True:
        info.rel_resid = _norm(r) / bnorm
        info.history.append(info.rel_resid)
        if info.rel_resid < tol:
            info.status = OK
            return x, info
        if info.iters >= maxit:
            info.status = NOT_CONVERGED
            return x, info
        x = x + M_inv(r)
        r = b - A(x)
        info.applies += 1
        info.iters += 1
