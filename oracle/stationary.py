"""SOR and SSOR preconditioners of the assembled sigma-form matrix (oracle;
test infrastructure only).

Sect. 2.3 of the paper splits A = D + L + U (diagonal, strictly lower and
strictly upper triangular parts) and, for 0 < omega < 2, defines

  * SOR:  P = D/omega + L   or   P = D/omega + U;
  * SSOR: P = omega/(2 - omega) * Lt @ Ut, a product of two triangular
    factors built from D/omega + L, D^{-1} and D/omega + U.

The experiments of Sect. 4.2 use the variant built on U, because of the
structure of A.  With omega = 1.5 for the Richardson iteration and
omega = 1 inside the Krylov methods, the readings below reproduce Tables 4
and 5 (``tests/test_oracle_stationary.py``).  They were chosen by that test
among the four combinations of unknown ordering and triangle:

  * unknowns ordered as the sigma-form vector, (sigma00_k, sigma20_k)
    interleaved per height, heights from the top;
  * SOR:  P = D/omega + U  (upper triangular);
  * SSOR: P = omega/(2 - omega) * (D/omega + U) @ D^{-1} @ (D/omega + L),
    i.e. the paper's product with the roles of L and U exchanged, consistent
    with its choice of U for SOR.  For omega = 1 it is the symmetric
    Gauss-Seidel preconditioner (D + U) D^{-1} (D + L).

The paper precomputes the action of P^{-1} (Sect. 4.2).  Here P is formed as
a dense matrix and P^{-1} v is a dense solve: plain, not fast.
"""
from __future__ import annotations

import numpy as np


def split(A: np.ndarray):
    """A = D + L + U: the diagonal (as a vector) and the strictly lower and
    upper triangular parts (Sect. 2.3)."""
    A = np.asarray(A, dtype=np.float64)
    return np.diag(A).copy(), np.tril(A, -1), np.triu(A, 1)


def sor_matrix(A: np.ndarray, omega: float) -> np.ndarray:
    """P = D/omega + U, the upper SOR variant the experiments use (Sect. 2.3,
    Sect. 4.2)."""
    d, _, U = split(A)
    return np.diag(d / omega) + U


def ssor_matrix(A: np.ndarray, omega: float) -> np.ndarray:
    """P = omega/(2-omega) (D/omega + U) D^{-1} (D/omega + L) (Sect. 2.3 with
    the upper factor first, see the module docstring)."""
    d, L, U = split(A)
    Lt = np.diag(d / omega) + U
    Ut = (np.diag(d / omega) + L) / d[:, None]
    return (omega / (2.0 - omega)) * (Lt @ Ut)


def inverse_action(P: np.ndarray):
    """v -> P^{-1} v by a dense solve."""
    P = np.asarray(P, dtype=np.float64)
    return lambda v: np.linalg.solve(P, np.asarray(v, dtype=np.float64))
