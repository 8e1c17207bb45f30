"""Operators of the discrete problem (oracle; test infrastructure only).

Notation of Sect. 3.2 of the paper:
  S = T sigma           Eq. (15): source functions from multipolar components
  I = Lambda S + t      Eq. (16): formal solution plus transmitted boundary radiation
  sigma = J I + c       Eq. (17): quadrature of the radiation field, c = [eps B, 0, ...]
  sigma-form            Eq. (18): (Id - J Lambda T) sigma = J t + c
  I-form                Eq. (19): (Id - Lambda T J) I = Lambda T c + t

Here J carries the factor xi = 1 - eps of Eq. (13)-(14) and the
polarizability factor W2 on the sigma^2_0 row (W2 = w^(2) = 1 in the paper).

Vector layouts
  I-form vector: x[s][k][m][p], s in {I, Q}, flattened C-order, length 2 N_s N_mu N_nu.
  sigma vector:  [sigma00(z_1), sigma20(z_1), sigma00(z_2), ...]  (Eq. 17), length 2 N_s.

Readings of points the paper leaves open (each is an option of rt_workloads.Atmosphere):
  * c generalises [eps, 0, eps, 0, ...] to [eps B_k, 0, ...] for a depth-dependent
    Planck function, and the bottom boundary value of I generalises 1 to B(tau_{N_s}).
  * "zero initial conditions" in Algorithm 1 means zero inflow at both ends.
"""
from __future__ import annotations

import numpy as np

from .formal import FormalSolver
from .grids import Grids


class Transfer:
    def __init__(self, at):
        self.at = at
        self.g = Grids(at)
        self.fs = FormalSolver(self.g)
        g = self.g
        self.shape = (2, g.Ns, g.Nmu, g.Nnu)
        self.N = 2 * g.Ns * g.Nmu * g.Nnu
        self.Nsig = 2 * g.Ns
        # hat-w_m hat-w_p on the (m, p) ray grid
        self.w_ray = g.wm_hat[:, None] * g.w_nu[None, :]

    # ------------------------------------------------------------------ J
    def radiation_moments(self, I: np.ndarray, Q: np.ndarray):
        """J00(z_k), J20(z_k) by the discrete Eq. (11)-(12)."""
        g = self.g
        J00 = np.einsum("kmp,mp->k", I, self.w_ray)
        J20 = (np.einsum("kmp,mp->k", I, self.w_ray * g.t201[:, None])
               + np.einsum("kmp,mp->k", Q, self.w_ray * g.t202[:, None]))
        return J00, J20

    def J_apply(self, x: np.ndarray):
        """Linear part of Eq. (17), per Eq. (13)-(14): (xi J00, xi W2 J20)."""
        I, Q = x.reshape(self.shape)
        J00, J20 = self.radiation_moments(I, Q)
        return self.g.xi * J00, self.g.xi * self.g.W2 * J20

    def c_vector(self):
        g = self.g
        return g.eps * g.B, np.zeros(g.Ns)

    # ------------------------------------------------------------------ T
    def T_apply(self, s00: np.ndarray, s20: np.ndarray):
        """Eq. (7)-(8): S_I = sigma00 + T201 sigma20, S_Q = T202 sigma20; shape (N_s, N_mu)."""
        g = self.g
        SI = s00[:, None] + g.t201[None, :] * s20[:, None]
        SQ = g.t202[None, :] * s20[:, None]
        return SI, SQ

    # ------------------------------------------------------------- Lambda
    def Lambda_apply(self, SI, SQ, boundary=False) -> np.ndarray:
        """Formal solution of Eq. (9)-(10); with boundary=True the incoming
        radiation of the boundary conditions is included (I = B_bottom, Q = 0
        for mu > 0 at the bottom; I = Q = 0 for mu < 0 at the top), i.e. the
        result is Lambda S + t."""
        g = self.g
        bottom = g.B[-1] if boundary else 0.0
        I = self.fs.solve(SI, inflow_top=0.0, inflow_bottom=bottom)
        Q = self.fs.solve(SQ, inflow_top=0.0, inflow_bottom=0.0)
        return np.stack([I, Q]).reshape(-1)

    def transmitted(self) -> np.ndarray:
        """t of Eq. (16): the boundary radiation propagated with S = 0."""
        g = self.g
        z = np.zeros((g.Ns, g.Nmu))
        return self.Lambda_apply(z, z, boundary=True)

    # ------------------------------------------------------------- I-form
    def apply_I(self, x: np.ndarray) -> np.ndarray:
        """y = (Id - Lambda T J) x, the I-form operator of Eq. (19)."""
        x = np.asarray(x, dtype=np.float64)
        s00, s20 = self.J_apply(x)
        SI, SQ = self.T_apply(s00, s20)
        return x - self.Lambda_apply(SI, SQ)

    def rhs_I(self) -> np.ndarray:
        """b = Lambda T c + t of Eq. (19) (one formal solve with boundaries)."""
        c00, c20 = self.c_vector()
        SI, SQ = self.T_apply(c00, c20)
        return self.Lambda_apply(SI, SQ, boundary=True)

    def jacobi_I(self) -> np.ndarray:
        """Diagonal of Id - Lambda T J (Jacobi P = D, Sect. 2.3).

        J and T are local in height, and Lambda couples S(z_k) into I(z_k) only
        through the last step of the ray, with the coefficient beta*:
          D_I = 1 - xi beta* hat-w_m hat-w_p (1 + W2 T201^2)
          D_Q = 1 - xi W2 beta* hat-w_m hat-w_p T202^2
        """
        g = self.g
        bs = self.fs.beta_star()
        w = self.w_ray[None, :, :]
        DI = 1.0 - g.xi * bs * w * (1.0 + g.W2 * g.t201[None, :, None] ** 2)
        DQ = 1.0 - g.xi * g.W2 * bs * w * g.t202[None, :, None] ** 2
        return np.stack([DI, DQ]).reshape(-1)

    # --------------------------------------------------------- sigma-form
    def apply_sigma(self, sig: np.ndarray) -> np.ndarray:
        """Algorithm 1: sigma_out = sigma_in - J Lambda T sigma_in (Eq. 18)."""
        sig = np.asarray(sig, dtype=np.float64).reshape(self.g.Ns, 2)
        SI, SQ = self.T_apply(sig[:, 0], sig[:, 1])
        I = self.Lambda_apply(SI, SQ)
        s00, s20 = self.J_apply(I)
        return (sig - np.stack([s00, s20], axis=1)).reshape(-1)

    def rhs_sigma(self) -> np.ndarray:
        """b = J t + c of Eq. (18)."""
        s00, s20 = self.J_apply(self.transmitted())
        c00, c20 = self.c_vector()
        return np.stack([s00 + c00, s20 + c20], axis=1).reshape(-1)

    def local_blocks_sigma(self) -> np.ndarray:
        """2x2 blocks M_k = Id - J_k Lambda*_k T_k of the sigma-form, per height.

        Lambda* keeps only the diagonal of Lambda (beta*), so the product is
        local in height.  diag(M_k) is the Jacobi diagonal of Eq. (18).
        Returns (N_s, 2, 2).
        """
        g = self.g
        bs = self.fs.beta_star()
        w = self.w_ray[None, :, :] * bs
        a0 = w.sum(axis=(1, 2))
        a1 = (w * g.t201[None, :, None]).sum(axis=(1, 2))
        a2 = (w * (g.t201 ** 2 + g.t202 ** 2)[None, :, None]).sum(axis=(1, 2))
        M = np.empty((g.Ns, 2, 2))
        M[:, 0, 0] = 1.0 - g.xi * a0
        M[:, 0, 1] = -g.xi * a1
        M[:, 1, 0] = -g.xi * g.W2 * a1
        M[:, 1, 1] = 1.0 - g.xi * g.W2 * a2
        return M

    def jacobi_sigma(self) -> np.ndarray:
        """Diagonal of Id - J Lambda T (the paper's Jacobi preconditioner on Eq. 18)."""
        M = self.local_blocks_sigma()
        return np.stack([M[:, 0, 0], M[:, 1, 1]], axis=1).reshape(-1)

    # ------------------------------------------- local-Lambda preconditioner
    def local_lambda_I(self, x: np.ndarray) -> np.ndarray:
        """P x = (Id - Lambda* T J) x: the I-form operator with Lambda replaced
        by its diagonal."""
        g = self.g
        s00, s20 = self.J_apply(x)
        SI, SQ = self.T_apply(s00, s20)
        bs = self.fs.beta_star()
        LS = np.stack([bs * SI[:, :, None], bs * SQ[:, :, None]]).reshape(-1)
        return x - LS

    def local_lambda_I_inverse(self, v: np.ndarray) -> np.ndarray:
        """P^{-1} v = v + Lambda* T M^{-1} J v (Woodbury identity), M_k the 2x2
        local blocks: the sigma-form block-Jacobi preconditioner lifted to the
        I-form.  The spectrum of A_I P^{-1} is that of A_sigma M^{-1} plus ones."""
        s00, s20 = self.J_apply(v)
        M = self.local_blocks_sigma()
        rhs = np.stack([s00, s20], axis=1)[:, :, None]
        u = np.linalg.solve(M, rhs)[:, :, 0]
        SI, SQ = self.T_apply(u[:, 0], u[:, 1])
        bs = self.fs.beta_star()
        return v + np.stack([bs * SI[:, :, None], bs * SQ[:, :, None]]).reshape(-1)

    # ------------------------------------------------- assembly, exact solve
    def assemble(self, apply, n: int) -> np.ndarray:
        """Dense matrix of a linear map, column by column on unit vectors
        (the column-by-column assembly of Sect. 3.3)."""
        A = np.empty((n, n))
        e = np.zeros(n)
        for j in range(n):
            e[j] = 1.0
            A[:, j] = apply(e)
            e[j] = 0.0
        return A

    def assemble_sigma(self) -> np.ndarray:
        return self.assemble(self.apply_sigma, self.Nsig)

    def assemble_I(self) -> np.ndarray:
        return self.assemble(self.apply_I, self.N)

    def exact_sigma(self) -> np.ndarray:
        """Direct LU solution of Eq. (18) on the assembled matrix (Sect. 4.4)."""
        return np.linalg.solve(self.assemble_sigma(), self.rhs_sigma())

    def lift(self, sig: np.ndarray) -> np.ndarray:
        """I = Lambda T sigma + t for a sigma-form solution (Eq. 16)."""
        sig = np.asarray(sig).reshape(self.g.Ns, 2)
        SI, SQ = self.T_apply(sig[:, 0], sig[:, 1])
        return self.Lambda_apply(SI, SQ, boundary=True)

    def exact_I(self) -> np.ndarray:
        """Exact discrete solution of Eq. (19), via the 2N_s LU solve of
        Eq. (18) and one formal solve: if sigma* solves (18), then
        I* = Lambda T sigma* + t solves (19)."""
        return self.lift(self.exact_sigma())
