"""Seeded synthetic inputs shared by the oracle tests, the CUDA-path tests and
the benchmark.

This module holds *inputs only*: atmospheres (optical-depth grids, Planck
values), grid sizes, physical parameters and seeded random vectors.  It holds
none of the method's arithmetic (no profile, no quadrature, no formal
solver); each side computes those itself from what is described here.

Workloads follow the benchmark of Sect. 3-4 of the paper (1D isothermal
slab, two-level atom J_u=1 -> J_l=0, CRD, Stokes I and Q), with the grid
sizes of the five synthetic workloads used to measure this build:

* ``slab70``      N_s=70,  N_mu=16 (half-range GL), N_nu=21,  line-centre tau 1e-4..1e6,  x in [-6,6]
* ``slab300``     N_s=300, N_mu=32 (half-range GL), N_nu=101, line-centre tau 1e-4..1e8,  x in [-8,8]
* ``sweep``       N_s in {100,250,500,1000,2000}, N_mu=64, N_nu=201, eps in {1e-2,1e-4,1e-6}, B=1 or 1+0.5 log10(1+tau)
* ``batch512``    512 uneven atmospheres drawn with splitmix64
* ``stream``      Poisson arrivals of requests drawn like ``batch512``
* ``paper``       the paper's own setting (Sect. 4.1): frequency-integrated tau 1e-5..1e4,
                  full-range GL on [-1,1], x in [-5,5].
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

# enumerations mirrored (by value) in include/rt_krylov.h
TAU_LINE_CENTER = 0
TAU_FREQ_INTEGRATED = 1
MU_GL_HALF = 0
MU_GL_FULL = 1
FS_DELO_LINEAR = 0
FS_IMPLICIT_EULER = 1
FS_TRAPEZOIDAL = 2
FS_DELO_PARABOLIC = 3
FS_DELOPAR = FS_DELO_PARABOLIC   # the same scheme under the paper's other name (no dichroism here)


@dataclasses.dataclass
class Atmosphere:
    """One problem instance (all arrays float64, host memory)."""

    Ns: int
    Nmu: int
    Nnu: int
    tau: np.ndarray          # (Ns,) strictly increasing optical depths, top -> bottom
    B: np.ndarray            # (Ns,) Planck function (Wien limit) at each height
    x_min: float
    x_max: float
    a: float = 1e-3          # Voigt damping
    eps: float = 1e-4        # thermalisation parameter (xi = 1 - eps)
    W2: float = 1.0          # polarizability factor multiplying sigma^2_0
    tau_kind: int = TAU_LINE_CENTER
    mu_quad: int = MU_GL_HALF
    formal_solver: int = FS_DELO_LINEAR
    freq_norm: int = 1       # 1: renormalise the spectral weights to sum 1
    name: str = ""

    @property
    def N(self) -> int:
        return 2 * self.Ns * self.Nmu * self.Nnu

    def with_(self, **kw) -> "Atmosphere":
        return dataclasses.replace(self, **kw)


def log_tau(tau_min: float, tau_max: float, Ns: int) -> np.ndarray:
    return np.logspace(math.log10(tau_min), math.log10(tau_max), Ns)


def planck_profile(tau: np.ndarray, B0: float = 1.0, Bc: float = 0.0) -> np.ndarray:
    """Depth-dependent Planck function B(tau) = B0 + Bc*log10(1+tau)."""
    return B0 + Bc * np.log10(1.0 + tau)


def slab(Ns, Nmu, Nnu, tau_min, tau_max, x_max, *, eps=1e-4, a=1e-3, W2=1.0,
         Bc=0.0, formal_solver=FS_DELO_LINEAR, name="") -> Atmosphere:
    tau = log_tau(tau_min, tau_max, Ns)
    return Atmosphere(Ns=Ns, Nmu=Nmu, Nnu=Nnu, tau=tau, B=planck_profile(tau, 1.0, Bc),
                      x_min=-x_max, x_max=x_max, a=a, eps=eps, W2=W2,
                      tau_kind=TAU_LINE_CENTER, mu_quad=MU_GL_HALF,
                      formal_solver=formal_solver, name=name)


def slab70(**kw) -> Atmosphere:
    """N_s=70, N_mu=16 (8 GL nodes per hemisphere), N_nu=21 in [-6,6] (47,040 unknowns)."""
    return slab(70, 16, 21, 1e-4, 1e6, 6.0, name="slab70", **kw)


def slab300(**kw) -> Atmosphere:
    """N_s=300, N_mu=32, N_nu=101 in [-8,8] (1,939,200 unknowns)."""
    return slab(300, 32, 101, 1e-4, 1e8, 8.0, name="slab300", **kw)


SWEEP_NS = (100, 250, 500, 1000, 2000)
SWEEP_EPS = (1e-2, 1e-4, 1e-6)


def sweep(Ns: int, eps: float = 1e-4, Bc: float = 0.0, **kw) -> Atmosphere:
    """Size-robustness sweep: N_mu=64, N_nu=201 in [-8,8], tau 1e-4..1e8."""
    return slab(Ns, 64, 201, 1e-4, 1e8, 8.0, eps=eps, Bc=Bc,
                name=f"sweep_Ns{Ns}_eps{eps:g}_Bc{Bc:g}", **kw)


def paper(Ns: int = 140, Nmu: int = 20, Nnu: int = 20, **kw) -> Atmosphere:
    """The paper's own setting (Sect. 4.1): frequency-integrated tau log-spaced
    1e-5..1e4, N_mu full-range Gauss-Legendre nodes, N_nu points in [-5,5]."""
    tau = log_tau(1e-5, 1e4, Ns)
    at = Atmosphere(Ns=Ns, Nmu=Nmu, Nnu=Nnu, tau=tau, B=np.ones(Ns), x_min=-5.0, x_max=5.0,
                    a=1e-3, eps=1e-4, W2=1.0, tau_kind=TAU_FREQ_INTEGRATED,
                    mu_quad=MU_GL_FULL, formal_solver=FS_DELO_LINEAR, name=f"paper_Ns{Ns}")
    return at.with_(**kw) if kw else at


def tiny(Ns=6, Nmu=4, Nnu=5, **kw) -> Atmosphere:
    """A very small slab for brute-force checks (dense matrices, eigenvalues)."""
    at = slab(Ns, Nmu, Nnu, 1e-3, 1e3, 4.0, name=f"tiny_{Ns}_{Nmu}_{Nnu}")
    return at.with_(**kw) if kw else at


# --------------------------------------------------------------------------
# splitmix64 (Steele, Lea & Flood 2014) for the uneven batch
# --------------------------------------------------------------------------
_M64 = (1 << 64) - 1


class SplitMix64:
    def __init__(self, seed: int):
        self.state = seed & _M64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _M64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def randint(self, lo: int, hi: int) -> int:
        """Uniform integer in [lo, hi]."""
        return lo + int(self.uniform() * (hi - lo + 1))


BATCH_SEED = 0x2110118730000001
STREAM_SEED = 0x2110118730000002


def batch_instances(count: int = 512, seed: int = BATCH_SEED) -> List[Atmosphere]:
    """Uneven atmospheres: N_s~U[50,400], N_nu~U{21,23,...,101}, N_mu~U{8,16,32},
    eps log-U[1e-6,1e-2], a log-U[1e-4,1e-2], B=1+c log10(1+tau), c~U[0,1];
    tau 1e-4..1e8 line-centre, x in [-8,8]."""
    g = SplitMix64(seed)
    out = []
    for i in range(count):
        Ns = g.randint(50, 400)
        Nnu = 21 + 2 * g.randint(0, 40)
        Nmu = (8, 16, 32)[g.randint(0, 2)]
        eps = 10.0 ** (-6.0 + 4.0 * g.uniform())
        a = 10.0 ** (-4.0 + 2.0 * g.uniform())
        c = g.uniform()
        at = slab(Ns, Nmu, Nnu, 1e-4, 1e8, 8.0, eps=eps, a=a, Bc=c, name=f"batch{i}")
        out.append(at)
    return out


def poisson_arrivals(rate_per_s: float, count: int, seed: int = STREAM_SEED) -> np.ndarray:
    """Arrival times (seconds) of a Poisson stream, drawn with splitmix64."""
    g = SplitMix64(seed ^ int(rate_per_s))
    t, out = 0.0, np.empty(count)
    for i in range(count):
        u = g.uniform()
        t += -math.log1p(-u) / rate_per_s
        out[i] = t
    return out


def random_vector(N: int, seed: int) -> np.ndarray:
    """Seeded standard-normal vector of length N (float64)."""
    return np.random.default_rng(seed).standard_normal(N)
