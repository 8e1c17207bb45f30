"""Helpers shared by the GPU parity tests (tests only)."""
import numpy as np
import torch

from paper_2110_11873_gb300 import Problem
from paper_2110_11873_gb300 import build as B

_built = False


def problem(atm, **kw) -> Problem:
    global _built
    if not _built:
        B.build()
        _built = True
    return Problem(atm, **kw)


def to_dev(x: np.ndarray, dtype=torch.float64) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def to_host(x: torch.Tensor) -> np.ndarray:
    return x.detach().double().cpu().numpy()


def stokes_blocks(n: int, layout: str):
    """Index sets of the Stokes I and Q parts of a vector of length n:
    "I" the I-form layout x[s][k][m][p] (first half I, second half Q),
    "sigma" the sigma-form layout (sigma00, sigma20 interleaved per height),
    "flat" the whole vector as one block."""
    if layout == "flat":
        return [("all", slice(None))]
    assert n % 2 == 0, f"a {layout}-form vector has even length, got {n}"
    if layout == "I":
        return [("I", slice(0, n // 2)), ("Q", slice(n // 2, n))]
    if layout == "sigma":
        return [("sigma00", slice(0, n, 2)), ("sigma20", slice(1, n, 2))]
    raise ValueError(layout)


def assert_close_scaled(got, ref, tol, what="", layout="I"):
    """Per Stokes block b: max_{i in b} |got_i - ref_i| <= tol * max_{i in b} |ref_i|.

    Each block is scaled by its own largest reference entry, so a Q part
    that is orders of magnitude below the I part is checked at the same
    relative accuracy.  A block whose reference is exactly zero is scaled
    by the whole vector's largest entry.  Returns the worst scaled error."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    whole = max(float(np.max(np.abs(ref))), 1e-300) if ref.size else 1.0
    worst = 0.0
    for name, ix in stokes_blocks(ref.size, layout):
        r, g = ref.reshape(-1)[ix], got.reshape(-1)[ix]
        if r.size == 0:
            continue
        scale = float(np.max(np.abs(r)))
        if scale == 0.0:
            scale = whole
        err = float(np.max(np.abs(g - r)))
        assert err <= tol * scale, f"{what} [{name}]: max err {err:.3e} > {tol:.1e} * {scale:.3e}"
        worst = max(worst, err / scale)
    return worst


def perturbed(b, seed):
    """b with every entry moved by about 1e-15 relative (seeded)."""
    return b * (1.0 + 1e-15 * np.random.default_rng(seed).standard_normal(b.size))


def assert_iterate(got, xo, xp, what, floor=1e-10):
    """Per Stokes block (I, then Q): max|got - xo| <= tol * max|xo| with
    tol = max(floor, 20 * the oracle's own change when b is perturbed by
    1e-15 relative, xp).  The Q part of a solution is about 1e-3 of the I
    part, so each block is scaled by its own largest entry."""
    n = xo.size // 2
    for name, sl in (("I", slice(0, n)), ("Q", slice(n, None))):
        scale = np.max(np.abs(xo[sl]))
        own = np.max(np.abs(xp[sl] - xo[sl])) / scale
        tol = max(floor, 20 * own)
        assert_close_scaled(got[sl], xo[sl], tol, f"{what} [{name}] (oracle's own change {own:.1e})",
                            layout="flat")
