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


def assert_close_scaled(got, ref, tol, what=""):
    """max_i |got_i - ref_i| <= tol * max_i |ref_i| (elementwise, scaled by the vector's size)."""
    got = np.asarray(got)
    ref = np.asarray(ref)
    assert got.shape == ref.shape, (got.shape, ref.shape)
    scale = max(np.max(np.abs(ref)), 1e-300)
    err = np.max(np.abs(got - ref))
    assert err <= tol * scale, f"{what}: max err {err:.3e} > {tol:.1e} * {scale:.3e}"
    return err / scale
