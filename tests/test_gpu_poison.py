"""Workspaces filled with NaN before first use change no result (GPU).

With RT_POISON=1 every device workspace the library allocates -- a
problem's tables and Krylov vectors, the batch server's buffers and every
block its arena hands out -- is filled with 0xFF bytes (NaN in FP64 and
FP32, -1 in integers) before it is returned.  A kernel that read memory
nothing had written would then turn a result into NaN or change it.  The
same operations on freshly created problems and a fresh server, with and
without the variable, must agree bit for bit (every reduction of the library
has a fixed order).
"""
import numpy as np
import pytest
import torch

import rt_workloads as W
from paper_2110_11873_gb300 import Server

from gpu_util import problem, to_dev, to_host

pytestmark = pytest.mark.gpu


def _runs():
    out = {}
    for name, at in (("slab70", W.slab70()), ("ragged", W.slab(37, 6, 33, 1e-4, 1e6, 6.0, Bc=0.3, eps=1e-3))):
        P = problem(at)
        b = P.rhs()
        out[name + ":rhs"] = to_host(b)
        out[name + ":diag"] = to_host(P.jacobi_diag())
        g = torch.Generator(device="cuda").manual_seed(5)
        x = torch.rand(P.N, dtype=torch.float64, device="cuda", generator=g)
        out[name + ":apply64"] = to_host(P.apply(x))
        out[name + ":apply32"] = to_host(P.apply_f32(x.float()))
        for key, method, kw in (("gmres-jacobi", "gmres", dict(precond="jacobi")),
                                ("gmres-ll-fp32", "gmres", dict(precond="local_lambda", precision="fp32_refine")),
                                ("bicgstab-ll", "bicgstab", dict(precond="local_lambda")),
                                ("cgs-jacobi", "cgs", dict(precond="jacobi"))):
            xs, info = P.solve(b, method, rtol=1e-8, **kw)
            out[f"{name}:{key}"] = to_host(xs)
            out[f"{name}:{key}:iters"] = np.array([info.iters])
        P.check()
        P.close()
    srv = Server(mem_budget_bytes=1 << 30, max_slots=4, precond="local_lambda", precision="fp32_refine")
    ats = [W.slab(20 + 7 * i, 8, 11 + 2 * i, 1e-4, 1e6, 6.0, eps=10.0 ** (-2 - i), name=f"p{i}") for i in range(4)]
    tickets = [srv.submit(a) for a in ats]
    done = {}
    while len(done) < len(tickets):
        for t in tickets:
            if t not in done:
                r = srv.poll(t)
                if r is not None:
                    done[t] = r
    srv.close()
    for i, t in enumerate(tickets):
        st, info, xb = done[t]
        assert st == 0
        out[f"batch{i}"] = xb
    return out


def test_poisoned_workspaces_change_no_result(monkeypatch):
    base = _runs()
    monkeypatch.setenv("RT_POISON", "1")
    poisoned = _runs()
    assert base.keys() == poisoned.keys()
    for k in base:
        assert np.all(np.isfinite(poisoned[k])), k
        np.testing.assert_array_equal(poisoned[k], base[k], err_msg=k)
