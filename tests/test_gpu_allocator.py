"""Caller-provided device memory (rt_problem_create_with_allocator,
rt_server_create_with_allocator), GPU.

The hook is PyTorch's caching allocator (api.TorchAllocator): every device
workspace of a problem or server comes from it, the solves give the same
results, bit for bit, as with the library's own cudaMalloc (the arithmetic
does not depend on where the buffers are), every block is handed back when
the problem or server is destroyed, and a hook that refuses a request makes
the call fail with RT_ENOMEM without leaking the blocks it had granted.
"""
import time

import numpy as np
import pytest
import torch

import rt_workloads as W
from oracle.transfer import Transfer
from paper_2110_11873_gb300 import Server, TorchAllocator
from paper_2110_11873_gb300 import _native as N

from gpu_util import problem, to_dev, to_host

pytestmark = pytest.mark.gpu


def test_solves_through_the_torch_caching_allocator():
    at = W.slab70()
    tr = Transfer(at)
    b_h = tr.rhs_I()
    x_ex = tr.exact_I()
    problem(at).close()   # builds the library
    torch.cuda.synchronize()
    m0 = torch.cuda.memory_allocated()
    A = TorchAllocator()
    P = problem(at, allocator=A)
    assert A.allocs > 0 and torch.cuda.memory_allocated() > m0   # the tables are PyTorch allocations
    Q = problem(at)                                               # the library's own cudaMalloc
    _same_solves(P, Q, tr, b_h)   # (its tensors are freed when it returns)
    n_live = len(A.live)
    assert n_live > 0 and A.allocs >= n_live
    P.close()
    Q.close()
    assert A.releases == A.allocs and not A.live
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == m0


def _same_solves(P, Q, tr, b_h):
    b = to_dev(b_h)
    runs = [("gmres", "jacobi", "fp64"), ("gmres", "local_lambda", "fp32_refine"), ("bicgstab", "jacobi", "fp64")]
    for method, prec, precision in runs:
        xa, ia = P.solve(b, method, precond=prec, precision=precision, rtol=1e-8, maxit=4000)
        xb, ib = Q.solve(b, method, precond=prec, precision=precision, rtol=1e-8, maxit=4000)
        assert ia.ok and ib.ok, (ia, ib)
        assert ia.iters == ib.iters
        assert torch.equal(xa, xb), method
        x = to_host(xa)
        assert np.linalg.norm(b_h - tr.apply_I(x)) / np.linalg.norm(b_h) < 2e-8


def test_a_refusing_hook_gives_enomem_and_leaks_nothing():
    at = W.slab70()
    problem(at).close()
    A = TorchAllocator(fail_after=3)
    with pytest.raises(N.RTError) as ei:
        problem(at, allocator=A)
    assert ei.value.status == N.RT_ENOMEM
    assert A.allocs == 3 and A.releases == 3 and not A.live


def test_server_memory_through_the_hook():
    ats = [W.slab(30, 8, 21, 1e-4, 1e6, 6.0, eps=1e-3, Bc=0.2 * i, name=f"h{i}") for i in range(3)]
    problem(ats[0]).close()
    A = TorchAllocator()
    srv = Server(mem_budget_bytes=64 << 20, max_slots=4, precond="local_lambda", allocator=A)
    assert A.allocs >= 1 and A.live
    tickets = [srv.submit(a) for a in ats]
    out = {}
    t0 = time.time()
    while len(out) < len(tickets):
        for t in tickets:
            if t not in out:
                r = srv.poll(t)
                if r is not None:
                    out[t] = r
        assert time.time() - t0 < 120
        time.sleep(0.002)
    for t, at in zip(tickets, ats):
        st, info, x = out[t]
        assert st == N.RT_OK, info
        tr = Transfer(at)
        b = tr.rhs_I()
        assert np.linalg.norm(b - tr.apply_I(x)) / np.linalg.norm(b) < 1e-8
    srv.close()
    assert A.releases == A.allocs and not A.live
