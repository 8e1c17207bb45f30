"""rt_arnoldi_mgs_static: the MGS Arnoldi step for callers that cannot
allocate device memory (stream capture, memory owned by another allocator,
service loops that cannot afford an allocation's synchronisation).  Its
scratch is a static device array inside the library; the step must give the
same result as rt_arnoldi_mgs, call after call, and allocate nothing.

Kept in a file of its own, collected last."""
import ctypes as C

import numpy as np
import pytest
import torch

import rt_workloads as W
from paper_2110_11873_gb300 import Problem
from paper_2110_11873_gb300 import _native as N
from paper_2110_11873_gb300 import build as B

pytestmark = pytest.mark.gpu

TOL = 1e-12   # the MGS step's tolerance in test_gpu_operator.py


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_no_alloc_step_matches_the_allocating_step_on_two_calls():
    B.build()
    lib = N.load()
    P = Problem(W.slab(37, 6, 33, 1e-4, 1e6, 6.0))
    n, j = P.N, 7
    rng = np.random.default_rng(11)
    Q, _ = np.linalg.qr(rng.standard_normal((n, j + 1)))
    V0 = np.zeros((j + 2) * n)
    V0[: (j + 1) * n] = Q.T.reshape(-1)
    w0 = rng.standard_normal(n)
    free_before = None
    for call in range(2):
        Va = torch.from_numpy(V0).cuda()
        wa = torch.from_numpy(w0).cuda()
        ha = P.arnoldi_mgs(Va, j, wa)
        Vb = torch.from_numpy(V0).cuda()
        wb = torch.from_numpy(w0).cuda()
        hb = torch.full((j + 2,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        if call == 1:
            free_before = torch.cuda.mem_get_info()[0]
        st = lib.rt_arnoldi_mgs_static(C.c_void_p(Vb.data_ptr()), n, j, C.c_void_p(wb.data_ptr()),
                                       C.c_void_p(hb.data_ptr()), _stream())
        assert st == N.RT_OK, N.last_error()
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free_before
        for got, ref in ((hb, ha), (Vb, Va), (wb, wa)):
            g, r = got.cpu().numpy(), ref.cpu().numpy()
            assert np.max(np.abs(g - r)) <= TOL * max(np.max(np.abs(r)), 1e-300)
    P.close()


def test_no_alloc_step_rejects_sizes_beyond_its_limits():
    lib = N.load()
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    p = C.c_void_p(x.data_ptr())
    assert lib.rt_arnoldi_mgs_static(p, 0, 0, p, p, _stream()) == N.RT_EINVAL
    assert "N must be" in N.last_error()
    assert lib.rt_arnoldi_mgs_static(p, 4, 64, p, p, _stream()) == N.RT_EINVAL
    assert "j must be" in N.last_error()
    assert lib.rt_arnoldi_mgs_static(p, (1 << 40) + 1, 0, p, p, _stream()) == N.RT_EINVAL
