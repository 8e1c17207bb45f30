"""The DELO-parabolic formal solver on the GPU (FP64 path).

Against the oracle at the FP64 tolerance 1e-10: the I-form operator, its
right-hand side, the Jacobi diagonal and the local-Lambda preconditioner
(both carry the extra e * gamma term of the Lambda diagonal), the sigma-form
operator, and converged solves.  The atmospheres cover one and several depth
tiles of the formal-solver kernel (the downwind node of a tile's last step
belongs to the next tile), partial ray groups, and thin and thick steps
(both branches of the coefficient series).  The FP32 paths refuse the
scheme.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import rt_workloads as W
from oracle.transfer import Transfer
from paper_2110_11873_gb300 import Server
from paper_2110_11873_gb300 import _native as N
from paper_2110_11873_gb300.api import _desc_of

from gpu_util import assert_close_scaled, problem, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
PARA = W.FS_DELO_PARABOLIC

CASES = [
    ("tiny", W.tiny(formal_solver=PARA)),
    ("ragged-37x6x33", W.slab(37, 6, 33, 1e-4, 1e6, 6.0, Bc=0.3, eps=1e-3, formal_solver=PARA)),
    ("slab70", W.slab70(formal_solver=PARA)),
    ("paper-60", W.paper(60, freq_norm=0, formal_solver=PARA)),
    ("slab300", W.slab300(formal_solver=PARA)),
]


@pytest.fixture(params=CASES, ids=[c[0] for c in CASES], scope="module")
def pair(request):
    name, at = request.param
    return name, at, problem(at), Transfer(at)


def test_apply_rhs_diagonal_and_preconditioner_match_the_oracle(pair):
    name, at, P, tr = pair
    x = W.random_vector(tr.N, 7)
    assert_close_scaled(to_host(P.apply(to_dev(x))), tr.apply_I(x), TOL64, name + " apply")
    assert_close_scaled(to_host(P.rhs()), tr.rhs_I(), TOL64, name + " rhs")
    assert_close_scaled(to_host(P.jacobi_diag()), tr.jacobi_I(), TOL64, name + " diag")
    assert_close_scaled(to_host(P.precond_local_lambda(to_dev(x))), tr.local_lambda_I_inverse(x), TOL64,
                        name + " local Lambda")


def test_sigma_form_apply_matches_the_oracle(pair):
    name, at, _, tr = pair
    Ps = problem(at, form="sigma")
    s = W.random_vector(2 * at.Ns, 8)
    assert_close_scaled(to_host(Ps.apply(to_dev(s))), tr.apply_sigma(s), TOL64, name + " sigma", layout="sigma")
    # the sigma20 part of b = J t + c is a near cancellation (T201 integrates to zero over a
    # hemisphere of isotropic radiation): it is checked on the scale of the whole vector
    assert_close_scaled(to_host(Ps.rhs()), tr.rhs_sigma(), TOL64, name + " sigma rhs", layout="flat")


@pytest.mark.parametrize("precond", ["jacobi", "local_lambda"])
def test_gmres_reaches_the_exact_solution(precond):
    at = W.slab70(formal_solver=PARA)
    tr = Transfer(at)
    P = problem(at)
    b = tr.rhs_I()
    x, info = P.solve(to_dev(b), "gmres", restart=30, precond=precond, rtol=1e-10, maxit=20000)
    assert info.status == 0, info
    xh = to_host(x)
    assert np.linalg.norm(b - tr.apply_I(xh)) / np.linalg.norm(b) < 1e-10
    x_ex = tr.exact_I()
    assert np.linalg.norm(xh - x_ex) / np.linalg.norm(x_ex) < 1e-6


def test_fp32_paths_refuse_the_parabolic_scheme():
    at = W.tiny(formal_solver=PARA)
    P = problem(at)
    with pytest.raises(N.RTError):
        P.apply_f32(torch.zeros(P.N, dtype=torch.float32, device="cuda"))
    with pytest.raises(N.RTError):
        P.solve(P.rhs(), "gmres", precond="local_lambda", precision="fp32_refine")
    srv = Server(mem_budget_bytes=64 << 20, max_slots=2)
    keep = []
    d = _desc_of(at, keep)
    t = C.c_uint64()
    assert srv.lib.rt_batch_submit(srv.handle, C.byref(d), None, C.byref(t)) == N.RT_EINVAL
    srv.close()
