"""GPU parity of the operator kernels against the oracle (C-ABI path).

Tolerances: FP64 paths 1e-10 relative to the largest entry (rounding of
sums over N_mu*N_nu rays and recurrences over N_s steps is ~1e-15; the two
sides also compute the Voigt profile by different algorithms, ~1e-13).
FP32 operator: 2e-5 relative (single precision, ~1e-7 per step over
N_s-step recurrences and N_mu*N_nu-term sums)."""
import numpy as np
import pytest
import torch

import rt_workloads as W
from oracle.transfer import Transfer

from gpu_util import assert_close_scaled, problem, to_dev, to_host

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 2e-5


def _cases():
    t = W.tiny()
    yield "tiny", t
    yield "tiny-euler-B", t.with_(formal_solver=W.FS_IMPLICIT_EULER, B=W.planck_profile(t.tau, 1.0, 0.7), eps=3e-2)
    yield "tiny-trap-W2=0", t.with_(formal_solver=W.FS_TRAPEZOIDAL, W2=0.0)
    yield "minimal-2x2x2", W.slab(2, 2, 2, 1e-2, 1e2, 3.0)
    yield "ragged-37x6x33", W.slab(37, 6, 33, 1e-4, 1e6, 6.0, Bc=0.3, eps=1e-3)
    yield "slab70", W.slab70()
    yield "slab70-euler", W.slab70(formal_solver=W.FS_IMPLICIT_EULER)
    yield "slab70-plain-trapezoid", W.slab70().with_(freq_norm=0)
    yield "paper-40-fullGL-freqint", W.paper(40, freq_norm=0)
    yield "batch-instance-3", W.batch_instances(4)[3]


CASES = list(_cases())
IDS = [c[0] for c in CASES]


@pytest.fixture(params=CASES, ids=IDS, scope="module")
def pair(request):
    name, at = request.param
    return name, at, problem(at), Transfer(at)


def test_grids_match(pair):
    name, at, P, tr = pair
    g = P.grids()
    np.testing.assert_allclose(g["mu"], tr.g.mu, rtol=0, atol=2e-15)
    np.testing.assert_allclose(g["w_mu"], tr.g.w_mu, rtol=1e-13)
    np.testing.assert_allclose(g["x"], tr.g.x, rtol=0, atol=1e-14)
    np.testing.assert_allclose(g["phi"], tr.g.phi, rtol=1e-12)
    np.testing.assert_allclose(g["w_nu"], tr.g.w_nu, rtol=1e-12)
    np.testing.assert_allclose(g["phi_hat"], tr.g.phi_hat, rtol=1e-12)


def test_apply_fp64(pair):
    name, at, P, tr = pair
    x = W.random_vector(tr.N, 11)
    y = to_host(P.apply(to_dev(x)))
    torch.cuda.synchronize()
    assert_close_scaled(y, tr.apply_I(x), TOL64, name)


def test_apply_is_linear_and_deterministic(pair):
    name, at, P, tr = pair
    x = to_dev(W.random_vector(tr.N, 12))
    y1 = P.apply(x)
    y2 = P.apply(x)
    assert torch.equal(y1, y2)
    y3 = P.apply(2.0 * x)
    assert torch.allclose(y3, 2.0 * y1, rtol=1e-14, atol=1e-300)


def test_rhs(pair):
    name, at, P, tr = pair
    assert_close_scaled(to_host(P.rhs()), tr.rhs_I(), TOL64, name)


def test_jacobi_diagonal(pair):
    name, at, P, tr = pair
    assert_close_scaled(to_host(P.jacobi_diag()), tr.jacobi_I(), TOL64, name)


def test_local_lambda_preconditioner(pair):
    name, at, P, tr = pair
    v = W.random_vector(tr.N, 13)
    assert_close_scaled(to_host(P.precond_local_lambda(to_dev(v))), tr.local_lambda_I_inverse(v), TOL64, name)


def test_apply_fp32(pair):
    name, at, P, tr = pair
    x = W.random_vector(tr.N, 14)
    y = to_host(P.apply_f32(to_dev(x, torch.float32)))
    ref = tr.apply_I(x.astype(np.float32).astype(np.float64))
    assert_close_scaled(y, ref, TOL32, name)


def test_point_source_columns_are_one_sided():
    """A column of A_I for a unit vector: zero upwind along the unit's own ray
    (Sect. 4.4), identical to the oracle's column."""
    at = W.slab(24, 8, 9, 1e-3, 1e4, 4.0)
    P, tr = problem(at), Transfer(at)
    for j in (5, tr.N // 2 + 17, tr.N - 3):
        e = np.zeros(tr.N)
        e[j] = 1.0
        col = to_host(P.apply(to_dev(e)))
        assert_close_scaled(col, tr.apply_I(e), TOL64, f"column {j}")


@pytest.mark.slow
def test_bench_size_slab300_full_vector():
    """The benchmark workload itself (1,939,200 unknowns), every element."""
    at = W.slab300()
    P, tr = problem(at), Transfer(at)
    x = W.random_vector(tr.N, 21)
    assert_close_scaled(to_host(P.apply(to_dev(x))), tr.apply_I(x), TOL64, "slab300")
    assert_close_scaled(to_host(P.rhs()), tr.rhs_I(), TOL64, "slab300 rhs")
    y32 = to_host(P.apply_f32(to_dev(x, torch.float32)))
    assert_close_scaled(y32, tr.apply_I(x.astype(np.float32).astype(np.float64)), TOL32, "slab300 fp32")


@pytest.mark.slow
def test_deep_sweep_atmosphere_ns2000():
    """Largest sweep atmosphere (N_s=2000, N_mu=64, N_nu=201: 51,456,000
    unknowns): full-vector parity of the FP64 and FP32 applies."""
    at = W.sweep(2000, eps=1e-6, Bc=0.5)
    P, tr = problem(at), Transfer(at)
    x = W.random_vector(tr.N, 22)
    assert_close_scaled(to_host(P.apply(to_dev(x))), tr.apply_I(x), TOL64, "sweep2000")
    y32 = to_host(P.apply_f32(to_dev(x, torch.float32)))
    assert_close_scaled(y32, tr.apply_I(x.astype(np.float32).astype(np.float64)), TOL32, "sweep2000 fp32")


def test_arnoldi_mgs_step_against_plain_mgs():
    """rt_arnoldi_mgs: h_i = <w, v_i>, w -= h_i v_i (i = 0..j), h_{j+1} = ||w||,
    v_{j+1} = w / h_{j+1}, compared with the same loop in numpy."""
    at = W.slab(37, 6, 33, 1e-4, 1e6, 6.0)
    P = problem(at)
    N = P.N
    j = 5
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((N, j + 1)))
    w0 = rng.standard_normal(N)
    V = np.zeros((j + 2) * N)
    V[: (j + 1) * N] = Q.T.reshape(-1)
    Vd = to_dev(V)
    wd = to_dev(w0)
    h = to_host(P.arnoldi_mgs(Vd, j, wd))
    w = w0.copy()
    href = np.zeros(j + 2)
    for i in range(j + 1):
        href[i] = np.dot(w, Q[:, i])
        w = w - href[i] * Q[:, i]
    href[j + 1] = np.linalg.norm(w)
    np.testing.assert_allclose(h, href, rtol=1e-12, atol=1e-14)
    np.testing.assert_allclose(to_host(Vd)[(j + 1) * N:], w / href[j + 1], rtol=1e-11, atol=1e-14)
    np.testing.assert_allclose(to_host(wd), w, rtol=1e-11, atol=1e-14)


@pytest.mark.parametrize("j", [0, 1, 2, 3, 4, 5, 6, 7, 8, 9, 15, 31, 63, 158, 159])
def test_arnoldi_block_mgs_step_against_plain_mgs(j):
    """rt_arnoldi_bmgs (the GMRES orthogonalisation): blocks of 4 basis vectors
    with the Gram correction give the MGS coefficients of the same loop in
    numpy, on a basis that is orthonormal only to rounding (its Gram rows
    computed in numpy), and write the Gram row of the new vector.  j covers
    every size of the last block, with and without a full block before it,
    and the last steps of the longest cycle (160)."""
    at = W.slab(37, 6, 33, 1e-4, 1e6, 6.0)
    P = problem(at)
    N = P.N
    rng = np.random.default_rng(7 + j)
    Q, _ = np.linalg.qr(rng.standard_normal((N, j + 1)))
    # a slightly non-orthogonal basis, so the Gram correction matters
    Q = Q + 1e-9 * rng.standard_normal(Q.shape)
    Q /= np.linalg.norm(Q, axis=0)
    gram = np.zeros((j + 2, 4))
    for i in range(1, j + 1):
        for d in range(1, 4):
            if i - d >= 0:
                gram[i, d] = Q[:, i] @ Q[:, i - d]
    w0 = rng.standard_normal(N)
    V = np.zeros((j + 2) * N)
    V[: (j + 1) * N] = Q.T.reshape(-1)
    Vd, wd, gd = to_dev(V), to_dev(w0), to_dev(gram.reshape(-1))
    h = to_host(P.arnoldi_bmgs(Vd, j, wd, gd))
    w = w0.copy()
    href = np.zeros(j + 2)
    for i in range(j + 1):
        href[i] = np.dot(w, Q[:, i])
        w = w - href[i] * Q[:, i]
    href[j + 1] = np.linalg.norm(w)
    np.testing.assert_allclose(h, href, rtol=1e-10, atol=1e-13)
    vnew = w / href[j + 1]
    np.testing.assert_allclose(to_host(Vd)[(j + 1) * N:], vnew, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(to_host(wd), w, rtol=1e-9, atol=1e-13)
    g_out = to_host(gd).reshape(j + 2, 4)
    for d in range(1, 4):   # the new row holds the entries of v_{j+1}'s own block
        if d <= (j + 1) % 4:
            assert abs(g_out[j + 1, d] - vnew @ Q[:, j + 1 - d]) < 1e-13
        else:
            assert g_out[j + 1, d] == gram[j + 1, d]   # left as it was
