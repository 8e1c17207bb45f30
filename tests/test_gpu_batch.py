"""Batched uneven instances and the serving loop (rt_server_*), GPU.

* every instance of a batch reaches ||b - A x||/||b|| < 1e-8 measured with the
  oracle's FP64 operator, and lies within 1e-7 of the oracle's exact (LU)
  solution (1e-6 with the FP32 operator inside FP64 refinement);
* GMRES iteration counts equal those of the single-instance GPU solver
  within 1 (same algorithm; reductions summed in a different order);
* an instance's result is bit-identical alone and in a mix (each instance's
  arithmetic depends only on its own data);
* admission by memory budget: more requests than the arena holds are solved
  as slots free up; one that cannot fit even alone fails with RT_ENOMEM.
"""
import time

import numpy as np
import torch
import pytest

import rt_workloads as W
from oracle import krylov as K
from oracle.transfer import Transfer
from paper_2110_11873_gb300 import Server
from paper_2110_11873_gb300 import _native as N

from gpu_util import problem, to_dev, to_host

pytestmark = pytest.mark.gpu


def _uneven(count=6, seed=7):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        Ns = int(rng.integers(20, 60))
        Nmu = int(rng.choice([4, 8, 16]))
        Nnu = int(2 * rng.integers(5, 16) + 1)
        eps = float(10 ** rng.uniform(-4, -2))
        a = float(10 ** rng.uniform(-4, -2))
        out.append(W.slab(Ns, Nmu, Nnu, 1e-4, 1e6, 6.0, eps=eps, a=a, Bc=float(rng.uniform(0, 1)),
                          name=f"u{i}"))
    return out


def _wait(srv, tickets, timeout=120.0):
    res = {}
    t0 = time.time()
    while len(res) < len(tickets):
        for t in tickets:
            if t not in res:
                r = srv.poll(t)
                if r is not None:
                    res[t] = r
        assert time.time() - t0 < timeout, "server did not finish"
        time.sleep(0.002)
    return res


@pytest.fixture(scope="module")
def cases():
    ats = _uneven()
    trs = [Transfer(a) for a in ats]
    return ats, trs, [t.rhs_I() for t in trs], [t.exact_I() for t in trs]


@pytest.mark.parametrize("precision,tol_exact", [("fp64", 1e-7), ("fp32_refine", 1e-6)])
def test_batch_solutions(cases, precision, tol_exact):
    ats, trs, bs, xs = cases
    problem(ats[0])   # builds the library
    srv = Server(mem_budget_bytes=1 << 30, max_slots=8, precond="local_lambda", precision=precision)
    tickets = [srv.submit(a) for a in ats]
    res = _wait(srv, tickets)
    for t, at, tr, b, x_ex in zip(tickets, ats, trs, bs, xs):
        st, info, x = res[t]
        assert st == N.RT_OK, (at.name, info)
        rel = np.linalg.norm(b - tr.apply_I(x)) / np.linalg.norm(b)
        assert rel < 1e-8, (at.name, rel)
        assert np.linalg.norm(x - x_ex) / np.linalg.norm(x_ex) < tol_exact
        # the Givens estimate of the instance's last Arnoldi step, relative to ||b||
        assert np.isfinite(info.err_est) and 0.0 < info.err_est < 1e-4, (at.name, info)
        if precision == "fp64":
            P = problem(at)
            _, si = P.solve(to_dev(b), "gmres", restart=30, precond="local_lambda", rtol=1e-8)
            assert abs(si.iters - info.iters) <= 1, (at.name, si.iters, info.iters)
    srv.close()


def test_result_is_the_same_alone_and_in_the_mix(cases):
    ats, trs, bs, xs = cases
    target = ats[2]
    srv = Server(mem_budget_bytes=1 << 30, max_slots=8, precond="local_lambda")
    (st, info_alone, x_alone), = _wait(srv, [srv.submit(target)]).values()
    tickets = [srv.submit(a) for a in ats[:2]]
    t_target = srv.submit(target)
    tickets += [srv.submit(a) for a in ats[3:]]
    res = _wait(srv, tickets + [t_target])
    st2, info_mix, x_mix = res[t_target]
    assert st == st2 == N.RT_OK
    assert info_alone.iters == info_mix.iters
    assert np.array_equal(x_alone, x_mix)
    srv.close()


@pytest.mark.parametrize("precond", ["jacobi", "none"])
def test_batch_other_preconditioners(cases, precond):
    ats, trs, bs, xs = cases
    srv = Server(mem_budget_bytes=1 << 30, max_slots=8, precond=precond)
    tickets = [srv.submit(a, maxit=20000) for a in ats[:3]]
    res = _wait(srv, tickets, timeout=300)
    for t, tr, b in zip(tickets, trs[:3], bs[:3]):
        st, info, x = res[t]
        assert st == N.RT_OK, info
        assert np.linalg.norm(b - tr.apply_I(x)) / np.linalg.norm(b) < 1e-8
    srv.close()


def test_admission_by_memory_budget_and_late_arrivals(cases):
    ats, trs, bs, xs = cases
    small = W.slab(30, 8, 21, 1e-4, 1e6, 6.0)
    tr = Transfer(small)
    b = tr.rhs_I()
    # an arena that holds one such instance at a time, and more slots than that
    srv = Server(mem_budget_bytes=6 << 20, max_slots=8, precond="local_lambda")
    first = [srv.submit(small) for _ in range(2)]
    time.sleep(0.01)
    late = [srv.submit(small) for _ in range(4)]   # arrive while the first ones are resident
    res = _wait(srv, first + late)
    xs_ = [res[t][2] for t in first + late]
    for st, info, x in res.values():
        assert st == N.RT_OK, info
        assert np.linalg.norm(b - tr.apply_I(x)) / np.linalg.norm(b) < 1e-8
    for x in xs_[1:]:
        assert np.array_equal(x, xs_[0])
    st_ = srv.stats()
    assert st_["completed"] == 6 and st_["resident"] == 0
    assert st_["arena_in_use"] == 0 and st_["arena_largest_free"] == 6 << 20   # every block returned
    # larger than the whole arena: rejected once nothing else is resident
    big = W.slab(300, 16, 61, 1e-4, 1e8, 8.0)
    t = srv.submit(big)
    (st, info, x), = _wait(srv, [t]).values()
    assert st == N.RT_ENOMEM
    srv.close()


def test_autotuned_grids_change_no_result(cases):
    """The server times candidate grids of its persistent kernels on the
    resident work before the first cycle and keeps the fastest; the batch's
    reductions do not depend on the grids, so the solutions are bit-identical
    with and without tuning."""
    ats, trs, bs, xs = cases
    out = {}
    for tune in (True, False):
        # tuning starts once all slots (or 64 instances) are resident
        srv = Server(mem_budget_bytes=1 << 30, max_slots=len(ats), precond="local_lambda", autotune=tune)
        tickets = [srv.submit(a) for a in ats]
        res = _wait(srv, tickets)
        st = srv.stats()
        assert st["tuned"] == (1 if tune else 0)
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        for key in ("grid_quad", "grid_formal", "grid_vec"):
            assert st[key] > 0 and st[key] % sms == 0, (key, st)
        out[tune] = [res[t] for t in tickets]
        srv.close()
    for (s1, i1, x1), (s2, i2, x2) in zip(out[True], out[False]):
        assert s1 == s2 == N.RT_OK
        assert i1.iters == i2.iters
        assert np.array_equal(x1, x2)


@pytest.mark.slow
def test_config4_size_instance_in_a_mix_matches_the_exact_solution(cases):
    """The largest atmosphere of the 512-instance benchmark batch (index 453:
    N_s=384, N_mu=32, N_nu=95, 2,334,720 unknowns), solved with the FP32
    operator inside FP64 refinement among the small uneven instances:
    ||b - A x||/||b|| < 1e-8 with the oracle's FP64 operator, within 1e-6 of
    the oracle's exact (LU-lifted) solution in norm, and per Stokes block
    (each scaled by its own largest entry) within 1e-6 or twice the error of
    the oracle's own FP64 local-Lambda GMRES(30) stopped by the same rule,
    whichever is larger: the stopping rule bounds the residual, not the
    error, and the Q block is about 1e-3 of the I block."""
    ats, trs, bs, xs = cases
    big = W.batch_instances(512)[453]
    assert (big.Ns, big.Nmu, big.Nnu) == (384, 32, 95)
    tr = Transfer(big)
    b = tr.rhs_I()
    x_ex = tr.exact_I()
    srv = Server(mem_budget_bytes=4 << 30, max_slots=8, precond="local_lambda", precision="fp32_refine")
    t_big = srv.submit(big)
    tickets = [srv.submit(a) for a in ats[:3]]
    res = _wait(srv, tickets + [t_big], timeout=300)
    st, info, x = res[t_big]
    srv.close()
    assert st == N.RT_OK, info
    assert np.linalg.norm(b - tr.apply_I(x)) / np.linalg.norm(b) < 1e-8
    assert np.linalg.norm(x - x_ex) / np.linalg.norm(x_ex) < 1e-6
    xo, io = K.gmres(tr.apply_I, b, M_inv=tr.local_lambda_I_inverse, restart=30, tol=1e-8)
    assert io.status == K.OK
    n = x.size // 2
    for name, sl in (("I", slice(0, n)), ("Q", slice(n, None))):
        scale = np.max(np.abs(x_ex[sl]))
        err = np.max(np.abs(x[sl] - x_ex[sl])) / scale
        own = np.max(np.abs(xo[sl] - x_ex[sl])) / scale
        assert err < max(1e-6, 2 * own), (name, err, own)


def test_direct_launches_give_the_graph_results(cases):
    """rt_server_opts.graphs = 0 launches every kernel of a restart cycle on
    the server's stream instead of one captured graph: the same solutions
    bit for bit, the same iteration counts, and the library's launch
    counter advances by at least the cycles' kernels."""
    from paper_2110_11873_gb300 import _native as NN
    ats, trs, bs, xs = cases
    problem(ats[0])
    lib = NN.load()
    out = {}
    for graphs in (True, False):
        srv = Server(mem_budget_bytes=1 << 30, max_slots=8, precond="local_lambda", precision="fp32_refine",
                     graphs=graphs, autotune=False)
        l0 = lib.rt_launch_count()
        tickets = [srv.submit(a) for a in ats]
        res = _wait(srv, tickets)
        out[graphs] = ([res[t][2] for t in tickets], [res[t][1].iters for t in tickets],
                       lib.rt_launch_count() - l0, srv.stats()["cycles"])
        srv.close()
    (xg, ig, lg, cg), (xd, id_, ld, cd) = out[True], out[False]
    assert ig == id_
    for a, b in zip(xg, xd):
        np.testing.assert_array_equal(a, b)
    assert ld >= cd > 0 and lg >= cg > 0, (lg, cg, ld, cd)



def _until(cond, timeout=60.0):
    t0 = time.time()
    while not cond():
        assert time.time() - t0 < timeout, "server state not reached"
        time.sleep(0.002)


def test_cancel_and_deadline(cases):
    """rt_batch_cancel ends a queued request at once (x zeros) and a resident
    one after the restart cycle in progress (x the iterate it reached); a
    request past deadline_ms ends the same way, whether resident or still
    queued; each reports RT_ECANCELED, and later requests on the same server
    are solved as usual."""
    ats, trs, bs, xs = cases
    # unpreconditioned GMRES(10) on a thick, strongly scattering slab: thousands of cycles
    slow = W.slab(120, 16, 41, 1e-4, 1e8, 8.0, eps=1e-6, name="slow")
    n_slow = 2 * 120 * 16 * 41
    srv = Server(mem_budget_bytes=1 << 30, max_slots=1, restart=10, precond="none", autotune=False)
    t_res = srv.submit(slow, rtol=1e-14, maxit=10 ** 7)
    t_q = srv.submit(slow, rtol=1e-14, maxit=10 ** 7)
    _until(lambda: srv.stats()["resident"] == 1 and srv.stats()["cycles"] >= 2)
    assert srv.stats()["queued"] == 1 and srv.poll(t_q) is None
    srv.cancel(t_q)
    st, info, x = srv.poll(t_q)        # finished by the cancel call itself
    assert st == N.RT_ECANCELED and info.status == N.RT_ECANCELED and info.iters == 0
    assert x.shape == (n_slow,) and not np.any(x)
    with pytest.raises(N.RTError):     # released by the poll that reported it
        srv.cancel(t_q)

    srv.cancel(t_res)
    (st, info, x), = _wait(srv, [t_res], timeout=30).values()
    assert st == N.RT_ECANCELED and info.iters >= 20 and info.restarts >= 2, info
    assert np.all(np.isfinite(x)) and np.any(x) and 0.0 < info.rel_resid < 1.0, info

    # deadline while resident
    t_d = srv.submit(slow, rtol=1e-14, maxit=10 ** 7, deadline_ms=300.0)
    (st, info, x), = _wait(srv, [t_d], timeout=30).values()
    assert st == N.RT_ECANCELED and info.t_total_ms >= 300.0 and info.iters > 0, info
    assert np.any(x)

    # deadline while queued behind a resident request
    t_hold = srv.submit(slow, rtol=1e-14, maxit=10 ** 7)
    _until(lambda: srv.stats()["resident"] == 1)
    t_qd = srv.submit(slow, rtol=1e-14, maxit=10 ** 7, deadline_ms=100.0)
    (st, info, x), = _wait(srv, [t_qd], timeout=30).values()
    assert st == N.RT_ECANCELED and info.iters == 0 and info.t_total_ms >= 100.0, info
    assert not np.any(x)
    assert srv.poll(t_hold) is None    # the resident request is untouched
    srv.cancel(t_hold)
    (st, info, x), = _wait(srv, [t_hold], timeout=30).values()
    assert st == N.RT_ECANCELED

    # the server goes on serving
    t_ok = srv.submit(ats[0], maxit=20000)
    (st, info, x), = _wait(srv, [t_ok], timeout=120).values()
    assert st == N.RT_OK, info
    assert np.linalg.norm(bs[0] - trs[0].apply_I(x)) / np.linalg.norm(bs[0]) < 1e-8
    s = srv.stats()
    assert s["completed"] == 6 and s["resident"] == 0 and s["queued"] == 0, s
    with pytest.raises(N.RTError):
        srv.submit(slow, deadline_ms=-1.0)
    srv.close()
