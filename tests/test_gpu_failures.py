"""Failure detection through the C ABI, with no GPU fault.

Each failure is made on the host or by a bounded device-side wait: a
NaN-poisoned right-hand side (RTE_ERR_DIVERGED), an iteration cap
(RTE_ERR_MAXITER), a problem larger than the device (RTE_ERR_NOMEM, refused
before anything is allocated) and a grid barrier that one block never
reaches (RTE_ERR_TIMEOUT, after a 1 ms wait limit).  After each, the same
handle, server or context must still solve a normal problem.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip('torch')


def small():
    return workloads.checkerboard(m=12, levels=1, g=0.6, ratio=0.9, blocks=2, nrhs=1)


def solve_ok(solver, p, tol=1e-8):
    """A normal solve on `solver`, judged in the oracle's operator."""
    q = solver.rhs(torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda'))
    u, info = solver.solve(q, tol=tol)
    assert info['status'] == 0, info
    disc = oracle.Discretisation(p.m, p.levels, p.sigma_t, p.sigma_s, p.g)
    ops = oracle.Operators(disc, n_plus=solver.options.n_plus,
                           n_minus=solver.options.n_minus)
    qr = disc.source(p.q_nodal[0])
    res = np.linalg.norm(ops.apply_EK(u[0].cpu().numpy()) - qr) / np.linalg.norm(qr)
    assert res <= 1.05 * tol, res


@pytest.mark.parametrize('prec', [0, 2])
def test_nan_rhs_diverges_and_handle_stays_usable(prec):
    import paper_2102_09038_gb300 as rte
    p = small()
    s = rte.Solver(p, n_plus=2, n_minus=3, precision=prec)
    q = s.rhs(torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda'))
    q[0, 5, 3] = float('nan')
    u, info = None, None
    with pytest.raises(rte.RteError) as e:
        s.solve(q, tol=1e-8)
    assert e.value.code == 3   # RTE_ERR_DIVERGED
    solve_ok(s, p)
    s.close()


def test_iteration_cap_and_handle_stays_usable():
    import paper_2102_09038_gb300 as rte
    p = small()
    s = rte.Solver(p, n_plus=2, n_minus=3, max_iter=2)
    q = s.rhs(torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda'))
    u, info = s.solve(q, tol=1e-14)
    assert info['status'] == 4 and info['iterations'] == 2, info   # RTE_ERR_MAXITER
    # the capped iterate is still the Richardson iterate: its residual fell
    assert info['history'][2] < info['history'][0]
    u, info = s.solve(q, tol=0.9)
    assert info['status'] == 0 and info['iterations'] <= 1, info
    s.close()
    solve_ok(rte.Solver(p, n_plus=2, n_minus=3), p)


def test_problem_beyond_device_memory_is_refused_before_allocation():
    import paper_2102_09038_gb300 as rte
    p = workloads.constant(64, 3, 0.5, 1.0, 0.5)
    free, total = torch.cuda.mem_get_info()
    nrhs = 1
    while rte.estimate_bytes(p, nrhs=nrhs) <= 2 * total:
        nrhs *= 2
    with pytest.raises(rte.RteError) as e:
        rte.Solver(p, max_rhs=nrhs)
    assert e.value.code == 2   # RTE_ERR_NOMEM
    assert 'MiB' in str(e.value)
    assert torch.cuda.mem_get_info()[0] >= free - (256 << 20)
    solve_ok(rte.Solver(small(), n_plus=2, n_minus=3), small())


def test_server_reports_failed_requests_and_keeps_serving():
    # a NaN source (DIVERGED) and an oversize request (NOMEM, run alone as
    # larger than the budget) fail on their own; the next request succeeds
    import paper_2102_09038_gb300 as rte
    p = small()
    sv = rte.Server(hbm_budget_bytes=8 << 30, slots=2, n_plus=2, n_minus=3)
    bad = p.q_nodal.copy()
    bad[0, 7] = np.nan
    big = workloads.constant(64, 3, 0.5, 1.0, 0.5)
    total = torch.cuda.mem_get_info()[1]
    nrhs = 1
    while rte.estimate_bytes(big, nrhs=nrhs) <= 2 * total:
        nrhs *= 2
    ids = [sv.submit(p, bad, tol=1e-8),
           sv.submit(big, np.ones((nrhs, big.n_nodes)), tol=1e-8),
           sv.submit(p, p.q_nodal, tol=1e-8)]
    codes = []
    for rid in ids[:2]:
        with pytest.raises(rte.RteError) as e:
            sv.wait(rid)
        codes.append(e.value.code)
    assert codes == [3, 2]
    u, info = sv.wait(ids[2])
    assert info['rel_residual'] <= 1e-8
    sv.close()


def test_barrier_wait_runs_out_and_context_stays_usable():
    # one block never reaches the barrier: the others give up after the
    # 1 ms limit, the kernel returns and the call reports RTE_ERR_TIMEOUT
    import paper_2102_09038_gb300 as rte
    rte.set_wait_limit(1e-3)
    try:
        rc, timed_out, passed = rte.barrier_selftest(8, skip_block=3, rounds=4)
        assert (rc, timed_out, passed) == (5, 1, 0)
        rc, timed_out, passed = rte.barrier_selftest(8, skip_block=-1, rounds=4)
        assert (rc, timed_out, passed) == (0, 0, 8)
    finally:
        rte.set_wait_limit(2.0)
    rc, timed_out, passed = rte.barrier_selftest(152, skip_block=-1, rounds=16)
    assert (rc, timed_out, passed) == (0, 0, 152)
    solve_ok(rte.Solver(small(), n_plus=2, n_minus=3), small())
