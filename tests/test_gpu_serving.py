"""The continuous-batching server: requests of different mesh and sphere
sizes, coefficients and anisotropy run concurrently on separate streams;
every result must equal the same problem solved alone (to the solve
tolerance) and satisfy the oracle's residual; a budget smaller than one
request serialises the requests without losing any.  The operator cache
lets requests with the operator of an idle handle skip the set-up, and
evicts idle handles to stay within the budget."""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip('torch')


def mix():
    rng = np.random.default_rng(5)
    out = []
    for i, (m, lv) in enumerate([(8, 1), (12, 2), (16, 1), (6, 2), (10, 1), (16, 2)]):
        g = float(rng.uniform(0.3, 0.9))
        st = float(np.exp(rng.uniform(np.log(0.5), np.log(20.0))))
        ratio = float(rng.uniform(0.5, 0.99))
        p = workloads.constant(m, lv, g, st, ratio * st, 1.0, nrhs=1 + i % 2)
        x, y = workloads.node_xy(m)
        p.q_nodal = np.stack([np.exp(-((x - 0.3 - 0.2 * r) ** 2 + (y - 0.5) ** 2) / 0.02)
                              for r in range(p.nrhs)])
        out.append(p)
    return out


@pytest.mark.parametrize('precision', [0, 2])
def test_mixed_requests_match_solves_alone(precision):
    import paper_2102_09038_gb300 as rte
    probs = mix()
    opts = dict(n_plus=2, n_minus=3, precision=precision)
    alone = []
    for p in probs:
        s = rte.Solver(p, max_rhs=p.nrhs, **opts)
        q = s.rhs(torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda'))
        u, info = s.solve(q, tol=1e-10)
        assert info['status'] == 0
        alone.append(u.cpu().numpy())
        s.close()
    sv = rte.Server(hbm_budget_bytes=64 << 30, slots=3, **opts)
    ids = [sv.submit(p, p.q_nodal, tol=1e-10) for p in probs]
    for p, rid, ua in zip(probs, ids, alone):
        u, info = sv.wait(rid)
        assert info['latency'] >= info['queue'] >= 0.0
        err = np.linalg.norm(u - ua) / np.linalg.norm(ua)
        assert err < 1e-8, (p.m, p.levels, err)
    sv.close()
    # and the served result solves the oracle's system
    p = probs[1]
    disc = oracle.Discretisation(p.m, p.levels, p.sigma_t, p.sigma_s, p.g)
    ops = oracle.Operators(disc, n_plus=2, n_minus=3)
    for r in range(p.nrhs):
        q = disc.source(p.q_nodal[r])
        res = np.linalg.norm(ops.apply_EK(alone[1][r]) - q) / np.linalg.norm(q)
        assert res < 1e-9


def test_budget_smaller_than_a_request_serialises():
    import paper_2102_09038_gb300 as rte
    probs = mix()[:3]
    sv = rte.Server(hbm_budget_bytes=1, slots=3, n_plus=2, n_minus=3)
    ids = [sv.submit(p, p.q_nodal, tol=1e-8) for p in probs]
    infos = [sv.wait(rid)[1] for rid in ids]
    sv.close()
    assert all(i['iterations'] > 0 for i in infos)
    # admitted one at a time, in order: every later request queued at least
    # as long as the earlier one ran
    assert infos[1]['queue'] > 0.0 and infos[2]['queue'] > infos[1]['queue']


def _sources(p, count, seed):
    rng = np.random.default_rng(seed)
    x, y = workloads.node_xy(p.m)
    return [np.stack([np.exp(-((x - c[0]) ** 2 + (y - c[1]) ** 2) / 0.02)
                      for c in rng.uniform(0.2, 0.8, (p.nrhs, 2))]) for _ in range(count)]


def _alone(p, q, **opts):
    import paper_2102_09038_gb300 as rte
    s = rte.Solver(p, max_rhs=p.nrhs, **opts)
    u, info = s.solve(s.rhs(torch.tensor(q, dtype=torch.float64, device='cuda')), tol=1e-10)
    assert info['status'] == 0
    out = u.cpu().numpy()
    s.close()
    return out


def test_operator_cache_reuses_set_up_handles():
    # requests with the operator of an idle handle take it and skip rte_setup:
    # one set-up for four sources of one operator, none for a repeat of it;
    # every result equals the problem solved alone
    import paper_2102_09038_gb300 as rte
    opts = dict(n_plus=2, n_minus=3, precision=2)
    p = workloads.checkerboard(m=16, levels=2, g=0.8, ratio=0.95, blocks=2, nrhs=2)
    srcs = _sources(p, 4, 7)
    sv = rte.Server(hbm_budget_bytes=64 << 30, slots=1, **opts)
    got = [sv.wait(sv.submit(p, q, tol=1e-10)) for q in srcs]
    hits, misses, idle = sv.cache_stats()
    assert (hits, misses) == (3, 1) and idle > 0
    # one right-hand side fits the cached handle of two; three do not
    one = workloads.checkerboard(m=16, levels=2, g=0.8, ratio=0.95, blocks=2, nrhs=1)
    three = workloads.checkerboard(m=16, levels=2, g=0.8, ratio=0.95, blocks=2, nrhs=3)
    u1, _ = sv.wait(sv.submit(one, one.q_nodal, tol=1e-10))
    u3, _ = sv.wait(sv.submit(three, three.q_nodal, tol=1e-10))
    assert sv.cache_stats()[:2] == (4, 2)
    sv.close()
    for q, (u, info) in zip(srcs, got):
        ua = _alone(p, q, **opts)
        assert np.linalg.norm(u - ua) / np.linalg.norm(ua) < 1e-8
    for pp, u in ((one, u1), (three, u3)):
        ua = _alone(pp, pp.q_nodal, **opts)
        assert np.linalg.norm(u - ua) / np.linalg.norm(ua) < 1e-8


def test_operator_cache_evicts_to_stay_within_the_budget():
    # a budget that holds one handle: each new operator evicts the idle one
    import paper_2102_09038_gb300 as rte
    opts = dict(n_plus=2, n_minus=3)
    a = workloads.constant(12, 2, 0.6, 2.0, 1.5)
    b = workloads.constant(12, 2, 0.7, 2.0, 1.5)
    budget = int(1.5 * rte.estimate_bytes(a, nrhs=1, **opts))
    sv = rte.Server(hbm_budget_bytes=budget, slots=1, **opts)
    res = [sv.wait(sv.submit(p, p.q_nodal, tol=1e-10))[0] for p in (a, b, a)]
    hits, misses, idle = sv.cache_stats()
    assert (hits, misses) == (0, 3) and 0 < idle <= budget
    sv.close()
    for p, u in zip((a, b, a), res):
        ua = _alone(p, p.q_nodal, **opts)
        assert np.linalg.norm(u - ua) / np.linalg.norm(ua) < 1e-8
