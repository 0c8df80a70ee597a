"""The continuous-batching server: requests of different mesh and sphere
sizes, coefficients and anisotropy run concurrently on separate streams;
every result must equal the same problem solved alone (to the solve
tolerance) and satisfy the oracle's residual; a budget smaller than one
request serialises the requests without losing any."""
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
