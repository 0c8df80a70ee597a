"""The inflow term of l^+ (Section 2.4) through the C ABI (rte_inflow).

* Element by element against the oracle's inflow functional, which
  integrates 2 |s.n| g over the incoming half of the sphere by its own
  quadrature, on random data whose outgoing halves are also random (they
  must not enter).
* A pure absorber with isotropic inflow c and source sigma_t c: the exact
  intensity is the constant c, and so is the discrete even solution.
* Solves with scattering and inflow reach the requested residual in the
  oracle's exact operator, with l^+ = source + inflow from the oracle.
"""
import numpy as np
import pytest

import oracle
import workloads
from test_oracle_inflow import tri_of

pytestmark = pytest.mark.gpu
torch = pytest.importorskip('torch')


def oracle_inflow(disc, data):
    """The oracle's functional for library-layout data [4][m+1][2 n_S^+]."""
    def g(face, j, s):
        k, half = tri_of(disc.an, s)
        return data[face, j, 2 * k + half]
    return disc.inflow(g)


@pytest.mark.parametrize('case', ['tiny', 'ragged'])
def test_inflow_term_matches_oracle(case):
    import paper_2102_09038_gb300 as rte
    p = (workloads.constant(5, 1, 0.5, 1.0, 0.9, nrhs=2) if case == 'tiny' else
         workloads.checkerboard(m=9, levels=2, g=0.7, ratio=0.95, blocks=3, nrhs=2))
    disc = oracle.Discretisation(p.m, p.levels, p.sigma_t, p.sigma_s, p.g)
    s = rte.Solver(p, n_plus=2, n_minus=3, max_rhs=2)
    data = np.random.default_rng(21).standard_normal((2, 4, p.m + 1, 2 * disc.nSp))
    q = s.rhs(torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda'))
    s.inflow(torch.tensor(data, dtype=torch.float64, device='cuda'), q)
    got = q.cpu().numpy()
    s.close()
    for r in range(2):
        ref = disc.source(p.q_nodal[r]) + oracle_inflow(disc, data[r])
        assert np.abs(got[r] - ref).max() <= 1e-13 * np.abs(ref).max()


def test_pure_absorber_with_constant_inflow_is_constant():
    import paper_2102_09038_gb300 as rte
    st, c = 2.5, 0.75
    p = workloads.constant(12, 2, 0.8, st, 0.0, q=st * c)
    s = rte.Solver(p, n_plus=2, n_minus=3)
    q = s.rhs(torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda'))
    g = torch.full((1, 4, p.m + 1, 2 * s.n_dirs), c, dtype=torch.float64, device='cuda')
    s.inflow(g, q)
    u, info = s.solve(q, tol=1e-13)
    s.close()
    assert info['status'] == 0, info
    assert np.abs(u.cpu().numpy() - c).max() <= 1e-11


@pytest.mark.parametrize('prec', [0, 2])
def test_solve_with_inflow_reaches_oracle_residual(prec):
    import paper_2102_09038_gb300 as rte
    p = workloads.checkerboard(m=9, levels=2, g=0.7, ratio=0.95, blocks=3, nrhs=2)
    disc = oracle.Discretisation(p.m, p.levels, p.sigma_t, p.sigma_s, p.g)
    ops = oracle.Operators(disc, n_plus=2, n_minus=3)
    rng = np.random.default_rng(5)
    data = rng.uniform(0.0, 2.0, (2, 4, p.m + 1, 2 * disc.nSp))
    s = rte.Solver(p, n_plus=2, n_minus=3, precision=prec, max_rhs=2)
    q = s.rhs(torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda'))
    s.inflow(torch.tensor(data, dtype=torch.float64, device='cuda'), q)
    u, info = s.solve(q, tol=1e-11)
    s.close()
    assert info['status'] == 0, info
    u = u.cpu().numpy()
    for r in range(2):
        ell = disc.source(p.q_nodal[r]) + oracle_inflow(disc, data[r])
        res = np.linalg.norm(ops.apply_EK(u[r]) - ell) / np.linalg.norm(ell)
        assert res <= 1e-10, res
