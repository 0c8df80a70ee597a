"""Pins of the oracle's H^2 approximation of S^+ and S^- (Section 5.2).

The approximation is pinned to things other than itself:

* its exact parts against the dense assembly (an independent loop in
  assemble.angular_matrices);
* with no admissible block (eta = 0) it is the dense matrix;
* with a kernel that tensor interpolation of degree p - 1 reproduces (a cubic
  polynomial in the coordinates), the approximation is exact at every depth
  of the block tree: a wrong basis, node, coupling orientation, sign of the
  mirror part or a missing/doubled block fails here;
* the blocks of each part partition the matrix;
* the error for the Henyey-Greenstein kernel falls geometrically with p
  (the interpolation estimate behind the Lemma's asymptotic smoothness), and
  at the paper's parameters (eta = 1.4, p = 4) stays below 3e-4 in the
  Frobenius norm;
* Chebyshev-Lagrange interpolation is cardinal at its nodes.
"""
import numpy as np
import pytest

from oracle import assemble, h2


def cubic_kernel(x, y):
    """A kernel that p >= 4 tensor interpolation reproduces exactly (degree
    3 in each coordinate of x and of y), with an odd part (the cubic)."""
    t = x @ y.T
    return t ** 3 + 0.5 * t ** 2 - 0.25 * t + 0.125


def test_lagrange_cardinal_and_reproduces_cubics():
    rng = np.random.default_rng(1)
    lo, hi = np.array([-0.3, 0.1, 0.5]), np.array([0.2, 0.4, 0.9])
    nodes = h2.chebyshev_nodes(lo, hi, 4)
    pts = h2.tensor_points(nodes)
    L = h2.lagrange(nodes, pts)
    assert np.abs(L - np.eye(64)).max() < 1e-12
    x = lo + (hi - lo) * rng.random((50, 3))
    f = lambda z: z[:, 0] ** 3 * z[:, 1] - 2 * z[:, 2] ** 2 * z[:, 0] + z[:, 1] ** 3 * z[:, 2] ** 3
    assert np.abs(h2.lagrange(nodes, x) @ f(pts) - f(x)).max() < 1e-12


def test_exact_parts_match_dense_assembly():
    an = assemble.angular_matrices(2, 0.6)
    H = h2.H2Scattering(2, 0.6)
    for parity, key in ((1, 'Splus'), (-1, 'Sminus')):
        D = H.dense(parity)
        D = 0.5 * (D + D.T)
        assert np.abs(D - an[key]).max() <= 1e-14 * np.abs(an[key]).max()


@pytest.fixture(scope='module')
def hier():
    # levels 3 with leaves of 4: far blocks at depths 1 and 2
    return h2.H2Scattering(3, 0.5, nmin=4)


def test_blocks_partition_each_part(hier):
    n = hier.n
    for sign in (1.0, -1.0):
        cover = np.zeros((n, n), dtype=int)
        for depth, t, c, s in hier.far + hier.near:
            if s != sign:
                continue
            rt, rc = hier.tree.members(depth, t), hier.tree.members(depth, c)
            cover[rt[0]:rt[-1] + 1, rc[0]:rc[-1] + 1] += 1
        assert cover.min() == 1 and cover.max() == 1
    depths = {b[0] for b in hier.far}
    assert depths == {1, 2}
    assert any(b[3] < 0 for b in hier.far) and any(b[3] > 0 for b in hier.far)


def test_no_admissible_block_is_dense():
    H = h2.H2Scattering(2, 0.7, eta=0.0, nmin=4)
    assert not H.far
    for parity in (1, -1):
        D = H.dense(parity)
        assert np.abs(H.approximate(parity) - D).max() <= 1e-15 * np.abs(D).max()


def test_cubic_kernel_reproduced_at_every_depth():
    H = h2.H2Scattering(3, 0.0, nmin=4, kernel=cubic_kernel, near_rule=False)
    assert len(H.far) > 1000
    for parity in (1, -1):
        D = H.dense(parity)
        A = H.approximate(parity)
        assert np.abs(A - D).max() <= 1e-12 * np.abs(D).max(), parity


def test_hg_error_falls_with_p():
    H = h2.H2Scattering(3, 0.5, nmin=16)
    for parity in (1, -1):
        D = H.dense(parity)
        errs = []
        for p in (2, 3, 4, 5):
            H.p = p
            errs.append(np.linalg.norm(H.approximate(parity) - D) / np.linalg.norm(D))
        assert all(b < a / 3 for a, b in zip(errs, errs[1:])), errs
        assert errs[2] < 3e-4, errs
