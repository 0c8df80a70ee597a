"""The seeded synthetic inputs match the recipe they stand for: the sizes,
coefficient fields, sources and tolerances of the benchmark configurations
(the paper's lattice geometry exists only as a figure, so these problems
take its structure: piecewise-constant coefficients on a uniform mesh,
strongly scattering media and forward-peaked scattering)."""
import numpy as np

import workloads


def test_plain_configuration():
    p = workloads.plain_fp64()
    assert (p.m, p.levels, p.g, p.tol) == (32, 2, 0.5, 1e-8)
    assert 8 * 4 ** p.levels == 128 and p.n_dirs == 64 and p.n_nodes == 33 * 33
    assert np.all(p.sigma_t == 1.0) and np.all(p.sigma_s == 0.5)
    assert p.q_nodal.shape == (1, 33 * 33) and np.all(p.q_nodal == 1.0)
    assert p.dofs == 69696


def test_checkerboard_benchmark_problem():
    p = workloads.checkerboard(m=128, levels=3, g=0.9, ratio=0.99, seed=0)
    assert (p.m, p.levels, p.g, p.tol) == (128, 3, 0.9, 1e-6)
    assert p.n_cells == 32768 and p.n_dirs == 256 and p.dofs == 4260096
    # sigma_t in {1, 10} on a 4 x 4 checkerboard of 32 x 32-square blocks,
    # both cells of a square alike, half the cells of each value
    I, J = workloads.cell_square(128)
    expect = np.where(((I // 32) + (J // 32)) % 2 == 0, 1.0, 10.0)
    assert np.array_equal(p.sigma_t, expect)
    assert np.array_equal(p.sigma_t[0::2], p.sigma_t[1::2])
    assert np.count_nonzero(p.sigma_t == 10.0) == p.n_cells // 2
    assert np.allclose(p.sigma_s, 0.99 * p.sigma_t, rtol=0, atol=1e-15)
    # one Gaussian source, standard deviation 0.1, centred in [0.2, 0.8]^2:
    # its nodal values peak next to the centre, and their spread is the
    # standard deviation (mildly cut by the square within two of them)
    q = p.q_nodal[0]
    assert q.shape == (129 * 129,) and np.all(q > 0) and q.max() <= 1.0
    x, y = workloads.node_xy(128)
    c = np.array([x[np.argmax(q)], y[np.argmax(q)]])
    assert np.all(c >= 0.2 - 1 / 128) and np.all(c <= 0.8 + 1 / 128)
    mean = np.array([np.sum(q * x), np.sum(q * y)]) / q.sum()
    var = np.array([np.sum(q * (x - mean[0]) ** 2), np.sum(q * (y - mean[1]) ** 2)]) / q.sum()
    assert np.all(np.abs(mean - c) <= 1 / 128 + 0.02)
    assert np.all(var > 0.8 * 0.01) and np.all(var < 1.02 * 0.01)
    # seeded: the same seed gives the same problem, another seed moves the source
    again = workloads.checkerboard(m=128, levels=3, g=0.9, ratio=0.99, seed=0)
    assert np.array_equal(again.q_nodal, p.q_nodal)
    other = workloads.checkerboard(m=128, levels=3, g=0.9, ratio=0.99, seed=1)
    assert not np.array_equal(other.q_nodal, p.q_nodal)


def test_precision_configuration():
    for g in (0.8, 0.95):
        p = workloads.precision_case(g=g)
        assert (p.m, p.levels, p.g) == (96, 4, g)
        assert 8 * 4 ** p.levels == 2048 and p.n_dirs == 1024 and p.dofs == 9634816
        assert np.all(p.sigma_t == 1.0) and np.allclose(p.sigma_s, 0.999)
        assert np.all(p.q_nodal == 1.0)


def test_batching_instances_cover_their_ranges():
    inst = workloads.batch_instances(64, seed=0)
    assert len(inst) == 64
    ms = np.array([p.m for p in inst])
    assert ms.min() >= 32 and ms.max() <= 128 and len(set(ms)) > 20
    assert {p.levels for p in inst} == {2, 3}     # 128 or 512 triangles
    for p in inst:
        assert 0.3 <= p.g <= 0.9
        st = p.sigma_t[0]
        assert 0.1 <= st <= 100.0 and np.all(p.sigma_t == st)
        ratio = p.sigma_s[0] / st
        assert 0.5 <= ratio <= 0.999 and np.allclose(p.sigma_s, ratio * st)
        assert 1 <= p.nrhs <= 8 and p.q_nodal.shape == (p.nrhs, (p.m + 1) ** 2)
        assert p.tol == 1e-6
    # sigma_t is log-uniform over four decades: values on both sides of 1
    sts = np.array([p.sigma_t[0] for p in inst])
    assert sts.min() < 1.0 < sts.max()
    again = workloads.batch_instances(64, seed=0)
    assert all(a.m == b.m and np.array_equal(a.q_nodal, b.q_nodal) for a, b in zip(inst, again))
