"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds only problem *inputs* (mesh size, sphere level, per-cell
sigma_t / sigma_s fields, the HG parameter g and nodal source values).  It
contains none of the method's arithmetic, so both the CUDA path and the
oracle may use it.

The paper's own workload (the lattice problem of Section 6) cannot be rebuilt:
its geometry is given only in a figure.  These synthetic problems stand in for
it, with the structure the paper's experiments have: piecewise-constant
coefficients on a uniform mesh, strongly scattering media (c close to 1) and
forward-peaked Henyey-Greenstein scattering.
"""
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Problem:
    name: str
    m: int                 # m x m squares, 2 m^2 cells, (m+1)^2 nodes
    levels: int            # sphere with 8 * 4**levels triangles
    g: float
    sigma_t: np.ndarray    # per cell, length 2 m^2
    sigma_s: np.ndarray
    q_nodal: np.ndarray    # (nrhs, (m+1)^2) nodal source values
    tol: float = 1e-6
    meta: dict = field(default_factory=dict)

    @property
    def n_nodes(self):
        return (self.m + 1) ** 2

    @property
    def n_cells(self):
        return 2 * self.m * self.m

    @property
    def n_dirs(self):
        return 4 * 4 ** self.levels

    @property
    def nrhs(self):
        return self.q_nodal.shape[0]

    @property
    def dofs(self):
        return self.n_nodes * self.n_dirs


def node_xy(m):
    xs = np.arange(m + 1) / m
    X, Y = np.meshgrid(xs, xs)
    return X.ravel(), Y.ravel()


def cell_square(m):
    """(I, J) square indices of each cell (two cells per square)."""
    q = np.arange(2 * m * m) // 2
    return q % m, q // m


def gaussian_source(m, centre, width):
    x, y = node_xy(m)
    return np.exp(-((x - centre[0]) ** 2 + (y - centre[1]) ** 2)
                  / (2.0 * width ** 2))


def constant(m, levels, g, sigma_t, sigma_s, q=1.0, nrhs=1, name='const',
             tol=1e-6):
    nc = 2 * m * m
    return Problem(name, m, levels, g, np.full(nc, float(sigma_t)),
                   np.full(nc, float(sigma_s)),
                   np.full((nrhs, (m + 1) ** 2), float(q)), tol)


def plain_fp64(m=32, levels=2):
    """Unit square, 32x32 mesh, 128-triangle sphere, g = 0.5, sigma_t = 1,
    sigma_s = 0.5, q = 1, vacuum inflow, tolerance 1e-8."""
    return constant(m, levels, 0.5, 1.0, 0.5, 1.0, name='plain_32x32_T128',
                    tol=1e-8)


def checkerboard(m=128, levels=3, g=0.9, ratio=0.99, blocks=4, seed=0,
                 width=0.1, nrhs=1):
    """Unit square m x m, sphere 8*4^levels triangles, HG g, sigma_t in
    {1, 10} on a blocks x blocks checkerboard, sigma_s = ratio * sigma_t,
    Gaussian source (standard deviation ``width``) centred at a seeded point
    of [0.2, 0.8]^2, tolerance 1e-6."""
    I, J = cell_square(m)
    bs = m // blocks
    odd = ((I // bs) + (J // bs)) % 2
    st = np.where(odd == 0, 1.0, 10.0)
    rng = np.random.default_rng(seed)
    q = np.stack([gaussian_source(m, rng.uniform(0.2, 0.8, 2), width)
                  for _ in range(nrhs)])
    return Problem('checker_%dx%d_T%d_g%.2f' % (m, m, 8 * 4 ** levels, g),
                   m, levels, g, st, ratio * st, q, 1e-6,
                   meta=dict(seed=seed))


def precision_case(m=96, levels=4, g=0.8, ratio=0.999):
    """96x96 mesh, 2048-triangle sphere, g in {0.8, 0.95}, sigma_s/sigma_t =
    0.999 with sigma_t = 1, q = 1."""
    return constant(m, levels, g, 1.0, ratio, 1.0,
                    name='precision_%dx%d_T%d_g%.2f' % (m, m, 8 * 4 ** levels, g))


def batch_instances(count=64, seed=0, m_range=(32, 128), levels=(2, 3),
                    g_range=(0.3, 0.9), st_range=(0.1, 100.0),
                    ratio_range=(0.5, 0.999), nrhs_range=(1, 8)):
    """Uneven instances for batched solves: m ~ U{m_range}, sphere level in
    ``levels``, g ~ U[g_range], sigma_t log-uniform, sigma_s / sigma_t
    uniform, 1-8 Gaussian sources each (width 0.1, seeded centres)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        lv = int(rng.choice(levels))
        g = float(rng.uniform(*g_range))
        st = float(np.exp(rng.uniform(np.log(st_range[0]),
                                      np.log(st_range[1]))))
        ratio = float(rng.uniform(*ratio_range))
        nrhs = int(rng.integers(nrhs_range[0], nrhs_range[1] + 1))
        q = np.stack([gaussian_source(m, rng.uniform(0.2, 0.8, 2), 0.1)
                      for _ in range(nrhs)])
        nc = 2 * m * m
        out.append(Problem('inst%02d' % i, m, lv, g, np.full(nc, st),
                           np.full(nc, ratio * st), q, 1e-6))
    return out
