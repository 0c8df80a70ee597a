"""Pins of the oracle's inflow functional (Section 2.4: the boundary part
2 (|s.n| g, w^+)_{dD_-} of l^+) against exact solutions of the transport
equation (Section 1, eq. rte1-rte2) that the discretisation reproduces.

With no scattering (sigma_s = 0) and constant sigma_t:

* u(s, r) = a.s (constant in space, linear and odd in s) solves
  s.grad u + sigma_t u = q for q = sigma_t a.s, with inflow data g = a.s.
  Its even part is 0 and a.s lies in the odd space, so the even-parity
  right-hand side l^+ + A^T (M^-)^{-1} l^- must vanish: the inflow term
  cancels A^T applied to the odd solution.  A wrong half of the sphere
  (s.n > 0 instead of < 0), a wrong normal or a lost factor 2 breaks it.
* u(s, r) = b.r + f(s) with f even and constant on every pair K u -K solves
  it for q = s.b + sigma_t (b.r + f), g = b.r + f.  b.r is P1 in space and
  f lies in the even space, so the discrete even solution is u^+ = b.r + f
  exactly.  A face's nodes in the wrong order, a wrong face mass or a wrong
  angular weight breaks it.
"""
import numpy as np

import oracle
import workloads


def tri_of(an, s):
    """(pair k, half) of each direction s (P x 3): half 0 for K_k, 1 for
    -K_k; the quadrature points lie strictly inside their triangles."""
    c = np.einsum('kij,pj->pki', an['Vinv'], s)
    plus = np.all(c > 0.0, axis=2)
    minus = np.all(c < 0.0, axis=2)
    k = np.where(plus.any(axis=1), plus.argmax(axis=1), minus.argmax(axis=1))
    assert np.all(plus.any(axis=1) ^ minus.any(axis=1))
    return k, minus.any(axis=1).astype(int)


def odd_coefficients(disc, a):
    """Coefficients of s -> a.s in the odd basis: its L2 projection (the
    oracle's quadrature) solved with M_S^-; a.s lies in the odd space."""
    an = disc.an
    pts, w = an['qpts'], an['qw']
    psi = np.einsum('kij,kpj->kpi', an['Vinv'], pts)
    rhs = 2.0 * np.einsum('kp,kp,kpi->ki', w, pts @ a, psi)
    return np.linalg.solve(an['MSm'], rhs[:, :, None])[:, :, 0].ravel()


def test_odd_linear_inflow_cancels_transport_of_the_odd_solution():
    p = workloads.constant(5, 1, 0.6, 2.0, 0.0)
    disc = oracle.Discretisation(p.m, p.levels, p.sigma_t, p.sigma_s, p.g)
    ops = oracle.Operators(disc, n_plus=2, n_minus=3)
    a = np.array([0.7, -1.3, 0.4])
    ca = odd_coefficients(disc, a)
    # nodal reading of the same coefficients: a.v_i at the vertices of K_k
    assert np.allclose(ca, (disc.an['reps'] @ a).ravel(), atol=1e-13)
    inflow = disc.inflow(lambda f, j, s: s @ a)
    # (M^-)^{-1} l^- = the odd solution's coefficients on every cell
    Z = np.tile(ca, (disc.nRm, 1))
    ell = inflow + ops.apply_AT(Z)
    assert np.abs(inflow).max() > 1e-2
    assert np.abs(ell).max() <= 1e-13 * np.abs(inflow).max()


def test_linear_in_space_plus_even_angular_inflow_is_reproduced():
    p = workloads.constant(4, 1, 0.3, 1.7, 0.0)
    disc = oracle.Discretisation(p.m, p.levels, p.sigma_t, p.sigma_s, p.g)
    ops = oracle.Operators(disc, n_plus=2, n_minus=3)
    st = 1.7
    rng = np.random.default_rng(4)
    f = rng.uniform(0.5, 2.0, disc.nSp)        # even: one value per pair
    b = np.array([0.8, -0.5])
    xy = disc.sp['nodes']
    br = xy @ b

    def g(face, j, s):
        k, _ = tri_of(disc.an, s)
        return br[disc.face_nodes(face)[j]] + f[k]

    # even source sigma_t (b.r + f): P1 in space, so its interpolant is exact
    ell = st * disc.source(br) + st * np.outer(disc.sp['M_plus_unit'] @ np.ones(disc.nRp),
                                               disc.an['m'] * f)
    ell = ell + disc.inflow(g)
    # odd source s.b: (M^-)^{-1} l^- = coefficients of s.b / sigma_t per cell
    cb = odd_coefficients(disc, np.array([b[0], b[1], 0.0])) / st
    ell = ell + ops.apply_AT(np.tile(cb, (disc.nRm, 1)))
    # no scattering: c = 0, so E_0 = E and its direct solve is E^{-1}
    u = ops.solve_E0(ell)
    exact = br[:, None] + f[None, :]
    assert np.abs(u - exact).max() <= 1e-12 * np.abs(exact).max()


def test_inflow_depends_only_on_incoming_directions():
    # data on the outgoing half of every face never enters: changing it
    # leaves the functional unchanged, changing the incoming half does not
    p = workloads.constant(3, 1, 0.5, 1.0, 0.5)
    disc = oracle.Discretisation(p.m, p.levels, p.sigma_t, p.sigma_s, p.g)
    rng = np.random.default_rng(9)
    vals = rng.standard_normal((4, p.m + 1, disc.nSp, 2))
    normals = [(0, -1.0), (0, 1.0), (1, -1.0), (1, 1.0)]

    def make(v):
        def g(face, j, s):
            k, half = tri_of(disc.an, s)
            return v[face, j, k, half]
        return g

    base = disc.inflow(make(vals))
    cen = disc.an['reps'].mean(axis=1)
    out_half = vals.copy()
    for face, (axis, sgn) in enumerate(normals):
        # half 0 (K_k) leaves through the face when its centroid has s.n > 0
        leaving0 = sgn * cen[:, axis] > 0
        out_half[face, :, leaving0, 0] += 5.0
        out_half[face, :, ~leaving0, 1] += 5.0
    assert np.abs(disc.inflow(make(out_half)) - base).max() <= 1e-14 * np.abs(base).max()
    in_half = vals.copy()
    in_half[0, 1, 0, :] += 1.0
    assert np.abs(disc.inflow(make(in_half)) - base).max() > 1e-3
