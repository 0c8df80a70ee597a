"""Meshes and quadrature for the oracle (test infrastructure only).

The oracle is the plain, slow FP64 CPU statement of the discretisation in the
paper's Section 4 and the iteration of Section 5.  Only ``tests/``, the smoke
entry point and the CPU-baseline leg of the benchmark may import it; the CUDA
product path never does.

Conventions (fixed readings of what the paper leaves open, shared with the
product only as a written specification, never as code):

* Spatial mesh (Section 4: quasi-uniform triangulation of R): the unit square
  split into m x m squares, each cut along the "/" diagonal.  Node (ix, iy)
  has index iy*(m+1)+ix.  Square (I, J) has index q = J*m+I and owns cells 2q
  (lower: (I,J),(I+1,J),(I+1,J+1)) and 2q+1 (upper: (I,J),(I+1,J+1),(I,J+1)).
* Sphere mesh (Section 6: octahedron, uniform refinement, new points projected
  to the sphere; Section 4: -K in the mesh for every K): only the four upper
  octahedron faces are refined, and they give the representatives K_k of the
  antipodal pairs K_k u (-K_k).  A face (a, b, c) splits into
  (a, ab, ca), (ab, b, bc), (ca, bc, c), (ab, bc, ca) with normalised edge
  midpoints; children of triangle t sit at 4t..4t+3.
"""
import numpy as np

UPPER_FACES = np.array([
    [[1, 0, 0], [0, 1, 0], [0, 0, 1]],
    [[0, 1, 0], [-1, 0, 0], [0, 0, 1]],
    [[-1, 0, 0], [0, -1, 0], [0, 0, 1]],
    [[0, -1, 0], [1, 0, 0], [0, 0, 1]],
], dtype=np.float64)


def square_mesh(m):
    """Uniform "/"-triangulation of (0,1)^2 (Section 4, T_h^R).

    Returns (nodes (n_R^+, 2), cells (n_R^-, 3) int array of node indices,
    listed counter-clockwise).
    """
    xs = np.arange(m + 1) / m
    X, Y = np.meshgrid(xs, xs)  # Y varies along axis 0
    nodes = np.stack([X.ravel(), Y.ravel()], axis=1)
    cells = np.zeros((2 * m * m, 3), dtype=np.int64)
    for J in range(m):
        for I in range(m):
            q = J * m + I
            n00 = J * (m + 1) + I
            n10 = n00 + 1
            n01 = n00 + (m + 1)
            n11 = n01 + 1
            cells[2 * q] = (n00, n10, n11)
            cells[2 * q + 1] = (n00, n11, n01)
    return nodes, cells


def _normalise(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


def refine_spherical(tris):
    """One uniform refinement of spherical triangles (t, 3 vertices, 3)."""
    a, b, c = tris[:, 0], tris[:, 1], tris[:, 2]
    ab = _normalise(a + b)
    bc = _normalise(b + c)
    ca = _normalise(c + a)
    kids = np.stack([
        np.stack([a, ab, ca], 1),
        np.stack([ab, b, bc], 1),
        np.stack([ca, bc, c], 1),
        np.stack([ab, bc, ca], 1),
    ], axis=1)  # (t, 4, 3, 3)
    return kids.reshape(-1, 3, 3)


def sphere_reps(levels):
    """Representative triangles K_k (n_S^+ = 4*4^levels) of the antipodal
    pairs, each a (3 vertices, 3) array of unit vectors."""
    tris = UPPER_FACES.copy()
    for _ in range(levels):
        tris = refine_spherical(tris)
    return tris


def spherical_area(tris):
    """Exact area of spherical triangles (Van Oosterom and Strackee's
    solid-angle formula)."""
    a, b, c = tris[..., 0, :], tris[..., 1, :], tris[..., 2, :]
    num = np.abs(np.einsum('...i,...i->...', a, np.cross(b, c)))
    den = (1.0 + np.einsum('...i,...i->...', a, b)
           + np.einsum('...i,...i->...', b, c)
           + np.einsum('...i,...i->...', c, a))
    return 2.0 * np.arctan2(num, den)


def quad_rule(tris, r):
    """Quadrature on spherical triangles: refine each triangle r more times;
    one node per sub-triangle at its normalised vertex mean, weighted by the
    sub-triangle's exact spherical area.  The weights of one triangle add up
    to its exact area.

    Returns (points (t, 4^r, 3), weights (t, 4^r)).
    """
    t = tris.shape[0]
    sub = tris
    for _ in range(r):
        sub = refine_spherical(sub)
    sub = sub.reshape(t, 4 ** r, 3, 3)
    pts = _normalise(sub.sum(axis=2))
    w = spherical_area(sub)
    return pts, w
