"""H^2-matrix approximation of the scattering matrices S^+ and S^- (Section
5.2) for the oracle.

Test infrastructure only: the CUDA product path never imports this module.

Section 5.2 applies S^+ and S^- through H^2-matrices obtained by polynomial
interpolation of the extension K(x~, y~) = k(x.y), x = x~/|x~|, y = y~/|y~|
(eq. HGextension) of the Henyey-Greenstein kernel, which the Lemma of that
section shows to be asymptotically smooth.  Its experiment (Section 6, the
table on compression) fixes the parameters: admissibility parameter
eta = 1.4, p = 4 interpolation points per coordinate, minimal block size
n_min = 64.  The construction itself is the textbook one; written out here
without any blocking or reordering:

1. cluster tree over the representatives K_k;
2. a bounding box per cluster;
3. the block tree: a pair of clusters is a far block when it is admissible,
   a near block when it is an inadmissible pair of leaves, and is split into
   all pairs of children otherwise;
4. far block (t, c): V_t K_tc V_c^T, with tensor Lagrange interpolation on
   the boxes, V_t[i, nu] = int_{K_i} phi_i L^t_nu ds and
   K_tc[nu, mu] = K(xi^t_nu, xi^c_mu);
5. near block: the exact entries, by the same quadrature as the dense
   assembly.

S^+ and S^- (see assemble.angular_matrices) are 2 (D + M) and 2 (D - M) in
the basis of the representatives, with D the integral of k(s.s') over
K_k x K_k' (the direct part) and M that of k(-s.s') (the mirror part,
K_k x (-K_k')).  Each part is a kernel matrix of its own: the direct part
uses K(x, y), the mirror part K(x, -y); each gets its own block tree.

Readings of what the paper leaves to the library (fixed here, and stated in
the design notes):

* Cluster tree: the refinement hierarchy of the representatives.  The four
  upper octahedron faces are the roots; the cluster (d, t) at depth d holds
  the 4^(levels-d) representatives t*4^(levels-d) ... (t+1)*4^(levels-d)-1
  (children of triangle t sit at 4t..4t+3).  Leaves: the shallowest depth
  whose clusters hold at most n_min representatives.
* Box: the axis-aligned bounding box of the far-rule quadrature points of
  the cluster's triangles (the points at which its basis is integrated).
  For the mirror part the column cluster's box is negated.
* Admissibility: max(diam B_t, diam B_c) <= eta dist(B_t, B_c), with diam
  the box diagonal and dist the Euclidean distance between the boxes.
* Interpolation: p Chebyshev points of the first kind per coordinate,
  c + h cos((2i + 1) pi / (2p)), i = 0..p-1, on each box (centre c,
  half-width h), tensor index nu = (i_x p + i_y) p + i_z.
* Quadrature: the far rule of the dense assembly (level R_FAR) for the
  interpolated integrals; near blocks take, per pair, the rule the dense
  assembly takes (R_NEAR when K_k' or -K_k' shares a vertex with K_k, else
  R_FAR), so that a near block equals the dense part exactly.
"""
import numpy as np

from . import geometry as geo
from .assemble import R_FAR, R_NEAR, _vertex_neighbours, hg_kernel

ETA, P, NMIN = 1.4, 4, 64


def hg_extension(g):
    """K(x~, y~) = k(x.y) with x, y the normalised arguments (eq.
    HGextension), for point sets x (a, 3) and y (b, 3): an (a, b) array.
    Every kernel of this module takes that pairwise form."""
    def K(x, y):
        xn = x / np.linalg.norm(x, axis=-1, keepdims=True)
        yn = y / np.linalg.norm(y, axis=-1, keepdims=True)
        return hg_kernel(xn @ yn.T, g)
    return K


class ClusterTree:
    """Clusters of the refinement hierarchy and their boxes."""

    def __init__(self, levels, pts, nmin=NMIN):
        self.levels = levels
        d = 0
        while 4 ** (levels - d) > nmin and d < levels:
            d += 1
        self.leaf_depth = d
        n = pts.shape[0]
        self.lo, self.hi = [], []
        for depth in range(d + 1):
            size = self.size(depth)
            P = pts.reshape(n // size, size * pts.shape[1], 3)
            self.lo.append(P.min(axis=1))
            self.hi.append(P.max(axis=1))

    def size(self, depth):
        return 4 ** (self.levels - depth)

    def count(self, depth):
        return 4 * 4 ** depth

    def members(self, depth, t):
        s = self.size(depth)
        return np.arange(t * s, (t + 1) * s)

    def box(self, depth, t, sign=1.0):
        lo, hi = self.lo[depth][t], self.hi[depth][t]
        return (lo, hi) if sign > 0 else (-hi, -lo)


def _diam(lo, hi):
    e = hi - lo
    return np.sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2])


def _dist(lo1, hi1, lo2, hi2):
    e = np.maximum(0.0, np.maximum(lo1 - hi2, lo2 - hi1))
    return np.sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2])


def admissible(tree, depth, t, c, sign, eta):
    lt, ht = tree.box(depth, t)
    lc, hc = tree.box(depth, c, sign)
    return max(_diam(lt, ht), _diam(lc, hc)) <= eta * _dist(lt, ht, lc, hc)


def block_tree(tree, eta):
    """Far and near blocks (depth, t, c, sign) of both parts; sign +1 is the
    direct part, -1 the mirror part."""
    far, near = [], []

    def visit(depth, t, c, sign):
        if admissible(tree, depth, t, c, sign, eta):
            far.append((depth, t, c, sign))
        elif depth == tree.leaf_depth:
            near.append((depth, t, c, sign))
        else:
            for a in range(4 * t, 4 * t + 4):
                for b in range(4 * c, 4 * c + 4):
                    visit(depth + 1, a, b, sign)

    for sign in (1.0, -1.0):
        for t in range(4):
            for c in range(4):
                visit(0, t, c, sign)
    return far, near


def chebyshev_nodes(lo, hi, p):
    """(p, 3) per-axis nodes on the box [lo, hi]."""
    i = np.arange(p)
    ref = np.cos((2 * i + 1) * np.pi / (2 * p))
    c, h = 0.5 * (lo + hi), 0.5 * (hi - lo)
    if np.any(h <= 0.0):
        raise ValueError('degenerate cluster box')
    return c[None, :] + h[None, :] * ref[:, None]


def tensor_points(nodes):
    """(p^3, 3) tensor points, index (i_x p + i_y) p + i_z."""
    p = nodes.shape[0]
    ix, iy, iz = np.meshgrid(np.arange(p), np.arange(p), np.arange(p), indexing='ij')
    return np.stack([nodes[ix.ravel(), 0], nodes[iy.ravel(), 1], nodes[iz.ravel(), 2]], axis=1)


def lagrange(nodes, x):
    """Tensor Lagrange basis of the per-axis nodes (p, 3) at points x
    (m, 3): (m, p^3)."""
    p = nodes.shape[0]
    per_axis = []
    for a in range(3):
        la = np.ones((x.shape[0], p))
        for i in range(p):
            for j in range(p):
                if j != i:
                    la[:, i] *= (x[:, a] - nodes[j, a]) / (nodes[i, a] - nodes[j, a])
        per_axis.append(la)
    return np.einsum('mi,mj,mk->mijk', *per_axis).reshape(x.shape[0], p ** 3)


class H2Scattering:
    """H^2 approximation of S^+ (parity +1) and S^- (parity -1) for the
    sphere of 8*4^levels triangles."""

    def __init__(self, levels, g, eta=ETA, p=P, nmin=NMIN, kernel=None, near_rule=True):
        """kernel: a pairwise kernel (default: the HG extension for g);
        near_rule=False integrates every pair by the far rule (for kernels
        whose interpolation is exact, so that the approximation must equal
        the dense matrix)."""
        self.levels, self.p, self.eta = levels, p, eta
        self.K = kernel if kernel is not None else hg_extension(g)
        self.use_near_rule = near_rule
        self._near_blocks, self._bases = {}, {}
        reps = geo.sphere_reps(levels)
        self.n = reps.shape[0]
        self.Vinv = np.linalg.inv(reps.transpose(0, 2, 1))
        self.pf, self.wf = geo.quad_rule(reps, R_FAR)
        self.pn, self.wn = geo.quad_rule(reps, R_NEAR)
        self.psif = np.einsum('kij,kpj->kpi', self.Vinv, self.pf)
        self.psin = np.einsum('kij,kpj->kpi', self.Vinv, self.pn)
        self.near_pairs = [set(a) | set(b) for a, b in
                           zip(_vertex_neighbours(reps, reps), _vertex_neighbours(reps, -reps))]
        self.tree = ClusterTree(levels, self.pf, nmin)
        self.far, self.near = block_tree(self.tree, eta)

    # ---------------------------------------------------------- pieces
    def nodes(self, depth, t):
        lo, hi = self.tree.box(depth, t)
        return chebyshev_nodes(lo, hi, self.p)

    def basis(self, depth, t, parity):
        """V_t: rows are the basis functions of the cluster's triangles (one
        per triangle for parity +1, three for -1), columns the p^3 Lagrange
        polynomials of its box."""
        key = (depth, t, parity, self.p)
        if key in self._bases:
            return self._bases[key]
        idx = self.tree.members(depth, t)
        nodes = self.nodes(depth, t)
        pts = self.pf[idx].reshape(-1, 3)
        L = lagrange(nodes, pts).reshape(len(idx), -1, self.p ** 3)    # (i, q, nu)
        if parity > 0:
            V = np.einsum('iq,iqn->in', self.wf[idx], L)
        else:
            V = np.einsum('iq,iqa,iqn->ian', self.wf[idx], self.psif[idx], L)
            V = V.reshape(3 * len(idx), -1)
        self._bases[key] = V
        return V

    def coupling(self, depth, t, c, sign):
        """K_tc[nu, mu] = K(xi^t_nu, sign xi^c_mu)."""
        xt = tensor_points(self.nodes(depth, t))
        xc = tensor_points(self.nodes(depth, c))
        return self.K(xt, sign * xc)

    def exact_part(self, rows, cols, sign, parity, chunk=32):
        """The dense part's entries for triangles rows x cols: the sum over
        the quadrature points of w w phi phi K(p, sign q), by the far rule
        for every pair, then by the near rule for the pairs the dense
        assembly integrates with it."""
        m = 1 if parity > 0 else 3
        qf = self.pf.shape[1]
        Q = self.pf[cols].reshape(-1, 3)
        wq = self.wf[cols].reshape(-1)
        out = np.zeros((len(rows), m, len(cols), m))
        for a0 in range(0, len(rows), chunk):
            r = rows[a0:a0 + chunk]
            ker = self.K(self.pf[r].reshape(-1, 3), sign * Q)
            ker *= np.outer(self.wf[r].reshape(-1), wq)
            ker = ker.reshape(len(r), qf, len(cols), qf)
            if parity > 0:
                out[a0:a0 + len(r), 0, :, 0] = ker.sum(axis=(1, 3))
            else:
                out[a0:a0 + len(r)] = np.einsum('iqa,iqjr,jrb->iajb', self.psif[r], ker,
                                                self.psif[cols])
        pos = {j: b for b, j in enumerate(cols)}
        for a, i in enumerate(rows if self.use_near_rule else []):
            for j in self.near_pairs[i]:
                b = pos.get(j)
                if b is None:
                    continue
                ker = self.K(self.pn[i], sign * self.pn[j]) * np.outer(self.wn[i], self.wn[j])
                if parity > 0:
                    out[a, 0, b, 0] = ker.sum()
                else:
                    out[a, :, b, :] = self.psin[i].T @ ker @ self.psin[j]
        return out.reshape(m * len(rows), m * len(cols))

    # ---------------------------------------------------------- matrices
    def approximate(self, parity):
        """The H^2 approximation of S^+ (parity +1) or S^- (parity -1) as a
        dense matrix: 2 (D^ + parity M^)."""
        m = 1 if parity > 0 else 3
        S = np.zeros((m * self.n, m * self.n))
        for depth, t, c, sign in self.far:
            rt = self.tree.members(depth, t)
            rc = self.tree.members(depth, c)
            blk = self.basis(depth, t, parity) @ self.coupling(depth, t, c, sign) @ \
                self.basis(depth, c, parity).T
            S[m * rt[0]:m * (rt[-1] + 1), m * rc[0]:m * (rc[-1] + 1)] += \
                2.0 * (sign if parity < 0 else 1.0) * blk
        for depth, t, c, sign in self.near:
            rt = self.tree.members(depth, t)
            rc = self.tree.members(depth, c)
            key = (parity, depth, t, c, sign)
            if key not in self._near_blocks:
                self._near_blocks[key] = self.exact_part(rt, rc, sign, parity)
            blk = self._near_blocks[key]
            S[m * rt[0]:m * (rt[-1] + 1), m * rc[0]:m * (rc[-1] + 1)] += \
                2.0 * (sign if parity < 0 else 1.0) * blk
        return S

    def dense(self, parity):
        """The exact 2 (D + parity M) by the dense assembly's rules (no
        compression; every pair by the far rule when near_rule is off)."""
        idx = np.arange(self.n)
        D = self.exact_part(idx, idx, 1.0, parity)
        M = self.exact_part(idx, idx, -1.0, parity)
        return 2.0 * (D + parity * M)
