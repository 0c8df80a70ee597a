"""Assembly of the discrete even/odd system (Section 4) for the oracle.

Test infrastructure only: the CUDA product path never imports this module.

Every matrix below is the definition in Section 4, eq. (bKebKo), (bMebMo),
(AR) and the entry formulas that follow them, written out plainly:

    K^+ = S^+ (x) M_s^+     K^- = S^- (x) M_s^-
    M^+ = M_S^+ (x) M_t^+   M^- = M_S^- (x) M_t^-
    A   = sum_n A_n (x) D_n R = blkdiag(R_k)

with the coefficient matrices U^+ (n_R^+ x n_S^+) and U^- (n_R^- x n_S^-)
stored row-major (spatial index slow, angular index fast), so that
(B (x) C) vec(U) = vec(C U B^T) (eq. tpmv) becomes C @ U @ B.T.

Readings of points the paper leaves open:

* Odd angular basis (Section 4: odd, piecewise linear): on the pair
  K_k u (-K_k) the three functions psi_{k,i}(s) = (V_k^{-1} s)_i, V_k the
  matrix whose columns are the vertices of K_k.  They are odd and nodal.
* Quadrature (Section 6 asks only for "higher-order" rules): the level-r rule
  of ``geometry.quad_rule``.  Single-triangle integrals (M_S^-, A_n, omega)
  use level R_NEAR; the double integrals of S^+/S^- over K_k x (+-K_k') use
  the tensor rule at level R_NEAR when K_k shares a vertex with K_k' or with
  -K_k' (self pairs included) and R_FAR otherwise; both signs of one pair use
  the same level.  S^+/S^- are symmetrised, (S + S^T)/2, afterwards.
* Boundary weight (Section 4 writes omega_k without the normal): on the square
  R = diag(omega^x) (x) B_x + diag(omega^y) (x) B_y with
  omega^x_k = int_S |s_x| mu_k^2 ds and B_x the P1 boundary mass on the faces
  x = 0 and x = 1 (B_y likewise).
* Two space dimensions, directions on S^2: A uses s_1 and s_2 only.
"""
import numpy as np
import scipy.sparse as sp

from . import geometry as geo

R_FAR = 2
R_NEAR = 4


def hg_kernel(mu, g):
    """Henyey-Greenstein phase function, eq. (HG-kernel1)."""
    return (1.0 - g * g) / (4.0 * np.pi) / (1.0 + g * g - 2.0 * g * mu) ** 1.5


# ----------------------------------------------------------------- spatial
def spatial_matrices(m, sigma_t, sigma_s):
    """Spatial FEM matrices of Section 4 on the m x m square mesh.

    sigma_t, sigma_s: per-cell values (length n_R^- = 2 m^2), piecewise
    constant.  Returns a dict with sparse CSR matrices
    Mt_plus, Ms_plus, M_plus_unit (P1 mass, weights sigma_t, sigma_s, 1),
    D1, D2 (n_R^- x n_R^+), Bx, By (boundary mass), and dense vectors
    Mt_minus, Ms_minus (diagonals of the P0 masses), area (cell areas).
    """
    nodes, cells = geo.square_mesh(m)
    nRp, nRm = nodes.shape[0], cells.shape[0]
    sigma_t = np.asarray(sigma_t, dtype=np.float64)
    sigma_s = np.asarray(sigma_s, dtype=np.float64)
    P = nodes[cells]  # (nRm, 3, 2)
    e1 = P[:, 1] - P[:, 0]
    e2 = P[:, 2] - P[:, 0]
    area = 0.5 * (e1[:, 0] * e2[:, 1] - e1[:, 1] * e2[:, 0])
    # gradient of the P1 hat function of local vertex a: perpendicular to the
    # opposite edge, length 1/height
    grad = np.zeros((nRm, 3, 2))
    for a in range(3):
        p1 = P[:, (a + 1) % 3]
        p2 = P[:, (a + 2) % 3]
        grad[:, a, 0] = (p1[:, 1] - p2[:, 1]) / (2 * area)
        grad[:, a, 1] = (p2[:, 0] - p1[:, 0]) / (2 * area)
    rows = np.repeat(np.arange(nRm), 3)
    cols = cells.ravel()
    D1 = sp.csr_matrix(((area[:, None] * grad[:, :, 0]).ravel(), (rows, cols)),
                       shape=(nRm, nRp))
    D2 = sp.csr_matrix(((area[:, None] * grad[:, :, 1]).ravel(), (rows, cols)),
                       shape=(nRm, nRp))
    loc = (np.ones((3, 3)) + np.eye(3)) / 12.0
    ii = np.repeat(cells, 3, axis=1).ravel()
    jj = np.tile(cells, (1, 3)).ravel()

    def p1_mass(weight):
        vals = (weight * area)[:, None, None] * loc[None]
        return sp.csr_matrix((vals.ravel(), (ii, jj)), shape=(nRp, nRp))

    h = 1.0 / m
    loc1 = np.array([[2.0, 1.0], [1.0, 2.0]]) * h / 6.0

    def face_mass(face_nodes_list):
        r, c, v = [], [], []
        for fn in face_nodes_list:
            for e in range(len(fn) - 1):
                pair = (fn[e], fn[e + 1])
                for a in range(2):
                    for b in range(2):
                        r.append(pair[a]); c.append(pair[b]); v.append(loc1[a, b])
        return sp.csr_matrix((v, (r, c)), shape=(nRp, nRp))

    idx = np.arange(nRp).reshape(m + 1, m + 1)  # [iy, ix]
    Bx = face_mass([idx[:, 0], idx[:, m]])
    By = face_mass([idx[0, :], idx[m, :]])
    return dict(
        nodes=nodes, cells=cells, area=area, grad=grad,
        Mt_plus=p1_mass(sigma_t), Ms_plus=p1_mass(sigma_s),
        M_plus_unit=p1_mass(np.ones(nRm)),
        Mt_minus=sigma_t * area, Ms_minus=sigma_s * area,
        D1=D1, D2=D2, Bx=Bx, By=By,
    )


# ----------------------------------------------------------------- angular
def _vertex_neighbours(reps, others):
    """For each triangle of ``reps``, the sorted indices of the triangles of
    ``others`` that share at least one vertex with it."""
    def key(v):
        return tuple(np.round(v * 1e9).astype(np.int64))
    owners = {}
    for j, tri in enumerate(others):
        for v in tri:
            owners.setdefault(key(v), set()).add(j)
    out = []
    for tri in reps:
        s = set()
        for v in tri:
            s |= owners.get(key(v), set())
        out.append(sorted(s))
    return out


def angular_matrices(levels, g, r_far=R_FAR, r_near=R_NEAR):
    """Angular FEM matrices of Section 4 for the sphere of 8*4^levels
    triangles.

    Returns a dict with m (diagonal of M_S^+, 2|K_k|), MSm (n_S^+, 3, 3)
    blocks of M_S^-, A1, A2 (n_S^+, 3): the nonzero 3x1 block column of A_n
    for direction pair k, omx, omy (boundary weights), Splus (n_S^+ square),
    Sminus (n_S^- square, index 3k+i), reps, Vinv.
    """
    reps = geo.sphere_reps(levels)
    n = reps.shape[0]
    V = reps.transpose(0, 2, 1)           # columns are vertices
    Vinv = np.linalg.inv(V)
    pn, wn = geo.quad_rule(reps, r_near)
    pf, wf = geo.quad_rule(reps, r_far)
    psin = np.einsum('kij,kpj->kpi', Vinv, pn)
    psif = np.einsum('kij,kpj->kpi', Vinv, pf)

    m = 2.0 * geo.spherical_area(reps)
    MSm = 2.0 * np.einsum('kp,kpi,kpj->kij', wn, psin, psin)
    A1 = 2.0 * np.einsum('kp,kp,kpi->ki', wn, pn[:, :, 0], psin)
    A2 = 2.0 * np.einsum('kp,kp,kpi->ki', wn, pn[:, :, 1], psin)
    omx = 2.0 * np.einsum('kp,kp->k', wn, np.abs(pn[:, :, 0]))
    omy = 2.0 * np.einsum('kp,kp->k', wn, np.abs(pn[:, :, 1]))

    # S^+_{kk'} = 2 sum_{p,p'} w w [k(p.p') + k(-p.p')]
    # S^-_{(k,i),(k',j)} = 2 sum_{p,p'} w w psi_i(p) psi_j(p') [k(p.p') - k(-p.p')]
    # the first term integrates K_k x K_k', the second K_k x (-K_k').
    near = [sorted(set(a) | set(b)) for a, b in
            zip(_vertex_neighbours(reps, reps), _vertex_neighbours(reps, -reps))]
    Sp = np.zeros((n, n))
    Sm = np.zeros((n, 3, n, 3))
    qf = pf.shape[1]
    pf_flat = pf.reshape(-1, 3)
    wf_flat = wf.reshape(-1)
    for k in range(n):
        mu = pf[k] @ pf_flat.T                       # (qf, n*qf)
        for sign in (1.0, -1.0):
            ker = hg_kernel(sign * mu, g) * wf_flat[None, :]
            row = (wf[k] @ ker).reshape(n, qf).sum(axis=1)
            Sp[k] += 2.0 * row
            t = np.einsum('p,pi,pq->iq', wf[k], psif[k], ker).reshape(3, n, qf)
            Sm[k] += 2.0 * sign * np.einsum('ikq,kqj->ikj', t, psif)
        # near pairs (K_k' or -K_k' shares a vertex with K_k): both terms by
        # the finer rule
        for kk in near[k]:
            mu_f = pf[k] @ pf[kk].T
            mu_n = pn[k] @ pn[kk].T
            for sign in (1.0, -1.0):
                ker_f = hg_kernel(sign * mu_f, g) * np.outer(wf[k], wf[kk])
                ker_n = hg_kernel(sign * mu_n, g) * np.outer(wn[k], wn[kk])
                Sp[k, kk] += 2.0 * (ker_n.sum() - ker_f.sum())
                Sm[k, :, kk, :] += 2.0 * sign * (
                    psin[k].T @ ker_n @ psin[kk] - psif[k].T @ ker_f @ psif[kk])
    Sm = Sm.reshape(3 * n, 3 * n)
    Sp = 0.5 * (Sp + Sp.T)
    Sm = 0.5 * (Sm + Sm.T)
    return dict(reps=reps, Vinv=Vinv, m=m, MSm=MSm, A1=A1, A2=A2,
                omx=omx, omy=omy, Splus=Sp, Sminus=Sm, qpts=pn, qw=wn)


# Faces of the unit square in the order the inflow data uses: (axis of the
# normal, coordinate of the face, sign of the outward normal along the axis):
# x = 0, x = 1, y = 0, y = 1.
FACES = ((0, 0.0, -1.0), (0, 1.0, 1.0), (1, 0.0, -1.0), (1, 1.0, 1.0))


def block_diag3(blocks):
    """Dense n_S^- x n_S^- matrix from (n, 3, 3) diagonal blocks."""
    n = blocks.shape[0]
    out = np.zeros((3 * n, 3 * n))
    for k in range(n):
        out[3 * k:3 * k + 3, 3 * k:3 * k + 3] = blocks[k]
    return out


def A_dense(col):
    """Dense n_S^- x n_S^+ matrix A_n from its 3x1 block columns (n, 3)."""
    n = col.shape[0]
    out = np.zeros((3 * n, n))
    for k in range(n):
        out[3 * k:3 * k + 3, k] = col[k]
    return out


class Discretisation:
    """All matrices of Section 4 for one problem (mesh m, sphere levels,
    sigma fields, HG parameter g)."""

    def __init__(self, m, levels, sigma_t, sigma_s, g,
                 r_far=R_FAR, r_near=R_NEAR):
        self.m, self.levels, self.g = m, levels, float(g)
        self.sp = spatial_matrices(m, sigma_t, sigma_s)
        self.an = angular_matrices(levels, g, r_far, r_near)
        self.sigma_t = np.asarray(sigma_t, dtype=np.float64)
        self.sigma_s = np.asarray(sigma_s, dtype=np.float64)
        self.nRp = self.sp['nodes'].shape[0]
        self.nRm = self.sp['cells'].shape[0]
        self.nSp = self.an['m'].shape[0]
        self.nSm = 3 * self.nSp
        self.A1 = A_dense(self.an['A1'])
        self.A2 = A_dense(self.an['A2'])
        self.MSm = block_diag3(self.an['MSm'])
        # c = ||sigma_s / sigma_t||_inf (Section 2.2)
        self.c = float(np.max(self.sigma_s / self.sigma_t))

    def face_nodes(self, f):
        """Node indices along boundary face f (order of FACES), in increasing
        coordinate along the face."""
        m = self.m
        idx = np.arange(self.nRp).reshape(m + 1, m + 1)   # [iy, ix]
        axis, coord, _ = FACES[f]
        c = 0 if coord == 0.0 else m
        return idx[:, c] if axis == 0 else idx[c, :]

    def inflow(self, g):
        """The inflow part of l^+ (Section 2.4, l^+(w^+) = (q, w^+) +
        2 (|s.n| g, w^+)_{dD_-}) for the test functions w^+ = phi_i mu_k:
        2 sum_faces int_face phi_i int_{K_k u -K_k, s.n < 0} |s.n| g ds dr,
        where dD_- = {(s, r): r on the boundary, s.n(r) < 0}.

        g(f, j, s): the inflow on face f at the face's node j (the data is P1
        along each face, so the space integral is the face's P1 mass) for the
        directions s (P x 3); returns P values.  The sphere integral runs over
        the quadrature points of both triangles of every pair (those of -K_k
        are the mirrored points of K_k) and keeps the points with s.n < 0."""
        m = self.m
        h = 1.0 / m
        pts, w = self.an['qpts'], self.an['qw']
        B = np.zeros((m + 1, m + 1))
        for e in range(m):
            B[e:e + 2, e:e + 2] += h / 6.0 * np.array([[2.0, 1.0], [1.0, 2.0]])
        out = np.zeros((self.nRp, self.nSp))
        for f, (axis, _, nsign) in enumerate(FACES):
            G = np.zeros((m + 1, self.nSp))
            for sgn in (1.0, -1.0):
                P = sgn * pts
                sn = nsign * P[:, :, axis]
                keep = sn < 0.0
                for j in range(m + 1):
                    vals = np.asarray(g(f, j, P.reshape(-1, 3))).reshape(P.shape[:2])
                    G[j] += np.sum(w * np.abs(sn) * keep * vals, axis=1)
            out[self.face_nodes(f)] += 2.0 * B @ G
        return out

    def source(self, q_nodal):
        """l^+ for an isotropic source given by nodal values and vacuum
        inflow: (q, phi_i mu_k) with q replaced by its P1 interpolant,
        = (M q)_i * m_k; l^- = (q, psi^-) = 0 because psi^- is odd."""
        Mq = self.sp['M_plus_unit'] @ np.asarray(q_nodal, dtype=np.float64)
        return np.outer(Mq, self.an['m'])
