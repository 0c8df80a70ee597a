"""Subspace correction and the preconditioned Richardson iteration
(Sections 5.4-5.5, Algorithm 3) for the oracle.

Test infrastructure only: the CUDA product path never imports this module.

Readings of the paper taken here:

* Correction right-hand side: q_c = W^T ((E - K^+) s - r) with
  r = (E - K^+) u_n - q, which is eq. (corr_discrete); the printed
  Algorithm 3 carries an extra "- q" under which the exact solution would not
  be a fixed point.
* P_1^l takes l steps (eq. applyP1, k < l), not the l+1 of the printed loop
  bound of Algorithm 2.
* E_c's transport block W^T A^T (M^- - K^-)^{-1} A W ("left to the reader" in
  Section 5.4) is formed exactly: per cell j it is
  sum_{n,m} D_n^T diag(H^{nm}(j)) D_m with
  H(j) = |T_j|^{-1} C^T (sigma_t,j M_S^- - sigma_s,j S^-)^{-1} C and
  C = [A_1 W_N, A_2 W_N].
* Stopping rule: ||r_n||_2 <= tol ||q||_2 (Euclidean norm of the coefficient
  vector).  The paper's energy-norm update size (eq. stop),
  ||u_n - u_{n-1}||_{E-K}^2 = (u_n - u_{n-1})^T (r_n - r_{n-1}), is recorded
  beside it.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def d_of(N):
    """Number of spherical harmonics of degree <= N of one parity,
    (N+1)(N+2)/2 (Section 5.1 and 5.4)."""
    return (N + 1) * (N + 2) // 2


class Coarse:
    """The Galerkin subspace W^+ = W_N^+ (x) I and its matrix
    E_c = W^T (E - K^+) W (Section 5.4)."""

    def __init__(self, ops, N=4, W=None):
        """W: optional basis of the angular subspace (n_S^+ x d_N); by
        default the eigenvectors of the d_N largest eigenvalues of
        (S^+, M_S^+) (Section 5.4)."""
        self.ops = ops
        self.N = N
        self.dN = d_of(N)
        lam, Wfull = ops.eig_plus()
        self.W = Wfull[:, :self.dN].copy() if W is None else np.array(W)
        self.lam = lam[:self.dN].copy()
        self.Ec = self.assemble()
        self._lu = None

    def assemble(self):
        ops, disc = self.ops, self.ops.d
        smat, an = disc.sp, disc.an
        W, dN = self.W, self.dN
        # W^T M^+ W = (W^T M_S^+ W) (x) M_t^+ and W^T K^+ W = (W^T S^+ W) (x)
        # M_s^+; for M_S^+-orthonormal eigenvectors these are I and Lambda_N
        # (Section 5.4), the general form serves any basis of the span.
        Ec = (sp.kron(smat['Mt_plus'], W.T @ (ops.m[:, None] * W))
              - sp.kron(smat['Ms_plus'], W.T @ ops.Sp @ W))
        # W^T R W: block (a,b) = sum_k R_k W(k,a) W(k,b)
        Ec = Ec + sp.kron(smat['Bx'], W.T @ (an['omx'][:, None] * W))
        Ec = Ec + sp.kron(smat['By'], W.T @ (an['omy'][:, None] * W))
        # transport block, per class of cells with equal (sigma_t, sigma_s)
        C = np.concatenate([ops.A1 @ W, ops.A2 @ W], axis=1)  # (nSm, 2 dN)
        Dn = [smat['D1'], smat['D2']]
        for c, (st, ss) in enumerate(ops.classes):
            rows = np.nonzero(ops.cell_class == c)[0]
            H = C.T @ sla.solve(st * ops.MSm - ss * ops.Sm, C, assume_a='pos')
            scale = sp.diags(1.0 / ops.area[rows])
            for a in range(2):
                for b in range(2):
                    Da = Dn[a][rows]
                    Db = Dn[b][rows]
                    spat = Da.T @ scale @ Db
                    Ec = Ec + sp.kron(spat, H[a * dN:(a + 1) * dN,
                                             b * dN:(b + 1) * dN])
        return Ec.tocsc()

    def restrict(self, T):
        """W^T t = vec(T W_N)."""
        return T @ self.W

    def prolong(self, Uc):
        """W u_c = vec(U_c W_N^T)."""
        return Uc @ self.W.T

    def solve(self, Qc):
        """E_c u_c = q_c by a sparse LU factorisation."""
        if self._lu is None:
            self._lu = spla.splu(self.Ec)
        x = self._lu.solve(Qc.ravel())
        return x.reshape(Qc.shape)


def richardson(ops, q, tol=1e-10, maxit=200, l=4, N=4, u0=None, coarse=None, p1='richardson'):
    """Algorithm 3 (eq. Richardson_discrete with the product preconditioner
    of eq. product_pre) with the readings in the module docstring.  p1 picks
    the realisation of P_1: 'richardson' (P_1^l, eq. applyP1) or 'pcg' (l
    PCG steps, the non-stationary choice of Section 5.3).

    Returns (u, info) where info holds the iteration count, the residual
    history ||r_n||/||q|| and the energy-norm update sizes."""
    if coarse is None and N >= 0:
        coarse = Coarse(ops, N)
    u = np.zeros_like(q) if u0 is None else u0.copy()
    nq = np.linalg.norm(q)
    hist, upd = [], []
    r_prev, u_prev = None, None
    it = 0
    for it in range(maxit + 1):
        r = ops.apply_EK(u) - q
        rel = np.linalg.norm(r) / nq
        hist.append(rel)
        if r_prev is not None:
            delta = u - u_prev
            upd.append(np.sqrt(max(np.vdot(delta, r - r_prev), 0.0)))
        if rel <= tol or it == maxit:
            break
        s = ops.apply_P1_pcg(r, l) if p1 == 'pcg' else ops.apply_P1(r, l)
        u_half = u - s
        if coarse is not None:
            t = ops.apply_EK(s) - r
            uc = coarse.solve(coarse.restrict(t))
            u_new = u_half + coarse.prolong(uc)
        else:
            u_new = u_half
        r_prev, u_prev = r, u
        u = u_new
    return u, dict(iterations=it, residuals=hist, updates=upd)
