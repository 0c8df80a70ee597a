"""Operator applications and solves of Section 5 for the oracle.

Test infrastructure only: the CUDA product path never imports this module.

Arrays are coefficient matrices stored row-major: U (n_R^+, n_S^+) for even
functions and Z (n_R^-, n_S^-) for odd ones, so the Kronecker operator
B (x) C of the paper acts as C @ U @ B.T (eq. tpmv).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla


class Operators:
    """Plain FP64 statements of A, A^T, M^+, R, K^+, M^- - K^-, E, E - K^+
    (Section 4 and eq. ep_discrete) for one ``Discretisation``."""

    def __init__(self, disc, n_plus=4, n_minus=5):
        self.d = disc
        sm, an = disc.sp, disc.an
        self.D1, self.D2 = sm['D1'], sm['D2']
        self.D1T, self.D2T = sm['D1'].T.tocsr(), sm['D2'].T.tocsr()
        self.A1, self.A2 = disc.A1, disc.A2
        self.m = an['m']
        self.Sp, self.Sm = an['Splus'], an['Sminus']
        self.MSm = disc.MSm
        self.area = sm['area']
        self.Mt_minus, self.Ms_minus = sm['Mt_minus'], sm['Ms_minus']
        # cells grouped by their (sigma_t, sigma_s) pair: M^- - K^- is block
        # diagonal per cell with block |T_j| (sigma_t M_S^- - sigma_s S^-)
        pairs = np.stack([disc.sigma_t, disc.sigma_s], axis=1)
        self.classes, self.cell_class = np.unique(pairs, axis=0,
                                                  return_inverse=True)
        self.cell_class = self.cell_class.ravel()
        self._chol = {}
        self.n_plus, self.n_minus = n_plus, n_minus
        self._e0 = None
        self._coarse = None

    # -------------------------------------------------------------- pieces
    def apply_A(self, U):
        """A u^+ with A = sum_n A_n (x) D_n (eq. AR): Z = sum_n D_n U A_n^T."""
        return self.D1 @ U @ self.A1.T + self.D2 @ U @ self.A2.T

    def apply_AT(self, Z):
        """A^T z = sum_n D_n^T Z A_n."""
        return self.D1T @ Z @ self.A1 + self.D2T @ Z @ self.A2

    def apply_Mplus(self, U):
        """M^+ u = (M_S^+ (x) M_t^+) u = M_t^+ U M_S^+ (M_S^+ diagonal)."""
        return (self.d.sp['Mt_plus'] @ U) * self.m[None, :]

    def apply_R(self, U):
        """R u = blkdiag(R_k) u, R_k = omega^x_k B_x + omega^y_k B_y."""
        an = self.d.an
        return ((self.d.sp['Bx'] @ U) * an['omx'][None, :]
                + (self.d.sp['By'] @ U) * an['omy'][None, :])

    def apply_Kplus(self, U):
        """K^+ u = (S^+ (x) M_s^+) u = M_s^+ U S^+ (eq. bKebKo)."""
        return self.d.sp['Ms_plus'] @ U @ self.Sp

    def apply_MKminus(self, Z):
        """(M^- - K^-) z = M_t^- Z M_S^- - M_s^- Z S^- (diagonal M_t^-, M_s^-)."""
        return (self.Mt_minus[:, None] * (Z @ self.MSm)
                - self.Ms_minus[:, None] * (Z @ self.Sm))

    def solve_MKminus(self, B):
        """(M^- - K^-)^{-1} b by a dense Cholesky factorisation of each
        distinct per-cell block sigma_t M_S^- - sigma_s S^-, scaled by the
        cell area."""
        X = np.empty_like(B)
        for c, (st, ss) in enumerate(self.classes):
            if c not in self._chol:
                self._chol[c] = sla.cho_factor(st * self.MSm - ss * self.Sm)
            rows = np.nonzero(self.cell_class == c)[0]
            X[rows] = sla.cho_solve(self._chol[c], B[rows].T).T
        return X / self.area[:, None]

    def apply_E(self, U):
        """E u = A^T (M^- - K^-)^{-1} A u + M^+ u + R u (eq. ep_discrete)."""
        return (self.apply_AT(self.solve_MKminus(self.apply_A(U)))
                + self.apply_Mplus(U) + self.apply_R(U))

    def apply_EK(self, U):
        """(E - K^+) u, the even-parity operator of eq. ep_discrete."""
        return self.apply_E(U) - self.apply_Kplus(U)

    # ------------------------------------------- Lemma apply_high_order_pre
    def eig_minus(self):
        """Generalised eigenpairs S^- W = M_S^- W Lambda^-, eigenvalues
        non-increasing, W^T M_S^- W = I (Section 5.1)."""
        if not hasattr(self, '_eigm'):
            lam, W = sla.eigh(self.Sm, self.MSm)
            self._eigm = (lam[::-1].copy(), W[:, ::-1].copy())
        return self._eigm

    def eig_plus(self):
        """Generalised eigenpairs S^+ W = M_S^+ W Lambda^+ (Section 5.4)."""
        if not hasattr(self, '_eigp'):
            lam, W = sla.eigh(self.Sp, np.diag(self.m))
            self._eigp = (lam[::-1].copy(), W[:, ::-1].copy())
        return self._eigp

    def precond_MKN(self, B, N=None):
        """x = (M^- - K^-_N)^{-1} b by eq. (MmKprecond), d_N = (N+1)(N+2)/2."""
        N = self.n_minus if N is None else N
        dN = (N + 1) * (N + 2) // 2
        lam, W = self.eig_minus()
        WN, lamN = W[:, :dN], lam[:dN]
        st = self.d.sigma_t[:, None]
        ss = self.d.sigma_s[:, None]
        F = 1.0 / (self.area[:, None] * (st - lamN[None, :] * ss))
        BW = B @ WN
        low = (BW * F) @ WN.T
        MSm_inv = np.linalg.inv(self.MSm)
        high = (B @ MSm_inv - BW @ WN.T) / self.Mt_minus[:, None]
        return low + high

    def pcg_MKminus(self, B, tol=1e-12, maxit=500, N=None):
        """Solve (M^- - K^-) x = b by PCG preconditioned with
        (M^- - K^-_N)^{-1} (Algorithm 1, first step).  Stops on
        ||r||_2 <= tol ||b||_2.  Returns (x, iterations)."""
        x = np.zeros_like(B)
        r = B.copy()
        nb = np.linalg.norm(B)
        if nb == 0.0:
            return x, 0
        z = self.precond_MKN(r, N)
        p = z.copy()
        rz = np.vdot(r, z)
        for it in range(1, maxit + 1):
            Ap = self.apply_MKminus(p)
            alpha = rz / np.vdot(p, Ap)
            x += alpha * p
            r -= alpha * Ap
            if np.linalg.norm(r) <= tol * nb:
                return x, it
            z = self.precond_MKN(r, N)
            rz_new = np.vdot(r, z)
            p = z + (rz_new / rz) * p
            rz = rz_new
        return x, maxit

    # ------------------------------------------------------------- E_0
    def e0_blocks(self):
        """Direction blocks of E_0 = (1-cg)^{-1} A^T (M^-)^{-1} A + R + M^+
        (eq. equivalence_bE_bE0).  Block k is
        (1-cg)^{-1} sum_{n,m} a_k^{nm} D_n^T (M_t^-)^{-1} D_m
          + omega^x_k B_x + omega^y_k B_y + m_k M_t^+
        with a_k^{nm} = [A_n^T (M_S^-)^{-1} A_m]_{kk}."""
        if self._e0 is None:
            an, smat = self.d.an, self.d.sp
            gamma = 1.0 / (1.0 - self.d.c * self.d.g)
            Minv = sp.diags(1.0 / self.Mt_minus)
            Dn = [self.D1, self.D2]
            K = [[(Dn[a].T @ Minv @ Dn[b]).tocsc() for b in range(2)]
                 for a in range(2)]
            acol = [an['A1'], an['A2']]
            MSinv = np.linalg.inv(an['MSm'])
            blocks = []
            for k in range(self.d.nSp):
                mat = (an['omx'][k] * smat['Bx'] + an['omy'][k] * smat['By']
                       + self.m[k] * smat['Mt_plus']).tocsc()
                for a in range(2):
                    for b in range(2):
                        akab = acol[a][k] @ MSinv[k] @ acol[b][k]
                        mat = mat + gamma * akab * K[a][b]
                blocks.append(mat.tocsc())
            self._e0 = dict(blocks=blocks, lu=[None] * len(blocks),
                            gamma=gamma)
        return self._e0

    def apply_E0(self, U):
        """E_0 u from its definition: (1-cg)^{-1} A^T (M^-)^{-1} A u + R u
        + M^+ u, with (M^-)^{-1} = (M_S^-)^{-1} (x) (M_t^-)^{-1}."""
        gamma = 1.0 / (1.0 - self.d.c * self.d.g)
        Z = self.apply_A(U)
        Z = (Z @ np.linalg.inv(self.MSm)) / self.Mt_minus[:, None]
        return gamma * self.apply_AT(Z) + self.apply_R(U) + self.apply_Mplus(U)

    def solve_E0(self, B):
        """E_0^{-1} b direction by direction with a sparse LU per block (the
        paper used a sparse direct solver for these blocks)."""
        e0 = self.e0_blocks()
        X = np.empty_like(B)
        for k in range(B.shape[1]):
            if e0['lu'][k] is None:
                e0['lu'][k] = spla.splu(e0['blocks'][k])
            X[:, k] = e0['lu'][k].solve(B[:, k])
        return X

    def apply_P1(self, B, l=4):
        """P_1^l b by eq. (applyP1): z_0 = 0, z_{k+1} = z_k - E_0^{-1}(E z_k - b),
        k < l.  The step from z_0 = 0 is z_1 = E_0^{-1} b."""
        z = self.solve_E0(B)
        for _ in range(1, l):
            z = z - self.solve_E0(self.apply_E(z) - B)
        return z

    def apply_P1_pcg(self, B, l=4):
        """The non-stationary P_1 named in Section 5.3 beside eq. (applyP1):
        l steps of the conjugate gradient method for E z = b with
        preconditioner E_0^{-1}, started from z = 0 (textbook PCG: residual
        r, preconditioned residual y = E_0^{-1} r, directions p, step length
        r.y / p.Ep, direction update with the ratio of successive r.y).
        Inner products are over all of b's coefficients."""
        z = np.zeros_like(B)
        r = B.copy()
        y = self.solve_E0(r)
        p = y.copy()
        ry = np.vdot(r, y)
        for k in range(l):
            w = self.apply_E(p)
            pw = np.vdot(p, w)
            alpha = ry / pw if pw != 0.0 else 0.0
            z = z + alpha * p
            if k + 1 == l:
                break
            r = r - alpha * w
            y = self.solve_E0(r)
            ry_new = np.vdot(r, y)
            p = y + (ry_new / ry if ry != 0.0 else 0.0) * p
            ry = ry_new
        return z
