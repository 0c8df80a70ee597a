"""Dense full-system statements for tiny problems (the plain definition).

Test infrastructure only: the CUDA product path never imports this module.

The even part u^+ of the solution of the mixed system eq. (mixed_discrete),

    [ R + M^+ - K^+   -A^T        ] [u^+]   [l^+]
    [ A               M^- - K^-   ] [u^-] = [l^-],

is the unique solution of (E - K^+) u^+ = q with E the Schur complement
(eq. ep_discrete).  Here every Kronecker product is formed densely.  With
row-major storage (spatial index slow) the paper's B (x) C becomes
numpy.kron(C, B).
"""
import numpy as np
import scipy.linalg as sla


def full_matrices(disc):
    an, smat = disc.an, disc.sp
    dense = lambda a: a.toarray() if hasattr(a, 'toarray') else np.asarray(a)
    Kp = np.kron(dense(smat['Ms_plus']), an['Splus'])
    Mp = np.kron(dense(smat['Mt_plus']), np.diag(an['m']))
    R = (np.kron(dense(smat['Bx']), np.diag(an['omx']))
         + np.kron(dense(smat['By']), np.diag(an['omy'])))
    A = (np.kron(dense(smat['D1']), disc.A1)
         + np.kron(dense(smat['D2']), disc.A2))
    Mm = np.kron(np.diag(smat['Mt_minus']), disc.MSm)
    Km = np.kron(np.diag(smat['Ms_minus']), an['Sminus'])
    return dict(Kp=Kp, Mp=Mp, R=R, A=A, Mm=Mm, Km=Km)


def mixed_solve(disc, lplus, lminus=None):
    """u^+, u^- from a dense LU solve of the mixed system."""
    f = full_matrices(disc)
    npl = f['Mp'].shape[0]
    nmi = f['Mm'].shape[0]
    top = np.concatenate([f['R'] + f['Mp'] - f['Kp'], -f['A'].T], axis=1)
    bot = np.concatenate([f['A'], f['Mm'] - f['Km']], axis=1)
    big = np.concatenate([top, bot], axis=0)
    rhs = np.concatenate([lplus.ravel(),
                          np.zeros(nmi) if lminus is None else lminus.ravel()])
    x = np.linalg.solve(big, rhs)
    return x[:npl], x[npl:]


def schur_matrix(disc):
    """E - K^+ formed densely: A^T (M^- - K^-)^{-1} A + M^+ + R - K^+."""
    f = full_matrices(disc)
    E = f['A'].T @ np.linalg.solve(f['Mm'] - f['Km'], f['A']) + f['Mp'] + f['R']
    return E - f['Kp'], E, f


def schur_solve(disc, q):
    """u^+ by a Cholesky solve with the dense Schur complement."""
    EK, _, _ = schur_matrix(disc)
    return sla.cho_solve(sla.cho_factor(EK), q.ravel())
