"""Direct parity of the mixed-precision kernels with the FP64 oracle.

The mixed modes (RTE_MIXED_FP32, RTE_MIXED_BF16) run E_0^{-1} as an FP32
multigrid-PCG kernel, the E_c solve with an FP32 V-cycle under FP64 CG
recurrences and the inner applies of E with FP32 stencils and BF16 or TF32
tensor-core GEMMs.  In a solve these are preconditioners under the FP64
outer residual, so a wrong kernel would only cost outer iterations; here
each is judged on its own:

* E_0^{-1} on mixed handles, by the FP32 direct factorisation and by the
  FP32 multigrid CG at a tight inner tolerance: every direction column's
  relative residual in the oracle's E_0 blocks, at 64, 256 and 1024 columns
  (the CG's quad kernel) and 1280 columns (its kernel for more columns than
  the quad kernel's per-block tables hold; the direct route's sweeps of
  four right-hand sides with a ragged last one);
* E_c^{-1} on mixed handles (direct and multigrid routes): relative
  residual in the oracle's E_c;
* E and E - K^+ in the mixed precision, element by element: max-norm error
  over the reference's max norm, against six unit roundoffs of the GEMM
  operand type (BF16 2^-9, TF32 2^-11), at 64, 256 and 1024 directions.
"""
import numpy as np
import pytest

import oracle
import workloads
from oracle.richardson import Coarse

pytestmark = pytest.mark.gpu
torch = pytest.importorskip('torch')

# (mesh, sphere levels, right-hand sides): 64, 256, 1024 and 1280 columns
COLS = {64: (10, 2, 1), 256: (12, 3, 1), 1024: (12, 3, 4), 1280: (12, 3, 5)}


def problem(m, levels, nrhs):
    return workloads.checkerboard(m=m, levels=levels, g=0.8, ratio=0.97, blocks=2,
                                  nrhs=nrhs)


_DISC = {}


def oracle_ops(p):
    """The oracle's assembly of p (cached: the 1024-direction sphere takes
    the oracle tens of seconds) and its operators with N^+ = 2, N^- = 3."""
    key = (p.m, p.levels, p.g, p.sigma_t.tobytes(), p.sigma_s.tobytes())
    if key not in _DISC:
        _DISC[key] = oracle.Discretisation(p.m, p.levels, p.sigma_t, p.sigma_s, p.g)
    disc = _DISC[key]
    return disc, oracle.Operators(disc, n_plus=2, n_minus=3)


def col_residuals(ops, x, b):
    """Relative residual of every (rhs, direction) column in the oracle's
    E_0 (its definition, applied in FP64)."""
    out = []
    for r in range(b.shape[0]):
        res = ops.apply_E0(x[r]) - b[r]
        out.append(np.linalg.norm(res, axis=0) / np.linalg.norm(b[r], axis=0))
    return np.concatenate(out)


@pytest.mark.parametrize('route', [1, 2], ids=['direct', 'multigrid'])
@pytest.mark.parametrize('prec', [1, 2], ids=['fp32', 'bf16'])
@pytest.mark.parametrize('ncols', sorted(COLS))
def test_mixed_e0_inverse_every_column(ncols, prec, route):
    # direct route: the FP32 factor's sweeps; multigrid route: the FP32 CG
    # to e0_tol
    import paper_2102_09038_gb300 as rte
    m, levels, nrhs = COLS[ncols]
    p = problem(m, levels, nrhs)
    disc, ops = oracle_ops(p)
    s = rte.Solver(p, n_plus=2, n_minus=3, precision=prec, max_rhs=nrhs, e0_tol=1e-5,
                   e0_route=route)
    assert s.n_dirs * nrhs == ncols
    b = np.random.default_rng(ncols + prec).standard_normal((nrhs, disc.nRp, disc.nSp))
    bt = torch.tensor(b, dtype=torch.float64, device='cuda')
    out = torch.zeros_like(bt)
    s.operator('E0_INV', bt, out)
    x = out.cpu().numpy()
    s.close()
    res = col_residuals(ops, x, b)
    assert res.size == ncols
    # the FP32 CG stops on its own recursively updated residual at 1e-5 (the
    # true residual of its FP32 iterate measured at most 9.7e-6); the FP32
    # direct sweeps are exact up to FP32 rounding
    assert res.max() <= 2e-5, res.max()


@pytest.mark.parametrize('route', [1, 2], ids=['direct', 'multigrid'])
@pytest.mark.parametrize('prec', [1, 2], ids=['fp32', 'bf16'])
def test_mixed_coarse_inverse(prec, route):
    # FP64 CG recurrences with an FP32 preconditioner (the FP32 sweeps of
    # E_c's factor, or an FP32 V-cycle): the FP32 preconditioner must not
    # limit the attainable accuracy
    import paper_2102_09038_gb300 as rte
    p = problem(17, 2, 2)
    disc, ops = oracle_ops(p)
    for tol in (1e-5, 1e-10):
        s = rte.Solver(p, n_plus=2, n_minus=3, precision=prec, max_rhs=2, coarse_tol=tol,
                       coarse_route=route)
        d = s.d_plus
        W = s.export('WpN').reshape(disc.nSp, d)
        co = Coarse(ops, 2, W=W)
        qc = np.random.default_rng(3).standard_normal((2, disc.nRp, d))
        qt = torch.tensor(qc, dtype=torch.float64, device='cuda')
        out = torch.zeros_like(qt)
        s.operator('EC_INV', qt, out)
        uc = out.cpu().numpy()
        s.close()
        for r in range(2):
            res = co.Ec @ uc[r].ravel() - qc[r].ravel()
            assert np.linalg.norm(res) / np.linalg.norm(qc[r]) <= 2 * tol


@pytest.mark.parametrize('prec', [1, 2], ids=['fp32', 'bf16'])
def test_mixed_coarse_inverse_at_the_default_tolerance(prec):
    # at the mixed modes' coarse tolerance 0.3 the coarse CG's own E_c
    # products run in FP32 on the multigrid's level 0: the result meets the
    # tolerance in the oracle's E_c, and it agrees with the FP64 handle's
    # (the same FP32 V-cycle, FP64 products) to far below the tolerance
    import paper_2102_09038_gb300 as rte
    p = problem(17, 2, 2)
    disc, ops = oracle_ops(p)
    outs, qc, W = {}, None, None
    for pr in (0, prec):
        s = rte.Solver(p, n_plus=2, n_minus=3, precision=pr, max_rhs=2, coarse_tol=0.3,
                       coarse_route=2)
        d = s.d_plus
        W = s.export('WpN').reshape(disc.nSp, d)
        if qc is None:
            qc = np.random.default_rng(5).standard_normal((2, disc.nRp, d))
        out = torch.zeros((2, disc.nRp, d), dtype=torch.float64, device='cuda')
        s.operator('EC_INV', torch.tensor(qc, dtype=torch.float64, device='cuda'), out)
        outs[pr] = out.cpu().numpy()
        s.close()
    co = Coarse(ops, 2, W=W)
    for r in range(2):
        res = co.Ec @ outs[prec][r].ravel() - qc[r].ravel()
        assert np.linalg.norm(res) / np.linalg.norm(qc[r]) <= 0.3 * 1.01
        diff = np.linalg.norm(outs[prec][r] - outs[0][r]) / np.linalg.norm(outs[0][r])
        assert diff <= 1e-4, diff


# element-wise bounds on max|got - ref| / max|ref| of one mixed apply: six
# unit roundoffs of the GEMM operand type (TF32 u = 2^-11, BF16 u = 2^-9),
# the operand roundings of the two eigenbasis contractions and of U S^+
# (measured: 1.1e-3 to 1.5e-3 TF32, 1.1e-3 to 2.4e-3 BF16)
BOUND = {1: 6 * 2.0 ** -11, 2: 6 * 2.0 ** -9}


@pytest.mark.parametrize('prec', [1, 2], ids=['tf32', 'bf16'])
@pytest.mark.parametrize('levels', [2, 3, 4], ids=['64dirs', '256dirs', '1024dirs'])
def test_mixed_applies_element_by_element(levels, prec):
    import paper_2102_09038_gb300 as rte
    m = {2: 8, 3: 6, 4: 4}[levels]
    p = problem(m, levels, 2)
    disc, ops = oracle_ops(p)
    s = rte.Solver(p, n_plus=2, n_minus=3, precision=prec, max_rhs=2)
    rng = np.random.default_rng(17 * levels + prec)
    # a smooth field plus noise: both the cancelling and the coherent parts
    # of the contractions are exercised
    x = rng.standard_normal((2, disc.nRp, disc.nSp)) + 2.0
    xt = torch.tensor(x, dtype=torch.float64, device='cuda')
    for op, fn in (('E_LO', ops.apply_E), ('EK_LO', ops.apply_EK)):
        out = torch.zeros_like(xt)
        s.operator(op, xt, out)
        got = out.cpu().numpy()
        ref = np.stack([fn(v) for v in x])
        err = np.abs(got - ref).max() / np.abs(ref).max()
        assert err <= BOUND[prec], (op, err)
    s.close()


@pytest.mark.parametrize('prec', [1, 2], ids=['fp32', 'bf16'])
def test_mixed_restriction_and_prolongation(prec):
    # on mixed handles the coarse restriction W^T x and prolongation W u_c
    # run in FP32 products (a preconditioner step): every entry within the
    # standard rounding bound (n + 1) u sum |x_k| |W_kj| of an n-term FP32
    # dot product (u = 2^-24; the operands' FP32 rounding included)
    import paper_2102_09038_gb300 as rte
    p = problem(9, 2, 2)
    disc, ops = oracle_ops(p)
    s = rte.Solver(p, n_plus=2, n_minus=3, precision=prec, max_rhs=2)
    d = s.d_plus
    W = s.export('WpN').reshape(disc.nSp, d)
    co = Coarse(ops, 2, W=W)
    u = 2.0 ** -24
    x = np.random.default_rng(11).standard_normal((2, disc.nRp, disc.nSp))
    qc = torch.zeros((2, disc.nRp, d), dtype=torch.float64, device='cuda')
    s.operator('RESTRICT', torch.tensor(x, device='cuda'), qc)
    got = qc.cpu().numpy()
    for r in range(2):
        ref = co.restrict(x[r]).reshape(disc.nRp, d)
        bound = (disc.nSp + 1) * u * (np.abs(x[r]) @ np.abs(W))
        assert np.all(np.abs(got[r] - ref) <= bound + 1e-300)
    uc = np.random.default_rng(12).standard_normal((2, disc.nRp, d))
    out = torch.zeros((2, disc.nRp, disc.nSp), dtype=torch.float64, device='cuda')
    s.operator('PROLONG', torch.tensor(uc, device='cuda'), out)
    got = out.cpu().numpy()
    s.close()
    for r in range(2):
        ref = co.prolong(uc[r]).reshape(disc.nRp, disc.nSp)
        bound = (d + 1) * u * (np.abs(uc[r]) @ np.abs(W).T)
        assert np.all(np.abs(got[r] - ref) <= bound + 1e-300)
