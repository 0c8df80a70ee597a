"""The FP64-accurate split GEMM (exact BF16 digit-slice products on the
tensor cores, summed in FP64) and the operators built on it.

Exactness: with one slice the digits of small integers are the integers
themselves and their tensor-core products sum exactly, so the result must
equal the FP64 product bit for bit.  Accuracy: with 7 slices the error is
bounded by about 2^-47 K relative to the operand scales; on random data the
normwise error must stay below 1e-12.  K above 1024 exercises the chunked
accumulation.
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip('torch')


@pytest.mark.parametrize('shape', [(128, 128, 64), (300, 192, 192), (1000, 768, 768),
                                   (257, 256, 128), (64, 16, 64), (2048, 768, 3072),
                                   (1089, 64, 64)])
def test_split_gemm_exact_on_small_integers(shape):
    import paper_2102_09038_gb300 as rte
    M, N, K = shape
    g = torch.Generator().manual_seed(M + 3 * N + 7 * K)
    A = torch.randint(-127, 128, (M, K), generator=g).double()
    B = torch.randint(-127, 128, (N, K), generator=g).double()
    C = rte.dgemm_split(A.cuda(), B.cuda(), slices=1).cpu()
    assert torch.equal(C, A @ B.T)


@pytest.mark.parametrize('K', [96, 768, 3072])
def test_split_gemm_fp64_accuracy(K):
    import paper_2102_09038_gb300 as rte
    M, N = 1500, 384
    g = torch.Generator().manual_seed(K)
    # rows with very different scales test the per-row exponents
    A = torch.randn(M, K, generator=g, dtype=torch.float64) * \
        torch.logspace(-6, 6, M, dtype=torch.float64)[:, None]
    B = torch.randn(N, K, generator=g, dtype=torch.float64)
    ref = A @ B.T
    C = rte.dgemm_split(A.cuda(), B.cuda(), slices=7).cpu()
    err = ((C - ref) / ref.abs().amax(dim=1, keepdim=True)).abs().max()
    assert err < 1e-12, float(err)


@pytest.fixture(scope='module')
def split_pair():
    import paper_2102_09038_gb300 as rte
    p = workloads.checkerboard(m=9, levels=2, g=0.7, ratio=0.95, blocks=3, nrhs=2)
    disc = oracle.Discretisation(p.m, p.levels, p.sigma_t, p.sigma_s, p.g)
    ops = oracle.Operators(disc, n_plus=2, n_minus=3)
    s = rte.Solver(p, n_plus=2, n_minus=3, dgemm=rte.DGEMM_SPLIT, max_rhs=3)
    yield p, disc, ops, s
    s.close()


def test_fp64_operators_with_split_gemm(split_pair):
    p, disc, ops, s = split_pair
    x = np.random.default_rng(3).standard_normal((2, disc.nRp, disc.nSp))
    xt = torch.tensor(x, dtype=torch.float64, device='cuda')
    y = s.apply(xt).cpu().numpy()
    ref = np.stack([ops.apply_EK(v) for v in x])
    assert np.abs(y - ref).max() / np.abs(ref).max() < 1e-11
    z = np.random.default_rng(4).standard_normal((2, disc.nRm, disc.nSm))
    zt = torch.tensor(z, dtype=torch.float64, device='cuda')
    out = torch.zeros_like(zt)
    s.operator('MK_INV', zt, out)
    ref = np.stack([ops.solve_MKminus(v) for v in z])
    assert np.abs(out.cpu().numpy() - ref).max() / np.abs(ref).max() < 1e-11


def test_fp64_solve_with_split_gemm(split_pair):
    p, disc, ops, s = split_pair
    q = s.rhs(torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda'))
    u, info = s.solve(q, tol=1e-11)
    assert info['status'] == 0, info
    qref = np.stack([disc.source(v) for v in p.q_nodal])
    for r in range(p.nrhs):
        res = np.linalg.norm(ops.apply_EK(u[r].cpu().numpy()) - qref[r]) / np.linalg.norm(qref[r])
        assert res < 1e-10, res
