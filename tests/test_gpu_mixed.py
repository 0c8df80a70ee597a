"""The tensor-core GEMM and the mixed-precision paths.

The tcgen05 GEMM is checked bit-exactly on integer-valued operands whose
products and sums are exact in FP32 (so any wrong operand, swizzle, K offset
or tail handling shows up as a mismatch), then on random data.  The
mixed-precision apply of E is compared with the FP64 oracle at the accuracy
its operand type allows, and the mixed-precision Richardson solve must reach
the same FP64 residual as the plain method (the outer residual is FP64, so
the loop acts as iterative refinement).
"""
import numpy as np
import pytest

import oracle
import workloads

pytestmark = pytest.mark.gpu
torch = pytest.importorskip('torch')

SHAPES = [(128, 128, 64), (300, 192, 192), (1000, 768, 768), (257, 256, 128),
          (64, 16, 64), (4096, 768, 768), (1089, 64, 64), (130, 136, 320)]


@pytest.mark.parametrize('bf16', [True, False])
@pytest.mark.parametrize('shape', SHAPES)
def test_tc_gemm_exact_on_integer_grid(shape, bf16):
    import paper_2102_09038_gb300 as rte
    M, N, K = shape
    if not bf16 and (K * 4) % 16:
        pytest.skip('TF32 rows must be 16-byte multiples')
    g = torch.Generator().manual_seed(M * 7 + N * 3 + K)
    # values j/64, |j| <= 64: exact in BF16 and TF32; products are multiples
    # of 2^-12 and every partial sum stays below 2^24 ulps, so FP32
    # accumulation is exact
    A = torch.randint(-64, 65, (M, K), generator=g).double() / 64
    B = torch.randint(-64, 65, (N, K), generator=g).double() / 64
    ref = A @ B.T
    dt = torch.bfloat16 if bf16 else torch.float32
    C = rte.gemm_lowp(A.to(dt).cuda(), B.to(dt).cuda())
    torch.cuda.synchronize()
    assert torch.equal(C.double().cpu(), ref)


@pytest.mark.parametrize('bf16', [True, False])
def test_tc_gemm_random_accuracy(bf16):
    import paper_2102_09038_gb300 as rte
    M, N, K = 2048, 768, 768
    g = torch.Generator().manual_seed(5)
    A = torch.randn(M, K, generator=g)
    B = torch.randn(N, K, generator=g)
    dt = torch.bfloat16 if bf16 else torch.float32
    C = rte.gemm_lowp(A.to(dt).cuda(), B.to(dt).cuda()).double().cpu()
    ref = A.to(dt).double() @ B.to(dt).double().T if bf16 else A.double() @ B.double().T
    err = (C - ref).norm() / ref.norm()
    # BF16: inputs exact in the reference, only FP32 accumulation differs;
    # TF32: the tensor core reads 10-bit mantissas of FP32 inputs
    assert err < (1e-6 if bf16 else 2e-3), err
    if bf16:
        Cb = rte.gemm_lowp(A.to(dt).cuda(), B.to(dt).cuda(), out_bf16=True)
        assert ((Cb.double().cpu() - ref).norm() / ref.norm()) < 5e-3


CASES = {
    'tiny': lambda: workloads.constant(3, 1, 0.5, 1.0, 0.9, 1.0),
    'ragged': lambda: workloads.checkerboard(m=9, levels=2, g=0.7, ratio=0.95,
                                             blocks=3, nrhs=2),
}
TOL = {1: 2e-3, 2: 2e-2}   # relative (Frobenius) error of one mixed apply


@pytest.fixture(scope='module', params=[(c, prec) for c in CASES for prec in (1, 2)],
                ids=lambda v: '%s-%s' % (v[0], 'tf32' if v[1] == 1 else 'bf16'))
def mixed(request):
    import paper_2102_09038_gb300 as rte
    name, prec = request.param
    p = CASES[name]()
    disc = oracle.Discretisation(p.m, p.levels, p.sigma_t, p.sigma_s, p.g)
    ops = oracle.Operators(disc, n_plus=2, n_minus=3)
    s = rte.Solver(p, n_plus=2, n_minus=3, precision=prec, max_rhs=3, l=4)
    yield p, disc, ops, s, prec
    s.close()


def test_mixed_apply_E(mixed):
    p, disc, ops, s, prec = mixed
    x = np.random.default_rng(11).standard_normal((2, disc.nRp, disc.nSp))
    xt = torch.tensor(x, dtype=torch.float64, device='cuda')
    for op, fn in (('E_LO', ops.apply_E), ('EK_LO', ops.apply_EK)):
        out = torch.zeros_like(xt)
        s.operator(op, xt, out)
        got = out.cpu().numpy()
        ref = np.stack([fn(v) for v in x])
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < TOL[prec], (op, err)


def test_mixed_solve_reaches_fp64_residual(mixed):
    p, disc, ops, s, prec = mixed
    qn = torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda')
    q = s.rhs(qn)
    u, info = s.solve(q, tol=1e-11)
    assert info['status'] == 0, info
    # every E_0^{-1} of P_1^l is counted; the active-column weighting lies
    # between one full V-cycle per launch (the first one visits every column)
    # and all of them
    assert info['e0_launches'] == 4 * info['iterations'], info
    assert info['e0_launches'] <= info['e0_active_vcycles'] <= info['e0_vcycles'], info
    qref = np.stack([disc.source(v) for v in p.q_nodal])
    u = u.cpu().numpy()
    for r in range(p.nrhs):
        res = np.linalg.norm(ops.apply_EK(u[r]) - qref[r]) / np.linalg.norm(qref[r])
        assert res < 1e-10, res
    # iterative refinement costs only a few more outer iterations
    _, io = oracle.richardson(ops, qref[0], tol=1e-11, l=4, N=2)
    assert info['iterations'] <= io['iterations'] + 6, (info['iterations'], io['iterations'])


@pytest.mark.parametrize('prec', [1, 2])
def test_autotuned_launch_shapes(prec):
    # the tuner picks one candidate per kernel shape (the fastest, unless the
    # default is within 3 % of it), and the picked shapes
    # give the same result as the fixed ones: each output is summed in the
    # same order whatever the block size or tile width
    import paper_2102_09038_gb300 as rte
    p = workloads.checkerboard(m=12, levels=2, g=0.8, ratio=0.9, blocks=2, nrhs=1)
    tuned = rte.Solver(p, n_plus=2, n_minus=3, precision=prec, autotune=1)
    fixed = rte.Solver(p, n_plus=2, n_minus=3, precision=prec, autotune=0)
    rep = rte.autotune_report()
    keys = [k for k in rep if 'm=12 ' in k or 'M=%d ' % (2 * 12 * 12) in k]
    assert any(k.startswith('apply_A') for k in keys)
    assert any(k.startswith('apply_even') for k in keys)
    assert any(k.startswith('tc_gemm %s' % ('bf16' if prec == 2 else 'tf32')) for k in rep)
    for choice, ms in rep.values():
        # the fastest, or the default shape within 3 % of the fastest
        assert 0 <= choice < len(ms) and ms[choice] > 0
        assert ms[choice] <= min(v for v in ms if v > 0) / 0.97 * (1 + 1e-6)
    x = torch.tensor(np.random.default_rng(5).standard_normal((1, tuned.n_nodes, tuned.n_dirs)),
                     dtype=torch.float64, device='cuda')
    for op in ('EK_LO', 'A'):
        shape = x.shape if op == 'EK_LO' else (1, tuned.n_cells, tuned.n_odd)
        a = torch.zeros(shape, dtype=torch.float64, device='cuda')
        b = torch.zeros_like(a)
        tuned.operator(op, x, a)
        fixed.operator(op, x, b)
        assert torch.equal(a, b), op
    tuned.close()
    fixed.close()


@pytest.mark.parametrize('prec', [0, 2])
def test_p1_pcg_route_solves(prec):
    # Algorithm 3 with P_1 as l PCG steps (RTE_P1_PCG) reaches the FP64
    # residual in FP64 and in the mixed BF16 mode; l left at 0 resolves to
    # two steps on this route (two E_0^{-1} per P_1)
    import paper_2102_09038_gb300 as rte
    p = workloads.checkerboard(m=24, levels=2, g=0.8, ratio=0.97, blocks=4, nrhs=2)
    disc = oracle.Discretisation(p.m, p.levels, p.sigma_t, p.sigma_s, p.g)
    ops = oracle.Operators(disc, n_plus=2, n_minus=3)
    s = rte.Solver(p, n_plus=2, n_minus=3, precision=prec, max_rhs=2, p1_route=rte.P1_PCG)
    q = s.rhs(torch.tensor(p.q_nodal, dtype=torch.float64, device='cuda'))
    u, info = s.solve(q, tol=1e-10)
    s.close()
    assert info['status'] == 0, info
    assert info['e0_launches'] == 2 * info['iterations'], info
    u = u.cpu().numpy()
    for r in range(p.nrhs):
        qr = disc.source(p.q_nodal[r])
        assert np.linalg.norm(ops.apply_EK(u[r]) - qr) / np.linalg.norm(qr) < 2e-10
