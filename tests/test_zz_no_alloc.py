"""The allocation-free split GEMM entry point, rte_dgemm_split_static.

Two calls in a row through the C ABI (different shapes, so a stale scratch
would show), each compared with the allocating entry point rte_dgemm_split
on the same operands: both run the same kernels, so they agree to FP64
rounding, and both match the FP64 product within the split GEMM's error
bound.  Operands beyond the fixed scratch are refused before any device
work.  The file name sorts last, so in a full run this also runs after
every other GPU test of the process."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip('torch')


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


def test_static_scratch_matches_allocating_entry_point_on_two_calls():
    import paper_2102_09038_gb300 as rte
    lib = rte.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, (M, N, K) in enumerate([(1000, 768, 768), (257, 130, 1032)]):
        g = torch.Generator().manual_seed(100 + call)
        A = torch.randn(M, K, generator=g, dtype=torch.float64) * \
            torch.logspace(-4, 4, M, dtype=torch.float64)[:, None]
        B = torch.randn(N, K, generator=g, dtype=torch.float64)
        Ad, Bd = A.cuda(), B.cuda()
        c_alloc = torch.full((M, N), float('nan'), dtype=torch.float64, device='cuda')
        c_static = torch.full_like(c_alloc, float('nan'))
        assert lib.rte_dgemm_split(_p(Ad), _p(Bd), _p(c_alloc), M, N, K, 7, stream) == 0
        assert lib.rte_dgemm_split_static(_p(Ad), _p(Bd), _p(c_static), M, N, K, 7,
                                          stream) == 0, lib.rte_last_error()
        torch.cuda.synchronize()
        ref = A @ B.T
        scale = ref.abs().amax(dim=1, keepdim=True)
        ca, cs = c_alloc.cpu(), c_static.cpu()
        assert torch.isfinite(cs).all()
        assert ((cs - ca) / scale).abs().max() <= 1e-15
        assert ((cs - ref) / scale).abs().max() < 1e-12


def test_static_scratch_edge_cases():
    import paper_2102_09038_gb300 as rte
    lib = rte.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # K = 0: C = 0 (the operands are not read; any non-null pointer will do)
    dummy = torch.zeros(1, dtype=torch.float64, device='cuda')
    C = torch.full((5, 3), 7.0, dtype=torch.float64, device='cuda')
    assert lib.rte_dgemm_split_static(_p(dummy), _p(dummy), _p(C), 5, 3, 0, 7, stream) == 0
    torch.cuda.synchronize()
    assert (C == 0).all()
    # operands beyond the scratch are refused and C is left as it was
    M = N = K = 2048
    A = torch.ones(M, K, dtype=torch.float64, device='cuda')
    C = torch.full((M, N), 7.0, dtype=torch.float64, device='cuda')
    assert lib.rte_dgemm_split_static(_p(A), _p(A), _p(C), M, N, K, 7, stream) == 1
    assert b'scratch' in lib.rte_last_error()
    torch.cuda.synchronize()
    assert (C == 7.0).all()
    # the binding, with a caller-provided output
    A = torch.randn(300, 192, dtype=torch.float64, device='cuda')
    B = torch.randn(64, 192, dtype=torch.float64, device='cuda')
    out = torch.empty(300, 64, dtype=torch.float64, device='cuda')
    got = rte.dgemm_split_static(A, B, out=out)
    assert got.data_ptr() == out.data_ptr()
    ref = rte.dgemm_split(A, B)
    assert ((got - ref).abs().max() / ref.abs().max()).item() <= 1e-15
