"""The allocation-free split GEMM entry point, rte_dgemm_split_static.

It is for callers that cannot allocate device memory when they call: a
process whose device memory already belongs to another allocator (a
framework's caching pool, a serving memory budget), or a latency-bound loop
in which an allocation could block or fail.

Two calls in a row through the C ABI (different shapes, so a stale scratch
would show), each compared with the allocating entry point rte_dgemm_split
on the same operands: both run the same kernels, so they agree to FP64
rounding, and both match the FP64 product within the split GEMM's error
bound.  The device's stream-ordered memory pool shows that the static entry
point draws nothing from it while the allocating one does.  Operands beyond
the fixed scratch, or with K not a multiple of 8, are refused before any
device work, and the binding refuses tensors of the wrong type or shape.
The file name sorts last, so in a full run this also runs after every other
GPU test of the process."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip('torch')


def _p(t):
    return ctypes.c_void_p(t.data_ptr())


# cudaMemPoolAttrUsedMemHigh of the CUDA runtime API
_USED_MEM_HIGH = 8


def _pool_high(lib, reset=False):
    """High watermark of the device's default stream-ordered memory pool
    (the pool cudaMallocAsync draws from), read through the CUDA runtime the
    library itself is linked against (dlsym on the library's handle searches
    its dependencies).  reset: restart the watermark at the current use."""
    pool = ctypes.c_void_p()
    assert lib.cudaDeviceGetDefaultMemPool(ctypes.byref(pool),
                                           torch.cuda.current_device()) == 0
    v = ctypes.c_uint64(0)
    if reset:
        assert lib.cudaMemPoolSetAttribute(pool, _USED_MEM_HIGH, ctypes.byref(v)) == 0
    assert lib.cudaMemPoolGetAttribute(pool, _USED_MEM_HIGH, ctypes.byref(v)) == 0
    return v.value


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


def test_static_entry_point_allocates_nothing():
    # the allocating entry point raises the pool's high watermark (its
    # temporaries come from cudaMallocAsync); the static one leaves it
    import paper_2102_09038_gb300 as rte
    lib = rte.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    M, N, K = 640, 384, 512
    A = torch.randn(M, K, dtype=torch.float64, device='cuda')
    B = torch.randn(N, K, dtype=torch.float64, device='cuda')
    C = torch.empty(M, N, dtype=torch.float64, device='cuda')
    torch.cuda.synchronize()
    base = _pool_high(lib, reset=True)
    assert lib.rte_dgemm_split(_p(A), _p(B), _p(C), M, N, K, 7, stream) == 0
    assert _pool_high(lib) > base
    base = _pool_high(lib, reset=True)
    for _ in range(2):
        assert lib.rte_dgemm_split_static(_p(A), _p(B), _p(C), M, N, K, 7, stream) == 0
    assert _pool_high(lib) <= base


def test_static_entry_point_refuses_bad_operands_before_device_work():
    import paper_2102_09038_gb300 as rte
    lib = rte.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # K not a multiple of 8: refused, C untouched
    A = torch.ones(16, 12, dtype=torch.float64, device='cuda')
    C = torch.full((16, 16), 7.0, dtype=torch.float64, device='cuda')
    assert lib.rte_dgemm_split_static(_p(A), _p(A), _p(C), 16, 16, 12, 7, stream) == 1
    assert b'multiple of 8' in lib.rte_last_error()
    torch.cuda.synchronize()
    assert (C == 7.0).all()
    # the binding refuses operands the library would read or write past
    A = torch.randn(64, 32, dtype=torch.float64, device='cuda')
    B = torch.randn(48, 32, dtype=torch.float64, device='cuda')
    for bad in (dict(A=A.float(), Bt=B), dict(A=A, Bt=B[:, :16].contiguous()),
                dict(A=A.cpu(), Bt=B.cpu())):
        with pytest.raises(ValueError):
            rte.dgemm_split_static(bad['A'], bad['Bt'])
        with pytest.raises(ValueError):
            rte.dgemm_split(bad['A'], bad['Bt'])
    for out in (torch.empty(64, 47, dtype=torch.float64, device='cuda'),
                torch.empty(64, 48, dtype=torch.float32, device='cuda'),
                torch.empty(48, 64, dtype=torch.float64, device='cuda').t()):
        with pytest.raises(ValueError):
            rte.dgemm_split_static(A, B, out=out)
