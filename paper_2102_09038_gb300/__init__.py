"""Python binding of librte, the GB300 library for the preconditioned
Richardson iteration of Dölz, Palii and Schlottbom (arXiv 2102.09038) for the
even-parity anisotropic radiative transfer equation.

The binding only marshals arguments: every step of the iteration runs in the
library's CUDA kernels (include/rte.h).  Device vectors are torch CUDA
tensors (float64, contiguous) passed by pointer; torch provides memory and
streams only.  There is no CPU fallback: constructing a ``Solver`` without
the built library or without a CUDA device raises.
"""
import ctypes
import os

__all__ = ['Solver', 'RteError', 'load', 'OPS', 'FP64', 'MIXED_FP32',
           'MIXED_BF16', 'MK_EIGEN', 'MK_PCG', 'P1_AUTO', 'P1_RICHARDSON',
           'P1_PCG', 'E0_AUTO', 'E0_DIRECT', 'E0_MULTIGRID', 'EC_AUTO', 'EC_DIRECT',
           'EC_MULTIGRID']

FP64, MIXED_FP32, MIXED_BF16 = 0, 1, 2
MK_EIGEN, MK_PCG = 0, 1
P1_AUTO, P1_RICHARDSON, P1_PCG = -1, 0, 1
DGEMM_AUTO, DGEMM_SIMT, DGEMM_SPLIT = 0, 1, 2
E0_AUTO, E0_DIRECT, E0_MULTIGRID = 0, 1, 2
EC_AUTO, EC_DIRECT, EC_MULTIGRID = 0, 1, 2
OPS = dict(A=1, AT=2, KPLUS=3, MK=4, MK_INV=5, MK_PREC=6, E=7, E0_INV=8,
           P1=9, RESTRICT=10, PROLONG=11, EC=12, EC_INV=13, E_LO=14, EK_LO=15)
EXPORTS = dict(Splus=0, Sminus=1, m=2, MSm=3, A1=4, A2=5, omx=6, omy=7,
               lamP=8, lamM=9, WpN=10, Ec=11)
ERRORS = {1: 'RTE_ERR_ARG', 2: 'RTE_ERR_NOMEM', 3: 'RTE_ERR_DIVERGED',
          4: 'RTE_ERR_MAXITER', 5: 'RTE_ERR_TIMEOUT', 6: 'RTE_ERR_CUDA'}

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, '_build', 'librte.so')


class RteError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__('%s: %s' % (ERRORS.get(code, code), msg))
        self.code = code


class _Problem(ctypes.Structure):
    _fields_ = [('mesh_m', ctypes.c_int), ('sphere_levels', ctypes.c_int),
                ('sigma_t', ctypes.POINTER(ctypes.c_double)),
                ('sigma_s', ctypes.POINTER(ctypes.c_double)),
                ('g', ctypes.c_double)]


class _Options(ctypes.Structure):
    _fields_ = [('l', ctypes.c_int), ('n_plus', ctypes.c_int),
                ('n_minus', ctypes.c_int), ('precision', ctypes.c_int),
                ('mk_route', ctypes.c_int), ('mk_tol', ctypes.c_double),
                ('mk_maxit', ctypes.c_int), ('e0_tol', ctypes.c_double),
                ('e0_maxit', ctypes.c_int), ('coarse_tol', ctypes.c_double),
                ('coarse_maxit', ctypes.c_int), ('max_iter', ctypes.c_int),
                ('max_rhs', ctypes.c_int), ('dgemm', ctypes.c_int),
                ('split_slices', ctypes.c_int), ('mg_sweeps', ctypes.c_int),
                ('autotune', ctypes.c_int), ('p1_route', ctypes.c_int),
                ('e0_route', ctypes.c_int), ('coarse_route', ctypes.c_int)]


class _Stats(ctypes.Structure):
    _fields_ = [('iterations', ctypes.c_int), ('rel_residual', ctypes.c_double),
                ('energy_update', ctypes.c_double),
                ('e0_iters_last', ctypes.c_int),
                ('coarse_iters_last', ctypes.c_int),
                ('mk_iters_last', ctypes.c_int),
                ('history', ctypes.POINTER(ctypes.c_double)),
                ('history_cap', ctypes.c_int), ('seconds', ctypes.c_double),
                ('e0_launches', ctypes.c_int), ('e0_vcycles', ctypes.c_double),
                ('e0_active_vcycles', ctypes.c_double)]


class _H2Options(ctypes.Structure):
    _fields_ = [('levels', ctypes.c_int), ('g', ctypes.c_double), ('eta', ctypes.c_double),
                ('p', ctypes.c_int), ('parities', ctypes.c_int), ('precisions', ctypes.c_int)]


class _H2Info(ctypes.Structure):
    _fields_ = [('n_plus', ctypes.c_int), ('leaves', ctypes.c_int), ('clusters', ctypes.c_int),
                ('far_blocks', ctypes.c_int * 2), ('near_blocks', ctypes.c_int * 2),
                ('near_matrices', ctypes.c_int), ('transfers', ctypes.c_int),
                ('bytes', ctypes.c_size_t),
                ('setup_ms', ctypes.c_double)]


_lib = None
EXPORTED = ['rte_default_options', 'rte_setup', 'rte_sizes', 'rte_rhs', 'rte_inflow',
            'rte_apply', 'rte_precond', 'rte_solve', 'rte_operator',
            'rte_export', 'rte_timing_enable', 'rte_timing_read',
            'rte_kernel_launches', 'rte_gemm_lowp', 'rte_dgemm_split',
            'rte_trace_enable', 'rte_estimate_bytes', 'rte_server_create',
            'rte_server_submit', 'rte_server_wait', 'rte_server_destroy', 'rte_solve_batch',
            'rte_trace_read', 'rte_destroy', 'rte_set_wait_limit', 'rte_barrier_selftest',
            'rte_set_stream', 'rte_server_cache_stats',
            'rte_h2_default_options', 'rte_h2_create', 'rte_h2_apply', 'rte_h2_get_info',
            'rte_h2_dense', 'rte_h2_destroy', 'rte_h2_plan_info',
            'rte_last_error']


def load(path=LIB_PATH):
    """Load librte.so and declare its signatures (no GPU needed)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError('librte.so not built: run __graft_entry__.build() '
                          '(expected at %s)' % path)
    lib = ctypes.CDLL(path)
    P, I, D, V = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, None
    lib.rte_default_options.argtypes = [ctypes.POINTER(_Options)]
    lib.rte_setup.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_Options),
                              P, ctypes.POINTER(P)]
    lib.rte_sizes.argtypes = [P] + [ctypes.POINTER(I)] * 6
    lib.rte_rhs.argtypes = [P, P, P, I]
    lib.rte_apply.argtypes = [P, P, P, I]
    lib.rte_inflow.argtypes = [P, P, P, I]
    lib.rte_precond.argtypes = [P, P, P, I, I]
    lib.rte_solve.argtypes = [P, P, P, I, D, ctypes.POINTER(_Stats)]
    lib.rte_operator.argtypes = [P, I, P, P, I]
    lib.rte_odd.argtypes = [P, P, P, P, I]
    lib.rte_rates.argtypes = [P, I, D, ctypes.c_ulonglong, ctypes.POINTER(D), ctypes.POINTER(D),
                              ctypes.POINTER(I)]
    lib.rte_export.argtypes = [P, I, ctypes.POINTER(D), ctypes.c_size_t]
    lib.rte_timing_enable.argtypes = [P, I]
    lib.rte_timing_read.argtypes = [P, ctypes.POINTER(ctypes.c_char_p),
                                    ctypes.POINTER(D),
                                    ctypes.POINTER(ctypes.c_longlong), I,
                                    ctypes.POINTER(I)]
    lib.rte_gemm_lowp.argtypes = [P, P, P, I, I, I, I, I, P]
    lib.rte_dgemm_split.argtypes = [P, P, P, I, I, I, I, P]
    lib.rte_autotune_report.argtypes = [ctypes.c_char_p, ctypes.c_size_t]
    lib.rte_autotune_report.restype = ctypes.c_size_t
    lib.rte_dgemm_split_static.argtypes = [P, P, P, I, I, I, I, P]
    lib.rte_estimate_bytes.argtypes = [ctypes.POINTER(_Problem), ctypes.POINTER(_Options), I]
    lib.rte_estimate_bytes.restype = ctypes.c_size_t
    lib.rte_server_create.argtypes = [ctypes.c_size_t, I, ctypes.POINTER(_Options),
                                      ctypes.POINTER(P)]
    lib.rte_server_submit.argtypes = [P, ctypes.POINTER(_Problem), ctypes.POINTER(D), I, D,
                                      ctypes.POINTER(ctypes.c_longlong)]
    lib.rte_server_wait.argtypes = [P, ctypes.c_longlong, D, ctypes.POINTER(D),
                                    ctypes.c_size_t, ctypes.POINTER(_Stats),
                                    ctypes.POINTER(D), ctypes.POINTER(D)]
    lib.rte_server_destroy.argtypes = [P]
    lib.rte_server_cache_stats.argtypes = [P, ctypes.POINTER(ctypes.c_longlong),
                                           ctypes.POINTER(ctypes.c_longlong),
                                           ctypes.POINTER(ctypes.c_size_t)]
    lib.rte_set_stream.argtypes = [P, P]
    lib.rte_server_destroy.restype = V
    lib.rte_setup_times.argtypes = [P, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(D), I,
                                    ctypes.POINTER(I)]
    lib.rte_trace_enable.argtypes = [P, I]
    lib.rte_trace_read.argtypes = [P, ctypes.POINTER(D), I, ctypes.POINTER(I)]
    lib.rte_set_wait_limit.argtypes = [D]
    lib.rte_barrier_selftest.argtypes = [I, I, I, P, ctypes.POINTER(I), ctypes.POINTER(I)]
    lib.rte_kernel_launches.argtypes = []
    lib.rte_kernel_launches.restype = ctypes.c_longlong
    lib.rte_destroy.argtypes = [P]
    lib.rte_destroy.restype = V
    lib.rte_h2_default_options.argtypes = [ctypes.POINTER(_H2Options)]
    lib.rte_h2_create.argtypes = [ctypes.POINTER(_H2Options), P, ctypes.POINTER(P)]
    lib.rte_h2_apply.argtypes = [P, I, I, P, P, I, P]
    lib.rte_h2_get_info.argtypes = [P, ctypes.POINTER(_H2Info)]
    lib.rte_h2_plan_info.argtypes = [ctypes.POINTER(_H2Options), ctypes.POINTER(_H2Info)]
    lib.rte_h2_dense.argtypes = [P, I, ctypes.POINTER(D), ctypes.c_size_t]
    lib.rte_h2_destroy.argtypes = [P]
    lib.rte_h2_destroy.restype = V
    lib.rte_last_error.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ('rte_destroy', 'rte_last_error', 'rte_kernel_launches',
                        'rte_estimate_bytes', 'rte_server_destroy', 'rte_h2_destroy'):
            getattr(lib, name).restype = I
    _lib = lib
    return lib


def kernel_launches():
    """Kernels launched by librte in this process so far."""
    return int(load().rte_kernel_launches())


def set_wait_limit(seconds):
    """Limit of every device-side wait of the library (rte_set_wait_limit):
    a wait that runs out makes the call return RTE_ERR_TIMEOUT."""
    _check(load().rte_set_wait_limit(float(seconds)))


def barrier_selftest(blocks, skip_block=-1, rounds=4, stream=None):
    """(status, timed_out, passed_blocks) of rte_barrier_selftest: a
    cooperative launch whose block skip_block never reaches the barrier."""
    import torch
    lib = load()
    st = stream if stream is not None else torch.cuda.current_stream()
    to, ok = ctypes.c_int(-1), ctypes.c_int(-1)
    rc = lib.rte_barrier_selftest(int(blocks), int(skip_block), int(rounds),
                                  ctypes.c_void_p(st.cuda_stream), ctypes.byref(to),
                                  ctypes.byref(ok))
    if rc not in (0, 5):
        _check(rc)
    return rc, to.value, ok.value


def gemm_lowp(A, Bt, out_bf16=False, stream=None):
    """C = A @ Bt.T on the tensor cores (A: M x K, Bt: N x K, both bfloat16
    or both float32 read as TF32; FP32 accumulation)."""
    import torch
    load()
    bf16 = A.dtype == torch.bfloat16
    if Bt.dtype != A.dtype or A.dtype not in (torch.bfloat16, torch.float32):
        raise ValueError('A and Bt must both be bfloat16 or both float32')
    M, K = A.shape
    N = Bt.shape[0]
    C = torch.empty((M, N), device=A.device,
                    dtype=torch.bfloat16 if (bf16 and out_bf16) else torch.float32)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(_lib.rte_gemm_lowp(_ptr(A.contiguous()), _ptr(Bt.contiguous()), _ptr(C), M, N,
                              K, int(bf16), int(out_bf16), ctypes.c_void_p(st.cuda_stream)))
    return C


def _split_operands(A, Bt):
    """Checks the operands of the split GEMMs before any library call: both
    2-D float64 tensors on one CUDA device with the same K."""
    import torch
    for name, t in (('A', A), ('Bt', Bt)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
                and t.dim() == 2):
            raise ValueError('%s must be a 2-D float64 CUDA tensor' % name)
    if A.device != Bt.device:
        raise ValueError('A and Bt must be on the same CUDA device')
    if A.shape[1] != Bt.shape[1]:
        raise ValueError('A is %s and Bt is %s: their K differ' % (tuple(A.shape),
                                                                    tuple(Bt.shape)))
    return A.contiguous(), Bt.contiguous()


def dgemm_split(A, Bt, slices=7, stream=None):
    """C = A @ Bt.T for float64 CUDA tensors by the exact BF16 digit-slice
    tensor-core GEMM."""
    import torch
    load()
    A, Bt = _split_operands(A, Bt)
    M, K = A.shape
    N = Bt.shape[0]
    C = torch.empty((M, N), device=A.device, dtype=torch.float64)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(_lib.rte_dgemm_split(_ptr(A), _ptr(Bt), _ptr(C), M, N, K, slices,
                                ctypes.c_void_p(st.cuda_stream)))
    return C


def autotune_report():
    """{kernel shape: (chosen candidate, [ms per candidate])} of the launch
    shapes the autotuner timed in this process."""
    load()
    n = _lib.rte_autotune_report(None, 0)
    buf = ctypes.create_string_buffer(n + 1)
    _lib.rte_autotune_report(buf, n + 1)
    out = {}
    for item in buf.value.decode().split(';'):
        if ' (ms' not in item:
            continue
        head, ms = item.rsplit(' (ms', 1)
        key, choice = head.rsplit('=', 1)
        out[key] = (int(choice), [float(v) for v in ms.strip(' )').split()])
    return out


def dgemm_split_static(A, Bt, slices=7, out=None, stream=None):
    """C = A @ Bt.T like dgemm_split, through the allocation-free entry point
    (temporaries in the library's fixed 32 MiB device scratch; calls must not
    overlap in time on one device).  Pass `out` (M x N float64, contiguous)
    so that nothing is allocated on this path at all."""
    import torch
    load()
    A, Bt = _split_operands(A, Bt)
    M, K = A.shape
    N = Bt.shape[0]
    if out is not None:
        if not (isinstance(out, torch.Tensor) and out.dtype == torch.float64
                and out.device == A.device and out.is_contiguous()
                and tuple(out.shape) == (M, N)):
            raise ValueError('out must be a contiguous float64 tensor of shape (%d, %d) on %s'
                             % (M, N, A.device))
    C = out if out is not None else torch.empty((M, N), device=A.device, dtype=torch.float64)
    st = stream if stream is not None else torch.cuda.current_stream()
    _check(_lib.rte_dgemm_split_static(_ptr(A), _ptr(Bt), _ptr(C), M, N, K, slices,
                                       ctypes.c_void_p(st.cuda_stream)))
    return C


def _check(rc):
    if rc != 0:
        raise RteError(rc, _lib.rte_last_error().decode())


def default_options(**kw):
    lib = load()
    o = _Options()
    _check(lib.rte_default_options(ctypes.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def _problem_struct(problem):
    import numpy as np
    st = np.ascontiguousarray(problem.sigma_t, dtype=np.float64)
    ss = np.ascontiguousarray(problem.sigma_s, dtype=np.float64)
    pr = _Problem(int(problem.m), int(problem.levels),
                  st.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                  ss.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(problem.g))
    return pr, (st, ss)


def estimate_bytes(problem, nrhs=1, **options):
    lib = load()
    pr, keep = _problem_struct(problem)
    o = default_options(**options)
    return int(lib.rte_estimate_bytes(ctypes.byref(pr), ctypes.byref(o), nrhs))


class Server:
    """Continuous-batching solve server on the current CUDA device (see
    rte_server_* in rte.h): requests are admitted in arrival order as worker
    slots and the HBM budget free up; their device work overlaps."""

    def __init__(self, hbm_budget_bytes, slots=4, **options):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError('librte needs a CUDA device; there is no CPU path')
        lib = load()
        self.options = default_options(**options)
        h = ctypes.c_void_p()
        _check(lib.rte_server_create(int(hbm_budget_bytes), int(slots),
                                     ctypes.byref(self.options), ctypes.byref(h)))
        self._h = h
        self._shapes = {}

    def submit(self, problem, q_nodal, tol=1e-6):
        """Queue a solve; q_nodal: host array (nrhs, (m+1)^2).  Returns an id."""
        import numpy as np
        q = np.ascontiguousarray(np.atleast_2d(q_nodal), dtype=np.float64)
        pr, keep = _problem_struct(problem)
        rid = ctypes.c_longlong()
        _check(_lib.rte_server_submit(self._h, ctypes.byref(pr),
                                      q.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                      q.shape[0], float(tol), ctypes.byref(rid)))
        self._shapes[rid.value] = (q.shape[0], (problem.m + 1) ** 2, 4 * 4 ** problem.levels)
        return rid.value

    def wait(self, rid, timeout=-1.0):
        """Wait for a request; returns (u, info) with u of shape
        (nrhs, n_R^+, n_S^+) and info holding stats and latency."""
        import numpy as np
        shape = self._shapes.pop(rid)
        u = np.empty(shape, dtype=np.float64)
        st = _Stats()
        lat, que = ctypes.c_double(), ctypes.c_double()
        rc = _lib.rte_server_wait(self._h, ctypes.c_longlong(rid), float(timeout),
                                  u.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), u.size,
                                  ctypes.byref(st), ctypes.byref(lat), ctypes.byref(que))
        if rc == 5:   # still running: keep the shape for the next wait
            self._shapes[rid] = shape
        _check(rc)
        return u, dict(iterations=st.iterations, rel_residual=st.rel_residual,
                       latency=lat.value, queue=que.value, seconds=st.seconds)

    def cache_stats(self):
        """(hits, misses, idle bytes) of the server's operator cache."""
        h, m, b = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_size_t()
        _check(_lib.rte_server_cache_stats(self._h, ctypes.byref(h), ctypes.byref(m),
                                           ctypes.byref(b)))
        return h.value, m.value, b.value

    def close(self):
        if getattr(self, '_h', None):
            _lib.rte_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def h2_plan_info(levels, eta=1.4, p=4):
    """Block counts of the H^2 compression for the sphere of 8 * 4^levels
    triangles, from the library's host plan alone (no GPU needed)."""
    lib = load()
    o = _H2Options()
    _check(lib.rte_h2_default_options(ctypes.byref(o)))
    o.levels, o.eta, o.p = int(levels), float(eta), int(p)
    inf = _H2Info()
    _check(lib.rte_h2_plan_info(ctypes.byref(o), ctypes.byref(inf)))
    return dict(n_plus=inf.n_plus, leaves=inf.leaves, clusters=inf.clusters,
                far_blocks=tuple(inf.far_blocks), near_blocks=tuple(inf.near_blocks),
                near_matrices=inf.near_matrices, transfers=inf.transfers)


class H2Scattering:
    """H^2-compressed S^+ and S^- (rte_h2_*) on the current CUDA device.

    levels: sphere refinement (n_S^+ = 4 * 4^levels, levels >= 3); g: HG
    asymmetry; eta, p: admissibility parameter and interpolation points per
    coordinate (defaults: the paper's 1.4 and 4); parities: 1 (S^+), 2 (S^-)
    or 3; precisions: a mask of 1 (FP64 apply), 2 (FP32) and 4 (BF16 on the
    tensor cores).
    """

    def __init__(self, levels, g, eta=1.4, p=4, parities=3, precisions=7, stream=None):
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError('librte needs a CUDA device; there is no CPU path')
        lib = load()
        o = _H2Options()
        _check(lib.rte_h2_default_options(ctypes.byref(o)))
        o.levels, o.g, o.eta, o.p = int(levels), float(g), float(eta), int(p)
        o.parities, o.precisions = int(parities), int(precisions)
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(lib.rte_h2_create(ctypes.byref(o), ctypes.c_void_p(self.stream.cuda_stream),
                                 ctypes.byref(h)))
        self._h = h
        self.n_plus = self.info()['n_plus']

    def info(self):
        inf = _H2Info()
        _check(_lib.rte_h2_get_info(self._h, ctypes.byref(inf)))
        return dict(n_plus=inf.n_plus, leaves=inf.leaves, clusters=inf.clusters,
                    far_blocks=tuple(inf.far_blocks), near_blocks=tuple(inf.near_blocks),
                    near_matrices=inf.near_matrices, transfers=inf.transfers, bytes=inf.bytes,
                    setup_ms=inf.setup_ms)

    def apply(self, X, parity=1, precision=FP64, out=None):
        """Y = X S^+ (parity +1) or X S^- (parity -1); X: float64 CUDA tensor
        (rows, n) with n = n_S^+ or 3 n_S^+."""
        torch = self.torch
        n = self.n_plus * (1 if parity > 0 else 3)
        if X.dtype != torch.float64 or not X.is_cuda or X.dim() != 2 or X.shape[1] != n:
            raise ValueError('X must be a float64 CUDA tensor of shape (rows, %d)' % n)
        X = X.contiguous()
        Y = out if out is not None else torch.empty_like(X)
        _check(_lib.rte_h2_apply(self._h, int(parity), int(precision), _ptr(X), _ptr(Y),
                                 int(X.shape[0]), ctypes.c_void_p(self.stream.cuda_stream)))
        return Y

    def dense(self, parity=1):
        """The dense S^+ or S^- by the library's quadrature (levels <= 5)."""
        import numpy as np
        n = self.n_plus * (1 if parity > 0 else 3)
        out = np.empty((n, n))
        _check(_lib.rte_h2_dense(self._h, int(parity),
                                 out.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), out.size))
        return out

    def close(self):
        if getattr(self, '_h', None):
            self.stream.synchronize()
            _lib.rte_h2_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """One assembled problem on the current CUDA device.

    problem: an object with m, levels, g, sigma_t, sigma_s (e.g.
    ``workloads.Problem``); options: keyword overrides of rte_options.
    """

    def __init__(self, problem, stream=None, **options):
        import numpy as np
        import torch
        if not torch.cuda.is_available():
            raise RuntimeError('librte needs a CUDA device; there is no CPU path')
        lib = load()
        self.torch = torch
        self._st = np.ascontiguousarray(problem.sigma_t, dtype=np.float64)
        self._ss = np.ascontiguousarray(problem.sigma_s, dtype=np.float64)
        pr = _Problem(int(problem.m), int(problem.levels),
                      self._st.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      self._ss.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                      float(problem.g))
        self.options = default_options(**options)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(lib.rte_setup(ctypes.byref(pr), ctypes.byref(self.options),
                             ctypes.c_void_p(self.stream.cuda_stream),
                             ctypes.byref(h)))
        self._h = h
        vals = [ctypes.c_int() for _ in range(6)]
        _check(lib.rte_sizes(h, *[ctypes.byref(v) for v in vals]))
        (self.n_nodes, self.n_cells, self.n_dirs, self.n_odd, self.d_plus,
         self.d_minus) = [v.value for v in vals]

    # ------------------------------------------------------------ shapes
    def even(self, nrhs=1):
        return self.torch.zeros((nrhs, self.n_nodes, self.n_dirs),
                                dtype=self.torch.float64, device='cuda')

    def odd_zeros(self, nrhs=1):
        # (odd(), below, recovers the odd part of a solution)
        return self.torch.zeros((nrhs, self.n_cells, self.n_odd),
                                dtype=self.torch.float64, device='cuda')

    def coarse(self, nrhs=1):
        return self.torch.zeros((nrhs, self.n_nodes, self.d_plus),
                                dtype=self.torch.float64, device='cuda')

    def _vec(self, t):
        if not (t.is_cuda and t.dtype == self.torch.float64 and t.is_contiguous()):
            raise ValueError('expected a contiguous float64 CUDA tensor')
        return _ptr(t)

    # --------------------------------------------------------------- ABI
    def rhs(self, q_nodal, out=None):
        q_nodal = q_nodal.reshape(-1, self.n_nodes)
        nrhs = q_nodal.shape[0]
        out = self.even(nrhs) if out is None else out
        _check(_lib.rte_rhs(self._h, self._vec(q_nodal), self._vec(out), nrhs))
        return out

    def inflow(self, g, q):
        """q += the inflow part of l^+ for data g of shape
        (nrhs, 4, m + 1, 2 n_S^+) (rte_inflow: faces x = 0, x = 1, y = 0,
        y = 1; nodes along each face; entry 2k on K_k, 2k + 1 on -K_k)."""
        m = int(round(self.n_nodes ** 0.5)) - 1
        nrhs = q.shape[0]
        if tuple(g.shape) != (nrhs, 4, m + 1, 2 * self.n_dirs):
            raise ValueError('inflow data must have shape (nrhs, 4, m + 1, 2 n_S^+)')
        _check(_lib.rte_inflow(self._h, self._vec(g), self._vec(q), nrhs))
        return q

    def apply(self, x, out=None):
        out = self.torch.empty_like(x) if out is None else out
        _check(_lib.rte_apply(self._h, self._vec(x), self._vec(out), x.shape[0]))
        return out

    def precond(self, r, with_p2=True, out=None):
        out = self.torch.empty_like(r) if out is None else out
        _check(_lib.rte_precond(self._h, self._vec(r), self._vec(out),
                                r.shape[0], int(with_p2)))
        return out

    def solve(self, q, u=None, tol=1e-8, history=256):
        u = self.torch.zeros_like(q) if u is None else u
        hist = (ctypes.c_double * history)()
        st = _Stats()
        st.history = ctypes.cast(hist, ctypes.POINTER(ctypes.c_double))
        st.history_cap = history
        rc = _lib.rte_solve(self._h, self._vec(q), self._vec(u), q.shape[0],
                            float(tol), ctypes.byref(st))
        info = dict(iterations=st.iterations, rel_residual=st.rel_residual,
                    energy_update=st.energy_update,
                    e0_iters=st.e0_iters_last,
                    coarse_iters=st.coarse_iters_last,
                    mk_iters=st.mk_iters_last, seconds=st.seconds,
                    e0_launches=st.e0_launches, e0_vcycles=st.e0_vcycles,
                    e0_active_vcycles=st.e0_active_vcycles,
                    history=list(hist[:min(history, st.iterations + 1)]),
                    status=rc)
        if rc not in (0, 4):
            _check(rc)
        return u, info

    def operator(self, name, x, out):
        _check(_lib.rte_operator(self._h, OPS[name], self._vec(x),
                                 self._vec(out), x.shape[0]))
        return out

    def odd(self, u_plus, l_minus=None):
        """u^- = (M^- - K^-)^{-1} (l^- - A u^+), the odd part of the solution
        (rte_odd); l_minus None means l^- = 0."""
        import torch
        nrhs = u_plus.shape[0]
        out = torch.empty((nrhs, self.n_cells, self.n_odd), dtype=torch.float64,
                          device=u_plus.device)
        lm = self._vec(l_minus) if l_minus is not None else None
        _check(_lib.rte_odd(self._h, self._vec(u_plus), lm, self._vec(out), nrhs))
        return out

    def rates(self, maxit=300, tol=1e-9, seed=1, rho=True, eta=True):
        """(rho, eta, steps): power-iteration estimates of the spectral radius
        and the energy norm of Algorithm 3's iteration matrix (rte_rates)."""
        r, e, it = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_int(0)
        _check(_lib.rte_rates(self._h, maxit, tol, seed, ctypes.byref(r) if rho else None,
                              ctypes.byref(e) if eta else None, ctypes.byref(it)))
        return (r.value if rho else None), (e.value if eta else None), it.value

    def export(self, name):
        """Host copy of an assembled matrix (see rte_export in rte.h)."""
        import numpy as np
        n, nm, dp = self.n_dirs, self.n_odd, self.d_plus
        size = dict(Splus=n * n, Sminus=nm * nm, m=n, MSm=9 * n, A1=3 * n,
                    A2=3 * n, omx=n, omy=n, lamP=n, lamM=nm, WpN=n * max(dp, 1))
        if name == 'Ec':
            count = 1
            while True:   # E_c block count is the stencil size: grow to fit
                buf = np.zeros(count * dp * dp, dtype=np.float64)
                rc = _lib.rte_export(self._h, EXPORTS[name],
                                     buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                     buf.size)
                if rc == 0:
                    return buf[:self._ec_blocks() * dp * dp]
                count *= 2
        buf = np.zeros(size[name], dtype=np.float64)
        _check(_lib.rte_export(self._h, EXPORTS[name],
                               buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                               buf.size))
        return buf

    def _ec_blocks(self):
        m = int(round(self.n_nodes ** 0.5)) - 1
        # 7-point stencil of the "/"-triangulation: (m+1)^2 diagonal entries,
        # 3 m (m+1) horizontal/vertical edge pairs and m^2 diagonal edges
        return (m + 1) ** 2 + 2 * (2 * m * (m + 1) + m * m)

    def timing(self, on=True):
        _check(_lib.rte_timing_enable(self._h, int(on)))

    def timing_read(self, cap=64):
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_double * cap)()
        cnt = (ctypes.c_longlong * cap)()
        n = ctypes.c_int()
        _check(_lib.rte_timing_read(self._h, names, ms, cnt, cap,
                                    ctypes.byref(n)))
        return {names[i].decode(): (ms[i], cnt[i]) for i in range(min(n.value, cap))}

    def setup_times(self):
        """{stage: wall-clock ms} of the setup that made this solver
        (rte_setup_times)."""
        cap = 32
        names = (ctypes.c_char_p * cap)()
        ms = (ctypes.c_double * cap)()
        n = ctypes.c_int()
        _check(_lib.rte_setup_times(self._h, names, ms, cap, ctypes.byref(n)))
        return {names[i].decode(): ms[i] for i in range(min(n.value, cap))}

    def trace(self, on=True):
        """Record per-barrier phase times of the next persistent solves."""
        _check(_lib.rte_trace_enable(self._h, int(on)))

    def trace_read(self, cap=65536):
        buf = (ctypes.c_double * cap)()
        n = ctypes.c_int()
        _check(_lib.rte_trace_read(self._h, buf, cap, ctypes.byref(n)))
        return list(buf[:min(n.value, cap)])

    def close(self):
        if getattr(self, '_h', None):
            _lib.rte_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
