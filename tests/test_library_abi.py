"""The C-ABI library builds, loads and exports every symbol that
include/rte.h declares (no GPU needed: no compute calls here)."""
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_2102_09038_gb300 import build
    return build.build()


def declared_symbols():
    src = open(os.path.join(ROOT, 'include', 'rte.h')).read()
    src = re.sub(r'/\*.*?\*/', '', src, flags=re.S)
    return sorted(set(re.findall(r'\b(rte_[a-z_0-9]+)\s*\(', src)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ('rte_setup', 'rte_apply', 'rte_precond', 'rte_solve',
                 'rte_rhs', 'rte_destroy'):
        assert name in syms


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(['nm', '-D', '--defined-only', lib_path],
                         capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r'\sT\s+(rte_\w+)', out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, missing


def test_binding_loads_without_gpu(lib_path):
    import paper_2102_09038_gb300 as rte
    lib = rte.load()
    for name in declared_symbols():
        assert hasattr(lib, name)
    o = rte.default_options()
    # Section 6 defaults; l = 0 resolves per P_1 route at set-up
    assert (o.l, o.n_plus, o.n_minus) == (0, 4, 5)


def test_solver_refuses_without_cuda(lib_path):
    import torch
    import paper_2102_09038_gb300 as rte
    import workloads
    if torch.cuda.is_available():
        pytest.skip('a GPU is present')
    with pytest.raises(RuntimeError):
        rte.Solver(workloads.constant(2, 0, 0.5, 1.0, 0.5))


def test_static_split_gemm_refuses_oversize_operands_on_the_host(lib_path):
    """The allocation-free split GEMM checks its operand sizes against the
    fixed scratch before any CUDA call, so this runs without a GPU (the
    pointers are never dereferenced)."""
    import ctypes
    import paper_2102_09038_gb300 as rte
    lib = rte.load()
    fake = ctypes.c_void_p(256)
    # 2 * 7 * (4096 + 4096) * 4096 bytes of slices, far above 32 MiB
    assert lib.rte_dgemm_split_static(fake, fake, fake, 4096, 4096, 4096, 7, None) == 1
    assert b'scratch' in lib.rte_last_error()
    # sizes whose byte count would overflow 64 bits
    big = 2 ** 31 - 1
    assert lib.rte_dgemm_split_static(fake, fake, fake, big, big, big, 9, None) == 1
    # just above the limit: M = N = 1024, K = 1176 needs 33,718,272 bytes of slices
    assert lib.rte_dgemm_split_static(fake, fake, fake, 1024, 1024, 1176, 7, None) == 1
    assert lib.rte_dgemm_split_static(fake, fake, fake, 1, 1, 1, 0, None) == 1
    # K not a multiple of 8 (16-byte rows of BF16 slices): refused up front,
    # by both split GEMM entry points
    assert lib.rte_dgemm_split_static(fake, fake, fake, 16, 16, 12, 7, None) == 1
    assert b'multiple of 8' in lib.rte_last_error()
    assert lib.rte_dgemm_split(fake, fake, fake, 16, 16, 12, 7, None) == 1
    assert b'multiple of 8' in lib.rte_last_error()


def test_failure_detection_arguments_refused_on_the_host(lib_path):
    """The wait-limit setter and the barrier self-test check their
    arguments before any CUDA call."""
    import paper_2102_09038_gb300 as rte
    lib = rte.load()
    for bad in (0.0, -1.0, 61.0, float('nan')):
        assert lib.rte_set_wait_limit(bad) == 1
    import ctypes
    a, b = ctypes.c_int(), ctypes.c_int()
    assert lib.rte_barrier_selftest(0, -1, 1, None, ctypes.byref(a), ctypes.byref(b)) == 1
    assert lib.rte_barrier_selftest(4, 4, 1, None, ctypes.byref(a), ctypes.byref(b)) == 1
    assert lib.rte_barrier_selftest(4, -1, 0, None, ctypes.byref(a), ctypes.byref(b)) == 1
    assert lib.rte_barrier_selftest(4, -1, 1, None, None, ctypes.byref(b)) == 1


def _c_layout(struct, fields, tmp_path):
    """sizeof and offsetof of a header struct, from a C program gcc builds."""
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "rte.h"',
             'int main(void) {', '  printf("%%zu\\n", sizeof(%s));' % struct]
    lines += ['  printf("%%zu\\n", offsetof(%s, %s));' % (struct, f) for f in fields]
    lines += ['  return 0;', '}']
    src = tmp_path / ('layout_%s.c' % struct)
    src.write_text('\n'.join(lines) + '\n')
    exe = tmp_path / ('layout_%s' % struct)
    subprocess.run(['gcc', '-I', os.path.join(ROOT, 'include'), str(src), '-o', str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout
    vals = [int(v) for v in out.split()]
    return vals[0], vals[1:]


@pytest.mark.parametrize('struct, mirror', [('rte_options', '_Options'),
                                            ('rte_stats', '_Stats'),
                                            ('rte_problem', '_Problem'),
                                            ('rte_h2_options', '_H2Options'),
                                            ('rte_h2_info', '_H2Info')])
def test_binding_structs_match_the_header_layout(struct, mirror, tmp_path):
    # the ctypes mirrors of the binding have the header's field order,
    # offsets and size (a field added on one side only would shift the rest)
    import ctypes
    import paper_2102_09038_gb300 as rte
    cls = getattr(rte, mirror)
    fields = [f[0] for f in cls._fields_]
    size, offs = _c_layout(struct, fields, tmp_path)
    assert ctypes.sizeof(cls) == size
    assert [getattr(cls, f).offset for f in fields] == offs


def test_default_options_through_the_library(lib_path):
    # rte_default_options fills the struct the binding reads back
    import paper_2102_09038_gb300 as rte
    o = rte.default_options()
    assert o.p1_route == rte.P1_AUTO and o.precision == rte.FP64
    assert o.e0_route == rte.E0_AUTO
    assert o.autotune == 1 and o.max_rhs >= 1
    o = rte.default_options(p1_route=rte.P1_PCG, precision=rte.MIXED_BF16)
    assert (o.p1_route, o.precision) == (rte.P1_PCG, rte.MIXED_BF16)


def _setup_rc(problem_kw=None, **opts):
    """rte_setup on arguments it must refuse on the host, before any CUDA
    call (so this runs without a GPU): (return code, error message)."""
    import ctypes
    import numpy as np
    import paper_2102_09038_gb300 as rte
    import workloads
    lib = rte.load()
    kw = dict(m=2, levels=1, g=0.5, sigma_t=1.0, sigma_s=0.5)
    kw.update(problem_kw or {})
    p = workloads.constant(kw['m'], kw['levels'], kw['g'], kw['sigma_t'], kw['sigma_s'])
    pr, keep = rte._problem_struct(p)
    if 'mesh_m' in kw:
        pr.mesh_m = kw['mesh_m']
    if 'sphere_levels' in kw:
        pr.sphere_levels = kw['sphere_levels']
    o = rte.default_options(**opts)
    h = ctypes.c_void_p()
    rc = lib.rte_setup(ctypes.byref(pr), ctypes.byref(o), None, ctypes.byref(h))
    assert not h.value
    return rc, lib.rte_last_error().decode()


@pytest.mark.parametrize('problem_kw, opts, words', [
    (dict(mesh_m=0), {}, 'mesh_m'),
    (dict(sphere_levels=6), {}, 'sphere_levels'),
    (dict(g=1.0), {}, 'g must'),
    (dict(sigma_s=1.0), {}, 'sigma_s < sigma_t'),
    (dict(sigma_t=-1.0, sigma_s=0.0), {}, 'sigma_s < sigma_t'),
    ({}, dict(l=-1), 'invalid options'),
    ({}, dict(n_minus=4), 'invalid options'),
    ({}, dict(n_plus=3), 'invalid options'),
    ({}, dict(max_rhs=0), 'invalid options'),
    ({}, dict(precision=7), 'precision'),
    ({}, dict(p1_route=5), 'P_1 route'),
    ({}, dict(mk_route=3), 'route'),
    ({}, dict(e0_route=7), 'E_0 route'),
    (dict(m=157), dict(e0_route=1), 'mesh_m <= 156'),
    ({}, dict(coarse_route=9), 'coarse route'),
    (dict(m=160), dict(e0_route=2, coarse_route=1), 'd^+ <= 2400'),
    (dict(levels=0), dict(n_plus=4), 'too large'),   # d^+ = 15 > 4 directions
])
def test_setup_refuses_bad_arguments_on_the_host(lib_path, problem_kw, opts, words):
    import paper_2102_09038_gb300 as rte
    rc, msg = _setup_rc(problem_kw, **opts)
    assert rte.ERRORS[rc] == 'RTE_ERR_ARG'
    assert words in msg, msg


def test_memory_estimate_grows_with_the_problem(lib_path):
    # rte_estimate_bytes (host only) drives the server's HBM admission: it
    # grows with the right-hand sides and the mesh, and counts the two extra
    # vectors of the PCG realisation of P_1
    import paper_2102_09038_gb300 as rte
    import workloads
    small = workloads.constant(16, 2, 0.5, 1.0, 0.5)
    big = workloads.constant(32, 2, 0.5, 1.0, 0.5)
    e = lambda p, n=1, **o: rte.estimate_bytes(p, nrhs=n, **o)
    assert 0 < e(small) < e(big)
    assert e(small, 1) < e(small, 4)
    ne = (16 + 1) ** 2 * 64 * 8      # one FP64 even vector
    rich = e(small, precision=rte.MIXED_BF16, p1_route=rte.P1_RICHARDSON)
    pcg = e(small, precision=rte.MIXED_BF16, p1_route=rte.P1_PCG)
    assert pcg - rich == 2 * ne
    assert e(small, precision=rte.MIXED_BF16) == pcg          # the mixed default
    assert e(small, precision=rte.FP64) == e(small, precision=rte.FP64,
                                             p1_route=rte.P1_RICHARDSON)
    # the split GEMM's reciprocal table 1 / (at - lam as) of the eigenbasis
    # route: n_R^- x n_S^- FP64 values, independent of the right-hand sides
    table = 2 * 16 * 16 * 3 * 64 * 8
    split = e(small, precision=rte.FP64, dgemm=rte.DGEMM_SPLIT)
    assert split - e(small, precision=rte.FP64) == table
    assert e(small, precision=rte.FP64, dgemm=rte.DGEMM_SPLIT, mk_route=rte.MK_PCG) == \
        e(small, precision=rte.FP64, mk_route=rte.MK_PCG)


@pytest.mark.parametrize('field, value, words', [
    ('levels', 2, 'levels must be in [3, 8]'),
    ('levels', 9, 'levels must be in [3, 8]'),
    ('g', 1.0, 'g must satisfy'),
    ('eta', 0.0, 'eta must be positive'),
    ('p', 5, 'p must be in [2, 4]'),
    ('parities', 0, 'parities'),
    ('precisions', 8, 'precisions')])
def test_h2_create_refuses_bad_options_on_the_host(lib_path, field, value, words):
    # rte_h2_create checks every option before touching the device
    import ctypes
    import paper_2102_09038_gb300 as rte
    lib = rte.load()
    o = rte._H2Options()
    assert lib.rte_h2_default_options(ctypes.byref(o)) == 0
    assert (o.eta, o.p, o.parities, o.precisions) == (1.4, 4, 3, 7)
    setattr(o, field, value)
    h = ctypes.c_void_p()
    rc = lib.rte_h2_create(ctypes.byref(o), None, ctypes.byref(h))
    assert rte.ERRORS[rc] == 'RTE_ERR_ARG'
    assert words in lib.rte_last_error().decode()
    assert not h.value
