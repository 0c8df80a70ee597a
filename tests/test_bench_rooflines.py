"""Host-side roofline arithmetic of the benchmark line: the algorithmic work
per launch of each timing scope against the measured peak of its bound, on
the benchmark's sizes (128 x 128 mesh, 512 triangles, d^+ = 15)."""
import math

import pytest

D = dict(nRp=129 * 129, nRm=2 * 128 * 128, nSp=256, nSm=768, e0_levels=5, mesh=128, dP=15)
PEAKS = dict(hbm_gbs=6689.8, bf16_tflops=1957.5)
INFO = dict(coarse_iters=5, e0_launches=32, e0_active_vcycles=32.0, e0_iters=1)


def _roof(name, total_ms, launches, tol=1e-6):
    import bench
    return bench.roofline_of(name, total_ms, launches, D, 1, INFO, PEAKS, 'measured',
                             lambda: 1.10, tol)


def test_split_slices_follow_the_tolerance():
    import bench
    # S 2^-7S <= tol / 1000, at least 3, at most the 7 slices set up
    assert bench.split_slices_for(1e-6) == 5
    assert bench.split_slices_for(1e-8) == 6
    assert bench.split_slices_for(1e-10) == 7
    assert bench.split_slices_for(1e-2) == 3
    assert bench.split_slices_for(1e-14) == 7


def test_split_gemm_scope_counts_the_slice_pair_products():
    # 15 pair products of 2 M N K at 5 slices; 1.06 ms per launch
    r = _roof('dgemm_split_mk1', 17 * 1.06, 17)
    flops = 15 * 2.0 * 32768 * 768 * 768
    assert r['bound'] == 'tensor' and r['unit'] == 'TFLOP/s'
    assert r['algorithmic_flops'] == pytest.approx(flops)
    assert r['achieved'] == pytest.approx(flops / 1.06e-3 / 1e12)
    assert r['frac'] == pytest.approx(r['achieved'] / 1957.5)
    assert 0.2 < r['frac'] < 0.4
    kp = _roof('dgemm_split_kplus', 17 * 0.1, 17)
    assert kp['algorithmic_flops'] == pytest.approx(15 * 2.0 * 16641 * 256 * 256)
    # without a tolerance the slice count is unknown: no roofline claimed
    assert _roof('dgemm_split_mk2', 1.0, 1, tol=None)['frac'] is None


def test_memory_bound_scopes_divide_algorithmic_bytes_by_time():
    r = _roof('coarse_cg', 16 * 2.4263, 16)
    per_it = 8 * (5 * 15 * D['nRp'] + 7 * 15 * 15 * D['nRp'])
    assert r['bound'] == 'hbm' and r['unit'] == 'GB/s'
    assert r['algorithmic_bytes'] == pytest.approx(5 * per_it)
    assert r['frac'] == pytest.approx(5 * per_it / 2.4263e-3 / 1e9 / 6689.8)
    e0 = _roof('e0_direct', 32 * 1.07, 32)
    b = 129
    alg = 2.0 * 256 * b ** 3 * 4 + 16.0 * D['nRp'] * 256
    assert e0['algorithmic_bytes'] == pytest.approx(alg)
    assert e0['frac'] == pytest.approx(alg / 1.07e-3 / 1e9 / 6689.8)
    assert 0.55 < e0['frac'] < 0.7
    assert e0['impl_bytes'] > alg


def test_fp64_scopes_use_the_measured_fp64_rate_and_unknown_scopes_stay_empty():
    r = _roof('gemm_mk_eig1', 10.0, 10)
    assert r['bound'] == 'alu' and r['peak'] == 1.10
    assert r['frac'] == pytest.approx(2.0 * 32768 * 768 * 768 / 1e-3 / 1e12 / 1.10)
    empty = _roof('axpy', 3.0, 100)
    assert empty['frac'] is None and empty['avg_ms'] == pytest.approx(0.03)
    assert not math.isnan(empty['avg_ms'])


def test_scope_rooflines_rank_the_timing_scopes():
    import bench
    # total ms and launches of one benchmark solve as the library's timing
    # scopes report them
    tim = {'coarse_cg': (38.8, 16), 'e0_direct': (34.4, 32), 'dgemm_split_mk1': (18.0, 17),
           'dgemm_split_mk2': (15.1, 17), 'apply_even': (11.0, 17), 'axpy': (5.1, 113),
           'tc_gemm_mk1': (7.5, 48)}
    roof, rows = bench.scope_rooflines(tim, D, 1, INFO, PEAKS, 'measured', lambda: 1.10, 1e-6)
    assert roof['kernel'] == 'coarse_cg' and roof['bound'] == 'hbm'
    assert [r['kernel'] for r in rows] == ['coarse_cg', 'e0_direct', 'dgemm_split_mk1',
                                           'dgemm_split_mk2']
    assert [r['bound'] for r in rows] == ['hbm', 'hbm', 'tensor', 'tensor']
    assert all(0 < r['frac'] < 1 for r in rows)
    assert rows[0] == roof
