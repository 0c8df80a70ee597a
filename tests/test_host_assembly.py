"""Host assembly of the library (csrc/setup_host.cpp) against the independent
FP64 oracle, on the CPU: the product's own C++ compiled with g++ into a small
driver that prints what build_host_system hands to the device.

Checked: the spatial stencil slots (sigma_t- and sigma_s-weighted P1 mass,
unit mass, the two boundary masses, the three parts D_n^T (M_t^-)^{-1} D_m)
against the oracle's sparse matrices; the angular vectors (m, omega^x,
omega^y); c and (1 - cg)^{-1}; and every E_0 direction block rebuilt from the
six per-direction weights and the stencil slots against the oracle's E_0
blocks (eq. equivalence_bE_bE0), which fixes the weights' convention.
"""
import os
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

import oracle
import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, 'paper_2102_09038_gb300', 'csrc')
CUDA_INC = '/usr/local/cuda/include'

DRIVER = r'''
#include <cstdio>
#include <string>
#include <vector>
#include "rte_internal.h"
namespace rte {
int fail(int c, const std::string& m) { std::fprintf(stderr, "%s\n", m.c_str()); return c; }
}
using namespace rte;
int main(int argc, char** argv) {
    FILE* f = std::fopen(argv[1], "r");
    int m, levels, nc;
    double g;
    if (std::fscanf(f, "%d %d %lf %d", &m, &levels, &g, &nc) != 4) return 3;
    std::vector<double> st(nc), ss(nc);
    for (auto& v : st) if (std::fscanf(f, "%lf", &v) != 1) return 3;
    for (auto& v : ss) if (std::fscanf(f, "%lf", &v) != 1) return 3;
    std::fclose(f);
    rte_problem p{m, levels, st.data(), ss.data(), g};
    rte_options o;
    o.l = 4; o.n_plus = 2; o.n_minus = 3; o.precision = RTE_FP64;
    HostSystem hs;
    if (build_host_system(p, o, hs)) return 2;
    const int nnz = (int)hs.st.col.size();
    std::printf("sizes %d %d %d %.17g %.17g\n", hs.nRp, hs.nSp, nnz, hs.c, hs.gamma);
    for (int i = 0; i < hs.nRp; ++i)
        for (int q = hs.st.ptr[i]; q < hs.st.ptr[i + 1]; ++q) {
            std::printf("S %d %d", i, hs.st.col[q]);
            for (int s = 0; s < kSlots; ++s) std::printf(" %.17g", hs.sval[(size_t)s * nnz + q]);
            std::printf("\n");
        }
    for (int k = 0; k < hs.nSp; ++k) {
        std::printf("K %.17g %.17g %.17g", hs.m_[k], hs.omx[k], hs.omy[k]);
        for (int q = 0; q < 6; ++q) std::printf(" %.17g", hs.e0s[6 * k + q]);
        std::printf("\n");
    }
    return 0;
}
'''


@pytest.fixture(scope='module')
def driver(tmp_path_factory):
    if not os.path.isdir(CUDA_INC):
        pytest.skip('CUDA headers not found')
    d = tmp_path_factory.mktemp('host_asm')
    src = d / 'drv.cpp'
    src.write_text(DRIVER)
    exe = d / 'drv'
    subprocess.run(['g++', '-std=c++17', '-O1', '-I', CSRC, '-I', CUDA_INC,
                    os.path.join(CSRC, 'setup_host.cpp'), str(src), '-o', str(exe)],
                   check=True, capture_output=True)
    return str(exe), d


def relerr(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize('case', ['checker', 'const'])
def test_host_assembly_matches_oracle(driver, case):
    exe, d = driver
    if case == 'checker':
        p = workloads.checkerboard(m=6, levels=1, g=0.7, ratio=0.9, blocks=2, nrhs=1)
    else:
        p = workloads.constant(5, 2, 0.4, 2.0, 1.1)
    inp = d / ('in_%s.txt' % case)
    with open(inp, 'w') as fh:
        fh.write('%d %d %.17g %d\n' % (p.m, p.levels, p.g, len(p.sigma_t)))
        fh.write(' '.join('%.17g' % v for v in p.sigma_t) + '\n')
        fh.write(' '.join('%.17g' % v for v in p.sigma_s) + '\n')
    out = subprocess.run([exe, str(inp)], capture_output=True, text=True,
                         check=True).stdout.splitlines()
    head = out[0].split()
    nRp, nSp, nnz = int(head[1]), int(head[2]), int(head[3])
    c, gamma = float(head[4]), float(head[5])
    rows = [ln.split() for ln in out if ln.startswith('S ')]
    assert len(rows) == nnz
    ii = np.array([int(r[1]) for r in rows])
    jj = np.array([int(r[2]) for r in rows])
    vals = np.array([[float(v) for v in r[3:]] for r in rows])
    slot = lambda s: sp.csr_matrix((vals[:, s], (ii, jj)), shape=(nRp, nRp)).toarray()
    kk = np.array([[float(v) for v in ln.split()[1:]] for ln in out if ln.startswith('K ')])

    disc = oracle.Discretisation(p.m, p.levels, p.sigma_t, p.sigma_s, p.g)
    ops = oracle.Operators(disc, n_plus=2, n_minus=3)
    sm, an = disc.sp, disc.an
    assert (nRp, nSp) == (disc.nRp, disc.nSp)
    assert abs(c - disc.c) < 1e-15 and abs(gamma - 1.0 / (1.0 - disc.c * disc.g)) < 1e-14
    Minv = sp.diags(1.0 / sm['Mt_minus'])
    K11 = (sm['D1'].T @ Minv @ sm['D1']).toarray()
    K22 = (sm['D2'].T @ Minv @ sm['D2']).toarray()
    K12 = (sm['D1'].T @ Minv @ sm['D2'] + sm['D2'].T @ Minv @ sm['D1']).toarray()
    want = [sm['Mt_plus'].toarray(), sm['Ms_plus'].toarray(), sm['M_plus_unit'].toarray(),
            sm['Bx'].toarray(), sm['By'].toarray(), K11, K12, K22]
    for s, W in enumerate(want):
        assert relerr(slot(s), W) < 1e-13, s
    assert relerr(kk[:, 0], an['m']) < 1e-13
    assert relerr(kk[:, 1], an['omx']) < 1e-13
    assert relerr(kk[:, 2], an['omy']) < 1e-13
    # E_0 direction blocks from the six weights (gamma a11, gamma a12,
    # gamma a22, omega^x, omega^y, m) and the stencil slots
    blocks = ops.e0_blocks()['blocks']
    parts = [slot(5), slot(6), slot(7), slot(3), slot(4), slot(0)]
    for k in range(nSp):
        Ek = sum(kk[k, 3 + q] * parts[q] for q in range(6))
        assert relerr(Ek, blocks[k].toarray()) < 1e-12, k
