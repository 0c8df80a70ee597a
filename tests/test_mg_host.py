"""Host logic of the library's multigrid hierarchy (csrc/mg_host.cpp), on the
CPU: the product's own C++ compiled with g++ into a small driver.

For even and odd meshes, and for scalar and block (bs = 3) operators with
several slots, the driver prints the prolongation, the restriction lists and
the operators of consecutive levels; the test checks that the prolongation
reproduces constants, that the restriction lists are its transpose, that
every coarse operator equals the Galerkin product P^T A P of the finer one
(dense, in NumPy), that the dense coarsest matrix is the slot-weighted sum,
and that the 7-point ELL form holds on every level.
"""
import os
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, 'paper_2102_09038_gb300', 'csrc')
CUDA_INC = '/usr/local/cuda/include'

DRIVER = r'''
#include <cstdio>
#include <random>
#include <string>
#include "mg_host.h"
namespace rte {
int fail(int c, const std::string& m) { std::fprintf(stderr, "%s\n", m.c_str()); return c; }
}
using namespace rte;
int main(int argc, char** argv) {
    const int m = std::atoi(argv[1]), slots = std::atoi(argv[2]), bs = std::atoi(argv[3]);
    const int maxc = std::atoi(argv[4]);
    Stencil st = stencil_of_square(m);
    const int n = (m + 1) * (m + 1), nnz = (int)st.col.size(), bb = bs * bs;
    // symmetric values on the pattern: v(i,j) block = transpose of v(j,i)
    std::mt19937_64 rng(7);
    std::uniform_real_distribution<double> U(-1.0, 1.0);
    std::vector<double> v((size_t)slots * nnz * bb);
    for (auto& x : v) x = U(rng);
    for (int s = 0; s < slots; ++s)
        for (int i = 0; i < n; ++i)
            for (int p = st.ptr[i]; p < st.ptr[i + 1]; ++p) {
                const int j = st.col[p];
                if (j < i) continue;
                int q = st.ptr[j];
                while (st.col[q] != i) ++q;
                for (int a = 0; a < bs; ++a)
                    for (int b = 0; b < bs; ++b) {
                        double& x = v[((size_t)s * nnz + p) * bb + a * bs + b];
                        if (j == i && b < a) x = v[((size_t)s * nnz + p) * bb + b * bs + a];
                        if (j != i) v[((size_t)s * nnz + q) * bb + b * bs + a] = x;
                    }
                if (j == i)
                    for (int a = 0; a < bs; ++a) v[((size_t)s * nnz + p) * bb + a * bs + a] += 8.0;
            }
    MGHost mh;
    if (build_hierarchy(m, st, v, slots, bs, maxc, mh)) return 2;
    std::printf("levels %zu coarse_nodes %d dense %d\n", mh.levels.size(), mh.coarse_nodes,
                (int)mh.dense_coarse);
    for (size_t l = 0; l < mh.levels.size(); ++l) {
        const MGHostLevel& L = mh.levels[l];
        const int nl = (L.m + 1) * (L.m + 1);
        std::printf("level %zu m %d n %d nnz %zu\n", l, L.m, nl, L.st.col.size());
        for (int i = 0; i < nl; ++i)
            for (int p = L.st.ptr[i]; p < L.st.ptr[i + 1]; ++p)
                for (int s = 0; s < slots; ++s)
                    for (int t = 0; t < bb; ++t)
                        std::printf("A %zu %d %d %d %d %.17g\n", l, s, i, L.st.col[p], t,
                                    L.vals[((size_t)s * L.st.col.size() + p) * bb + t]);
        if (!L.p0.empty()) {
            for (int i = 0; i < nl; ++i) {
                std::printf("P %zu %d %d %.17g\n", l, i, L.p0[i], (double)L.w0[i]);
                if (L.p1[i] >= 0) std::printf("P %zu %d %d %.17g\n", l, i, L.p1[i], (double)L.w1[i]);
            }
            const int nc = (int)L.rptr.size() - 1;
            for (int I = 0; I < nc; ++I)
                for (int k = L.rptr[I]; k < L.rptr[I + 1]; ++k)
                    std::printf("R %zu %d %d %.17g\n", l, I, L.ridx[k], (double)L.rw[k]);
        }
        std::vector<double> ell;
        std::printf("ell %zu %d\n", l, to_ell(L, slots, bs, ell));
        std::vector<float> dinv;
        if (block_diag_inverse(L, bs, dinv) == 0)
            for (size_t k = 0; k < dinv.size(); ++k) std::printf("I %zu %zu %.9g\n", l, k, (double)dinv[k]);
    }
    std::vector<double> wts(slots);
    for (int s = 0; s < slots; ++s) wts[s] = 1.0 + s;
    std::vector<double> D;
    coarse_dense_matrix(mh.levels.back(), wts, slots, bs, D);
    for (size_t k = 0; k < D.size(); ++k) std::printf("D %zu %.17g\n", k, D[k]);
    return 0;
}
'''


@pytest.fixture(scope='module')
def driver(tmp_path_factory):
    if not os.path.isdir(CUDA_INC):
        pytest.skip('CUDA headers not found')
    d = tmp_path_factory.mktemp('mg_host')
    src = d / 'drv.cpp'
    src.write_text(DRIVER)
    exe = d / 'drv'
    subprocess.run(['g++', '-std=c++17', '-O1', '-I', CSRC, '-I', CUDA_INC,
                    os.path.join(CSRC, 'mg_host.cpp'), os.path.join(CSRC, 'setup_host.cpp'),
                    str(src), '-o', str(exe)], check=True, capture_output=True)
    return str(exe)


def run(exe, m, slots, bs, maxc):
    out = subprocess.run([exe, str(m), str(slots), str(bs), str(maxc)], capture_output=True,
                         text=True, check=True).stdout.splitlines()
    info = dict(levels=[], A={}, P={}, R={}, ell={}, D=[], I={})
    for ln in out:
        t = ln.split()
        if t[0] == 'levels':
            info['nlev'], info['coarse_nodes'], info['dense'] = int(t[1]), int(t[3]), int(t[5])
        elif t[0] == 'level':
            info['levels'].append((int(t[3]), int(t[5])))
        elif t[0] == 'A':
            info['A'].setdefault(int(t[1]), []).append(
                (int(t[2]), int(t[3]), int(t[4]), int(t[5]), float(t[6])))
        elif t[0] in ('P', 'R'):
            info[t[0]].setdefault(int(t[1]), []).append((int(t[2]), int(t[3]), float(t[4])))
        elif t[0] == 'ell':
            info['ell'][int(t[1])] = int(t[2])
        elif t[0] == 'D':
            info['D'].append(float(t[2]))
        elif t[0] == 'I':
            info['I'].setdefault(int(t[1]), []).append(float(t[3]))
    return info


def dense(entries, n, slots, bs):
    A = np.zeros((slots, n * bs, n * bs))
    for s, i, j, t, v in entries:
        A[s, i * bs + t // bs, j * bs + t % bs] = v
    return A


@pytest.mark.parametrize('m, slots, bs, maxc', [(8, 2, 1, 30), (9, 2, 1, 30), (35, 1, 1, 100),
                                                (7, 1, 3, 20), (12, 3, 1, 30)])
def test_hierarchy_is_galerkin(driver, m, slots, bs, maxc):
    info = run(driver, m, slots, bs, maxc)
    levels = info['levels']
    assert levels[0][0] == m
    for (mf, nf), (mc, nc) in zip(levels, levels[1:]):
        assert mc == mf // 2 and nf == (mf + 1) ** 2 and nc == (mc + 1) ** 2
    mlast, nlast = levels[-1]
    # coarsening stops at <= maxc nodes (or a mesh too small to halve)
    assert nlast <= maxc or mlast < 4
    assert info['dense'] == int(nlast <= maxc)
    for l in range(len(levels) - 1):
        nf, nc = levels[l][1], levels[l + 1][1]
        P = np.zeros((nf, nc))
        for i, c, w in info['P'][l]:
            P[i, c] += w
        # constants are reproduced: every row of P sums to one
        assert np.abs(P.sum(1) - 1.0).max() < 1e-6
        # linear interpolation on the nested coarse mesh: a linear function
        # of the node indices is reproduced, the last fine column and row of
        # an odd mesh taking the values of the ones before them
        mf, mc = levels[l][0], levels[l + 1][0]
        xf, yf = np.arange(nf) % (mf + 1), np.arange(nf) // (mf + 1)
        xc, yc = np.arange(nc) % (mc + 1), np.arange(nc) // (mc + 1)
        lin = lambda x, y: 0.3 + 1.7 * x - 0.9 * y
        want = lin(np.minimum(xf, 2 * mc), np.minimum(yf, 2 * mc))
        assert np.abs(P @ lin(2 * xc, 2 * yc) - want).max() < 1e-5 * np.abs(want).max()
        R = np.zeros((nc, nf))
        for I, i, w in info['R'][l]:
            R[I, i] += w
        assert np.array_equal(R, P.T)
        Pk = np.kron(P, np.eye(bs))
        Af = dense(info['A'][l], nf, slots, bs)
        Ac = dense(info['A'][l + 1], nc, slots, bs)
        for s in range(slots):
            G = Pk.T @ Af[s] @ Pk
            assert np.abs(Ac[s] - G).max() <= 1e-12 * np.abs(G).max()
            assert np.abs(Ac[s] - Ac[s].T).max() <= 1e-12 * np.abs(Ac[s]).max()
    assert all(v == 0 for v in info['ell'].values())     # 7-point pattern on every level
    # inverses of the diagonal blocks of slot 0 (the block-Jacobi smoother), FP32
    for l, (ml, nl) in enumerate(levels):
        A0 = dense(info['A'][l], nl, slots, bs)[0]
        Dv = np.array(info['I'][l]).reshape(nl, bs, bs)
        for i in range(nl):
            blk = A0[i * bs:(i + 1) * bs, i * bs:(i + 1) * bs]
            assert np.abs(Dv[i] @ blk - np.eye(bs)).max() < 1e-5
    Al = dense(info['A'][len(levels) - 1], nlast, slots, bs)
    D = np.array(info['D']).reshape(nlast * bs, nlast * bs)
    Ws = sum((1.0 + s) * Al[s] for s in range(slots))
    assert np.abs(D - Ws).max() <= 1e-13 * np.abs(Ws).max()
