// Geometric multigrid hierarchy on the "/"-triangulations of the unit
// square, used to precondition the conjugate-gradient solves of the E_0
// direction blocks and of the coarse Galerkin system E_c.
//
// Coarse level of an m-mesh: the floor(m/2)-mesh.  For even m, refining the
// coarse mesh by edge midpoints gives exactly the fine mesh, and the
// prolongation is linear interpolation: a fine node that is also a coarse
// node keeps its value, a fine node at the midpoint of a coarse edge
// (horizontal, vertical or the "/" diagonal) takes the mean of the edge's two
// ends.  For odd m the fine nodes of the last column (and row) take the
// values of the column (row) before them, x -> min(x, m - 1): the coarse
// space is then the interpolants on [0, (m-1)/m]^2 extended constantly over
// the last fine cell, and every fine coupling still lands inside the coarse
// 7-point pattern.  Coarse operators are Galerkin products P^T A P of the
// fine ones.
#include <algorithm>
#include <cmath>
#include <set>
#include <vector>

#include "mg_host.h"
#include "rte_internal.h"

namespace rte {

Stencil stencil_of_square(int m) {
    const SquareMesh M = make_square(m);
    std::vector<std::set<int>> nb(M.n_nodes);
    for (int j = 0; j < M.n_cells; ++j)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                nb[M.cell_nodes[3 * j + a]].insert(M.cell_nodes[3 * j + b]);
    Stencil st;
    st.ptr.assign(M.n_nodes + 1, 0);
    st.diag.resize(M.n_nodes);
    for (int i = 0; i < M.n_nodes; ++i) {
        st.ptr[i + 1] = st.ptr[i] + (int)nb[i].size();
        for (int c : nb[i]) {
            if (c == i) st.diag[i] = (int)st.col.size();
            st.col.push_back(c);
        }
    }
    return st;
}

// Prolongation from the floor(m/2)-mesh to the m-mesh: up to two coarse
// nodes per fine node with weights.
static void prolongation(int mf, std::vector<int>& p0, std::vector<int>& p1,
                         std::vector<float>& w0, std::vector<float>& w1) {
    const int mc = mf / 2, nf = (mf + 1) * (mf + 1);
    p0.assign(nf, 0); p1.assign(nf, -1); w0.assign(nf, 0.f); w1.assign(nf, 0.f);
    auto cid = [&](int x, int y) { return y * (mc + 1) + x; };
    for (int yf = 0; yf <= mf; ++yf)
        for (int xf = 0; xf <= mf; ++xf) {
            const int f = yf * (mf + 1) + xf;
            const int x = std::min(xf, 2 * mc), y = std::min(yf, 2 * mc);
            if (x % 2 == 0 && y % 2 == 0) {
                p0[f] = cid(x / 2, y / 2); w0[f] = 1.f;
            } else if (x % 2 == 1 && y % 2 == 0) {        // horizontal edge
                p0[f] = cid((x - 1) / 2, y / 2); p1[f] = cid((x + 1) / 2, y / 2);
                w0[f] = w1[f] = 0.5f;
            } else if (x % 2 == 0 && y % 2 == 1) {        // vertical edge
                p0[f] = cid(x / 2, (y - 1) / 2); p1[f] = cid(x / 2, (y + 1) / 2);
                w0[f] = w1[f] = 0.5f;
            } else {                                      // "/" diagonal
                p0[f] = cid((x - 1) / 2, (y - 1) / 2); p1[f] = cid((x + 1) / 2, (y + 1) / 2);
                w0[f] = w1[f] = 0.5f;
            }
        }
}

static int find_pos(const Stencil& st, int row, int col) {
    const int* b = st.col.data() + st.ptr[row];
    const int* e = st.col.data() + st.ptr[row + 1];
    const int* it = std::lower_bound(b, e, col);
    if (it == e || *it != col) return -1;
    return (int)(it - st.col.data());
}

// A_c = P^T A_f P for `slots` value arrays of bs x bs blocks on the stencils.
static bool galerkin(const Stencil& sf, const Stencil& sc, const std::vector<int>& p0,
                     const std::vector<int>& p1, const std::vector<float>& w0,
                     const std::vector<float>& w1, const std::vector<double>& vf, int slots,
                     int bs, std::vector<double>& vc) {
    const size_t nnzf = sf.col.size(), nnzc = sc.col.size(), bb = (size_t)bs * bs;
    vc.assign((size_t)slots * nnzc * bb, 0.0);
    const int nf = (int)sf.ptr.size() - 1;
    for (int i = 0; i < nf; ++i) {
        const int Ii[2] = {p0[i], p1[i]};
        const double wi[2] = {w0[i], w1[i]};
        for (int q = sf.ptr[i]; q < sf.ptr[i + 1]; ++q) {
            const int j = sf.col[q];
            const int Jj[2] = {p0[j], p1[j]};
            const double wj[2] = {w0[j], w1[j]};
            for (int a = 0; a < 2; ++a) {
                if (Ii[a] < 0) continue;
                for (int b = 0; b < 2; ++b) {
                    if (Jj[b] < 0) continue;
                    const int pos = find_pos(sc, Ii[a], Jj[b]);
                    if (pos < 0) return false;
                    const double w = wi[a] * wj[b];
                    for (int s = 0; s < slots; ++s) {
                        const double* src = &vf[((size_t)s * nnzf + q) * bb];
                        double* dst = &vc[((size_t)s * nnzc + pos) * bb];
                        for (size_t t = 0; t < bb; ++t) dst[t] += w * src[t];
                    }
                }
            }
        }
    }
    return true;
}

static bool invert(int n, std::vector<double>& A) {
    std::vector<double> I((size_t)n * n, 0.0);
    for (int i = 0; i < n; ++i) I[(size_t)i * n + i] = 1.0;
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (std::fabs(A[(size_t)r * n + c]) > std::fabs(A[(size_t)piv * n + c])) piv = r;
        if (!(std::fabs(A[(size_t)piv * n + c]) > 0)) return false;
        if (piv != c)
            for (int k = 0; k < n; ++k) {
                std::swap(A[(size_t)c * n + k], A[(size_t)piv * n + k]);
                std::swap(I[(size_t)c * n + k], I[(size_t)piv * n + k]);
            }
        const double inv = 1.0 / A[(size_t)c * n + c];
        for (int k = 0; k < n; ++k) {
            A[(size_t)c * n + k] *= inv;
            I[(size_t)c * n + k] *= inv;
        }
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            const double f = A[(size_t)r * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < n; ++k) {
                A[(size_t)r * n + k] -= f * A[(size_t)c * n + k];
                I[(size_t)r * n + k] -= f * I[(size_t)c * n + k];
            }
        }
    }
    A.swap(I);
    return true;
}

int build_hierarchy(int m, const Stencil& fine, const std::vector<double>& vals0, int slots,
                    int bs, int max_coarse_nodes, MGHost& out) {
    out.levels.clear();
    out.bs = bs;
    out.slots = slots;
    MGHostLevel L0;
    L0.m = m;
    L0.st = fine;
    L0.vals = vals0;
    out.levels.push_back(std::move(L0));
    // coarsen while the level is not yet small
    while (true) {
        MGHostLevel& f = out.levels.back();
        const int nf = (f.m + 1) * (f.m + 1);
        if (f.m < 4 || nf <= max_coarse_nodes) break;
        MGHostLevel c;
        c.m = f.m / 2;
        c.st = stencil_of_square(c.m);
        prolongation(f.m, f.p0, f.p1, f.w0, f.w1);
        if (!galerkin(f.st, c.st, f.p0, f.p1, f.w0, f.w1, f.vals, slots, bs, c.vals))
            return fail(RTE_ERR_ARG, "Galerkin product left the coarse stencil");
        // restriction = P^T as CSR over coarse nodes
        const int nc = (c.m + 1) * (c.m + 1);
        f.rptr.assign(nc + 1, 0);
        for (int i = 0; i < nf; ++i) {
            f.rptr[f.p0[i] + 1]++;
            if (f.p1[i] >= 0) f.rptr[f.p1[i] + 1]++;
        }
        for (int I = 0; I < nc; ++I) f.rptr[I + 1] += f.rptr[I];
        f.ridx.resize(f.rptr[nc]);
        f.rw.resize(f.rptr[nc]);
        std::vector<int> fill(f.rptr.begin(), f.rptr.end() - 1);
        for (int i = 0; i < nf; ++i) {
            f.ridx[fill[f.p0[i]]] = i;
            f.rw[fill[f.p0[i]]++] = f.w0[i];
            if (f.p1[i] >= 0) {
                f.ridx[fill[f.p1[i]]] = i;
                f.rw[fill[f.p1[i]]++] = f.w1[i];
            }
        }
        out.levels.push_back(std::move(c));
    }
    const MGHostLevel& cl = out.levels.back();
    out.coarse_nodes = (cl.m + 1) * (cl.m + 1);
    out.dense_coarse = out.coarse_nodes <= max_coarse_nodes;
    return RTE_OK;
}

void coarse_dense_matrix(const MGHostLevel& L, const std::vector<double>& weights, int slots,
                         int bs, std::vector<double>& A) {
    const int n = (L.m + 1) * (L.m + 1);
    const int N = n * bs;
    const size_t nnz = L.st.col.size(), bb = (size_t)bs * bs;
    A.assign((size_t)N * N, 0.0);
    for (int i = 0; i < n; ++i)
        for (int q = L.st.ptr[i]; q < L.st.ptr[i + 1]; ++q) {
            const int j = L.st.col[q];
            for (int s = 0; s < slots; ++s) {
                const double w = weights.empty() ? 1.0 : weights[s];
                if (w == 0.0) continue;
                const double* v = &L.vals[((size_t)s * nnz + q) * bb];
                for (int a = 0; a < bs; ++a)
                    for (int b = 0; b < bs; ++b)
                        A[(size_t)(i * bs + a) * N + j * bs + b] += w * v[a * bs + b];
            }
        }
}

int block_diag_inverse(const MGHostLevel& L, int bs, std::vector<float>& dinv) {
    const int n = (L.m + 1) * (L.m + 1);
    const size_t bb = (size_t)bs * bs;
    dinv.assign((size_t)n * bb, 0.f);
    for (int i = 0; i < n; ++i) {
        std::vector<double> A(L.vals.begin() + (size_t)L.st.diag[i] * bb,
                              L.vals.begin() + (size_t)(L.st.diag[i] + 1) * bb);
        if (!invert(bs, A)) return fail(RTE_ERR_ARG, "singular multigrid diagonal block");
        for (size_t t = 0; t < bb; ++t) dinv[(size_t)i * bb + t] = (float)A[t];
    }
    return RTE_OK;
}

int to_ell(const MGHostLevel& L, int slots, int bs, std::vector<double>& out) {
    const int m = L.m, n = (m + 1) * (m + 1);
    const size_t nnz = L.st.col.size(), bb = (size_t)bs * bs;
    out.assign((size_t)slots * 7 * n * bb, 0.0);
    for (int i = 0; i < n; ++i)
        for (int q = L.st.ptr[i]; q < L.st.ptr[i + 1]; ++q) {
            const int off = L.st.col[q] - i;
            int dir = -1;
            if (off == 0) dir = 0;
            else if (off == 1) dir = 1;
            else if (off == -1) dir = 2;
            else if (off == m + 1) dir = 3;
            else if (off == -(m + 1)) dir = 4;
            else if (off == m + 2) dir = 5;
            else if (off == -(m + 2)) dir = 6;
            if (dir < 0) return fail(RTE_ERR_ARG, "stencil entry outside the 7-point pattern");
            for (int s = 0; s < slots; ++s)
                for (size_t t = 0; t < bb; ++t)
                    out[(((size_t)s * 7 + dir) * n + i) * bb + t] =
                        L.vals[((size_t)s * nnz + q) * bb + t];
        }
    return RTE_OK;
}

}  // namespace rte
