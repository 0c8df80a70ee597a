// Host-side assembly of the discrete system of Section 4: meshes, the sparse
// spatial matrices, the angular mass/transport/boundary matrices and the
// quadrature rules used by the device assembly of S^+ and S^-.
#include <algorithm>
#include <cmath>
#include <map>
#include <set>
#include <tuple>

#include "rte_internal.h"

namespace rte {

SquareMesh make_square(int m) {
    SquareMesh M;
    M.m = m;
    M.n_nodes = (m + 1) * (m + 1);
    M.n_cells = 2 * m * m;
    M.cell_nodes.resize(3 * M.n_cells);
    M.area.resize(M.n_cells);
    M.grad.resize(6 * M.n_cells);
    const double h = 1.0 / m;
    for (int J = 0; J < m; ++J)
        for (int I = 0; I < m; ++I) {
            const int q = J * m + I;
            const int n00 = J * (m + 1) + I, n10 = n00 + 1;
            const int n01 = n00 + (m + 1), n11 = n01 + 1;
            const int tri[2][3] = {{n00, n10, n11}, {n00, n11, n01}};
            for (int t = 0; t < 2; ++t) {
                const int c = 2 * q + t;
                double x[3], y[3];
                for (int a = 0; a < 3; ++a) {
                    M.cell_nodes[3 * c + a] = tri[t][a];
                    x[a] = (tri[t][a] % (m + 1)) * h;
                    y[a] = (tri[t][a] / (m + 1)) * h;
                }
                const double A = 0.5 * ((x[1] - x[0]) * (y[2] - y[0]) -
                                        (y[1] - y[0]) * (x[2] - x[0]));
                M.area[c] = A;
                for (int a = 0; a < 3; ++a) {
                    const int b = (a + 1) % 3, d = (a + 2) % 3;
                    // gradient of the hat function of vertex a
                    M.grad[6 * c + a] = (y[b] - y[d]) / (2 * A);
                    M.grad[6 * c + 3 + a] = (x[d] - x[b]) / (2 * A);
                }
            }
        }
    return M;
}

static void normalise3(double* v) {
    const double r = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
    v[0] /= r; v[1] /= r; v[2] /= r;
}

SphereMesh make_sphere(int levels) {
    SphereMesh S;
    S.levels = levels;
    S.verts = {1, 0, 0, 0, 1, 0, -1, 0, 0, 0, -1, 0, 0, 0, 1};
    // upper octahedron faces, counter-clockwise seen from outside
    S.tri = {0, 1, 4, 1, 2, 4, 2, 3, 4, 3, 0, 4};
    for (int lv = 0; lv < levels; ++lv) {
        std::map<std::pair<int, int>, int> mid;
        auto midpoint = [&](int a, int b) {
            auto key = std::make_pair(std::min(a, b), std::max(a, b));
            auto it = mid.find(key);
            if (it != mid.end()) return it->second;
            double v[3];
            for (int i = 0; i < 3; ++i) v[i] = S.verts[3 * a + i] + S.verts[3 * b + i];
            normalise3(v);
            const int id = (int)S.verts.size() / 3;
            S.verts.insert(S.verts.end(), v, v + 3);
            mid[key] = id;
            return id;
        };
        std::vector<int> nt;
        nt.reserve(4 * S.tri.size());
        for (size_t t = 0; t < S.tri.size() / 3; ++t) {
            const int a = S.tri[3 * t], b = S.tri[3 * t + 1], c = S.tri[3 * t + 2];
            const int ab = midpoint(a, b), bc = midpoint(b, c), ca = midpoint(c, a);
            const int kids[4][3] = {{a, ab, ca}, {ab, b, bc}, {ca, bc, c}, {ab, bc, ca}};
            for (auto& k : kids) nt.insert(nt.end(), k, k + 3);
        }
        S.tri.swap(nt);
    }
    S.n = (int)S.tri.size() / 3;
    return S;
}

// Exact area of the spherical triangle (a, b, c) (solid angle formula of
// Van Oosterom and Strackee).
static double sph_area(const double* a, const double* b, const double* c) {
    const double bxc[3] = {b[1] * c[2] - b[2] * c[1], b[2] * c[0] - b[0] * c[2],
                           b[0] * c[1] - b[1] * c[0]};
    const double num = std::fabs(a[0] * bxc[0] + a[1] * bxc[1] + a[2] * bxc[2]);
    const double den = 1.0 + (a[0] * b[0] + a[1] * b[1] + a[2] * b[2]) +
                       (b[0] * c[0] + b[1] * c[1] + b[2] * c[2]) +
                       (c[0] * a[0] + c[1] * a[1] + c[2] * a[2]);
    return 2.0 * std::atan2(num, den);
}

// Level-r rule on one spherical triangle: refine r times (normalised edge
// midpoints), one node per sub-triangle at its normalised vertex mean with
// the sub-triangle's exact area as weight.
void quad_one(const double* a, const double* b, const double* c, int r, double* pts, double* w,
              int& count) {
    if (r == 0) {
        double p[3] = {a[0] + b[0] + c[0], a[1] + b[1] + c[1], a[2] + b[2] + c[2]};
        normalise3(p);
        pts[3 * count] = p[0]; pts[3 * count + 1] = p[1]; pts[3 * count + 2] = p[2];
        w[count] = sph_area(a, b, c);
        ++count;
        return;
    }
    double ab[3], bc[3], ca[3];
    for (int i = 0; i < 3; ++i) {
        ab[i] = a[i] + b[i]; bc[i] = b[i] + c[i]; ca[i] = c[i] + a[i];
    }
    normalise3(ab); normalise3(bc); normalise3(ca);
    quad_one(a, ab, ca, r - 1, pts, w, count);
    quad_one(ab, b, bc, r - 1, pts, w, count);
    quad_one(ca, bc, c, r - 1, pts, w, count);
    quad_one(ab, bc, ca, r - 1, pts, w, count);
}

bool inv3(const double* A, double* Ai) {
    const double det = A[0] * (A[4] * A[8] - A[5] * A[7]) -
                       A[1] * (A[3] * A[8] - A[5] * A[6]) +
                       A[2] * (A[3] * A[7] - A[4] * A[6]);
    if (!(std::fabs(det) > 0)) return false;
    Ai[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    Ai[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    Ai[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    Ai[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    Ai[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    Ai[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    Ai[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    Ai[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    Ai[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    return true;
}

// Pairs (k, k') where K_k' or -K_k' shares a vertex with K_k: the pairs whose
// double integrals take the near rule.
void sphere_near_pairs(const SphereMesh& S, std::vector<int>& ptr, std::vector<int>& idx) {
    const int n = S.n;
    std::map<std::tuple<long long, long long, long long>, int> vid;
    auto key = [](const double* v) {
        return std::make_tuple(std::llround(v[0] * 1e9), std::llround(v[1] * 1e9),
                               std::llround(v[2] * 1e9));
    };
    const int nv = (int)S.verts.size() / 3;
    for (int v = 0; v < nv; ++v) vid[key(&S.verts[3 * v])] = v;
    std::vector<int> anti(nv, -1);
    for (int v = 0; v < nv; ++v) {
        const double w[3] = {-S.verts[3 * v], -S.verts[3 * v + 1], -S.verts[3 * v + 2]};
        auto it = vid.find(key(w));
        if (it != vid.end()) anti[v] = it->second;
    }
    std::vector<std::vector<int>> owners(nv);
    for (int k = 0; k < n; ++k)
        for (int a = 0; a < 3; ++a) owners[S.tri[3 * k + a]].push_back(k);
    ptr.assign(n + 1, 0);
    idx.clear();
    for (int k = 0; k < n; ++k) {
        std::set<int> s;
        for (int a = 0; a < 3; ++a) {
            const int v = S.tri[3 * k + a];
            for (int kk : owners[v]) s.insert(kk);
            if (anti[v] >= 0)
                for (int kk : owners[anti[v]]) s.insert(kk);
        }
        idx.insert(idx.end(), s.begin(), s.end());
        ptr[k + 1] = (int)idx.size();
    }
}

int build_host_system(const rte_problem& p, const rte_options& o, HostSystem& hs) {
    if (p.mesh_m < 1 || p.mesh_m > 4096)
        return fail(RTE_ERR_ARG, "mesh_m must be in [1, 4096]");
    if (p.sphere_levels < 0 || p.sphere_levels > 5)
        return fail(RTE_ERR_ARG, "sphere_levels must be in [0, 5]");
    if (!(p.g >= 0.0 && p.g < 1.0))
        return fail(RTE_ERR_ARG, "g must satisfy 0 <= g < 1");
    if (!p.sigma_t || !p.sigma_s) return fail(RTE_ERR_ARG, "sigma arrays are NULL");
    hs.m = p.mesh_m;
    hs.levels = p.sphere_levels;
    hs.g = p.g;
    hs.mesh = make_square(p.mesh_m);
    hs.sphere = make_sphere(p.sphere_levels);
    const SquareMesh& M = hs.mesh;
    hs.nRp = M.n_nodes;
    hs.nRm = M.n_cells;
    hs.nSp = hs.sphere.n;
    hs.nSm = 3 * hs.nSp;
    hs.dP = o.n_plus >= 0 ? (o.n_plus + 1) * (o.n_plus + 2) / 2 : 0;
    hs.dM = (o.n_minus + 1) * (o.n_minus + 2) / 2;
    if (hs.dP > hs.nSp || hs.dM > hs.nSm)
        return fail(RTE_ERR_ARG, "N^+ or N^- too large for the sphere mesh");

    // sigma fields, c = ||sigma_s / sigma_t||_inf (Section 2.2)
    double c = 0.0;
    hs.cell_at.resize(hs.nRm);
    hs.cell_as.resize(hs.nRm);
    for (int j = 0; j < hs.nRm; ++j) {
        const double st = p.sigma_t[j], ss = p.sigma_s[j];
        if (!(st > 0.0) || !(ss >= 0.0) || !(ss < st) || !std::isfinite(st))
            return fail(RTE_ERR_ARG, "need 0 <= sigma_s < sigma_t per cell");
        c = std::max(c, ss / st);
        hs.cell_at[j] = st * M.area[j];
        hs.cell_as[j] = ss * M.area[j];
    }
    hs.c = c;
    hs.gamma = 1.0 / (1.0 - c * p.g);

    // ---------------------------------------------------- node stencil
    std::vector<std::set<int>> nb(hs.nRp);
    for (int j = 0; j < hs.nRm; ++j)
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                nb[M.cell_nodes[3 * j + a]].insert(M.cell_nodes[3 * j + b]);
    hs.st.ptr.assign(hs.nRp + 1, 0);
    hs.st.diag.resize(hs.nRp);
    for (int i = 0; i < hs.nRp; ++i) {
        hs.st.ptr[i + 1] = hs.st.ptr[i] + (int)nb[i].size();
        for (int col : nb[i]) {
            if (col == i) hs.st.diag[i] = (int)hs.st.col.size();
            hs.st.col.push_back(col);
        }
    }
    const int nnz = (int)hs.st.col.size();
    hs.sval.assign((size_t)kSlots * nnz, 0.0);
    auto slot = [&](int s, int row, int col) -> double& {
        const int* b = hs.st.col.data() + hs.st.ptr[row];
        const int* e = hs.st.col.data() + hs.st.ptr[row + 1];
        const int pos = (int)(std::lower_bound(b, e, col) - hs.st.col.data());
        return hs.sval[(size_t)s * nnz + pos];
    };
    hs.cell_D.resize(6 * hs.nRm);
    for (int j = 0; j < hs.nRm; ++j) {
        const double A = M.area[j];
        const double st = p.sigma_t[j], ss = p.sigma_s[j];
        const int* nd = &M.cell_nodes[3 * j];
        const double* gx = &M.grad[6 * j];
        const double* gy = &M.grad[6 * j + 3];
        for (int a = 0; a < 3; ++a) {
            hs.cell_D[6 * j + a] = A * gx[a];       // (D_1)_{j, nd[a]}
            hs.cell_D[6 * j + 3 + a] = A * gy[a];   // (D_2)_{j, nd[a]}
            for (int b = 0; b < 3; ++b) {
                const double mass = A * (a == b ? 2.0 : 1.0) / 12.0;
                slot(kMt, nd[a], nd[b]) += st * mass;
                slot(kMs, nd[a], nd[b]) += ss * mass;
                slot(kMu, nd[a], nd[b]) += mass;
                // (D_n^T (M_t^-)^{-1} D_m)_{ab} = A^2 g_n,a g_m,b / (sigma_t A)
                slot(kK11, nd[a], nd[b]) += A * gx[a] * gx[b] / st;
                slot(kK12, nd[a], nd[b]) += A * (gx[a] * gy[b] + gy[a] * gx[b]) / st;
                slot(kK22, nd[a], nd[b]) += A * gy[a] * gy[b] / st;
            }
        }
    }
    // boundary mass on the four faces: 1-D P1 mass (h/6)[2 1; 1 2]
    const int m = hs.m;
    const double h = 1.0 / m;
    for (int e = 0; e < m; ++e) {
        const int faces[4][2] = {
            {e * (m + 1), (e + 1) * (m + 1)},                   // x = 0
            {e * (m + 1) + m, (e + 1) * (m + 1) + m},           // x = 1
            {e, e + 1},                                         // y = 0
            {m * (m + 1) + e, m * (m + 1) + e + 1}};            // y = 1
        for (int f = 0; f < 4; ++f) {
            const int s = f < 2 ? kBx : kBy;
            const int u = faces[f][0], v = faces[f][1];
            slot(s, u, u) += h / 3.0;
            slot(s, v, v) += h / 3.0;
            slot(s, u, v) += h / 6.0;
            slot(s, v, u) += h / 6.0;
        }
    }
    // node -> incident cells
    hs.adj_ptr.assign(hs.nRp + 1, 0);
    for (int j = 0; j < hs.nRm; ++j)
        for (int a = 0; a < 3; ++a) hs.adj_ptr[M.cell_nodes[3 * j + a] + 1]++;
    for (int i = 0; i < hs.nRp; ++i) hs.adj_ptr[i + 1] += hs.adj_ptr[i];
    hs.adj_cell.resize(3 * hs.nRm);
    hs.adj_loc.resize(3 * hs.nRm);
    {
        std::vector<int> fill(hs.adj_ptr.begin(), hs.adj_ptr.end() - 1);
        for (int j = 0; j < hs.nRm; ++j)
            for (int a = 0; a < 3; ++a) {
                const int i = M.cell_nodes[3 * j + a];
                hs.adj_cell[fill[i]] = j;
                hs.adj_loc[fill[i]] = a;
                fill[i]++;
            }
    }

    // ------------------------------------------------------- angular
    const SphereMesh& S = hs.sphere;
    const int n = hs.nSp;
    const int qn = 1 << (2 * kRNear), qf = 1 << (2 * kRFar);
    hs.quad_near_pts.resize((size_t)n * qn * 3);
    hs.quad_near_w.resize((size_t)n * qn);
    hs.quad_far_pts.resize((size_t)n * qf * 3);
    hs.quad_far_w.resize((size_t)n * qf);
    hs.quad_near_psi.resize((size_t)n * qn * 3);
    hs.quad_far_psi.resize((size_t)n * qf * 3);
    hs.m_.resize(n); hs.omx.resize(n); hs.omy.resize(n);
    hs.A1.resize(3 * n); hs.A2.resize(3 * n);
    hs.MSm.resize(9 * n); hs.MSm_inv.resize(9 * n); hs.e0s.resize(6 * n);
    for (int k = 0; k < n; ++k) {
        const double* a = &S.verts[3 * S.tri[3 * k]];
        const double* b = &S.verts[3 * S.tri[3 * k + 1]];
        const double* cc = &S.verts[3 * S.tri[3 * k + 2]];
        int cnt = 0;
        quad_one(a, b, cc, kRNear, &hs.quad_near_pts[(size_t)k * qn * 3],
                 &hs.quad_near_w[(size_t)k * qn], cnt);
        cnt = 0;
        quad_one(a, b, cc, kRFar, &hs.quad_far_pts[(size_t)k * qf * 3],
                 &hs.quad_far_w[(size_t)k * qf], cnt);
        hs.m_[k] = 2.0 * sph_area(a, b, cc);
        // V has the vertices as columns; psi_i(s) = (V^{-1} s)_i
        const double V[9] = {a[0], b[0], cc[0], a[1], b[1], cc[1], a[2], b[2], cc[2]};
        double Vi[9];
        if (!inv3(V, Vi)) return fail(RTE_ERR_ARG, "degenerate sphere triangle");
        double Mk[9] = {0}, a1[3] = {0}, a2[3] = {0}, ox = 0, oy = 0;
        for (int q = 0; q < qn; ++q) {
            const double* s = &hs.quad_near_pts[((size_t)k * qn + q) * 3];
            const double w = hs.quad_near_w[(size_t)k * qn + q];
            double psi[3];
            for (int i = 0; i < 3; ++i)
                psi[i] = Vi[3 * i] * s[0] + Vi[3 * i + 1] * s[1] + Vi[3 * i + 2] * s[2];
            for (int i = 0; i < 3; ++i) {
                for (int jj = 0; jj < 3; ++jj) Mk[3 * i + jj] += 2.0 * w * psi[i] * psi[jj];
                a1[i] += 2.0 * w * s[0] * psi[i];
                a2[i] += 2.0 * w * s[1] * psi[i];
            }
            ox += 2.0 * w * std::fabs(s[0]);
            oy += 2.0 * w * std::fabs(s[1]);
        }
        for (int lvl = 0; lvl < 2; ++lvl) {
            const int nq = lvl ? qf : qn;
            const double* P = lvl ? &hs.quad_far_pts[(size_t)k * qf * 3]
                                  : &hs.quad_near_pts[(size_t)k * qn * 3];
            double* Psi = lvl ? &hs.quad_far_psi[(size_t)k * qf * 3]
                              : &hs.quad_near_psi[(size_t)k * qn * 3];
            for (int q = 0; q < nq; ++q)
                for (int i = 0; i < 3; ++i)
                    Psi[3 * q + i] = Vi[3 * i] * P[3 * q] + Vi[3 * i + 1] * P[3 * q + 1] +
                                     Vi[3 * i + 2] * P[3 * q + 2];
        }
        double Mi[9];
        if (!inv3(Mk, Mi)) return fail(RTE_ERR_ARG, "singular odd mass block");
        for (int i = 0; i < 9; ++i) { hs.MSm[9 * k + i] = Mk[i]; hs.MSm_inv[9 * k + i] = Mi[i]; }
        for (int i = 0; i < 3; ++i) { hs.A1[3 * k + i] = a1[i]; hs.A2[3 * k + i] = a2[i]; }
        hs.omx[k] = ox;
        hs.omy[k] = oy;
        // a_k^{nm} = A_n(k)^T M_k^{-1} A_m(k)
        double t1[3], t2[3];
        for (int i = 0; i < 3; ++i) {
            t1[i] = Mi[3 * i] * a1[0] + Mi[3 * i + 1] * a1[1] + Mi[3 * i + 2] * a1[2];
            t2[i] = Mi[3 * i] * a2[0] + Mi[3 * i + 1] * a2[1] + Mi[3 * i + 2] * a2[2];
        }
        const double a11 = a1[0] * t1[0] + a1[1] * t1[1] + a1[2] * t1[2];
        const double a12 = a1[0] * t2[0] + a1[1] * t2[1] + a1[2] * t2[2];
        const double a22 = a2[0] * t2[0] + a2[1] * t2[1] + a2[2] * t2[2];
        hs.e0s[6 * k + 0] = hs.gamma * a11;
        hs.e0s[6 * k + 1] = hs.gamma * a12;
        hs.e0s[6 * k + 2] = hs.gamma * a22;
        hs.e0s[6 * k + 3] = ox;
        hs.e0s[6 * k + 4] = oy;
        hs.e0s[6 * k + 5] = hs.m_[k];
    }
    sphere_near_pairs(S, hs.near_ptr, hs.near_idx);
    return RTE_OK;
}

}  // namespace rte
