// Host plan of the H^2 compression of S^+ and S^- (Section 5.2): cluster
// tree, bounding boxes, interpolation nodes, block tree and the block lists
// of the apply.  Compiled without floating-point contraction so that the
// admissibility test rounds the same way on every host.
#include "h2.h"

#include <algorithm>
#include <cmath>
#include <functional>
#include <map>
#include <utility>

namespace rte {

namespace {

double diam(const double* lo, const double* hi) {
    const double ex = hi[0] - lo[0], ey = hi[1] - lo[1], ez = hi[2] - lo[2];
    return std::sqrt(ex * ex + ey * ey + ez * ez);
}

double dist(const double* lo1, const double* hi1, const double* lo2, const double* hi2) {
    double e[3];
    for (int a = 0; a < 3; ++a) e[a] = std::max(0.0, std::max(lo1[a] - hi2[a], lo2[a] - hi1[a]));
    return std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
}

}  // namespace

bool h2_plan(int levels, double eta, int p, const std::vector<double>& far_pts, int qf,
             H2Plan& P) {
    P.levels = levels;
    P.n = 4 << (2 * levels);
    P.p = p;
    P.k = p * p * p;
    P.eta = eta;
    // leaves: the shallowest depth whose clusters hold at most n_min = 64
    int ld = 0;
    while ((1 << (2 * (levels - ld))) > kH2Leaf && ld < levels) ++ld;
    P.ld = ld;

    // boxes at every depth (far-rule points of the cluster's triangles)
    std::vector<std::vector<double>> lo(ld + 1), hi(ld + 1);
    for (int d = 0; d <= ld; ++d) {
        const int cnt = 4 << (2 * d), size = 1 << (2 * (levels - d));
        lo[d].assign(3 * (size_t)cnt, 0.0);
        hi[d].assign(3 * (size_t)cnt, 0.0);
        for (int t = 0; t < cnt; ++t) {
            double l[3] = {1e300, 1e300, 1e300}, h[3] = {-1e300, -1e300, -1e300};
            const size_t q0 = (size_t)t * size * qf, q1 = q0 + (size_t)size * qf;
            for (size_t q = q0; q < q1; ++q)
                for (int a = 0; a < 3; ++a) {
                    l[a] = std::min(l[a], far_pts[3 * q + a]);
                    h[a] = std::max(h[a], far_pts[3 * q + a]);
                }
            for (int a = 0; a < 3; ++a) {
                lo[d][3 * (size_t)t + a] = l[a];
                hi[d][3 * (size_t)t + a] = h[a];
            }
        }
    }

    // block tree of both parts: sign +1 direct, -1 mirror (column box negated)
    P.far.clear();
    P.near.clear();
    std::function<void(int, int, int, int)> visit = [&](int d, int t, int c, int sign) {
        const double* lt = &lo[d][3 * (size_t)t];
        const double* ht = &hi[d][3 * (size_t)t];
        double lc[3], hc[3];
        for (int a = 0; a < 3; ++a) {
            lc[a] = sign > 0 ? lo[d][3 * (size_t)c + a] : -hi[d][3 * (size_t)c + a];
            hc[a] = sign > 0 ? hi[d][3 * (size_t)c + a] : -lo[d][3 * (size_t)c + a];
        }
        if (std::max(diam(lt, ht), diam(lc, hc)) <= eta * dist(lt, ht, lc, hc)) {
            P.far.push_back({d, t, c, sign});
        } else if (d == ld) {
            P.near.push_back({d, t, c, sign});
        } else {
            for (int a = 4 * t; a < 4 * t + 4; ++a)
                for (int b = 4 * c; b < 4 * c + 4; ++b) visit(d + 1, a, b, sign);
        }
    };
    for (int sign : {1, -1})
        for (int t = 0; t < 4; ++t)
            for (int c = 0; c < 4; ++c) visit(0, t, c, sign);

    P.dmin = ld;
    for (const auto& b : P.far) P.dmin = std::min(P.dmin, b.depth);
    P.depth_off.clear();
    P.ncl = 0;
    for (int d = P.dmin; d <= ld; ++d) {
        P.depth_off.push_back(P.ncl);
        P.ncl += P.count(d);
    }

    // per-cluster boxes, nodes and normalised tensor points
    P.lo.assign(3 * (size_t)P.ncl, 0.0);
    P.hi.assign(3 * (size_t)P.ncl, 0.0);
    P.nodes.assign((size_t)P.ncl * p * 3, 0.0);
    P.xi.assign((size_t)P.ncl * kH2B * 3, 0.0);
    const double pi = 3.14159265358979323846;
    for (int d = P.dmin; d <= ld; ++d)
        for (int t = 0; t < P.count(d); ++t) {
            const int id = P.id(d, t);
            for (int a = 0; a < 3; ++a) {
                const double l = lo[d][3 * (size_t)t + a], h = hi[d][3 * (size_t)t + a];
                P.lo[3 * (size_t)id + a] = l;
                P.hi[3 * (size_t)id + a] = h;
                const double c = 0.5 * (l + h), w = 0.5 * (h - l);
                if (!(w > 0.0)) return false;
                for (int i = 0; i < p; ++i)
                    P.nodes[((size_t)id * p + i) * 3 + a] =
                        c + w * std::cos((2 * i + 1) * pi / (2 * p));
            }
            const double* nd = &P.nodes[(size_t)id * p * 3];
            for (int ix = 0; ix < p; ++ix)
                for (int iy = 0; iy < p; ++iy)
                    for (int iz = 0; iz < p; ++iz) {
                        const int nu = (ix * p + iy) * p + iz;
                        double v[3] = {nd[3 * ix], nd[3 * iy + 1], nd[3 * iz + 2]};
                        const double r = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
                        if (!(r > 0.0)) return false;
                        for (int a = 0; a < 3; ++a)
                            P.xi[((size_t)id * kH2B + nu) * 3 + a] = v[a] / r;
                    }
        }

    // near blocks with both parts merged per leaf pair
    std::map<std::pair<int, int>, int> flags;
    for (const auto& b : P.near) flags[{b.t, b.c}] |= (b.sign > 0 ? 1 : 2);
    P.nearm.clear();
    for (const auto& kv : flags) P.nearm.push_back({kv.first.first, kv.first.second, kv.second});
    return true;
}

H2Pool h2_pool(const H2Plan& P, int m) {
    H2Pool pl;
    pl.m = m;
    pl.leaf0 = 0;
    pl.transfer0 = (long long)P.leaves() * m;
    pl.near0 = pl.transfer0 + (P.ncl - P.count(P.dmin));
    pl.total = pl.near0 + (long long)P.nearm.size() * m * m;
    return pl;
}

void h2_lists(const H2Plan& P, const H2Pool& pool, H2Lists& L) {
    const int m = pool.m, ld = P.ld;
    auto open = [](H2List& l) {
        l = H2List();
        l.ptr.push_back(0);
    };
    auto row = [](H2List& l, int out) { l.out_blk.push_back(out); };
    auto entry = [](H2List& l, int in, long long mat) {
        l.in_blk.push_back(in);
        l.mat.push_back((int)mat);
    };
    auto close = [](H2List& l) { l.ptr.push_back((int)l.in_blk.size()); };

    open(L.up_leaf);
    for (int t = 0; t < P.leaves(); ++t) {
        row(L.up_leaf, P.id(ld, t));
        for (int a = 0; a < m; ++a) entry(L.up_leaf, t * m + a, pool.leaf(t, a));
        close(L.up_leaf);
    }
    L.up.assign(ld - P.dmin, H2List());
    L.down.assign(ld - P.dmin, H2List());
    for (int d = P.dmin; d < ld; ++d) {
        H2List& u = L.up[d - P.dmin];
        open(u);
        for (int t = 0; t < P.count(d); ++t) {
            row(u, P.id(d, t));
            for (int c = 4 * t; c < 4 * t + 4; ++c) entry(u, P.id(d + 1, c), pool.transfer(P, d + 1, c));
            close(u);
        }
        H2List& w = L.down[d - P.dmin];
        open(w);
        for (int c = 0; c < P.count(d + 1); ++c) {
            row(w, P.id(d + 1, c));
            entry(w, P.id(d, c / 4), pool.transfer(P, d + 1, c));
            close(w);
        }
    }
    // couplings grouped by row cluster (depth, t)
    std::map<std::pair<int, int>, std::vector<std::pair<int, int>>> rows;
    for (const auto& b : P.far) rows[{b.depth, b.t}].push_back({b.c, b.sign});
    open(L.couple);
    for (const auto& kv : rows) {
        row(L.couple, P.id(kv.first.first, kv.first.second));
        for (const auto& cs : kv.second) entry(L.couple, P.id(kv.first.first, cs.first), cs.second);
        close(L.couple);
    }
    open(L.down_leaf);
    for (int t = 0; t < P.leaves(); ++t)
        for (int a = 0; a < m; ++a) {
            row(L.down_leaf, t * m + a);
            entry(L.down_leaf, P.id(ld, t), pool.leaf(t, a));
            close(L.down_leaf);
        }
    // near field, grouped by row leaf
    std::vector<std::vector<int>> by_t(P.leaves());
    for (int i = 0; i < (int)P.nearm.size(); ++i) by_t[P.nearm[i].t].push_back(i);
    open(L.near);
    for (int t = 0; t < P.leaves(); ++t)
        for (int a = 0; a < m; ++a) {
            row(L.near, t * m + a);
            for (int i : by_t[t])
                for (int b = 0; b < m; ++b) entry(L.near, P.nearm[i].c * m + b, pool.nearb(i, a, b));
            close(L.near);
        }
}

}  // namespace rte
