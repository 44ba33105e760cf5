// Host assembly of the field operators (Sec. II.C) for the implicit field step.
//   [*eps]  edge mass     M_T(ab,cd) = eps |T|/20 [ (gb.gd)(1+d_ac) - (gb.gc)(1+d_ad)
//                                                  - (ga.gd)(1+d_bc) + (ga.gc)(1+d_bd) ]
//           (from int_T l_x l_y = |T| (1 + d_xy) / 20 and W1_ab = l_a g_b - l_b g_a)
//   [*S]    curl-curl     S_T(ab,cd) = (4 |T| / mu) (ga x gb).(gc x gd)   (curl W1_ab = 2 ga x gb)
//   L       node Laplacian L_T(a,b) = eps |T| ga.gb  (= [grad]^T [*eps] [grad] for Whitney forms)
// PEC walls: rows and columns of boundary edges (boundary nodes for L) are removed; a
// boundary row keeps a unit diagonal so the full-length vectors can be used everywhere.
#include <algorithm>
#include <cmath>

#include "field.cuh"

namespace fempic {

namespace {

const int kLE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};

double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// sparsity of a "DOF x DOF within a tet" operator with free DOFs only
void pattern(int64_t n, int64_t nt, int k, const int32_t* tdofs, const std::vector<uint8_t>& fixed,
             std::vector<int32_t>* rp, std::vector<int32_t>* col) {
    // dof -> tets
    std::vector<int32_t> cnt(n + 1, 0), d2t;
    for (int64_t t = 0; t < nt; ++t)
        for (int a = 0; a < k; ++a) cnt[tdofs[k * t + a] + 1]++;
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    d2t.resize(cnt[n]);
    {
        std::vector<int32_t> fill(cnt.begin(), cnt.end() - 1);
        for (int64_t t = 0; t < nt; ++t)
            for (int a = 0; a < k; ++a) d2t[fill[tdofs[k * t + a]]++] = (int32_t)t;
    }
    rp->assign(n + 1, 0);
    col->clear();
    std::vector<int32_t> row;
    for (int64_t i = 0; i < n; ++i) {
        row.clear();
        if (fixed[i]) {
            row.push_back((int32_t)i);
        } else {
            for (int32_t j = cnt[i]; j < cnt[i + 1]; ++j) {
                const int32_t t = d2t[j];
                for (int b = 0; b < k; ++b) {
                    const int32_t c = tdofs[k * (int64_t)t + b];
                    if (!fixed[c]) row.push_back(c);
                }
            }
            std::sort(row.begin(), row.end());
            row.erase(std::unique(row.begin(), row.end()), row.end());
        }
        col->insert(col->end(), row.begin(), row.end());
        (*rp)[i + 1] = (int32_t)col->size();
    }
}

int64_t find(const std::vector<int32_t>& rp, const std::vector<int32_t>& col, int32_t i, int32_t j) {
    auto b = col.begin() + rp[i], e = col.begin() + rp[i + 1];
    auto it = std::lower_bound(b, e, j);
    return (it != e && *it == j) ? (int64_t)(it - col.begin()) : -1;
}

}  // namespace

void assemble_fields(const HostComplex& hc, double eps, double mu, bool pec, HostFields* hf) {
    const int64_t nt = hc.nt, ne = hc.ne, nn = hc.nn;
    // PEC: edges and nodes of boundary faces are fixed at zero (natural boundary: none is)
    hf->node_fixed.assign(nn, 0);
    hf->edge_fixed.assign(ne, 0);
    for (int64_t f = 0; f < hc.nf && pec; ++f) {
        if (!hc.bface[f]) continue;
        for (int k = 0; k < 3; ++k) hf->node_fixed[hc.faces[3 * f + k]] = 1;
    }
    for (int64_t t = 0; t < nt && pec; ++t)
        for (int kf = 0; kf < 4; ++kf) {
            if (!hc.bface[hc.tf[4 * t + kf]]) continue;
            for (int a = 0; a < 6; ++a)  // the edges of face kf avoid its opposite vertex kf
                if (kLE[a][0] != kf && kLE[a][1] != kf) hf->edge_fixed[hc.te[6 * t + a]] = 1;
        }
    pattern(ne, nt, 6, hc.te.data(), hf->edge_fixed, &hf->e_rp, &hf->e_col);
    pattern(nn, nt, 4, hc.tv.data(), hf->node_fixed, &hf->n_rp, &hf->n_col);
    hf->M.assign(hf->e_col.size(), 0.0);
    hf->S.assign(hf->e_col.size(), 0.0);
    hf->L.assign(hf->n_col.size(), 0.0);
    for (int64_t i = 0; i < ne; ++i)
        if (hf->edge_fixed[i]) hf->M[hf->e_rp[i]] = 1.0;  // unit diagonal on PEC rows
    for (int64_t i = 0; i < nn; ++i)
        if (hf->node_fixed[i]) hf->L[hf->n_rp[i]] = 1.0;
    for (int64_t t = 0; t < nt; ++t) {
        const TetGeo& G = hc.geo[t];
        double g[4][3];
        for (int i = 0; i < 3; ++i) {
            g[1][i] = G.g[i];
            g[2][i] = G.g[3 + i];
            g[3][i] = G.g[6 + i];
            g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
        }
        // |T| = 1 / (6 |det G|)
        double c12[3];
        cross3(g[2], g[3], c12);
        const double vol = 1.0 / (6.0 * std::fabs(dot3(g[1], c12)));
        double gg[4][4];
        for (int a = 0; a < 4; ++a)
            for (int b = 0; b < 4; ++b) gg[a][b] = dot3(g[a], g[b]);
        double cw[6][3];
        for (int a = 0; a < 6; ++a) cross3(g[kLE[a][0]], g[kLE[a][1]], cw[a]);
        const int32_t* E = &hc.te[6 * t];
        for (int r = 0; r < 6; ++r) {
            if (hf->edge_fixed[E[r]]) continue;
            const int a = kLE[r][0], b = kLE[r][1];
            for (int s = 0; s < 6; ++s) {
                if (hf->edge_fixed[E[s]]) continue;
                const int c = kLE[s][0], d = kLE[s][1];
                const double m = eps * vol / 20.0 *
                                 (gg[b][d] * (1.0 + (a == c)) - gg[b][c] * (1.0 + (a == d)) -
                                  gg[a][d] * (1.0 + (b == c)) + gg[a][c] * (1.0 + (b == d)));
                const double sv = 4.0 * vol / mu * dot3(cw[r], cw[s]);
                const int64_t pos = find(hf->e_rp, hf->e_col, E[r], E[s]);
                hf->M[pos] += m;
                hf->S[pos] += sv;
            }
        }
        const int32_t* V = &hc.tv[4 * t];
        for (int a = 0; a < 4; ++a) {
            if (hf->node_fixed[V[a]]) continue;
            for (int b = 0; b < 4; ++b) {
                if (hf->node_fixed[V[b]]) continue;
                hf->L[find(hf->n_rp, hf->n_col, V[a], V[b])] += eps * vol * gg[a][b];
            }
        }
    }
}

double jacobi_lambda_max(const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                         const std::vector<double>& val, int steps) {
    const int64_t n = (int64_t)rp.size() - 1;
    if (n <= 0) return 1.0;
    std::vector<double> dis(n, 1.0);
    for (int64_t i = 0; i < n; ++i)
        for (int32_t j = rp[i]; j < rp[i + 1]; ++j)
            if (col[j] == i && val[j] > 0.0) dis[i] = 1.0 / std::sqrt(val[j]);
    std::vector<double> v(n), vp(n, 0.0), w(n), al, be;
    // fixed start vector with all modes present: 1 + a deterministic perturbation
    double nv = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        v[i] = 1.0 + 0.5 * std::sin(0.7 * (double)i + 0.3);
        nv += v[i] * v[i];
    }
    nv = std::sqrt(nv);
    for (double& x : v) x /= nv;
    double bprev = 0.0;
    for (int k = 0; k < steps && k < n; ++k) {
        for (int64_t i = 0; i < n; ++i) {
            double t = 0.0;
            for (int32_t j = rp[i]; j < rp[i + 1]; ++j) t += val[j] * dis[col[j]] * v[col[j]];
            w[i] = dis[i] * t;
        }
        double a = 0.0;
        for (int64_t i = 0; i < n; ++i) a += w[i] * v[i];
        double b = 0.0;
        for (int64_t i = 0; i < n; ++i) {
            w[i] -= a * v[i] + bprev * vp[i];
            b += w[i] * w[i];
        }
        b = std::sqrt(b);
        al.push_back(a);
        if (!(b > 1e-12 * std::fabs(a))) break;
        be.push_back(b);
        for (int64_t i = 0; i < n; ++i) {
            vp[i] = v[i];
            v[i] = w[i] / b;
        }
        bprev = b;
    }
    // largest eigenvalue of the tridiagonal (al, be) by bisection on Sturm counts
    const int m = (int)al.size();
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < m; ++i) {
        const double r = (i > 0 ? std::fabs(be[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(be[i]) : 0.0);
        lo = std::min(lo, al[i] - r);
        hi = std::max(hi, al[i] + r);
    }
    auto below = [&](double x) {  // number of eigenvalues < x
        int cnt = 0;
        double q = 1.0;
        for (int i = 0; i < m; ++i) {
            const double off = i > 0 ? be[i - 1] * be[i - 1] : 0.0;
            q = al[i] - x - (i > 0 ? off / q : 0.0);
            if (q == 0.0) q = -1e-300;
            if (q < 0.0) ++cnt;
        }
        return cnt;
    };
    for (int it = 0; it < 200 && hi - lo > 1e-12 * std::fabs(hi); ++it) {
        const double mid = 0.5 * (lo + hi);
        if (below(mid) == m) hi = mid; else lo = mid;
    }
    return hi;
}

}  // namespace fempic
