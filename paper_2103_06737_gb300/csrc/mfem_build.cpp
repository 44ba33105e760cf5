// Host assembly of the face mass [*mu^-1] and of [curl]^T for the first-order mixed FEM.
//
// On a tet with barycentric gradients g_0..g_3, the Whitney-2 function of the face with
// (sorted) vertices a < b < c is
//     W2_abc = 2 (l_a g_b x g_c + l_b g_c x g_a + l_c g_a x g_b),
// the unit-flux function oriented like the face's circulation a -> b -> c, which is the
// orientation [curl] = D1 gives the global face (i<j<k) since the tet's vertices are sorted by
// global id.  With int_T l_p l_q = |T| (1 + d_pq) / 20 the element matrix is exact:
//     [*mu^-1]_T(f, h) = (|T| / (5 mu)) sum_{p in f} sum_{q in h} (1 + d_pq) C_f(p) . C_h(q),
// C_f(a) = g_b x g_c, C_f(b) = g_c x g_a, C_f(c) = g_a x g_b.  No face is fixed: under PEC
// the boundary faces' fluxes never change, and their couplings to interior faces still enter
// Ampere's law on the interior edges.
#include <algorithm>
#include <cmath>

#include "mfem.cuh"

namespace fempic {

namespace {

void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

// vertices of local face k (the face opposite vertex k), ascending
const int kFaceVerts[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

}  // namespace

void assemble_mfem(const HostComplex& hc, double mu, HostMfem* hm) {
    const int64_t nt = hc.nt, nf = hc.nf, ne = hc.ne, nn = hc.nn;
    // face -> tets (one or two)
    std::vector<int32_t> f2t(2 * nf, -1);
    for (int64_t t = 0; t < nt; ++t)
        for (int k = 0; k < 4; ++k) {
            const int32_t f = hc.tf[4 * t + k];
            f2t[2 * f + (f2t[2 * f] < 0 ? 0 : 1)] = (int32_t)t;
        }
    // pattern: the faces of the tets each face belongs to
    hm->f_rp.assign(nf + 1, 0);
    hm->f_col.clear();
    std::vector<int32_t> row;
    for (int64_t f = 0; f < nf; ++f) {
        row.clear();
        for (int s = 0; s < 2; ++s) {
            const int32_t t = f2t[2 * f + s];
            if (t < 0) continue;
            for (int k = 0; k < 4; ++k) row.push_back(hc.tf[4 * (int64_t)t + k]);
        }
        std::sort(row.begin(), row.end());
        row.erase(std::unique(row.begin(), row.end()), row.end());
        hm->f_col.insert(hm->f_col.end(), row.begin(), row.end());
        hm->f_rp[f + 1] = (int32_t)hm->f_col.size();
    }
    hm->Fm.assign(hm->f_col.size(), 0.0);
    auto slot = [&](int32_t i, int32_t j) -> int64_t {
        auto b = hm->f_col.begin() + hm->f_rp[i], e = hm->f_col.begin() + hm->f_rp[i + 1];
        return std::lower_bound(b, e, j) - hm->f_col.begin();
    };
    for (int64_t t = 0; t < nt; ++t) {
        const TetGeo& G = hc.geo[t];
        double g[4][3];
        for (int i = 0; i < 3; ++i) {
            g[1][i] = G.g[i];
            g[2][i] = G.g[3 + i];
            g[3][i] = G.g[6 + i];
            g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
        }
        double c23[3];
        cross3(g[2], g[3], c23);
        const double vol = 1.0 / (6.0 * std::fabs(dot3(g[1], c23)));
        double C[4][3][3];  // C[k][p]: coefficient of l_{kFaceVerts[k][p]} in W2 of local face k
        for (int k = 0; k < 4; ++k) {
            const int a = kFaceVerts[k][0], b = kFaceVerts[k][1], c = kFaceVerts[k][2];
            cross3(g[b], g[c], C[k][0]);
            cross3(g[c], g[a], C[k][1]);
            cross3(g[a], g[b], C[k][2]);
        }
        const double scale = vol / (5.0 * mu);
        for (int k = 0; k < 4; ++k) {
            const int32_t fk = hc.tf[4 * t + k];
            for (int l = 0; l < 4; ++l) {
                double s = 0.0;
                for (int p = 0; p < 3; ++p)
                    for (int q = 0; q < 3; ++q) {
                        const double w = kFaceVerts[k][p] == kFaceVerts[l][q] ? 2.0 : 1.0;
                        s += w * dot3(C[k][p], C[l][q]);
                    }
                hm->Fm[slot(fk, hc.tf[4 * t + l])] += scale * s;
            }
        }
    }
    // [curl]^T: edge -> faces, with the face's sign for that edge
    std::vector<int64_t> ekey(ne);
    for (int64_t e = 0; e < ne; ++e) ekey[e] = (int64_t)hc.edges[2 * e] * nn + hc.edges[2 * e + 1];
    auto edge_of = [&](int32_t i, int32_t j) -> int32_t {
        const int64_t k = (int64_t)i * nn + j;
        return (int32_t)(std::lower_bound(ekey.begin(), ekey.end(), k) - ekey.begin());
    };
    std::vector<int32_t> fe(3 * nf);
    for (int64_t f = 0; f < nf; ++f) {
        const int32_t i = hc.faces[3 * f], j = hc.faces[3 * f + 1], k = hc.faces[3 * f + 2];
        fe[3 * f] = edge_of(i, j);
        fe[3 * f + 1] = edge_of(j, k);
        fe[3 * f + 2] = edge_of(i, k);
    }
    const int8_t sgn[3] = {1, 1, -1};
    hm->ef_rp.assign(ne + 1, 0);
    for (int64_t f = 0; f < nf; ++f)
        for (int s = 0; s < 3; ++s) hm->ef_rp[fe[3 * f + s] + 1]++;
    for (int64_t e = 0; e < ne; ++e) hm->ef_rp[e + 1] += hm->ef_rp[e];
    hm->ef_col.assign(hm->ef_rp[ne], 0);
    hm->ef_sgn.assign(hm->ef_rp[ne], 0);
    std::vector<int32_t> fill(hm->ef_rp.begin(), hm->ef_rp.end() - 1);
    for (int64_t f = 0; f < nf; ++f)  // faces in ascending order: each edge's list is sorted
        for (int s = 0; s < 3; ++s) {
            const int32_t e = fe[3 * f + s];
            hm->ef_col[fill[e]] = (int32_t)f;
            hm->ef_sgn[fill[e]++] = sgn[s];
        }
}

}  // namespace fempic
