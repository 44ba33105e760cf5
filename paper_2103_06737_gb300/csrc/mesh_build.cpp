// Host construction of the discrete complex K = {N, E, F, T} (Sec. II.C) and of the
// per-tet tables the kernels read.  Runs once per mesh in fem_pic_create.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <utility>

#include "internal.cuh"

namespace fempic {

namespace {

const int kLE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
const int kLF[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

struct FaceKey {
    int32_t a, b, c;
    bool operator<(const FaceKey& o) const {
        if (a != o.a) return a < o.a;
        if (b != o.b) return b < o.b;
        return c < o.c;
    }
    bool operator==(const FaceKey& o) const { return a == o.a && b == o.b && c == o.c; }
};

}  // namespace

fp_status build_complex(const fp_mesh* mesh, HostComplex* hc, std::string* err) {
    const int64_t nn = mesh->n_nodes, nt = mesh->n_tets;
    if (nn < 4 || nt < 1 || !mesh->xyz || !mesh->tet) {
        *err = "fem_pic_create: empty mesh or NULL arrays";
        return FP_EINVAL;
    }
    if (nn > INT32_MAX || 6 * nt > INT32_MAX) {
        *err = "fem_pic_create: mesh too large for 32-bit ids";
        return FP_EINVAL;
    }
    hc->nn = nn;
    hc->nt = nt;
    hc->xyz.assign(mesh->xyz, mesh->xyz + 3 * nn);
    hc->tv.resize(4 * nt);
    hc->orient.resize(nt);
    hc->geo.resize(nt);
    for (int64_t t = 0; t < nt; ++t) {
        int32_t v[4];
        for (int k = 0; k < 4; ++k) {
            v[k] = mesh->tet[4 * t + k];
            if (v[k] < 0 || v[k] >= nn) {
                *err = "fem_pic_create: tet " + std::to_string(t) + " has a node id out of range";
                return FP_EINVAL;
            }
        }
        std::sort(v, v + 4);
        if (v[0] == v[1] || v[1] == v[2] || v[2] == v[3]) {
            *err = "fem_pic_create: tet " + std::to_string(t) + " repeats a node";
            return FP_EGEOM;
        }
        std::memcpy(&hc->tv[4 * t], v, sizeof v);
        const double* x0 = &hc->xyz[3 * (int64_t)v[0]];
        double e[3][3];  // columns of the Jacobian: e[c] = x_{c+1} - x0
        for (int c = 0; c < 3; ++c)
            for (int i = 0; i < 3; ++i) e[c][i] = hc->xyz[3 * (int64_t)v[c + 1] + i] - x0[i];
        // rows of the inverse Jacobian: (e2 x e3, e3 x e1, e1 x e2) / det
        double r[3][3];
        const int cyc[3][2] = {{1, 2}, {2, 0}, {0, 1}};
        for (int k = 0; k < 3; ++k) {
            const double* a = e[cyc[k][0]];
            const double* b = e[cyc[k][1]];
            r[k][0] = a[1] * b[2] - a[2] * b[1];
            r[k][1] = a[2] * b[0] - a[0] * b[2];
            r[k][2] = a[0] * b[1] - a[1] * b[0];
        }
        double det = e[0][0] * r[0][0] + e[0][1] * r[0][1] + e[0][2] * r[0][2];
        if (!(std::fabs(det) > 0.0) || !std::isfinite(det)) {
            *err = "fem_pic_create: tet " + std::to_string(t) + " has zero volume";
            return FP_EGEOM;
        }
        hc->orient[t] = det > 0 ? 1 : -1;
        TetGeo& G = hc->geo[t];
        for (int i = 0; i < 3; ++i) G.o[i] = x0[i];
        for (int k = 0; k < 3; ++k)
            for (int i = 0; i < 3; ++i) G.g[3 * k + i] = r[k][i] / det;
    }

    // edges: unique sorted pairs in lexicographic order
    {
        std::vector<std::pair<uint64_t, int32_t>> keys(6 * nt);
        for (int64_t t = 0; t < nt; ++t)
            for (int k = 0; k < 6; ++k) {
                uint64_t i = (uint64_t)hc->tv[4 * t + kLE[k][0]], j = (uint64_t)hc->tv[4 * t + kLE[k][1]];
                keys[6 * t + k] = {i * (uint64_t)nn + j, (int32_t)(6 * t + k)};
            }
        std::sort(keys.begin(), keys.end());
        hc->te.resize(6 * nt);
        hc->edges.clear();
        int64_t id = -1;
        uint64_t last = ~0ull;
        for (auto& kv : keys) {
            if (kv.first != last) {
                ++id;
                last = kv.first;
                hc->edges.push_back((int32_t)(kv.first / (uint64_t)nn));
                hc->edges.push_back((int32_t)(kv.first % (uint64_t)nn));
            }
            hc->te[kv.second] = (int32_t)id;
        }
        hc->ne = id + 1;
    }
    // faces: unique sorted triples, face k opposite local vertex k
    std::vector<int32_t> face_t0, face_t1;
    {
        std::vector<std::pair<FaceKey, int32_t>> keys(4 * nt);
        for (int64_t t = 0; t < nt; ++t)
            for (int k = 0; k < 4; ++k) {
                const int32_t* v = &hc->tv[4 * t];
                keys[4 * t + k] = {{v[kLF[k][0]], v[kLF[k][1]], v[kLF[k][2]]}, (int32_t)(4 * t + k)};
            }
        std::sort(keys.begin(), keys.end(),
                  [](const std::pair<FaceKey, int32_t>& x, const std::pair<FaceKey, int32_t>& y) {
                      if (x.first == y.first) return x.second < y.second;
                      return x.first < y.first;
                  });
        hc->tf.resize(4 * nt);
        hc->faces.clear();
        int64_t id = -1;
        for (size_t i = 0; i < keys.size(); ++i) {
            if (i == 0 || !(keys[i].first == keys[i - 1].first)) {
                ++id;
                hc->faces.push_back(keys[i].first.a);
                hc->faces.push_back(keys[i].first.b);
                hc->faces.push_back(keys[i].first.c);
                face_t0.push_back(keys[i].second / 4);
                face_t1.push_back(-1);
            } else {
                if (face_t1[id] >= 0) {
                    *err = "fem_pic_create: a face is shared by more than two tets";
                    return FP_EGEOM;
                }
                face_t1[id] = keys[i].second / 4;
            }
            hc->tf[keys[i].second] = (int32_t)id;
        }
        hc->nf = id + 1;
    }
    hc->nb.resize(4 * nt);
    hc->bface.assign(hc->nf, 0);
    for (int64_t f = 0; f < hc->nf; ++f) hc->bface[f] = face_t1[f] < 0;
    for (int64_t t = 0; t < nt; ++t)
        for (int k = 0; k < 4; ++k) {
            int32_t f = hc->tf[4 * t + k];
            int32_t o = face_t0[f] == t ? face_t1[f] : face_t0[f];
            hc->nb[4 * t + k] = o;
        }
    return FP_OK;
}

static int32_t edge_id(const HostComplex& hc, int32_t i, int32_t j) {
    // edges are lexicographic: binary search
    int64_t lo = 0, hi = hc.ne - 1;
    while (lo <= hi) {
        int64_t mid = (lo + hi) / 2;
        int32_t a = hc.edges[2 * mid], b = hc.edges[2 * mid + 1];
        if (a == i && b == j) return (int32_t)mid;
        if (a < i || (a == i && b < j))
            lo = mid + 1;
        else
            hi = mid - 1;
    }
    return -1;
}

void incidence_csr(const HostComplex& hc, int which, std::vector<int32_t>* row_ptr,
                   std::vector<int32_t>* col, std::vector<int8_t>* val) {
    row_ptr->clear();
    col->clear();
    val->clear();
    if (which == 0) {  // D0: edge (i<j): -1 at i, +1 at j
        row_ptr->push_back(0);
        for (int64_t e = 0; e < hc.ne; ++e) {
            col->push_back(hc.edges[2 * e]);
            val->push_back(-1);
            col->push_back(hc.edges[2 * e + 1]);
            val->push_back(1);
            row_ptr->push_back((int32_t)col->size());
        }
    } else if (which == 1) {  // D1: face (i<j<k): +(i,j) +(j,k) -(i,k); sorted: (i,j)<(i,k)<(j,k)
        row_ptr->push_back(0);
        for (int64_t f = 0; f < hc.nf; ++f) {
            int32_t i = hc.faces[3 * f], j = hc.faces[3 * f + 1], k = hc.faces[3 * f + 2];
            col->push_back(edge_id(hc, i, j));
            val->push_back(1);
            col->push_back(edge_id(hc, i, k));
            val->push_back(-1);
            col->push_back(edge_id(hc, j, k));
            val->push_back(1);
            row_ptr->push_back((int32_t)col->size());
        }
    } else {  // D2: tet with orientation s: s*(-1)^k on face k, columns sorted
        row_ptr->push_back(0);
        for (int64_t t = 0; t < hc.nt; ++t) {
            std::pair<int32_t, int8_t> c[4];
            for (int k = 0; k < 4; ++k)
                c[k] = {hc.tf[4 * t + k], (int8_t)(hc.orient[t] * ((k & 1) ? -1 : 1))};
            std::sort(c, c + 4);
            for (int k = 0; k < 4; ++k) {
                col->push_back(c[k].first);
                val->push_back(c[k].second);
            }
            row_ptr->push_back((int32_t)col->size());
        }
    }
}

}  // namespace fempic
