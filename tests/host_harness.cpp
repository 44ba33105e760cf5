// The library's host-side assembly (discrete complex, field operators, face mass and [curl]^T)
// compiled without CUDA, with a small C interface, so that the CPU tests can hold it against
// the oracle.  Test infrastructure: built by tests/test_host_assembly.py with g++.
#include <algorithm>
#include <cstring>

#include "../paper_2103_06737_gb300/csrc/field.cuh"
#include "../paper_2103_06737_gb300/csrc/mfem.cuh"

using namespace fempic;

namespace {
HostComplex g_hc;
HostFields g_hf;
HostMfem g_hm;
std::string g_err;

template <typename T>
void put(const std::vector<T>& v, T* out) {
    if (out) std::copy(v.begin(), v.end(), out);
}
}  // namespace

extern "C" {

// Build the complex of a mesh and assemble every host operator; returns the fp_status.
int hh_build(int64_t nn, int64_t nt, const double* xyz, const int32_t* tet, double eps, double mu, int pec) {
    fp_mesh m{};
    m.n_nodes = nn;
    m.n_tets = nt;
    m.xyz = xyz;
    m.tet = tet;
    g_hc = HostComplex();
    g_hf = HostFields();
    g_hm = HostMfem();
    const fp_status st = build_complex(&m, &g_hc, &g_err);
    if (st != FP_OK) return (int)st;
    assemble_fields(g_hc, eps, mu, pec != 0, &g_hf);
    assemble_mfem(g_hc, mu, &g_hm);
    return 0;
}

const char* hh_error() { return g_err.c_str(); }

// N_n, N_e, N_f, N_t, nnz of the edge pattern, of the node pattern, of the face mass, of [curl]^T
void hh_sizes(int64_t* s) {
    s[0] = g_hc.nn;
    s[1] = g_hc.ne;
    s[2] = g_hc.nf;
    s[3] = g_hc.nt;
    s[4] = (int64_t)g_hf.e_col.size();
    s[5] = (int64_t)g_hf.n_col.size();
    s[6] = (int64_t)g_hm.f_col.size();
    s[7] = (int64_t)g_hm.ef_col.size();
}

void hh_complex(int32_t* edges, int32_t* faces, int32_t* tet_faces, uint8_t* bface) {
    put(g_hc.edges, edges);
    put(g_hc.faces, faces);
    put(g_hc.tf, tet_faces);
    put(g_hc.bface, bface);
}

void hh_fields(int32_t* e_rp, int32_t* e_col, double* M, double* S, int32_t* n_rp, int32_t* n_col, double* L,
               uint8_t* edge_fixed, uint8_t* node_fixed) {
    put(g_hf.e_rp, e_rp);
    put(g_hf.e_col, e_col);
    put(g_hf.M, M);
    put(g_hf.S, S);
    put(g_hf.n_rp, n_rp);
    put(g_hf.n_col, n_col);
    put(g_hf.L, L);
    put(g_hf.edge_fixed, edge_fixed);
    put(g_hf.node_fixed, node_fixed);
}

void hh_mfem(int32_t* f_rp, int32_t* f_col, double* Fm, int32_t* ef_rp, int32_t* ef_col, int8_t* ef_sgn) {
    put(g_hm.f_rp, f_rp);
    put(g_hm.f_col, f_col);
    put(g_hm.Fm, Fm);
    put(g_hm.ef_rp, ef_rp);
    put(g_hm.ef_col, ef_col);
    put(g_hm.ef_sgn, ef_sgn);
}

// D0 (which 0), D1 (1) or D2 (2) in CSR; returns nnz (arrays may be NULL to size them)
int64_t hh_incidence(int which, int32_t* row_ptr, int32_t* col, int8_t* val) {
    std::vector<int32_t> rp, c;
    std::vector<int8_t> v;
    incidence_csr(g_hc, which, &rp, &c, &v);
    put(rp, row_ptr);
    put(c, col);
    put(v, val);
    return (int64_t)c.size();
}

// per tet: neighbours across faces 0..3 (-1 wall), the gradients of lambda_1..3 (rows) and the
// origin (the lowest-id vertex)
void hh_tets(int32_t* nb, double* grad, double* origin) {
    put(g_hc.nb, nb);
    for (size_t t = 0; t < g_hc.geo.size(); ++t) {
        if (grad) std::memcpy(grad + 9 * t, g_hc.geo[t].g, 9 * sizeof(double));
        if (origin) std::memcpy(origin + 3 * t, g_hc.geo[t].o, 3 * sizeof(double));
    }
}

// The Lanczos estimate of the largest eigenvalue of D^-1 A that sets the Chebyshev interval of
// the inner solves: which = 0 the Newmark operator [*eps] + dt^2/4 [*S], 1 the node Laplacian.
double hh_lambda_max(int which, double dt, int steps) {
    if (which == 0) {
        std::vector<double> A(g_hf.M.size());
        for (size_t k = 0; k < A.size(); ++k) A[k] = g_hf.M[k] + 0.25 * dt * dt * g_hf.S[k];
        return jacobi_lambda_max(g_hf.e_rp, g_hf.e_col, A, steps);
    }
    return jacobi_lambda_max(g_hf.n_rp, g_hf.n_col, g_hf.L, steps);
}

}  // extern "C"
