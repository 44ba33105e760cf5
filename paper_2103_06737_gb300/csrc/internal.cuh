// Internal declarations of the FEM-PIC library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/fem_pic.h"

namespace fempic {

// Per-tet FP64 geometry: origin = position of the lowest-id vertex v0, and the
// gradients of the barycentric coordinates lambda_1..3 (rows of the inverse of
// the Jacobian [x1-x0 | x2-x0 | x3-x0]); grad lambda_0 = -(g1+g2+g3).
struct __align__(16) TetGeo {
    double o[3];
    double g[9];
};
static_assert(sizeof(TetGeo) == 96, "TetGeo layout");

// Per-tet topology: sorted vertex ids, the 6 local edges (01,02,03,12,13,23),
// the 4 faces (face k opposite vertex k), the neighbour across face k (-1 wall).
struct __align__(16) TetTopo {
    int32_t node[4];
    int32_t edge[6];
    int32_t face[4];
    int32_t nb[4];
    int32_t pad[2];
};
static_assert(sizeof(TetTopo) == 80, "TetTopo layout");

// Per-tet record read by the FP32 particle kernel: one 128-byte line holding what a
// particle that stays in its tet needs.  node/edge ids and FP32 barycentric gradients
// are static; the affine field coefficients are rewritten from e, b at every push:
//   E(off) = E0 + W x off          (W = sum_ab e_ab grad l_a x grad l_b, half the curl of E)
//   B(off) = B0 + beta off         (lowest-order W2 fields: divergence 3 beta)
// where off is the position minus the tet's vertex v0.
struct __align__(128) TetHot {
    int32_t node[4];
    int32_t edge[6];
    float g[9];
    float E0[3];
    float W[3];
    float B0[3];
    float beta;
    float pad[3];
};
static_assert(sizeof(TetHot) == 128, "TetHot layout");

// bits of the device status word
enum : int32_t { ST_WALK = 1, ST_INVAL = 2 };

struct HostComplex {
    int64_t nn = 0, ne = 0, nf = 0, nt = 0;
    std::vector<double> xyz;          // [3 nn]
    std::vector<int32_t> tv;          // [4 nt] sorted vertex ids
    std::vector<int8_t> orient;       // [nt] sign of the sorted tet's volume
    std::vector<int32_t> edges;       // [2 ne] (i<j), lexicographic
    std::vector<int32_t> faces;       // [3 nf] (i<j<k), lexicographic
    std::vector<int32_t> te;          // [6 nt]
    std::vector<int32_t> tf;          // [4 nt]
    std::vector<int32_t> nb;          // [4 nt]
    std::vector<uint8_t> bface;       // [nf] 1 = boundary (PEC) face
    std::vector<TetGeo> geo;          // [nt]
};

// Builds the discrete complex on the host.  Returns FP_OK or an error with text.
fp_status build_complex(const fp_mesh* mesh, HostComplex* hc, std::string* err);
// CSR of D0 / D1 / D2 with sorted columns.
void incidence_csr(const HostComplex& hc, int which, std::vector<int32_t>* row_ptr,
                   std::vector<int32_t>* col, std::vector<int8_t>* val);

}  // namespace fempic

struct fem_pic {
    int device = 0;
    int precision = FP_FP64;
    fempic::HostComplex hc;
    // device tables
    fempic::TetGeo* d_geo = nullptr;
    fempic::TetTopo* d_topo = nullptr;
    double* d_xyz = nullptr;
    int32_t* d_edges = nullptr;       // [2 ne]
    int32_t* d_faces = nullptr;       // [3 nf]
    int32_t* d_n2e_ptr = nullptr;     // node -> incident edges (D0^T as CSR)
    int32_t* d_n2e_col = nullptr;
    int8_t* d_n2e_sgn = nullptr;
    int8_t* d_orient = nullptr;       // [nt]
    fempic::TetHot* d_hot = nullptr;  // [nt]
    int32_t* d_status = nullptr;
    // particles deferred to the FP64 walk (near or across a face)
    int32_t* d_slow_idx = nullptr;    // [slow_cap]
    int32_t* d_slow_count = nullptr;  // [1]
    int64_t slow_cap = 0;
    uint8_t* d_node_wall = nullptr;   // [nn] 1 = node on the PEC boundary
    // sort scratch
    int32_t* d_sort_count = nullptr;  // [nt + 2]
    int32_t* d_sort_block = nullptr;  // block sums
    int32_t* d_sort_rank = nullptr;   // [cap]
    int64_t sort_cap = 0;
    std::string err;
};

#define FP_CUDA_TRY(ctx, call)                                                             \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess) {                                                           \
            if (ctx) (ctx)->err = std::string(#call ": ") + cudaGetErrorString(_e);        \
            return FP_ECUDA;                                                               \
        }                                                                                  \
    } while (0)

// launchers implemented in the .cu files
namespace fempic {
fp_status launch_push_deposit(fem_pic* ctx, const double* e, const double* b, const fp_particles* p,
                              double dt, int max_cross, void* dG, void* Q, int flags,
                              cudaStream_t s);
fp_status launch_deposit_charge(fem_pic* ctx, const fp_particles* p, void* Q, int flags,
                                cudaStream_t s);
fp_status launch_sort(fem_pic* ctx, const fp_particles* src, fp_particles* dst, cudaStream_t s);
fp_status launch_residuals(fem_pic* ctx, const void* dG, const void* Qn, const void* Qo,
                           const double* b, double* out, cudaStream_t s);
}  // namespace fempic
