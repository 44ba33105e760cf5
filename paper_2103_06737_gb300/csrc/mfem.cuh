// Internal declarations of the field solve's comparison systems (not part of the C ABI):
// the first-order mixed FEM and the wave-equation FEM without the Gauss-law projection.
#pragma once

#include "internal.cuh"

namespace fempic {

struct HostMfem {
    std::vector<int32_t> f_rp, f_col;    // face-face pattern (faces that share a tet), all faces
    std::vector<double> Fm;              // [*mu^-1] on that pattern
    std::vector<int32_t> ef_rp, ef_col;  // edge -> the faces it bounds ([curl]^T as CSR)
    std::vector<int8_t> ef_sgn;          // the [curl] entry of (face, edge): +1 or -1
};

// [*mu^-1]_fg = integral of W2_f . mu^-1 W2_g over the mesh (Sec. II.C), every face free,
// and the transpose of [curl] = D1 (face (i<j<k): +1 on (i,j) and (j,k), -1 on (i,k)).
void assemble_mfem(const HostComplex& hc, double mu, HostMfem* hm);

}  // namespace fempic
