// Internal declarations of the implicit field step (not part of the C ABI).
#pragma once

#include "internal.cuh"

namespace fempic {

struct HostFields {
    std::vector<uint8_t> edge_fixed, node_fixed;   // PEC DOFs
    std::vector<int32_t> e_rp, e_col;              // edge-edge pattern (free DOFs)
    std::vector<double> M, S;                      // [*eps], [*S] on that pattern
    std::vector<int32_t> n_rp, n_col;              // node-node pattern
    std::vector<double> L;                         // D0^T [*eps] D0
};

void assemble_fields(const HostComplex& hc, double eps, double mu, HostFields* hf);

}  // namespace fempic
