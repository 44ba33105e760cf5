// Internal declarations of the implicit field step (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>

#include "internal.cuh"

// FP_COL16=1: the mixed solver's streamed FP32 operators read their columns as 16-bit offsets
// from a per-slice-position base (Sell::cb, Sell::cd) where every offset fits, a quarter fewer
// operator bytes per product.  Measured on the 96^3 mesh (both operators streamed), Jacobi-CG
// per solve: Newmark 17.8 -> 18.1 ms and Gauss-law 6.3 -> 6.8 ms in the bench; with the L2
// prefetch of the operator, field-only, Newmark 19.5 -> 19.6 ms and Gauss-law 3.7 -> 4.2 ms.
// The extra base load per entry costs more than the bytes it saves; off by default.
#ifndef FP_COL16
#define FP_COL16 0
#endif

namespace fempic {

struct HostFields {
    std::vector<uint8_t> edge_fixed, node_fixed;   // PEC DOFs
    std::vector<int32_t> e_rp, e_col;              // edge-edge pattern (free DOFs)
    std::vector<double> M, S;                      // [*eps], [*S] on that pattern
    std::vector<int32_t> n_rp, n_col;              // node-node pattern
    std::vector<double> L;                         // D0^T [*eps] D0
};

// pec: boundary edges and nodes fixed at zero; else the natural boundary (nothing fixed)
void assemble_fields(const HostComplex& hc, double eps, double mu, bool pec, HostFields* hf);

// Largest eigenvalue of D^-1 A (A symmetric CSR with positive diagonal), estimated by
// `steps` Lanczos steps on D^-1/2 A D^-1/2 from a fixed start vector (a lower bound that
// converges quickly for the top of the spectrum).
double jacobi_lambda_max(const std::vector<int32_t>& rp, const std::vector<int32_t>& col,
                         const std::vector<double>& val, int steps);

struct LearnedDev;  // learned correction (learned.cu)

struct FieldDev {
    double dt = 0, eps = 0, mu = 0;
    int bc = FP_BC_PEC;             // field boundary condition
    // natural boundary: the W0 integrals alpha (device) and their sum, for the projection's
    // zero-mean constraint; partial sums of its two reductions
    double* alpha = nullptr;
    double alpha_sum = 0.0;
    double* msum = nullptr;
    int64_t ne = 0, nn = 0, nf = 0;
    HostFields host;
    int32_t *e_rp = nullptr, *e_col = nullptr, *n_rp = nullptr, *n_col = nullptr;
    double *Mv = nullptr, *Sv = nullptr, *Av = nullptr, *Adinv = nullptr, *Lv = nullptr, *Ldinv = nullptr;
    uint8_t *edge_fixed = nullptr, *node_fixed = nullptr;
    int32_t* face_edges = nullptr;  // [3 nf]: (i,j), (j,k), (i,k) of face (i<j<k)
    double *r = nullptr, *z = nullptr, *p = nullptr, *q = nullptr, *rhs = nullptr, *tmp = nullptr,
           *delta = nullptr, *qd = nullptr;
    float *Av32 = nullptr, *Adinv32 = nullptr, *Lv32 = nullptr, *Ldinv32 = nullptr;  // FP32 copies
    // sliced ELLPACK (slices of 32 rows, column-major inside a slice): coalesced loads of the
    // values and columns of 32 consecutive rows
    int32_t *se_ptr = nullptr, *se_w = nullptr, *se_col = nullptr, *sn_ptr = nullptr, *sn_w = nullptr,
            *sn_col = nullptr;
    double *se_M = nullptr, *se_S = nullptr, *se_A = nullptr, *sn_L = nullptr;
    float *se_A32 = nullptr, *sn_L32 = nullptr;
    float *r32 = nullptr, *z32 = nullptr, *p32 = nullptr, *q32 = nullptr, *c32 = nullptr;
    float *s32 = nullptr, *d32[2] = {nullptr, nullptr};  // Chebyshev preconditioner scratch
    double lmax[2] = {2.0, 2.0};    // estimated largest eigenvalue of D^-1 A, Newmark and Gauss systems
    // FP32 operators held in shared memory by the mixed solver (per system): column offsets
    // col - row as int16 in the SELL layout, and the slots per block (0: not held)
    int16_t *se_d16 = nullptr, *sn_d16 = nullptr;
    // the 16-bit column encoding of the mixed solver's streamed operators (Sell::cb, Sell::cd):
    // Newmark in the solver's row order, Gauss law (null when some offset does not fit)
    int32_t *pe_cb = nullptr, *sn_cb = nullptr;
    int16_t *pe_cd = nullptr, *sn_cd = nullptr;
    // The mixed solver's copy of the Newmark operator in its own row order: solver row r is
    // edge perm_e[r] (rows and columns renumbered alike).  Right-hand side and guess are
    // gathered into pb / px before each solve and the solution scattered back after it.
    // se_d16 and hptr / slots_total of the Newmark system describe this copy.
    int32_t *pe_ptr = nullptr, *pe_w = nullptr, *pe_col = nullptr, *perm_e = nullptr;
    double* pe_A = nullptr;
    float *pe_A32 = nullptr, *pe_dinv32 = nullptr;
    double *pb = nullptr, *px = nullptr;
    int64_t sectors_e[2] = {0, 0};  // gathered 32-byte sectors per product: edge order, solver order
    int64_t slots_total[2] = {0, 0};
    int sm_slots[2] = {0, 0};
    int sm_learned[2] = {0, 0};     // the learned preconditioner's values fit in shared memory too
    std::vector<int32_t> hptr[2];   // host copies of the SELL slice starts (Newmark, Gauss)
    double* red = nullptr;          // reduction partials
    double* out = nullptr;          // [8] solver outputs (iterations, rr, bb) of the last two solves
    int grid = 0;                   // co-resident blocks (cooperative launch limit)
    int grid_e = 0, grid_n = 0;     // grids of the edge and node systems
    int bs_e = 256, bs_n = 256;     // and their block sizes
    int last_fp64[2] = {0, 0};      // solver used by the last solve in each info slot
    LearnedDev* learned[2] = {nullptr, nullptr};  // per system (Newmark, Gauss)
    int learned_sys = FP_SYS_NEWMARK;              // system the fem_pic_learned_* calls address
    bool learned_used[2] = {false, false};         // the last solve in each info slot used its network
    int slot_sys[2] = {FP_SYS_NEWMARK, FP_SYS_GAUSS};  // system of the last solve in each info slot
};

#ifdef __CUDACC__
struct Sell {
    const int32_t* ptr;   // [slices] start of each slice
    const int32_t* w;     // [slices] width (longest row) of each slice
    const int32_t* col;   // padded entries point at the row itself with value 0
    // the same columns in 16 bits (null when not built): column = cb[ptr/32 + j] + lane + cd,
    // one 32-bit base per slice position j (the 32 lanes' j-th entries), a 16-bit offset per entry
    const int32_t* cb = nullptr;
    const int16_t* cd = nullptr;
};

// row i of a SELL-32 matrix times x; the 32 lanes of a warp take the 32 rows of a slice.
// The entries are taken in chunks of kSellChunk: the column indices of a chunk are loaded
// together, then the values and the gathered x, so a thread has a chunk of independent
// loads in flight instead of one dependent index -> x pair at a time.
#ifndef FP_SELL_CHUNK
#define FP_SELL_CHUNK 8
#endif
constexpr int kSellChunk = FP_SELL_CHUNK;

// Operator entries are read once per product and streamed: with FP_SELL_STREAM (the default)
// they are loaded with the evict-first hint so that they do not push the gathered vector out
// of L2 (96^3 mesh: Gauss-law solve 5.6 -> 4.3 ms, Newmark 19.9 -> 19.4 ms).
#ifndef FP_SELL_STREAM
#define FP_SELL_STREAM 1
#endif
template <typename T>
__device__ __forceinline__ T ld_op(const T* p) {
#if FP_SELL_STREAM
    return __ldcs(p);
#else
    return __ldg(p);
#endif
}

template <typename V, typename X>
__device__ __forceinline__ X sell_row(const Sell& S, const V* __restrict__ val, const X* __restrict__ x,
                                      int64_t i) {
    const int64_t sl = i >> 5;
    const int32_t* cp = S.col + __ldg(S.ptr + sl) + (i & 31);
    const V* vp = val + __ldg(S.ptr + sl) + (i & 31);
    const int w = __ldg(S.w + sl);
    X s = X(0);
    for (int j0 = 0; j0 < w; j0 += kSellChunk) {
        int c[kSellChunk];
        V a[kSellChunk];
        X xv[kSellChunk];
#pragma unroll
        for (int u = 0; u < kSellChunk; ++u) c[u] = j0 + u < w ? ld_op(cp + 32 * (j0 + u)) : -1;
#pragma unroll
        for (int u = 0; u < kSellChunk; ++u) a[u] = j0 + u < w ? ld_op(vp + 32 * (j0 + u)) : V(0);
#pragma unroll
        for (int u = 0; u < kSellChunk; ++u) xv[u] = c[u] >= 0 ? __ldcg(x + c[u]) : X(0);
#pragma unroll
        for (int u = 0; u < kSellChunk; ++u) s += (X)a[u] * xv[u];
    }
    return s;
}

// sell_row with the 16-bit column encoding (S.cd, S.cb non-null): 2 bytes per entry and one
// base per 32 entries instead of 4 bytes per entry; the base is one broadcast load per warp
template <typename V, typename X>
__device__ __forceinline__ X sell_row16(const Sell& S, const V* __restrict__ val, const X* __restrict__ x,
                                        int64_t i) {
    const int64_t sl = i >> 5;
    const int32_t p0 = __ldg(S.ptr + sl);
    const int16_t* dp = S.cd + p0 + (i & 31);
    const int32_t* bp = S.cb + (p0 >> 5);
    const V* vp = val + p0 + (i & 31);
    const int w = __ldg(S.w + sl);
    const int lane = (int)(i & 31);
    X s = X(0);
    for (int j0 = 0; j0 < w; j0 += kSellChunk) {
        int c[kSellChunk];
        V a[kSellChunk];
        X xv[kSellChunk];
#pragma unroll
        for (int u = 0; u < kSellChunk; ++u)
            c[u] = j0 + u < w ? ld_op(bp + j0 + u) + lane + (int)ld_op(dp + 32 * (j0 + u)) : -1;
#pragma unroll
        for (int u = 0; u < kSellChunk; ++u) a[u] = j0 + u < w ? ld_op(vp + 32 * (j0 + u)) : V(0);
#pragma unroll
        for (int u = 0; u < kSellChunk; ++u) xv[u] = c[u] >= 0 ? __ldcg(x + c[u]) : X(0);
#pragma unroll
        for (int u = 0; u < kSellChunk; ++u) s += (X)a[u] * xv[u];
    }
    return s;
}

// the FP32 products of the mixed solver: 16-bit columns where built
template <typename V, typename X>
__device__ __forceinline__ X sell_row_any(const Sell& S, const V* __restrict__ val, const X* __restrict__ x,
                                          int64_t i) {
    return S.cd ? sell_row16<V, X>(S, val, x, i) : sell_row<V, X>(S, val, x, i);
}

#endif

// learned correction hooks (learned.cu)
void learned_free(FieldDev* F);
void learned_free(FieldDev* F, int sys);
fp_status learned_guess(fem_pic* ctx, int sys, const double* rhs, double* x0, cudaStream_t s);
bool learned_active(const FieldDev* F, int sys);
int* learned_flag(FieldDev* F, int sys);
// the learned preconditioner's correction (solver SELL layout) when it is active and built, else null
const __nv_bfloat16* learned_precond(const FieldDev* F, int sys);
bool learned_precond_ready(const FieldDev* F, int sys);   // model FP_LEARNED_PRECOND, built
int learned_model(const FieldDev* F, int sys);            // -1: no network
void learned_set_active(FieldDev* F, int sys, bool on);

}  // namespace fempic
