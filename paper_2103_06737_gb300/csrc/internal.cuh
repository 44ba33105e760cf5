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
    float gsum;      // sum of |g| over g[0..8] (written with the field coefficients)
    float pad[2];
};
static_assert(sizeof(TetHot) == 128, "TetHot layout");

// bits of the device status word
// ST_NONFINITE: a particle's position or velocity (given, or after its push) was not finite;
// the particle was removed (cell -1) with nothing deposited
enum : int32_t { ST_WALK = 1, ST_INVAL = 2, ST_NOCONV = 4, ST_TIMEOUT = 8, ST_NONFINITE = 16 };

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

namespace fempic {
struct FieldDev;
void field_free(fem_pic* ctx);
// phases timed by the optional profiler (fem_pic_profile_*)
enum Phase : int { PH_PREP = 0, PH_FAST = 1, PH_WALK = 2, PH_PUSH64 = 3, PH_CHARGE = 4, PH_SORT = 5,
                   PH_RESID = 6, PH_SOLVE = 7, PH_CG_NEWMARK = 8, PH_CG_GAUSS = 9, PH_LEARNED = 10,
                   PH_ADAMS = 11, PH_ADAMS_WALK = 12, PH_COUNT = 16 };
struct ProfRec {
    int phase;
    cudaEvent_t a, b;
};
}  // namespace fempic

struct fem_pic {
    int device = 0;
    int sm_count = 152;
    fempic::FieldDev* field = nullptr;  // implicit field step (fem_pic_field_setup)
    int solver_fp64 = 0;                // 1: plain FP64 PCG, 0: mixed-precision refinement
    int solver_sys[2] = {-1, -1};       // per-system override (FP_PC_JACOBI / _FP64), -1 = as requested
    double inner_tol = 1e-5;            // mixed solver: residual reduction of each FP32 inner solve
    int poly_deg[2] = {1, 1};           // mixed solver: Chebyshev degree of the Jacobi preconditioner per system
    double poly_ratio[2] = {30.0, 30.0};  // and lambda_max / lambda_low of its interval
    // profiler: events recorded on the launch stream around each kernel when enabled
    bool prof_on = false;
    std::vector<fempic::ProfRec> prof_pending;
    std::vector<cudaEvent_t> prof_pool;
    double prof_ms[fempic::PH_COUNT] = {0};
    int64_t prof_n[fempic::PH_COUNT] = {0};
    int precision = FP_FP64;
    int dG64 = 0;  // FP32 mode: dG is a double array (fem_pic_set_deposit_precision)
    int Q64 = 0;   // FP32 mode: Q is a double array (fem_pic_set_deposit_precision, _charge_precision)
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
    double* d_field64 = nullptr;      // [10 nt] FP64 mode: per tet E0, W, B0, beta (affine fields)
    int4* d_tet_faces = nullptr;      // [nt] face ids of each tet (face k opposite vertex k)
    int32_t* d_status = nullptr;
    // particles deferred to the FP64 walk (near or across a face)
    int32_t* d_slow_idx = nullptr;    // [slow_cap]
    int32_t* d_slow_count = nullptr;  // [1]
    int64_t slow_cap = 0;
    // device address of the allocation-free push's fixed queue in this handle's context
    int32_t* d_static_queue = nullptr;
    // co-resident blocks of the staged push kernels (0: not queried yet): bulk-copy pipeline,
    // warp-specialised Boris push, warp-specialised Adams push
    int tma_blocks_per_sm = 0;
    int ws_blocks_per_sm = 0;
    int run_blocks_per_sm[4] = {0, 0, 0, 0};  // per (dG double) + 2 (Q double)
    int ws_adams_blocks_per_sm = 0;
    uint8_t* d_node_wall = nullptr;   // [nn] 1 = node on the PEC boundary
    // sort scratch
    int32_t* d_sort_count = nullptr;  // [nt + 2]
    int32_t* d_sort_block = nullptr;  // block sums
    int32_t* d_sort_rank = nullptr;   // [cap]
    int64_t sort_cap = 0;
    std::string err;
};

// dG / Q are float arrays (FP32 mode with FP32 deposits), else double
inline bool dG_f32(const fem_pic* ctx) { return ctx->precision == FP_FP32 && !ctx->dG64; }
inline bool Q_f32(const fem_pic* ctx) { return ctx->precision == FP_FP32 && !ctx->Q64; }

#define FP_CUDA_TRY(ctx, call)                                                             \
    do {                                                                                   \
        cudaError_t _e = (call);                                                           \
        if (_e != cudaSuccess) {                                                           \
            if (ctx) (ctx)->err = std::string(#call ": ") + cudaGetErrorString(_e);        \
            return FP_ECUDA;                                                               \
        }                                                                                  \
    } while (0)

namespace fempic {
#ifdef __CUDACC__
// Conversions between float and double with integer operations only.  On GB300 the
// FP64 pipe (which also executes F2F conversions) issues 2 thread-operations per clock
// per SM, so the particle and residual kernels convert through the bit patterns.
// f2d is exact for normal floats, zeros, infinities and NaN; float subnormals become
// signed zero.  d2f rounds to nearest, ties to even, like __double2float_rn, for
// results in the normal float range; results below it become signed zero, above it
// signed infinity; NaN stays NaN.
__device__ __forceinline__ double f2d(float f) {
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    const unsigned long long sgn = (unsigned long long)(u >> 31) << 63;
    const unsigned long long man = (unsigned long long)(u & 0x7fffffu) << 29;
    const unsigned long long ex = e == 0xffu ? 0x7ffull : (unsigned long long)(e + (1023u - 127u));
    const unsigned long long bits = e == 0u ? sgn : (sgn | (ex << 52) | man);
    return __longlong_as_double((long long)bits);
}

__device__ __forceinline__ float d2f(double d) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(d);
    const unsigned sign = (unsigned)(u >> 63) << 31;
    const int e = (int)((u >> 52) & 0x7ffull);
    const unsigned long long m = u & 0xfffffffffffffull;
    const int ef = e - 1023 + 127;
    const unsigned rem = (unsigned)(m & 0x1fffffffull);  // the 29 bits dropped
    unsigned r = ((unsigned)(ef & 0xff) << 23) | (unsigned)(m >> 29);
    r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;  // carry may raise the exponent
    r = ef <= 0 ? 0u : (ef >= 255 ? 0x7f800000u : r);
    r = e == 0x7ff ? (0x7f800000u | (m ? 0x400000u : 0u)) : r;
    return __uint_as_float(r | sign);
}

// A deposit contribution in the element type of its array: a float goes into a double array
// through f2d (so a float subnormal contribution, below 1.2e-38 in magnitude, adds zero);
// a double (FP64 mode) or a float into a float array is passed as it is.
template <typename D>
__device__ __forceinline__ D dep_cast(float x) {
    if constexpr (sizeof(D) == 8) return f2d(x);
    else return x;
}
template <typename D>
__device__ __forceinline__ D dep_cast(double x) {
    static_assert(sizeof(D) == 8, "double contributions go into double arrays");
    return x;
}

// x < 0 strictly (and not NaN-with-sign), from the bit pattern
__device__ __forceinline__ bool neg_strict(double x) {
    const long long b = __double_as_longlong(x);
    return b < 0 && b != (long long)0x8000000000000000ull;
}
// x is neither infinite nor NaN (exponent field not all ones), from the bit pattern
__device__ __forceinline__ bool finite_bits(double x) {
    return ((__double_as_longlong(x) >> 52) & 0x7ff) != 0x7ff;
}
__device__ __forceinline__ bool finite_bits(float x) {
    return ((__float_as_uint(x) >> 23) & 0xffu) != 0xffu;
}
// x > 0 strictly, from the bit pattern (NaN with a clear sign bit counts as > 0)
__device__ __forceinline__ bool pos_strict(double x) {
    return __double_as_longlong(x) > 0;
}
#endif
}  // namespace fempic

// launchers implemented in the .cu files
namespace fempic {
// Records an event pair around the launches in its scope when profiling is on.
struct PhaseTimer {
    fem_pic* c;
    int ph;
    cudaStream_t s;
    cudaEvent_t a = nullptr;
    static cudaEvent_t get(fem_pic* c) {
        if (!c->prof_pool.empty()) {
            cudaEvent_t e = c->prof_pool.back();
            c->prof_pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        return e;
    }
    PhaseTimer(fem_pic* c_, int ph_, cudaStream_t s_) : c(c_), ph(ph_), s(s_) {
        if (c->prof_on) {
            a = get(c);
            if (a) cudaEventRecord(a, s);
        }
    }
    ~PhaseTimer() {
        if (!a) return;
        cudaEvent_t b = get(c);
        if (!b) {
            c->prof_pool.push_back(a);
            return;
        }
        cudaEventRecord(b, s);
        c->prof_pending.push_back({ph, a, b});
    }
};
fp_status launch_push_deposit(fem_pic* ctx, const double* e, const double* b, const fp_particles* p,
                              double dt, int max_cross, void* dG, void* Q, int flags,
                              cudaStream_t s);
fp_status launch_push_adams(fem_pic* ctx, const double* e, const double* b, const fp_particles* p, void* hist,
                            int64_t step, double dt, int max_cross, void* dG, void* Q, int flags, cudaStream_t s);
fp_status static_queue_lookup(fem_pic* ctx);
fp_status launch_wait_selftest(fem_pic* ctx, double limit_s, cudaStream_t s);
fp_status launch_deposit_charge(fem_pic* ctx, const fp_particles* p, void* Q, int flags,
                                cudaStream_t s);
fp_status launch_sort(fem_pic* ctx, const fp_particles* src, fp_particles* dst, cudaStream_t s,
                      const void* cols_src = nullptr, void* cols_dst = nullptr, int ncols = 0);
fp_status launch_residuals(fem_pic* ctx, const void* dG, const void* Qn, const void* Qo,
                           const double* b, double* out, cudaStream_t s);
}  // namespace fempic
