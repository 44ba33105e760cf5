// Implicit field step on the GPU (FP64): Newmark wave-equation update, Gauss-law
// projection, Faraday update (Sec. II.C, IV.A-B), with a Jacobi-preconditioned CG that
// runs as one cooperative kernel (convergence decided on the device, no host round trip).
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "async_copy.cuh"
#include "field.cuh"

namespace cg = cooperative_groups;


namespace fempic {


namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kBlock = 256;
// Cooperative solvers: up to 2 co-resident blocks per SM (1 for 1024-thread blocks); the block
// size is chosen per system from kSolverBlocks at setup.
constexpr int kSolverPerSm = 2;
// fraction of the outer threshold an inner solve aims for when that needs less than
// inner_tol (the FP32 recurrence residual can differ slightly from the FP64 one)
constexpr double kInnerMargin = 0.2;

__device__ __forceinline__ double as_f64(float x) { return f2d(x); }
__device__ __forceinline__ double as_f64(double x) { return x; }

// Deterministic grid-wide sum of NV values, result valid in every thread.  Warp sums go to
// sh[k][warp]; thread 0 writes the block's partial to part[NV * block + k]; after the grid
// barrier warp 0 of every block adds all partials in block order and broadcasts through
// sh[k][BS / 32].  Two block barriers and one grid barrier per call.  Consecutive calls must
// use different `part` buffers (a block may write the next partials while another block
// still reads these).
template <int BS, int NV, typename T>
__device__ __forceinline__ void grid_sum(T v[NV], T* part, cg::grid_group& g, T (*sh)[BS / 32 + 1]) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(kFull, v[k], o);
    }
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k][wid] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            T t = T(0);
#pragma unroll
            for (int w = 0; w < BS / 32; ++w) t += sh[k][w];
            part[NV * blockIdx.x + k] = t;
        }
    g.sync();
    if (wid == 0) {
        T t[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) t[k] = T(0);
        for (int b = lane; b < (int)gridDim.x; b += 32)
#pragma unroll
            for (int k = 0; k < NV; ++k) t[k] += __ldcg(part + NV * b + k);
#pragma unroll
        for (int k = 0; k < NV; ++k) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) t[k] += __shfl_xor_sync(kFull, t[k], o);
        }
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < NV; ++k) sh[k][BS / 32] = t[k];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < NV; ++k) v[k] = sh[k][BS / 32];
}

struct PcgArgs {
    Sell S;
    const double* val;
    const double* dinv;
    int64_t n;
    const double* b;
    double* x;
    double *r, *z, *p, *q;
    double* red;
    double tol;
    const double* scale_vec;  // non-null: stop at ||r|| <= tol ||scale_vec||, else at ||r|| <= tol ||b||
    int max_iter;
    double* out;     // [iterations, ||r||^2, ||b||^2]
    int32_t* status;
};

// Jacobi-preconditioned conjugate gradients in one cooperative launch (FP64).  Every
// block takes the same decisions from the same grid-wide sums (deterministic: partials
// summed in block order), so all blocks run the same number of grid barriers; the loop is
// bounded by max_iter.  A p is carried as q = A z + beta q, two barriers per iteration.
template <int BS>
__global__ void __launch_bounds__(BS, BS >= 1024 ? 1 : kSolverPerSm) k_pcg(PcgArgs a) {
    cg::grid_group g = cg::this_grid();
    __shared__ double sh[4][BS / 32 + 1];
    // rows [r0, r1) of this block: contiguous runs of whole 32-row slices, so the columns a
    // block gathers (neighbouring DOFs) stay within a window that its SM's L1 can hold
    const int64_t chunk = ((a.n + gridDim.x - 1) / gridDim.x + 31) & ~(int64_t)31;
    const int64_t r0 = min(a.n, (int64_t)blockIdx.x * chunk), r1 = min(a.n, r0 + chunk);
    const int64_t stride = BS;
    const int64_t t0 = r0 + threadIdx.x;
    double* part0 = a.red;                    // 4 values per block
    double* part1 = a.red + 4 * gridDim.x;    // 2 values per block
    double* part2 = a.red + 6 * gridDim.x;    // 2 values per block
    double v[4] = {0.0, 0.0, 0.0, 0.0};  // r.r, b.b, s.s
    for (int64_t i = t0; i < r1; i += stride) {
        const double bi = a.b[i];
        const double ri = bi - sell_row<double, double>(a.S, a.val, a.x, i);
        a.r[i] = ri;
        a.z[i] = a.dinv[i] * ri;
        v[0] += ri * ri;
        v[1] += bi * bi;
        if (a.scale_vec) v[2] += a.scale_vec[i] * a.scale_vec[i];
    }
    grid_sum<BS, 4, double>(v, part0, g, sh);  // also makes z visible to every block
    double rr = v[0];
    const double bb = a.scale_vec ? v[2] : v[1];
    const double thr = a.tol * a.tol * bb;
    int it = 0;
    if (rr > thr && a.max_iter > 0) {
        // p = z, q = A z; rz, pq
        double u[2] = {0.0, 0.0};
        for (int64_t i = t0; i < r1; i += stride) {
            const double w = sell_row<double, double>(a.S, a.val, a.z, i);
            const double zi = a.z[i];
            a.p[i] = zi;
            a.q[i] = w;
            u[0] += a.r[i] * zi;
            u[1] += zi * w;
        }
        grid_sum<BS, 2, double>(u, part1, g, sh);
        double rz = u[0], pq = u[1];
        for (;;) {
            if (!(pq > 0.0)) break;  // breakdown (same decision in every block)
            const double alpha = rz / pq;
            double w2[2] = {0.0, 0.0};  // r.z, r.r
            for (int64_t i = t0; i < r1; i += stride) {
                a.x[i] += alpha * a.p[i];
                const double ri = a.r[i] - alpha * a.q[i];
                const double zi = a.dinv[i] * ri;
                a.r[i] = ri;
                a.z[i] = zi;
                w2[0] += ri * zi;
                w2[1] += ri * ri;
            }
            grid_sum<BS, 2, double>(w2, part2, g, sh);
            ++it;
            rr = w2[1];
            if (!(rr > thr) || it >= a.max_iter) break;
            const double beta = w2[0] / rz;
            rz = w2[0];
            double u2[2] = {0.0, 0.0};
            for (int64_t i = t0; i < r1; i += stride) {
                const double w = sell_row<double, double>(a.S, a.val, a.z, i);
                const double pi = a.z[i] + beta * a.p[i];
                const double qi = w + beta * a.q[i];
                a.p[i] = pi;
                a.q[i] = qi;
                u2[0] += pi * qi;
            }
            grid_sum<BS, 2, double>(u2, part1, g, sh);
            pq = u2[0];
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.out[0] = (double)it;
        a.out[1] = rr;
        a.out[2] = bb;      // squared norm the residual is measured against
        a.out[3] = 0.0;
        if (rr > thr) atomicOr(a.status, ST_NOCONV);
    }
}

// ---------------------------------------------------------------- mixed-precision solver
// Iterative refinement: the residual r = b - A x and its norm are FP64; each correction
// A c = r / |r| is solved approximately by Jacobi-PCG on FP32 copies of A and of the
// vectors, with FP32 dot products and grid sums (until its own residual drops by inner_tol,
// or by less when that already meets the outer tolerance), then x += |r| c in FP64.  FP64
// work is one product per refinement.  Two grid barriers per inner iteration (A p is
// carried as q = A z + beta q).

struct MixedArgs {
    Sell S;
    const double* val;     // FP64 operator (outer residual)
    const float* val32;    // FP32 copy (inner solves)
    const float* dinv32;
    int64_t n;
    const double* b;
    double* x;
    double* r64;
    float *r, *z, *p, *q, *c;
    // Chebyshev preconditioner of degree deg (1: plain Jacobi) on [theta - delta, theta + delta]
    int deg;
    float theta, delta;
    float *s, *d0, *d1;    // its residual and two buffers of its step (deg > 1)
    // FP32 operator in shared memory: sm_slots > 0 slots per block (values, then int16
    // column offsets), copied from val32 / d16 at the start of the launch
    const int16_t* d16;
    int sm_slots;
    int64_t slots_total;
    double* red;
    double tol;            // outer: ||b - A x|| <= tol ||ref||
    double inner_tol;      // inner: residual reduction per refinement
    const double* scale_vec;
    int max_iter;          // total inner iterations
    int max_outer;
    double* out;
    int32_t* status;
    // learned preconditioner (null: off): z = D^-1 r + Dl r with Dl on the operator's SELL
    // pattern, BF16 (replaces the Chebyshev polynomial); with sm_l the block's slots of Dl are
    // held in shared memory after the operator's; lflag (may be null) is set to 1 when the
    // solve fell back to Jacobi because r.z was not positive
    const __nv_bfloat16* dl16;
    int sm_l;
    int* lflag;
};

// This block's rows of the FP32 operator in shared memory (when the launch holds it there).
struct SmemOp {
    const float* v;       // values, SELL order, slots [base, base + count) of the global layout
    const int16_t* d;     // column - row
    int64_t base;
    const __nv_bfloat16* l;   // the learned preconditioner's values of the same slots (or null)
};

// A block's streamed product runs through its rows in steps of BS rows (thread 0 holds each
// step's first row).  With FP_SELL_PREFETCH = D > 0, thread 0 asks the TMA engine at every step
// to bring the SELL entries (columns and values) of the step D steps ahead into L2, so that the
// dependent column -> x gathers of the rows wait on L2 rather than HBM latency.  Rows of a step
// are whole 32-row slices; a slice's entries are 32 w slots from ptr, so the range is
// 128-byte aligned.
#ifndef FP_SELL_PREFETCH
#define FP_SELL_PREFETCH 1
#endif
__device__ __forceinline__ void sell_prefetch(const Sell& S, const void* val, int vbytes, int64_t i, int64_t r1,
                                              int64_t stride) {
#if FP_SELL_PREFETCH
    if (threadIdx.x != 0) return;
    const int64_t r0 = i + FP_SELL_PREFETCH * stride;
    if (r0 >= r1) return;
    const int64_t re = r0 + stride < r1 ? r0 + stride : r1;
    const int64_t s0 = r0 >> 5, s1 = (re - 1) >> 5;
    const int64_t k0 = __ldg(S.ptr + s0), k1 = (int64_t)__ldg(S.ptr + s1) + 32 * (int64_t)__ldg(S.w + s1);
    if (k1 <= k0) return;
    bulk_prefetch_l2(S.col + k0, (uint32_t)((k1 - k0) * 4));
    bulk_prefetch_l2(static_cast<const char*>(val) + k0 * vbytes, (uint32_t)((k1 - k0) * vbytes));
#endif
}

// row i of the FP32 operator times x: from shared memory (sm_slots > 0) or from the global
// SELL copy; chunks of CH independent loads (as in sell_row)
template <int CH>
__device__ __forceinline__ float row_product32(const MixedArgs& a, const SmemOp& so, const float* __restrict__ x,
                                               int64_t i) {
    if (a.sm_slots == 0) return sell_row_any<float, float>(a.S, a.val32, x, i);
    const int64_t sl = i >> 5;
    const int64_t base = __ldg(a.S.ptr + sl) - so.base + (i & 31);
    const int w = __ldg(a.S.w + sl);
    float s = 0.f;
    for (int j0 = 0; j0 < w; j0 += CH) {
        int c[CH];
        float av[CH], xv[CH];
#pragma unroll
        for (int u = 0; u < CH; ++u) {
            const bool in = j0 + u < w;
            c[u] = in ? (int)i + so.d[base + 32 * (j0 + u)] : -1;
            av[u] = in ? so.v[base + 32 * (j0 + u)] : 0.f;
        }
#pragma unroll
        for (int u = 0; u < CH; ++u) xv[u] = c[u] >= 0 ? __ldcg(x + c[u]) : 0.f;
#pragma unroll
        for (int u = 0; u < CH; ++u) s += av[u] * xv[u];
    }
    return s;
}

// entries per chunk of the mixed solver's products: 16 where the block size leaves the
// registers for them (blocks of at most 256 threads: up to 96 registers a thread), else the
// SELL default
#ifndef FP_SMALL_BLOCK_CHUNK
#define FP_SMALL_BLOCK_CHUNK 16
#endif
template <int BS>
struct ProductChunk {
    static constexpr int value = BS <= 256 ? FP_SMALL_BLOCK_CHUNK : kSellChunk;
};

// z = P(r) for the rows [t0, r1) of this block, P the Chebyshev polynomial of degree deg in
// B = D^-1 A applied to f = D^-1 r (three-term recurrence on [theta - delta, theta + delta]):
//   d_0 = f / theta, z = d_0, s = f;
//   k = 1..deg-1:  s <- s - B d_{k-1},  d_k = rho_k rho_{k-1} d_{k-1} + (2 rho_k / delta) s,
//                  z <- z + d_k,  rho_0 = delta / theta,  rho_k = 1 / (2 theta / delta - rho_{k-1}).
// P is positive on (0, theta + delta] and beyond it up to 2 theta, so PCG with it stays a
// symmetric positive definite method.  Each step's product needs the previous d of every
// block: one grid barrier per step, d in two buffers.  z is published by the caller's next
// grid barrier.
template <int CH>
__device__ __forceinline__ void chebyshev_apply(const MixedArgs& a, const SmemOp& so, int64_t t0, int64_t r1,
                                                int64_t stride, cg::grid_group& g) {
    const float th = a.theta, de = a.delta, sig = th / de;
    float rho = 1.f / sig;
    for (int64_t i = t0; i < r1; i += stride) {
        const float f = a.dinv32[i] * a.r[i];
        const float d = f / th;
        a.d0[i] = d;
        a.z[i] = d;
        a.s[i] = f;
    }
    float* dc = a.d0;
    float* dn = a.d1;
    for (int k = 1; k < a.deg; ++k) {
        g.sync();
        const float rn = 1.f / (2.f * sig - rho);
        const float c1 = rn * rho, c2 = 2.f * rn / de;
        for (int64_t i = t0; i < r1; i += stride) {
            if (a.sm_slots == 0) sell_prefetch(a.S, a.val32, 4, i, r1, stride);
            const float bd = a.dinv32[i] * row_product32<CH>(a, so, dc, i);
            const float sk = a.s[i] - bd;
            const float dk = c1 * dc[i] + c2 * sk;
            a.s[i] = sk;
            dn[i] = dk;
            a.z[i] += dk;
        }
        rho = rn;
        float* t = dc;
        dc = dn;
        dn = t;
    }
}

// z = D^-1 r + Dl r for the rows [t0, r1) of this block (the learned preconditioner); the
// product needs every block's r: one grid barrier first.  z is published by the caller's
// next grid barrier.  With rz_rr, r.z and r.r of these rows are added to rz_rr[0], rz_rr[1].
__device__ __forceinline__ void learned_apply(const MixedArgs& a, const SmemOp& so, int64_t t0, int64_t r1,
                                              int64_t stride, cg::grid_group& g, float* rz_rr = nullptr) {
    g.sync();
    if (so.l) {   // Dl and the column offsets from shared memory
        for (int64_t i = t0; i < r1; i += stride) {
            const int64_t sl = i >> 5;
            const int64_t base = __ldg(a.S.ptr + sl) - so.base + (i & 31);
            const int w = __ldg(a.S.w + sl);
            float t = 0.f;
            for (int j0 = 0; j0 < w; j0 += kSellChunk) {
                int c[kSellChunk];
                float lv[kSellChunk], xv[kSellChunk];
#pragma unroll
                for (int u = 0; u < kSellChunk; ++u) {
                    const bool in = j0 + u < w;
                    c[u] = in ? (int)i + so.d[base + 32 * (j0 + u)] : -1;
                    lv[u] = in ? __bfloat162float(so.l[base + 32 * (j0 + u)]) : 0.f;
                }
#pragma unroll
                for (int u = 0; u < kSellChunk; ++u) xv[u] = c[u] >= 0 ? __ldcg(a.r + c[u]) : 0.f;
#pragma unroll
                for (int u = 0; u < kSellChunk; ++u) t += lv[u] * xv[u];
            }
            const float ri = a.r[i], zi = a.dinv32[i] * ri + t;
            a.z[i] = zi;
            if (rz_rr) {
                rz_rr[0] += ri * zi;
                rz_rr[1] += ri * ri;
            }
        }
        return;
    }
    for (int64_t i = t0; i < r1; i += stride) {
        sell_prefetch(a.S, a.dl16, 2, i, r1, stride);
        const float ri = a.r[i], zi = a.dinv32[i] * ri + sell_row_any<__nv_bfloat16, float>(a.S, a.dl16, a.r, i);
        a.z[i] = zi;
        if (rz_rr) {
            rz_rr[0] += ri * zi;
            rz_rr[1] += ri * ri;
        }
    }
}

// Inner CG in the Chronopoulos-Gear form (one grid sum per iteration instead of two)
#ifndef FP_CG_ONE_SUM
#define FP_CG_ONE_SUM 0
#endif

template <int BS>
__global__ void __launch_bounds__(BS, BS >= 1024 ? 1 : kSolverPerSm) k_pcg_mixed(MixedArgs a) {
    cg::grid_group g = cg::this_grid();
    __shared__ double sh[4][BS / 32 + 1];
    __shared__ float shf[3][BS / 32 + 1];
    // rows [r0, r1) of this block: contiguous runs of whole 32-row slices, so the columns a
    // block gathers (neighbouring DOFs) stay within a window that its SM's L1 can hold
    const int64_t chunk = ((a.n + gridDim.x - 1) / gridDim.x + 31) & ~(int64_t)31;
    const int64_t r0 = min(a.n, (int64_t)blockIdx.x * chunk), r1 = min(a.n, r0 + chunk);
    const int64_t stride = BS;
    const int64_t t0 = r0 + threadIdx.x;
    // this block's slots of the FP32 operator into shared memory (whole 32-row slices)
    extern __shared__ __align__(16) unsigned char dsm[];
    SmemOp so{reinterpret_cast<const float*>(dsm),
              reinterpret_cast<const int16_t*>(dsm + 4 * (size_t)a.sm_slots), 0,
              a.sm_l && a.dl16 ? reinterpret_cast<const __nv_bfloat16*>(dsm + 6 * (size_t)a.sm_slots) : nullptr};
    if (a.sm_slots > 0) {
        const int64_t ns = (a.n + 31) >> 5, s0 = r0 >> 5, s1 = (r1 + 31) >> 5;
        const int64_t b0 = r0 < r1 ? __ldg(a.S.ptr + s0) : 0;
        const int64_t b1 = r0 < r1 ? (s1 < ns ? __ldg(a.S.ptr + s1) : a.slots_total) : 0;
        so.base = b0;
        float* v = reinterpret_cast<float*>(dsm);
        int16_t* d = reinterpret_cast<int16_t*>(dsm + 4 * (size_t)a.sm_slots);
        __nv_bfloat16* l = so.l ? reinterpret_cast<__nv_bfloat16*>(dsm + 6 * (size_t)a.sm_slots) : nullptr;
        for (int64_t k = threadIdx.x; k < b1 - b0; k += BS) {
            v[k] = __ldg(a.val32 + b0 + k);
            d[k] = __ldg(a.d16 + b0 + k);
            if (l) l[k] = a.dl16[b0 + k];
        }
        __syncthreads();
    }
    double* part0 = a.red;                               // 4 FP64 values per block
    float* part1 = (float*)(a.red + 4 * gridDim.x);      // 3 FP32 values per block
    float* part2 = part1 + 3 * gridDim.x;                // 2 FP32 values per block
    int total = 0, outer = 0;
    double rr64 = 0.0, ref2 = 0.0, thr = 0.0;
    bool use_l = a.dl16 != nullptr;   // every block takes the same fallback decision (grid sums)
    if (use_l && a.lflag && blockIdx.x == 0 && threadIdx.x == 0) *a.lflag = 0;
    for (;;) {
        // ---- outer residual in FP64: r = b - A x; its norm and the reference norm
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        for (int64_t i = t0; i < r1; i += stride) {
            const double bi = a.b[i];
            const double ri = bi - sell_row<double, double>(a.S, a.val, a.x, i);
            a.r64[i] = ri;
            a.c[i] = 0.f;
            v[0] += ri * ri;
            v[1] += bi * bi;
            if (a.scale_vec) v[2] += a.scale_vec[i] * a.scale_vec[i];
        }
        grid_sum<BS, 4, double>(v, part0, g, sh);
        rr64 = v[0];
        if (outer == 0) {
            ref2 = a.scale_vec ? v[2] : v[1];
            thr = a.tol * a.tol * ref2;
        }
        if (!(rr64 > thr) || total >= a.max_iter || outer >= a.max_outer) break;
        ++outer;
        // ---- inner FP32 Jacobi-PCG on A c = r / ||r||: vectors, products, dot products and
        // their grid sums all in FP32 (an inner solve only has to reduce its residual by
        // inner_tol; the FP64 outer residual corrects what FP32 loses)
        const double rnorm = sqrt(rr64), rinv = 1.0 / rnorm;
        for (int64_t i = t0; i < r1; i += stride) {
            const float ri = d2f(a.r64[i] * rinv);
            a.r[i] = ri;
            a.z[i] = a.dinv32[i] * ri;
        }
        if (use_l)
            learned_apply(a, so, t0, r1, stride, g);
        else if (a.deg > 1)
            chebyshev_apply<ProductChunk<BS>::value>(a, so, t0, r1, stride, g);
        g.sync();
        float u[3] = {0.f, 0.f, 0.f};  // r.z, p.q, r.r
        for (int64_t i = t0; i < r1; i += stride) {
            if (a.sm_slots == 0) sell_prefetch(a.S, a.val32, 4, i, r1, stride);
            const float w = row_product32<ProductChunk<BS>::value>(a, so, a.z, i);
            const float zi = a.z[i], ri = a.r[i];
            a.p[i] = zi;
            a.q[i] = w;
            u[0] += ri * zi;
            u[1] += zi * w;
            u[2] += ri * ri;
        }
        grid_sum<BS, 3, float>(u, part1, g, shf);
        if (use_l && !(u[0] > 0.f)) {   // the learned operator is not positive on r: Jacobi from here on
            use_l = false;
            if (a.lflag && blockIdx.x == 0 && threadIdx.x == 0) *a.lflag = 1;
            g.sync();
            continue;                   // c is still 0: the refinement restarts with Jacobi
        }
        float rz = u[0], pq = u[1];
        // the inner solve stops at a reduction of inner_tol, or earlier when a smaller
        // reduction (with a margin of kInnerMargin) already meets the outer tolerance
        const double need = kInnerMargin * sqrt(thr / rr64);
        const float red = (float)(need > a.inner_tol ? need : a.inner_tol);
        const float ithr = red * red * u[2];
#if FP_CG_ONE_SUM
        // Chronopoulos-Gear form: one grid sum per iteration.  After the update of c and r
        // and z = P(r), w = A z is formed behind a plain grid barrier, then r.z, r.r and z.w
        // are summed together; beta = (r.z)/(r.z)_old, p.q = z.w - beta (r.z) / alpha_old
        // (= p.A p), p = z + beta p, q = w + beta q (= A p).  w is kept in s (free between
        // applications of the preconditioner).
        float alpha = pq > 0.f ? rz / pq : 0.f;
        for (;;) {
            if (!(pq > 0.f) || total >= a.max_iter) break;
            float v3[3] = {0.f, 0.f, 0.f};  // r.z, r.r, z.w
            if (use_l) {
                for (int64_t i = t0; i < r1; i += stride) {
                    a.c[i] += alpha * a.p[i];
                    a.r[i] -= alpha * a.q[i];
                }
                learned_apply(a, so, t0, r1, stride, g);
            } else if (a.deg <= 1) {
                for (int64_t i = t0; i < r1; i += stride) {
                    a.c[i] += alpha * a.p[i];
                    const float ri = a.r[i] - alpha * a.q[i];
                    a.r[i] = ri;
                    a.z[i] = a.dinv32[i] * ri;
                }
            } else {
                for (int64_t i = t0; i < r1; i += stride) {
                    a.c[i] += alpha * a.p[i];
                    a.r[i] -= alpha * a.q[i];
                }
                chebyshev_apply<ProductChunk<BS>::value>(a, so, t0, r1, stride, g);
            }
            g.sync();   // z of every block before its product
            for (int64_t i = t0; i < r1; i += stride) {
                const float zi = a.z[i], ri = a.r[i];
                const float w = row_product32<ProductChunk<BS>::value>(a, so, a.z, i);
                a.s[i] = w;
                v3[0] += ri * zi;
                v3[1] += ri * ri;
                v3[2] += zi * w;
            }
            grid_sum<BS, 3, float>(v3, part1, g, shf);
            ++total;
            if (!(v3[1] > ithr)) break;
            if (use_l && !(v3[0] > 0.f)) {   // not positive on this r: keep c, Jacobi from here on
                use_l = false;
                if (a.lflag && blockIdx.x == 0 && threadIdx.x == 0) *a.lflag = 1;
                break;
            }
            const float beta = v3[0] / rz;
            pq = v3[2] - beta * v3[0] / alpha;
            rz = v3[0];
            alpha = pq > 0.f ? rz / pq : 0.f;
            for (int64_t i = t0; i < r1; i += stride) {
                a.p[i] = a.z[i] + beta * a.p[i];
                a.q[i] = a.s[i] + beta * a.q[i];
            }
        }
#else
        for (;;) {
            if (!(pq > 0.f) || total >= a.max_iter) break;
            const float alpha = rz / pq;
            float w2[2] = {0.f, 0.f};  // r.z, r.r
            if (use_l) {
                // r.z and r.r come with z; c += alpha p waits for the product loop, which
                // reads p anyway (or for the exit below)
                for (int64_t i = t0; i < r1; i += stride) a.r[i] -= alpha * a.q[i];
                learned_apply(a, so, t0, r1, stride, g, w2);
            } else if (a.deg <= 1) {
                for (int64_t i = t0; i < r1; i += stride) {
                    a.c[i] += alpha * a.p[i];
                    const float ri = a.r[i] - alpha * a.q[i];
                    const float zi = a.dinv32[i] * ri;
                    a.r[i] = ri;
                    a.z[i] = zi;
                    w2[0] += ri * zi;
                    w2[1] += ri * ri;
                }
            } else {
                for (int64_t i = t0; i < r1; i += stride) {
                    a.c[i] += alpha * a.p[i];
                    a.r[i] -= alpha * a.q[i];
                }
                chebyshev_apply<ProductChunk<BS>::value>(a, so, t0, r1, stride, g);
                for (int64_t i = t0; i < r1; i += stride) {
                    const float ri = a.r[i];
                    w2[0] += ri * a.z[i];
                    w2[1] += ri * ri;
                }
            }
            grid_sum<BS, 2, float>(w2, part2, g, shf);
            ++total;
            const bool l_step = use_l;   // this iteration deferred c += alpha p
            if (!(w2[1] > ithr) || (use_l && !(w2[0] > 0.f))) {
                if (use_l && !(w2[0] > 0.f)) {   // not positive on this r: keep c, Jacobi from here on
                    use_l = false;
                    if (a.lflag && blockIdx.x == 0 && threadIdx.x == 0) *a.lflag = 1;
                }
                if (l_step)
                    for (int64_t i = t0; i < r1; i += stride) a.c[i] += alpha * a.p[i];
                break;
            }
            const float beta = w2[0] / rz;
            rz = w2[0];
            float u2[1] = {0.f};
            for (int64_t i = t0; i < r1; i += stride) {
                if (a.sm_slots == 0) sell_prefetch(a.S, a.val32, 4, i, r1, stride);
                const float w = row_product32<ProductChunk<BS>::value>(a, so, a.z, i);
                if (l_step) a.c[i] += alpha * a.p[i];
                const float pi = a.z[i] + beta * a.p[i];
                const float qi = w + beta * a.q[i];
                a.p[i] = pi;
                a.q[i] = qi;
                u2[0] += pi * qi;
            }
            grid_sum<BS, 1, float>(u2, part1, g, shf);
            pq = u2[0];
        }
#endif
        for (int64_t i = t0; i < r1; i += stride) a.x[i] += rnorm * f2d(a.c[i]);
        g.sync();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.out[0] = (double)total;
        a.out[1] = rr64;
        a.out[2] = ref2;
        a.out[3] = (double)outer;
        if (rr64 > thr) atomicOr(a.status, ST_NOCONV);
    }
}

// Newmark right-hand side and the extrapolated initial guess 2E^n - E^{n-1}, in two passes
// so that the SELL pass does two FP64 multiply-adds per stored entry:
//   u = 2E^n - E^{n-1} (also the guess), v = -dt^2 (E^n / 2 + E^{n-1} / 4)   (per row)
//   rhs = [*eps] u + [*S] v - (dG^{n+1/2} - dG^{n-1/2})                      (SELL)
__global__ void k_newmark_uv(const uint8_t* __restrict__ fixed, const double* __restrict__ En,
                             const double* __restrict__ Em, double dt2, int64_t n, double* __restrict__ u,
                             double* __restrict__ v) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const double en = En[i], em = Em[i];
        u[i] = fixed[i] ? 0.0 : 2.0 * en - em;
        v[i] = -dt2 * (0.5 * en + 0.25 * em);
    }
}

template <typename Real>
__global__ void k_newmark_rhs(Sell Sl, const double* __restrict__ Mv, const double* __restrict__ Sv,
                              const uint8_t* __restrict__ fixed, const double* __restrict__ u,
                              const double* __restrict__ v, const Real* __restrict__ dGh,
                              const Real* __restrict__ dGp, int64_t n, double* __restrict__ rhs) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t sl = i >> 5;
        const int64_t base = __ldg(Sl.ptr + sl) + (i & 31);
        const int w = __ldg(Sl.w + sl);
        double s = 0.0;
        for (int j0 = 0; j0 < w; j0 += kSellChunk) {   // chunks of independent loads, as in sell_row
            int c[kSellChunk];
#pragma unroll
            for (int q = 0; q < kSellChunk; ++q) c[q] = j0 + q < w ? __ldg(Sl.col + base + 32 * (j0 + q)) : -1;
#pragma unroll
            for (int q = 0; q < kSellChunk; ++q) {
                if (c[q] < 0) continue;
                const int64_t k = base + 32 * (int64_t)(j0 + q);
                s = fma(__ldg(Mv + k), u[c[q]], s);
                s = fma(__ldg(Sv + k), v[c[q]], s);
            }
        }
        if (fixed[i]) {
            rhs[i] = 0.0;
            continue;
        }
        const double gh = dGh ? as_f64(dGh[i]) : 0.0, gp = dGp ? as_f64(dGp[i]) : 0.0;
        rhs[i] = s - (gh - gp);
    }
}

__global__ void k_spmv(Sell Sl, const double* __restrict__ val, const double* __restrict__ x, int64_t n,
                       double* __restrict__ y) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        y[i] = sell_row<double, double>(Sl, val, x, i);
}

// g_n = (D0^T [*eps] E)_n + Q_n on free nodes (ME = [*eps] E), 0 on PEC nodes
template <typename Real>
__global__ void k_gauss_rhs(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                            const int8_t* __restrict__ sgn, const uint8_t* __restrict__ fixed,
                            const double* __restrict__ ME, const Real* __restrict__ Q, int64_t nn,
                            double* __restrict__ g, double* __restrict__ qd) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += stride) {
        if (fixed[i]) {
            g[i] = 0.0;
            qd[i] = 0.0;
            continue;
        }
        double s = Q ? as_f64(Q[i]) : 0.0;
        qd[i] = s;
        for (int j = ptr[i]; j < ptr[i + 1]; ++j) s += sgn[j] > 0 ? ME[col[j]] : -ME[col[j]];
        g[i] = s;
    }
}

// E_e <- E_e - (d_j - d_i) on free edges: the Gauss-law projection E - D0 d
__global__ void k_project(const int32_t* __restrict__ edges, const uint8_t* __restrict__ fixed,
                          const double* __restrict__ d, const double* __restrict__ EN, int64_t ne,
                          double* __restrict__ E) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += stride)
        E[e] = fixed[e] ? 0.0 : EN[e] - (d[edges[2 * e + 1]] - d[edges[2 * e]]);
}

// b <- b - dt D1 (E1 + E0)/2, face (i<j<k): +(i,j) +(j,k) -(i,k)
__global__ void k_faraday(const int32_t* __restrict__ fe, const double* __restrict__ E1,
                          const double* __restrict__ E0, double half_dt, int64_t nf, double* __restrict__ b) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += stride) {
        const int ij = fe[3 * f], jk = fe[3 * f + 1], ik = fe[3 * f + 2];
        const double c = (E1[ij] + E0[ij]) + (E1[jk] + E0[jk]) - (E1[ik] + E0[ik]);
        b[f] -= half_dt * c;
    }
}

constexpr int kSolverBlocks[4] = {128, 256, 512, 1024};
// largest per-block share of an FP32 operator (4-byte values + 2-byte column offsets) that the
// mixed solver keeps in shared memory
constexpr size_t kSmemOperatorBytes = 200 * 1024;

void* solver_kernel(int bs, bool fp64) {
    switch (bs) {
        case 128: return fp64 ? (void*)k_pcg<128> : (void*)k_pcg_mixed<128>;
        case 256: return fp64 ? (void*)k_pcg<256> : (void*)k_pcg_mixed<256>;
        case 1024: return fp64 ? (void*)k_pcg<1024> : (void*)k_pcg_mixed<1024>;
        default: return fp64 ? (void*)k_pcg<512> : (void*)k_pcg_mixed<512>;
    }
}

int grid_of(const fem_pic* ctx, int64_t n) {
    int64_t g = (n + kBlock - 1) / kBlock, cap = (int64_t)ctx->sm_count * 8;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

template <typename T>
fp_status up(fem_pic* ctx, T** d, const std::vector<T>& h) {
    FP_CUDA_TRY(ctx, cudaMalloc((void**)d, h.size() * sizeof(T) + 16));
    if (!h.empty()) FP_CUDA_TRY(ctx, cudaMemcpy(*d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    return FP_OK;
}

// b and x into the solver's row order (row r is DOF perm[r]), and the solution back
__global__ void k_perm_gather(const int32_t* __restrict__ perm, const double* __restrict__ b,
                              const double* __restrict__ x, double* __restrict__ pb, double* __restrict__ px,
                              int64_t n) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = __ldg(perm + r);
        pb[r] = __ldg(b + k);
        px[r] = __ldg(x + k);
    }
}

// ... and, when ax is given, A x = b - r from the solve's last FP64 residual r (the mixed
// solver stops right after computing it for the final x), back in DOF order as well
__global__ void k_perm_scatter(const int32_t* __restrict__ perm, const double* __restrict__ px,
                               double* __restrict__ x, const double* __restrict__ pb,
                               const double* __restrict__ r64, double* __restrict__ ax, int64_t n) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t k = __ldg(perm + r);
        x[k] = px[r];
        if (ax) ax[k] = pb[r] - r64[r];
    }
}

// ax (Newmark system only, may be null): also A x for the final x, in DOF order, when the
// mixed solver ran (F->last_fp64[slot] == 0 afterwards); the FP64 solver leaves it alone
fp_status run_pcg(fem_pic* ctx, int system, const double* rhs, double* x, double tol, const double* scale_vec,
                  int max_iter, int slot, cudaStream_t s, double* ax = nullptr) {
    FieldDev* F = ctx->field;
    int use64 = ctx->solver_fp64;
    if (ctx->solver_sys[system] >= 0) use64 = ctx->solver_sys[system] == FP_PC_JACOBI_FP64;
    const int ph = system == FP_SYS_NEWMARK ? PH_CG_NEWMARK : PH_CG_GAUSS;
    F->last_fp64[slot] = use64;
    F->slot_sys[slot] = system;
    if (!use64) {
        MixedArgs m;
        if (system == FP_SYS_NEWMARK) {   // the solver's own row order (gathered in and scattered out below)
            m.S = Sell{F->pe_ptr, F->pe_w, F->pe_col, F->pe_cb, F->pe_cd}, m.val = F->pe_A, m.val32 = F->pe_A32,
            m.dinv32 = F->pe_dinv32, m.n = F->ne;
        } else {
            m.S = Sell{F->sn_ptr, F->sn_w, F->sn_col, F->sn_cb, F->sn_cd}, m.val = F->sn_L, m.val32 = F->sn_L32,
            m.dinv32 = F->Ldinv32, m.n = F->nn;
        }
        m.b = rhs, m.x = x, m.r64 = F->q;
        m.r = F->r32, m.z = F->z32, m.p = F->p32, m.q = F->q32, m.c = F->c32, m.red = F->red;
        {
            // Chebyshev interval [b / ratio, b] with b 5% above the Lanczos estimate of lambda_max
            const double bmax = 1.05 * F->lmax[system], blo = bmax / ctx->poly_ratio[system];
            m.deg = ctx->poly_deg[system];
            m.theta = (float)(0.5 * (bmax + blo));
            m.delta = (float)(0.5 * (bmax - blo));
            m.s = F->s32, m.d0 = F->d32[0], m.d1 = F->d32[1];
        }
        m.tol = tol, m.inner_tol = ctx->inner_tol, m.scale_vec = scale_vec, m.max_iter = max_iter, m.max_outer = 12;
        m.out = F->out + 4 * slot, m.status = ctx->d_status;
        m.dl16 = learned_precond(F, system);
        m.lflag = m.dl16 ? learned_flag(F, system) : nullptr;
        m.sm_l = 0;
        void* args[] = {&m};
        m.d16 = system == FP_SYS_NEWMARK ? F->se_d16 : F->sn_d16;
        m.sm_slots = F->sm_slots[system];
        m.slots_total = F->slots_total[system];
        // the learned preconditioner's BF16 values join the operator in shared memory when
        // the block's slots still fit (8 bytes per slot in all) with the launch co-resident
        if (m.dl16 && m.sm_slots > 0) m.sm_l = F->sm_learned[system];
        PhaseTimer pt(ctx, ph, s);
        const int grid = system == FP_SYS_NEWMARK ? F->grid_e : F->grid_n;
        const int bs = system == FP_SYS_NEWMARK ? F->bs_e : F->bs_n;
        const size_t smem = (size_t)m.sm_slots * (m.sm_l ? 8 : 6);
        if (system == FP_SYS_NEWMARK) {
            k_perm_gather<<<grid_of(ctx, F->ne), kBlock, 0, s>>>(F->perm_e, rhs, x, F->pb, F->px, F->ne);
            m.b = F->pb, m.x = F->px;
        }
        FP_CUDA_TRY(ctx, cudaLaunchCooperativeKernel(solver_kernel(bs, false), dim3(grid), dim3(bs), args, smem, s));
        if (system == FP_SYS_NEWMARK)
            k_perm_scatter<<<grid_of(ctx, F->ne), kBlock, 0, s>>>(F->perm_e, F->px, x, F->pb, F->q, ax, F->ne);
        FP_CUDA_TRY(ctx, cudaGetLastError());
        return FP_OK;
    }
    PcgArgs a;
    if (system == FP_SYS_NEWMARK) {
        a.S = Sell{F->se_ptr, F->se_w, F->se_col}, a.val = F->se_A, a.dinv = F->Adinv, a.n = F->ne;
    } else {
        a.S = Sell{F->sn_ptr, F->sn_w, F->sn_col}, a.val = F->sn_L, a.dinv = F->Ldinv, a.n = F->nn;
    }
    a.b = rhs, a.x = x, a.r = F->r, a.z = F->z, a.p = F->p, a.q = F->q, a.red = F->red;
    a.tol = tol, a.scale_vec = scale_vec, a.max_iter = max_iter, a.out = F->out + 4 * slot, a.status = ctx->d_status;
    void* args[] = {&a};
    PhaseTimer pt(ctx, ph, s);
    const int grid = system == FP_SYS_NEWMARK ? F->grid_e : F->grid_n;
    const int bs = system == FP_SYS_NEWMARK ? F->bs_e : F->bs_n;
    FP_CUDA_TRY(ctx, cudaLaunchCooperativeKernel(solver_kernel(bs, true), dim3(grid), dim3(bs), args, 0, s));
    return FP_OK;
}

fp_status fill_info(fem_pic* ctx, int slot, fp_solve_info* info, cudaStream_t s, float ms) {
    if (!info) return FP_OK;
    double o[4];
    FP_CUDA_TRY(ctx, cudaMemcpyAsync(o, ctx->field->out + 4 * slot, sizeof o, cudaMemcpyDeviceToHost, s));
    FP_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    info->iters = (int32_t)o[0];
    info->outer = (int32_t)o[3];
    info->rel_res = o[2] > 0 ? sqrt(o[1] / o[2]) : sqrt(o[1]);
    info->abs_res = sqrt(o[1]);
    info->ms = ms;
    info->precond = ctx->field->last_fp64[slot] ? FP_PC_JACOBI_FP64 : FP_PC_JACOBI;
    info->fell_back = 0;
    if (ctx->field->learned_used[slot]) {
        int fl = 0;
        FP_CUDA_TRY(ctx, cudaMemcpyAsync(&fl, learned_flag(ctx->field, ctx->field->slot_sys[slot]), sizeof(int),
                                         cudaMemcpyDeviceToHost, s));
        FP_CUDA_TRY(ctx, cudaStreamSynchronize(s));
        info->precond = FP_PC_LEARNED;
        info->fell_back = fl;
    }
    return FP_OK;
}

// Natural boundary (Eq. zero_mean_constraint): the projection solves L d = g - (sum g / sum
// alpha) alpha (L is singular, its null space the constants; the net charge is spread as
// alpha) and takes the solution with alpha^T d = 0, the d = C_z y of the constrained system.
// Both use a deterministic reduction: per-block partial sums, then every block adds the
// partials in block order before it updates its entries.
constexpr int kMeanBlocks = 128;

// part[b] = sum over block b's entries of v (w == nullptr) or of w v
__global__ void __launch_bounds__(256) k_dot_partial(const double* __restrict__ v, const double* __restrict__ w,
                                                     int64_t n, double* __restrict__ part) {
    __shared__ double sh[8];
    double t = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        t += w ? w[i] * v[i] : v[i];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = t;
    __syncthreads();
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int k = 0; k < 8; ++k) u += sh[k];
        part[blockIdx.x] = u;
    }
}

// y -= (scale sum_b part[b]) dir  (dir == nullptr: the constant vector 1)
__global__ void __launch_bounds__(256) k_sub_scaled(const double* __restrict__ part, int np, double scale,
                                                    const double* __restrict__ dir, int64_t n, double* __restrict__ y) {
    __shared__ double c;
    if (threadIdx.x == 0) {
        double u = 0.0;
        for (int k = 0; k < np; ++k) u += part[k];
        c = scale * u;
    }
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        y[i] -= dir ? c * dir[i] : c;
}

// the projection's right-hand side made consistent (natural boundary only)
fp_status neumann_rhs(fem_pic* ctx, cudaStream_t s) {
    FieldDev* F = ctx->field;
    if (F->bc != FP_BC_NEUMANN) return FP_OK;
    k_dot_partial<<<kMeanBlocks, 256, 0, s>>>(F->rhs, nullptr, F->nn, F->msum);
    k_sub_scaled<<<kMeanBlocks, 256, 0, s>>>(F->msum, kMeanBlocks, 1.0 / F->alpha_sum, F->alpha, F->nn, F->rhs);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}

// the projection's solution shifted to alpha^T d = 0 (natural boundary only)
fp_status neumann_gauge(fem_pic* ctx, cudaStream_t s) {
    FieldDev* F = ctx->field;
    if (F->bc != FP_BC_NEUMANN) return FP_OK;
    k_dot_partial<<<kMeanBlocks, 256, 0, s>>>(F->delta, F->alpha, F->nn, F->msum);
    k_sub_scaled<<<kMeanBlocks, 256, 0, s>>>(F->msum, kMeanBlocks, 1.0 / F->alpha_sum, nullptr, F->nn, F->delta);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}

fp_status field_step_impl(fem_pic_t* ctx, const double* E_prev, const double* E_cur, double* E_next,
                          double* b, const void* dG_half, const void* dG_prev, const void* Q_new, double tol,
                          int max_iter, cudaStream_t s) {
    FieldDev* F = ctx->field;
    const bool f32 = dG_f32(ctx), q32 = Q_f32(ctx);   // dG, Q are float arrays
    const int ge = grid_of(ctx, F->ne), gn = grid_of(ctx, F->nn);
    {
        PhaseTimer pt(ctx, PH_SOLVE, s);
        // u = 2E^n - E^{n-1} goes straight into E_next: it is also the solver's starting guess
        k_newmark_uv<<<ge, kBlock, 0, s>>>(F->edge_fixed, E_cur, E_prev, F->dt * F->dt, F->ne, E_next, F->tmp);
        if (f32)
            k_newmark_rhs<float><<<ge, kBlock, 0, s>>>(Sell{F->se_ptr, F->se_w, F->se_col}, F->se_M, F->se_S,
                                                       F->edge_fixed, E_next, F->tmp, (const float*)dG_half,
                                                       (const float*)dG_prev, F->ne, F->rhs);
        else
            k_newmark_rhs<double><<<ge, kBlock, 0, s>>>(Sell{F->se_ptr, F->se_w, F->se_col}, F->se_M, F->se_S,
                                                        F->edge_fixed, E_next, F->tmp, (const double*)dG_half,
                                                        (const double*)dG_prev, F->ne, F->rhs);
        FP_CUDA_TRY(ctx, cudaGetLastError());
    }
    // learned correction of the guess (with fallback), and/or collection of its residual
    if (learned_active(F, FP_SYS_NEWMARK)) {
        fp_status sl = learned_guess(ctx, FP_SYS_NEWMARK, F->rhs, E_next, s);
        if (sl != FP_OK) return sl;
    }
    // Newmark solve for E^N from the guess 2E^n - E^{n-1} (written into E_next above)
    fp_status st = run_pcg(ctx, FP_SYS_NEWMARK, F->rhs, E_next, tol, nullptr, max_iter, 0, s, F->tmp);
    if (st != FP_OK) return st;
    // Gauss-law projection: L d = D0^T M E^N + Q on interior nodes, to ||r|| <= tol ||Q||.
    // D0^T M E^N = D0^T A E^N, since D0^T S = (S D0)^T = 0 (curl grad = 0) on the rows the
    // interior nodes touch; the mixed solver hands back A E^N = b - r from its last residual,
    // so M E^N needs its own product only after the FP64 solver.
    {
        PhaseTimer pt(ctx, PH_SOLVE, s);
        if (F->last_fp64[0])
            k_spmv<<<ge, kBlock, 0, s>>>(Sell{F->se_ptr, F->se_w, F->se_col}, F->se_M, E_next, F->ne, F->tmp);
        if (q32)
            k_gauss_rhs<float><<<gn, kBlock, 0, s>>>(ctx->d_n2e_ptr, ctx->d_n2e_col, ctx->d_n2e_sgn, F->node_fixed,
                                                     F->tmp, (const float*)Q_new, F->nn, F->rhs, F->qd);
        else
            k_gauss_rhs<double><<<gn, kBlock, 0, s>>>(ctx->d_n2e_ptr, ctx->d_n2e_col, ctx->d_n2e_sgn,
                                                      F->node_fixed, F->tmp, (const double*)Q_new, F->nn, F->rhs,
                                                      F->qd);
        FP_CUDA_TRY(ctx, cudaMemsetAsync(F->delta, 0, F->nn * sizeof(double), s));
        FP_CUDA_TRY(ctx, cudaGetLastError());
        fp_status sn = neumann_rhs(ctx, s);
        if (sn != FP_OK) return sn;
    }
    // learned correction of the projection's zero starting point (node graph), with fallback
    if (learned_active(F, FP_SYS_GAUSS)) {
        fp_status sl = learned_guess(ctx, FP_SYS_GAUSS, F->rhs, F->delta, s);
        if (sl != FP_OK) return sl;
    }
    st = run_pcg(ctx, FP_SYS_GAUSS, F->rhs, F->delta, tol, F->qd, max_iter, 1, s);
    if (st != FP_OK) return st;
    {
        PhaseTimer pt(ctx, PH_SOLVE, s);
        st = neumann_gauge(ctx, s);
        if (st != FP_OK) return st;
        FP_CUDA_TRY(ctx, cudaMemcpyAsync(F->tmp, E_next, F->ne * sizeof(double), cudaMemcpyDeviceToDevice, s));
        k_project<<<ge, kBlock, 0, s>>>(ctx->d_edges, F->edge_fixed, F->delta, F->tmp, F->ne, E_next);
        if (b) k_faraday<<<grid_of(ctx, F->nf), kBlock, 0, s>>>(F->face_edges, E_next, E_cur, 0.5 * F->dt, F->nf, b);
        FP_CUDA_TRY(ctx, cudaGetLastError());
    }
    return FP_OK;
}

}  // namespace

void field_free(fem_pic* ctx) {
    FieldDev* F = ctx->field;
    if (!F) return;
    learned_free(F);
    void* ptrs[] = {F->e_rp, F->e_col, F->n_rp, F->n_col, F->Mv, F->Sv, F->Av, F->Adinv, F->Lv, F->Ldinv,
                    F->edge_fixed, F->node_fixed, F->face_edges, F->r, F->z, F->p, F->q, F->rhs, F->tmp,
                    F->delta, F->qd, F->red, F->out, F->Av32, F->Adinv32, F->Lv32, F->Ldinv32, F->r32,
                    F->z32, F->p32, F->q32, F->c32, F->s32, F->d32[0], F->d32[1], F->se_d16, F->sn_d16, F->pe_ptr, F->pe_w, F->pe_col, F->perm_e, F->pe_A, F->pe_A32, F->pe_dinv32, F->pb, F->px, F->alpha, F->msum, F->se_ptr, F->se_w, F->se_col, F->sn_ptr, F->sn_w,
                    F->sn_col, F->se_M, F->se_S, F->se_A, F->sn_L, F->se_A32, F->sn_L32, F->pe_cb, F->sn_cb,
                    F->pe_cd, F->sn_cd};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete F;
    ctx->field = nullptr;
}

}  // namespace fempic

using namespace fempic;

extern "C" {

fp_status fem_pic_field_setup(fem_pic_t* ctx, double dt, double eps, double mu) {
    return fem_pic_field_setup_bc(ctx, dt, eps, mu, FP_BC_PEC);
}

fp_status fem_pic_field_setup_bc(fem_pic_t* ctx, double dt, double eps, double mu, int bc) {
    if (!ctx || !(dt > 0.0) || !(eps > 0.0) || !(mu > 0.0) || (bc != FP_BC_PEC && bc != FP_BC_NEUMANN)) {
        if (ctx) ctx->err = "fem_pic_field_setup: dt, eps and mu must be positive, bc FP_BC_PEC or FP_BC_NEUMANN";
        return FP_EINVAL;
    }
    field_free(ctx);
    FieldDev* F = new FieldDev();
    ctx->field = F;
    const HostComplex& hc = ctx->hc;
    F->dt = dt, F->eps = eps, F->mu = mu, F->ne = hc.ne, F->nn = hc.nn, F->nf = hc.nf, F->bc = bc;
    assemble_fields(hc, eps, mu, bc == FP_BC_PEC, &F->host);
    const HostFields& H = F->host;
    std::vector<double> A(H.M.size()), Ad(hc.ne), Ld(hc.nn);
    for (size_t k = 0; k < A.size(); ++k) A[k] = H.M[k] + 0.25 * dt * dt * H.S[k];
    for (int64_t i = 0; i < hc.ne; ++i)
        for (int32_t j = H.e_rp[i]; j < H.e_rp[i + 1]; ++j)
            if (H.e_col[j] == i) Ad[i] = 1.0 / A[j];
    for (int64_t i = 0; i < hc.nn; ++i)
        for (int32_t j = H.n_rp[i]; j < H.n_rp[i + 1]; ++j)
            if (H.n_col[j] == i) Ld[i] = 1.0 / H.L[j];
    // top of the Jacobi-scaled spectra, for the Chebyshev preconditioner of the inner solves
    F->lmax[FP_SYS_NEWMARK] = jacobi_lambda_max(H.e_rp, H.e_col, A, 40);
    F->lmax[FP_SYS_GAUSS] = jacobi_lambda_max(H.n_rp, H.n_col, H.L, 40);
    // face -> edges (i,j), (j,k), (i,k)
    std::vector<int32_t> fe(3 * hc.nf);
    {
        std::vector<int32_t> rp, col;
        std::vector<int8_t> val;
        incidence_csr(hc, 1, &rp, &col, &val);  // columns sorted: (i,j) < (i,k) < (j,k)
        for (int64_t f = 0; f < hc.nf; ++f) {
            fe[3 * f] = col[3 * f];
            fe[3 * f + 1] = col[3 * f + 2];
            fe[3 * f + 2] = col[3 * f + 1];
        }
    }
    fp_status st = FP_OK;
    if (st == FP_OK) st = up(ctx, &F->e_rp, H.e_rp);
    if (st == FP_OK) st = up(ctx, &F->e_col, H.e_col);
    if (st == FP_OK) st = up(ctx, &F->n_rp, H.n_rp);
    if (st == FP_OK) st = up(ctx, &F->n_col, H.n_col);
    if (st == FP_OK) st = up(ctx, &F->Mv, H.M);
    if (st == FP_OK) st = up(ctx, &F->Sv, H.S);
    if (st == FP_OK) st = up(ctx, &F->Av, A);
    if (st == FP_OK) st = up(ctx, &F->Adinv, Ad);
    if (st == FP_OK) st = up(ctx, &F->Lv, H.L);
    if (st == FP_OK) st = up(ctx, &F->Ldinv, Ld);
    if (st == FP_OK) st = up(ctx, &F->edge_fixed, H.edge_fixed);
    if (st == FP_OK) st = up(ctx, &F->node_fixed, H.node_fixed);
    if (st == FP_OK) st = up(ctx, &F->face_edges, fe);
    {
        std::vector<float> a32(A.begin(), A.end()), ad32(Ad.begin(), Ad.end()), l32(H.L.begin(), H.L.end()),
            ld32(Ld.begin(), Ld.end());
        if (st == FP_OK) st = up(ctx, &F->Av32, a32);
        if (st == FP_OK) st = up(ctx, &F->Adinv32, ad32);
        if (st == FP_OK) st = up(ctx, &F->Lv32, l32);
        if (st == FP_OK) st = up(ctx, &F->Ldinv32, ld32);
    }
    {
        // SELL-32 copies of the operators (the CSR stays on the host for export)
        auto sell = [](const std::vector<int32_t>& rp, const std::vector<int32_t>& col, int64_t n,
                       std::vector<int32_t>* ptr, std::vector<int32_t>* w, std::vector<int32_t>* scol,
                       std::vector<int64_t>* map) {
            const int64_t ns = (n + 31) / 32;
            ptr->assign(ns, 0);
            w->assign(ns, 0);
            int64_t off = 0;
            for (int64_t sl = 0; sl < ns; ++sl) {
                int wmax = 0;
                for (int64_t r = 32 * sl; r < 32 * sl + 32 && r < n; ++r) wmax = std::max(wmax, rp[r + 1] - rp[r]);
                (*ptr)[sl] = (int32_t)off;
                (*w)[sl] = wmax;
                off += 32 * (int64_t)wmax;
            }
            scol->assign(off, 0);
            map->assign(off, -1);
            for (int64_t sl = 0; sl < ns; ++sl)
                for (int64_t lane = 0; lane < 32; ++lane) {
                    const int64_t r = 32 * sl + lane;
                    const int64_t base = (*ptr)[sl] + lane;
                    for (int j = 0; j < (*w)[sl]; ++j) {
                        const int64_t k = base + 32 * (int64_t)j;
                        if (r < n && j < rp[r + 1] - rp[r]) {
                            (*scol)[k] = col[rp[r] + j];
                            (*map)[k] = rp[r] + j;
                        } else {
                            (*scol)[k] = (int32_t)(r < n ? r : 0);  // padding: zero value
                        }
                    }
                }
        };
        auto gather = [](const std::vector<int64_t>& map, const std::vector<double>& v) {
            std::vector<double> o(map.size(), 0.0);
            for (size_t k = 0; k < map.size(); ++k)
                if (map[k] >= 0) o[k] = v[map[k]];
            return o;
        };
        std::vector<int32_t> ptr, w, scol;
        std::vector<int64_t> map;
        // column offsets col - row as int16 (empty when some offset does not fit)
        // (the lanes past the last row of a partial slice are never computed: offset 0)
        auto offsets16 = [](const std::vector<int32_t>& scol, const std::vector<int32_t>& sptr,
                            const std::vector<int32_t>& sw, int64_t n) {
            std::vector<int16_t> d(scol.size());
            for (size_t sl = 0; sl < sptr.size(); ++sl)
                for (int64_t j = 0; j < sw[sl]; ++j)
                    for (int64_t lane = 0; lane < 32; ++lane) {
                        const int64_t k = sptr[sl] + 32 * j + lane;
                        const int64_t row = (int64_t)(32 * sl + lane);
                        const int64_t off = row < n ? (int64_t)scol[k] - row : 0;
                        if (off < -32768 || off > 32767) return std::vector<int16_t>();
                        d[k] = (int16_t)off;
                    }
            return d;
        };
        // columns as a 32-bit base per slice position plus lane plus a 16-bit offset (Sell::cb,
        // Sell::cd); false when some offset does not fit.  The base is the middle of the lanes'
        // col - lane at that position: in an order where the 32 rows of a slice have the same
        // stencil (consecutive rows, consecutive neighbours) the offsets stay near 0.
        auto columns16 = [](const std::vector<int32_t>& scol, const std::vector<int32_t>& sptr,
                            const std::vector<int32_t>& sw, int64_t n, std::vector<int32_t>* cb,
                            std::vector<int16_t>* cd) {
            cb->assign(scol.size() / 32, 0);
            cd->assign(scol.size(), 0);
            for (size_t sl = 0; sl < sptr.size(); ++sl)
                for (int64_t j = 0; j < sw[sl]; ++j) {
                    int64_t lo = INT64_MAX, hi = INT64_MIN;
                    for (int64_t lane = 0; lane < 32 && 32 * (int64_t)sl + lane < n; ++lane) {
                        const int64_t v = (int64_t)scol[sptr[sl] + 32 * j + lane] - lane;
                        lo = std::min(lo, v);
                        hi = std::max(hi, v);
                    }
                    if (lo > hi) continue;   // no row (never computed)
                    const int64_t base = lo + (hi - lo) / 2;
                    if (hi - base > 32767 || lo - base < -32768) return false;
                    (*cb)[sptr[sl] / 32 + j] = (int32_t)base;
                    for (int64_t lane = 0; lane < 32 && 32 * (int64_t)sl + lane < n; ++lane) {
                        const int64_t k = sptr[sl] + 32 * j + lane;
                        (*cd)[k] = (int16_t)((int64_t)scol[k] - lane - base);
                    }
                }
            return true;
        };
        sell(H.e_rp, H.e_col, hc.ne, &ptr, &w, &scol, &map);
        std::vector<double> sM = gather(map, H.M), sS = gather(map, H.S), sA = gather(map, A);
        std::vector<float> sA32(sA.begin(), sA.end());
        if (st == FP_OK) st = up(ctx, &F->se_ptr, ptr);
        if (st == FP_OK) st = up(ctx, &F->se_w, w);
        if (st == FP_OK) st = up(ctx, &F->se_col, scol);
        if (st == FP_OK) st = up(ctx, &F->se_M, sM);
        if (st == FP_OK) st = up(ctx, &F->se_S, sS);
        if (st == FP_OK) st = up(ctx, &F->se_A, sA);
        if (st == FP_OK) st = up(ctx, &F->se_A32, sA32);
        {
            // Row order of the mixed solver's Newmark operator.  Edge ids are lexicographic in
            // (i, j), so the edges leaving a node are consecutive and a 32-row slice mixes edges
            // of several directions: lane l's k-th neighbour lies far from lane l+1's, and a
            // product gathers about one useful value per 32-byte sector of x.  Renumbered by
            // (block of kPermNodes first nodes, rank of the edge among its first node's edges,
            // first node), a slice holds same-rank edges of consecutive nodes, whose neighbours
            // are again consecutive.  Of the two orders the one whose products gather fewer
            // sectors (counted over its SELL layout) is kept, so a mesh without that structure
            // keeps the edge order; so is the edge order when the other's column offsets do
            // not fit in 16 bits.
            constexpr int32_t kPermNodes = 256;
            const int64_t ne = hc.ne;
            std::vector<int32_t> ident(ne), blocked(ne), rank(ne, 0);
            for (int64_t k = 0; k < ne; ++k) {
                ident[k] = (int32_t)k;
                if (k > 0 && hc.edges[2 * k] == hc.edges[2 * (k - 1)]) rank[k] = rank[k - 1] + 1;
            }
            blocked = ident;
            std::sort(blocked.begin(), blocked.end(), [&](int32_t a, int32_t b) {
                const int32_t ia = hc.edges[2 * a], ib = hc.edges[2 * b];
                if (ia / kPermNodes != ib / kPermNodes) return ia / kPermNodes < ib / kPermNodes;
                if (rank[a] != rank[b]) return rank[a] < rank[b];
                return ia != ib ? ia < ib : a < b;
            });
            // CSR of P A P^T (columns sorted) for perm (solver row -> edge)
            auto permuted = [&](const std::vector<int32_t>& perm, std::vector<int32_t>* rp2, std::vector<int32_t>* col2,
                                std::vector<double>* val2) {
                std::vector<int32_t> inv(ne);
                for (int64_t r = 0; r < ne; ++r) inv[perm[r]] = (int32_t)r;
                rp2->assign(ne + 1, 0);
                col2->resize(H.e_col.size());
                val2->resize(H.e_col.size());
                std::vector<std::pair<int32_t, double>> row;
                int64_t o = 0;
                for (int64_t r = 0; r < ne; ++r) {
                    const int32_t e0 = perm[r];
                    row.clear();
                    for (int32_t j = H.e_rp[e0]; j < H.e_rp[e0 + 1]; ++j) row.emplace_back(inv[H.e_col[j]], A[j]);
                    std::sort(row.begin(), row.end(),
                              [](const std::pair<int32_t, double>& a, const std::pair<int32_t, double>& b) {
                                  return a.first < b.first;
                              });
                    for (const auto& pr : row) (*col2)[o] = pr.first, (*val2)[o] = pr.second, ++o;
                    (*rp2)[r + 1] = (int32_t)o;
                }
            };
            // distinct 32-byte sectors of x that the lanes of each slice gather per entry
            auto sectors = [](const std::vector<int32_t>& rp, const std::vector<int32_t>& col, int64_t n) {
                int64_t total = 0;
                int32_t sec[32];
                for (int64_t r0 = 0; r0 < n; r0 += 32) {
                    const int64_t r1 = std::min<int64_t>(n, r0 + 32);
                    int w = 0;
                    for (int64_t r = r0; r < r1; ++r) w = std::max(w, rp[r + 1] - rp[r]);
                    for (int j = 0; j < w; ++j) {
                        int m = 0;
                        for (int64_t r = r0; r < r1; ++r)
                            if (j < rp[r + 1] - rp[r]) sec[m++] = col[rp[r] + j] >> 3;
                        std::sort(sec, sec + m);
                        total += (int64_t)(std::unique(sec, sec + m) - sec);
                    }
                }
                return total;
            };
            std::vector<int32_t> rp2, col2;
            std::vector<double> val2;
            permuted(blocked, &rp2, &col2, &val2);
            F->sectors_e[0] = sectors(H.e_rp, H.e_col, ne);
            F->sectors_e[1] = sectors(rp2, col2, ne);
            const std::vector<int32_t>* perm = &blocked;
            std::vector<int16_t> d16;
#ifndef FP_SOLVER_ORDER
#define FP_SOLVER_ORDER 1
#endif
            bool blocked_order = false;
            if (FP_SOLVER_ORDER && F->sectors_e[1] < F->sectors_e[0]) {
                // the solver order gathers fewer sectors; its 16-bit column offsets (for the
                // shared-memory operator) may not fit on large meshes, the order is kept anyway
                sell(rp2, col2, ne, &ptr, &w, &scol, &map);
                d16 = offsets16(scol, ptr, w, ne);
                blocked_order = true;
            }
            if (!blocked_order) {   // the edge order
                perm = &ident;
                F->sectors_e[1] = F->sectors_e[0];
                permuted(ident, &rp2, &col2, &val2);
                sell(rp2, col2, ne, &ptr, &w, &scol, &map);
                d16 = offsets16(scol, ptr, w, ne);
            }
            std::vector<double> pA = gather(map, val2);
            std::vector<float> pA32(pA.begin(), pA.end()), pdinv(ne);
            for (int64_t r = 0; r < ne; ++r) pdinv[r] = (float)Ad[(*perm)[r]];
#ifdef FP_SMEM_REPORT
            fprintf(stderr, "newmark solver order: %s, sectors %lld (edge order %lld), SELL slots %lld, nonzeros %lld\n",
                    perm == &blocked ? "blocked" : "edge", (long long)F->sectors_e[1], (long long)F->sectors_e[0],
                    (long long)scol.size(), (long long)H.e_col.size());
#endif
            if (!d16.empty() && st == FP_OK) st = up(ctx, &F->se_d16, d16);
            F->hptr[FP_SYS_NEWMARK] = ptr;
            F->slots_total[FP_SYS_NEWMARK] = (int64_t)scol.size();
            if (st == FP_OK) st = up(ctx, &F->perm_e, *perm);
            if (st == FP_OK) st = up(ctx, &F->pe_ptr, ptr);
            if (st == FP_OK) st = up(ctx, &F->pe_w, w);
            if (st == FP_OK) st = up(ctx, &F->pe_col, scol);
            {
                std::vector<int32_t> cb;
                std::vector<int16_t> cd;
                if (FP_COL16 && columns16(scol, ptr, w, ne, &cb, &cd)) {
                    if (st == FP_OK) st = up(ctx, &F->pe_cb, cb);
                    if (st == FP_OK) st = up(ctx, &F->pe_cd, cd);
                }
            }
            if (st == FP_OK) st = up(ctx, &F->pe_A, pA);
            if (st == FP_OK) st = up(ctx, &F->pe_A32, pA32);
            if (st == FP_OK) st = up(ctx, &F->pe_dinv32, pdinv);
            if (st == FP_OK) FP_CUDA_TRY(ctx, cudaMalloc((void**)&F->pb, ne * sizeof(double)));
            if (st == FP_OK) FP_CUDA_TRY(ctx, cudaMalloc((void**)&F->px, ne * sizeof(double)));
        }
        sell(H.n_rp, H.n_col, hc.nn, &ptr, &w, &scol, &map);
        std::vector<double> sL = gather(map, H.L);
        std::vector<float> sL32(sL.begin(), sL.end());
        {
            const std::vector<int16_t> d16 = offsets16(scol, ptr, w, hc.nn);
            if (!d16.empty() && st == FP_OK) st = up(ctx, &F->sn_d16, d16);
            F->hptr[FP_SYS_GAUSS] = ptr;
            F->slots_total[FP_SYS_GAUSS] = (int64_t)scol.size();
        }
        if (st == FP_OK) st = up(ctx, &F->sn_ptr, ptr);
        if (st == FP_OK) st = up(ctx, &F->sn_w, w);
        if (st == FP_OK) st = up(ctx, &F->sn_col, scol);
        {
            std::vector<int32_t> cb;
            std::vector<int16_t> cd;
            if (FP_COL16 && columns16(scol, ptr, w, hc.nn, &cb, &cd)) {
                if (st == FP_OK) st = up(ctx, &F->sn_cb, cb);
                if (st == FP_OK) st = up(ctx, &F->sn_cd, cd);
            }
        }
        if (st == FP_OK) st = up(ctx, &F->sn_L, sL);
        if (st == FP_OK) st = up(ctx, &F->sn_L32, sL32);
    }
    const int64_t nmax = hc.ne > hc.nn ? hc.ne : hc.nn;
    float** vecs32[] = {&F->r32, &F->z32, &F->p32, &F->q32, &F->c32, &F->s32, &F->d32[0], &F->d32[1]};
    for (float** v : vecs32)
        if (st == FP_OK) FP_CUDA_TRY(ctx, cudaMalloc((void**)v, nmax * sizeof(float)));
    double** vecs[] = {&F->r, &F->z, &F->p, &F->q, &F->rhs, &F->tmp, &F->delta, &F->qd};
    for (double** v : vecs)
        if (st == FP_OK) FP_CUDA_TRY(ctx, cudaMalloc((void**)v, nmax * sizeof(double)));
    // cooperative grids: all blocks co-resident, at most kSolverPerSm per SM.  Per system the
    // block size whose block count (one row per thread) is closest to one block per SM: the
    // grid barriers and reductions cost more with more blocks, the SpMV and vector passes
    // less with more SMs busy.
    auto pick = [&](int64_t rows, int force, int* bs, int* grid) -> fp_status {
        double best = 1e30;
        for (int b : kSolverBlocks) {
            const double d = std::fabs(std::log((double)((rows + b - 1) / b) / (double)ctx->sm_count));
            if (d < best) best = d, *bs = b;
        }
        if (force > 0) *bs = force;
        int per_sm = 0, per_sm2 = 0;
        FP_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, solver_kernel(*bs, true), *bs, 0));
        FP_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, solver_kernel(*bs, false), *bs, 0));
        per_sm = std::min(std::min(per_sm, per_sm2), kSolverPerSm);
        if (per_sm < 1) {
            ctx->err = "fem_pic_field_setup: the solver kernel cannot be co-resident";
            return FP_ECUDA;
        }
        const int64_t need = std::max<int64_t>(1, (rows + *bs - 1) / *bs);
        *grid = (int)std::min<int64_t>(need, (int64_t)ctx->sm_count * per_sm);
        return FP_OK;
    };
#ifndef FP_SOLVER_BS_E
#define FP_SOLVER_BS_E 0
#endif
#ifndef FP_SOLVER_BS_N
#define FP_SOLVER_BS_N 0
#endif
    if (st == FP_OK) st = pick(hc.ne, FP_SOLVER_BS_E, &F->bs_e, &F->grid_e);
    if (st == FP_OK) st = pick(hc.nn, FP_SOLVER_BS_N, &F->bs_n, &F->grid_n);
    // Shared-memory residency of the FP32 operator in the mixed solver: the slots of a
    // block's rows (its whole 32-row slices, as the kernel partitions them) must fit; the
    // launch then stays co-resident with that much shared memory per block.
    auto residency = [&](int sys, int64_t rows, int bs, int grid) -> fp_status {
        F->sm_slots[sys] = 0;
        const int16_t* d16 = sys == FP_SYS_NEWMARK ? F->se_d16 : F->sn_d16;
        if (!d16 || grid < 1) return FP_OK;
        const std::vector<int32_t>& ptr = F->hptr[sys];
        const int64_t ns = (int64_t)ptr.size();
        const int64_t chunk = ((rows + grid - 1) / grid + 31) & ~(int64_t)31;
        int64_t most = 0;
        for (int b = 0; b < grid; ++b) {
            const int64_t r0 = std::min<int64_t>(rows, (int64_t)b * chunk), r1 = std::min<int64_t>(rows, r0 + chunk);
            if (r0 >= r1) continue;
            const int64_t s0 = r0 >> 5, s1 = (r1 + 31) >> 5;
            const int64_t b1 = s1 < ns ? ptr[s1] : F->slots_total[sys];
            most = std::max<int64_t>(most, b1 - ptr[s0]);
        }
        const int64_t slots = (most + 7) & ~(int64_t)7;        // int16 part starts 16-byte aligned
        const size_t bytes = (size_t)slots * 6;
        if (bytes > kSmemOperatorBytes) return FP_OK;
        void* k = solver_kernel(bs, false);
        // the attribute is per kernel, shared by every context: set it to the device's limit
        // (less room for the kernel's static shared memory) so that no context lowers it below
        // what another one launches with
        int optin = 0;
        FP_CUDA_TRY(ctx, cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
        if (bytes + 4096 > (size_t)optin) return FP_OK;
        FP_CUDA_TRY(ctx, cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - 4096));
        int per_sm = 0;
        FP_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, bs, bytes));
        if ((int64_t)per_sm * ctx->sm_count < grid) return FP_OK;
        F->sm_slots[sys] = (int)slots;
        // room for the learned preconditioner's BF16 values beside them (8 bytes per slot)?
        F->sm_learned[sys] = 0;
        if ((size_t)slots * 8 <= kSmemOperatorBytes + 24 * 1024 && (size_t)slots * 8 + 4096 <= (size_t)optin) {
            int per_sm8 = 0;
            FP_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm8, k, bs, (size_t)slots * 8));
            F->sm_learned[sys] = (int64_t)per_sm8 * ctx->sm_count >= grid ? 1 : 0;
        }
        return FP_OK;
    };
#ifndef FP_SMEM_OPERATOR
#define FP_SMEM_OPERATOR 1
#endif
    if (FP_SMEM_OPERATOR && st == FP_OK) st = residency(FP_SYS_NEWMARK, hc.ne, F->bs_e, F->grid_e);
    if (FP_SMEM_OPERATOR && st == FP_OK) st = residency(FP_SYS_GAUSS, hc.nn, F->bs_n, F->grid_n);
    if (st == FP_OK) {
        F->grid = std::max(F->grid_e, F->grid_n);
        FP_CUDA_TRY(ctx, cudaMalloc((void**)&F->red, 9 * (size_t)F->grid * sizeof(double)));
        FP_CUDA_TRY(ctx, cudaMalloc((void**)&F->out, 16 * sizeof(double)));
        FP_CUDA_TRY(ctx, cudaMemset(F->out, 0, 16 * sizeof(double)));
    }
    if (st == FP_OK && bc == FP_BC_NEUMANN) {
        std::vector<double> a(hc.nn);
        st = fem_pic_whitney0_integrals(ctx, a.data());
        F->alpha_sum = 0.0;
        for (double v : a) F->alpha_sum += v;
        if (st == FP_OK) st = up(ctx, &F->alpha, a);
        if (st == FP_OK) FP_CUDA_TRY(ctx, cudaMalloc((void**)&F->msum, kMeanBlocks * sizeof(double)));
    }
    return st;
}

fp_status fem_pic_field_options(fem_pic_t* ctx, int newmark_solver, int gauss_solver, double inner_tol) {
    if (!ctx) return FP_EINVAL;
    auto ok = [](int v) { return v == -1 || v == FP_PC_JACOBI || v == FP_PC_JACOBI_FP64; };
    if (!ok(newmark_solver) || !ok(gauss_solver) || !(inner_tol > 0.0 && inner_tol < 1.0)) {
        ctx->err = "fem_pic_field_options: bad solver code or inner tolerance";
        return FP_EINVAL;
    }
    ctx->solver_sys[FP_SYS_NEWMARK] = newmark_solver;
    ctx->solver_sys[FP_SYS_GAUSS] = gauss_solver;
    ctx->inner_tol = inner_tol;
    return FP_OK;
}

fp_status fem_pic_field_poly(fem_pic_t* ctx, int system, int degree, double ratio) {
    if (!ctx || (system != FP_SYS_NEWMARK && system != FP_SYS_GAUSS) || degree < 1 || degree > 16 ||
        !(ratio > 1.0)) {
        if (ctx) ctx->err = "fem_pic_field_poly: system, degree in [1, 16] or ratio > 1 out of range";
        return FP_EINVAL;
    }
    ctx->poly_deg[system] = degree;
    ctx->poly_ratio[system] = ratio;
    return FP_OK;
}

fp_status fem_pic_field_last_info(fem_pic_t* ctx, fp_solve_info info[2], void* stream) {
    if (!ctx || !ctx->field || !info) return FP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    fp_status st = fill_info(ctx, 0, &info[0], s, 0.f);
    if (st == FP_OK) st = fill_info(ctx, 1, &info[1], s, 0.f);
    return st;
}

fp_status fem_pic_whitney0_integrals(const fem_pic_t* ctx, double* alpha) {
    if (!ctx || !alpha) return FP_EINVAL;
    const HostComplex& hc = ctx->hc;
    std::vector<double> a(hc.nn, 0.0);
    for (int64_t t = 0; t < hc.nt; ++t) {
        const double* g = hc.geo[t].g;
        // |T| = 1 / (6 |det G|), G = rows grad l1..3
        const double det = g[0] * (g[4] * g[8] - g[5] * g[7]) - g[1] * (g[3] * g[8] - g[5] * g[6]) +
                           g[2] * (g[3] * g[7] - g[4] * g[6]);
        const double q = 1.0 / (24.0 * std::fabs(det));  // |T| / 4
        for (int k = 0; k < 4; ++k) a[hc.tv[4 * t + k]] += q;
    }
    std::memcpy(alpha, a.data(), a.size() * sizeof(double));
    return FP_OK;
}

fp_status fem_pic_field_nnz(const fem_pic_t* ctx, int64_t nnz[2]) {
    if (!ctx || !ctx->field || !nnz) return FP_EINVAL;
    nnz[0] = (int64_t)ctx->field->host.e_col.size();
    nnz[1] = (int64_t)ctx->field->host.n_col.size();
    return FP_OK;
}

fp_status fem_pic_field_matrix(const fem_pic_t* ctx, int which, int32_t* row_ptr, int32_t* col, double* val) {
    if (!ctx || !ctx->field || which < 0 || which > 3) return FP_EINVAL;
    const FieldDev* F = ctx->field;
    const HostFields& H = F->host;
    const bool node = which == 3;
    const std::vector<int32_t>& rp = node ? H.n_rp : H.e_rp;
    const std::vector<int32_t>& c = node ? H.n_col : H.e_col;
    if (row_ptr) std::memcpy(row_ptr, rp.data(), rp.size() * 4);
    if (col) std::memcpy(col, c.data(), c.size() * 4);
    if (val) {
        for (size_t k = 0; k < c.size(); ++k) {
            double v = which == 0 ? H.M[k] : which == 1 ? H.S[k] : which == 2 ? H.M[k] + 0.25 * F->dt * F->dt * H.S[k]
                                                                             : H.L[k];
            val[k] = v;
        }
    }
    return FP_OK;
}

fp_status fem_pic_field_solve(fem_pic_t* ctx, int system, const double* rhs, double* x, double tol,
                              int max_iter, int precond, fp_solve_info* info, void* stream) {
    if (!ctx || !ctx->field || !rhs || !x || (system != FP_SYS_NEWMARK && system != FP_SYS_GAUSS) ||
        !(tol > 0.0) || max_iter < 0 ||
        (precond != FP_PC_JACOBI && precond != FP_PC_JACOBI_FP64 && precond != FP_PC_LEARNED)) {
        if (ctx) ctx->err = "fem_pic_field_solve: bad argument (or fem_pic_field_setup not called)";
        return FP_EINVAL;
    }
    if (precond == FP_PC_LEARNED && !learned_precond_ready(ctx->field, system)) {
        ctx->err = "fem_pic_field_solve: FP_PC_LEARNED needs a built FP_LEARNED_PRECOND network for the system";
        return FP_EINVAL;
    }
    ctx->solver_fp64 = precond == FP_PC_JACOBI_FP64;
    learned_set_active(ctx->field, system, precond == FP_PC_LEARNED);
    ctx->field->learned_used[0] = precond == FP_PC_LEARNED;
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t a = nullptr, b = nullptr;
    if (info) {
        FP_CUDA_TRY(ctx, cudaEventCreate(&a));
        FP_CUDA_TRY(ctx, cudaEventCreate(&b));
        FP_CUDA_TRY(ctx, cudaEventRecord(a, s));
    }
    fp_status st = run_pcg(ctx, system, rhs, x, tol, nullptr, max_iter, 0, s);
    if (info && st == FP_OK) {
        float ms = 0.f;
        cudaEventRecord(b, s);
        cudaEventSynchronize(b);
        cudaEventElapsedTime(&ms, a, b);
        st = fill_info(ctx, 0, info, s, ms);
        if (st == FP_OK && info->rel_res > tol) st = FP_ENOCONV;
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    return st;
}

fp_status fem_pic_field_step(fem_pic_t* ctx, const double* E_prev, const double* E_cur, double* E_next,
                             double* b, const void* dG_half, const void* dG_prev, const void* Q_new, double tol,
                             int max_iter, int precond, fp_solve_info info[2], void* stream) {
    if (!ctx || !ctx->field || !E_prev || !E_cur || !E_next || !Q_new || !(tol > 0.0) || max_iter < 0 ||
        (precond & ~(FP_PC_LEARNED | FP_PC_JACOBI_FP64 | FP_PC_LEARNED_GAUSS)) != 0 ||
        E_next == E_cur || E_next == E_prev) {
        if (ctx) ctx->err = "fem_pic_field_step: bad argument (or fem_pic_field_setup not called)";
        return FP_EINVAL;
    }
    const bool use[2] = {(precond & FP_PC_LEARNED) != 0, (precond & FP_PC_LEARNED_GAUSS) != 0};
    for (int k = 0; k < 2; ++k)
        if (use[k] && (!ctx->field->learned[k] || (learned_model(ctx->field, k) == FP_LEARNED_PRECOND &&
                                                    !learned_precond_ready(ctx->field, k)))) {
            ctx->err = "fem_pic_field_step: a learned correction needs fem_pic_learned_init for its system "
                       "(and fem_pic_learned_build for a learned preconditioner)";
            return FP_EINVAL;
        }
    ctx->solver_fp64 = (precond & FP_PC_JACOBI_FP64) != 0;
    for (int k = 0; k < 2; ++k) {
        learned_set_active(ctx->field, k, use[k]);
        ctx->field->learned_used[k] = use[k];
    }
    cudaStream_t s = (cudaStream_t)stream;
    fp_status st = field_step_impl(ctx, E_prev, E_cur, E_next, b, dG_half, dG_prev, Q_new, tol, max_iter, s);
    if (st != FP_OK || !info) return st;
    st = fill_info(ctx, 0, &info[0], s, 0.f);
    if (st == FP_OK) st = fill_info(ctx, 1, &info[1], s, 0.f);
    if (st == FP_OK && (info[0].rel_res > tol || info[1].rel_res > tol)) st = FP_ENOCONV;
    return st;
}

fp_status fem_pic_field_initial(fem_pic_t* ctx, const void* Q, double* E, double tol, int max_iter,
                                fp_solve_info* info, void* stream) {
    if (!ctx || !ctx->field || !Q || !E || !(tol > 0.0) || max_iter < 0) {
        if (ctx) ctx->err = "fem_pic_field_initial: bad argument (or fem_pic_field_setup not called)";
        return FP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    FieldDev* F = ctx->field;
    const bool f32 = Q_f32(ctx);   // Q is a float array
    const int gn = grid_of(ctx, F->nn), ge = grid_of(ctx, F->ne);
    FP_CUDA_TRY(ctx, cudaMemsetAsync(F->tmp, 0, F->ne * sizeof(double), s));
    if (f32)
        k_gauss_rhs<float><<<gn, kBlock, 0, s>>>(ctx->d_n2e_ptr, ctx->d_n2e_col, ctx->d_n2e_sgn, F->node_fixed, F->tmp,
                                                 (const float*)Q, F->nn, F->rhs, F->qd);
    else
        k_gauss_rhs<double><<<gn, kBlock, 0, s>>>(ctx->d_n2e_ptr, ctx->d_n2e_col, ctx->d_n2e_sgn, F->node_fixed,
                                                  F->tmp, (const double*)Q, F->nn, F->rhs, F->qd);
    FP_CUDA_TRY(ctx, cudaMemsetAsync(F->delta, 0, F->nn * sizeof(double), s));
    fp_status st = neumann_rhs(ctx, s);
    if (st == FP_OK) st = run_pcg(ctx, FP_SYS_GAUSS, F->rhs, F->delta, tol, F->qd, max_iter, 1, s);
    if (st == FP_OK) st = neumann_gauge(ctx, s);
    if (st != FP_OK) return st;
    k_project<<<ge, kBlock, 0, s>>>(ctx->d_edges, F->edge_fixed, F->delta, F->tmp, F->ne, E);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    if (info) {
        st = fill_info(ctx, 1, info, s, 0.f);
        if (st == FP_OK && info->rel_res > tol) st = FP_ENOCONV;
    }
    return st;
}

}  // extern "C"
