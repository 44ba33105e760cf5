// Periodic counting sort of the particle SoA by cell, and the FP64 invariant residuals.
#include "internal.cuh"

namespace fempic {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kScanTile = 1024;

int grid_cap(int64_t n, int block, int per_sm, int sms) {
    int64_t g = (n + block - 1) / block, cap = (int64_t)sms * per_sm;
    if (g > cap) g = cap;
    return g < 1 ? 1 : (int)g;
}

// histogram of cell ids (dead particles go to bucket nt) and the rank of each
// particle inside its bucket; one atomic per run of equal keys in a warp
__global__ void k_sort_count(const int32_t* __restrict__ cell, int64_t n, int32_t nt,
                             int32_t* __restrict__ count, int32_t* __restrict__ rank) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride) {
        const int64_t p = base + lane;
        int key = -1;
        if (p < n) {
            int c = cell[p];
            key = (c >= 0 && c < nt) ? c : nt;
        }
        int prev = __shfl_up_sync(kFull, key, 1);
        bool head = lane == 0 || prev != key;
        unsigned heads = __ballot_sync(kFull, head);
        unsigned above = heads & ~((2u << lane) - 1u);
        int end = above ? __ffs(above) - 1 : 32;
        int start = 31 - __clz(heads & ((2u << lane) - 1u));
        int old = 0;
        if (head && key >= 0) old = atomicAdd(count + key, end - lane);
        old = __shfl_sync(kFull, old, start);
        if (p < n) rank[p] = old + (lane - start);
    }
}

// exclusive scan, phase 1: per-tile scan and tile totals
__global__ void __launch_bounds__(kScanTile) k_scan_tiles(int32_t* __restrict__ a, int64_t m,
                                                          int32_t* __restrict__ tile_sum) {
    __shared__ int32_t warp_tot[32];
    const int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int32_t x = i < m ? a[i] : 0, incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int32_t t = warp_tot[lane], ti = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(kFull, ti, o);
            if (lane >= o) ti += y;
        }
        warp_tot[lane] = ti - t;  // exclusive warp offsets
        if (lane == 31) tile_sum[blockIdx.x] = ti;
    }
    __syncthreads();
    if (i < m) a[i] = incl - x + warp_tot[wid];
}

// phase 2: one block scans the tile totals (exclusive), sequentially in chunks
__global__ void __launch_bounds__(kScanTile) k_scan_sums(int32_t* __restrict__ s, int64_t nt_) {
    __shared__ int32_t warp_tot[32];
    __shared__ int32_t carry;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t b0 = 0; b0 < nt_; b0 += kScanTile) {
        const int64_t i = b0 + threadIdx.x;
        int32_t x = i < nt_ ? s[i] : 0, incl = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) warp_tot[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int32_t t = warp_tot[lane], ti = t;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                int32_t y = __shfl_up_sync(kFull, ti, o);
                if (lane >= o) ti += y;
            }
            warp_tot[lane] = ti - t;
        }
        __syncthreads();
        const int32_t c0 = carry;
        if (i < nt_) s[i] = c0 + incl - x + warp_tot[wid];
        __syncthreads();
        if (threadIdx.x == kScanTile - 1) carry = c0 + warp_tot[wid] + incl;
        __syncthreads();
    }
}

// phase 3: add the scanned tile totals
__global__ void k_scan_add(int32_t* __restrict__ a, int64_t m, const int32_t* __restrict__ tile_off) {
    const int64_t i = (int64_t)blockIdx.x * kScanTile + threadIdx.x;
    if (i < m) a[i] += tile_off[blockIdx.x];
}

template <typename Real>
__global__ void k_sort_scatter(const int32_t* __restrict__ cell, const Real* __restrict__ off,
                               const Real* __restrict__ vel, int64_t n, int32_t nt,
                               const int32_t* __restrict__ start, const int32_t* __restrict__ rank,
                               int32_t* __restrict__ cell_o, Real* __restrict__ off_o,
                               Real* __restrict__ vel_o) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        int c = cell[p];
        int key = (c >= 0 && c < nt) ? c : nt;
        int64_t q = (int64_t)start[key] + rank[p];
        cell_o[q] = (c >= 0 && c < nt) ? c : -1;
        off_o[q] = off[p];
        off_o[n + q] = off[n + p];
        off_o[2 * n + q] = off[2 * n + p];
        vel_o[q] = vel[p];
        vel_o[n + q] = vel[n + p];
        vel_o[2 * n + q] = vel[2 * n + p];
    }
}

// extra planar columns (ncols x n) moved with the same permutation as the particle state
template <typename Real>
__global__ void k_sort_scatter_cols(const int32_t* __restrict__ cell, int64_t n, int32_t nt,
                                    const int32_t* __restrict__ start, const int32_t* __restrict__ rank,
                                    const Real* __restrict__ src, Real* __restrict__ dst, int ncols) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < n; p += stride) {
        const int c = cell[p];
        const int key = (c >= 0 && c < nt) ? c : nt;
        const int64_t q = (int64_t)start[key] + rank[p];
        for (int k = 0; k < ncols; ++k) dst[k * n + q] = src[k * n + p];
    }
}

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    // for non-negative doubles the IEEE bit pattern orders like the value
    atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}


__device__ __forceinline__ double as_f64(float x) { return f2d(x); }
__device__ __forceinline__ double as_f64(double x) { return x; }
__device__ __forceinline__ float as_f32(float x) { return x; }
__device__ __forceinline__ float as_f32(double x) { return d2f(x); }

// |x| of a double as its bit pattern: for non-negative doubles the pattern orders like the value
__device__ __forceinline__ unsigned long long abs_bits(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long u = __shfl_xor_sync(kFull, v, o);
        v = u > v ? u : v;
    }
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    unsigned long long r = 0;
    if (wid == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0ull;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            unsigned long long u = __shfl_xor_sync(kFull, r, o);
            r = u > r ? u : r;
        }
    }
    __syncthreads();
    return r;
}

// One launch for both invariants.  The residual sums are FP64; the maxima are taken
// on bit patterns and the scales in FP32, so the FP64 pipe only does the sums.
//   blocks [0, nb_cont): continuity r_n = (D0^T dG)_n - (Q_new - Q_old)_n, a thread per node;
//   blocks [nb_cont, ...): magnetic Gauss law r_t = (D2 b)_t, a thread per tet.
template <typename Real, typename RealQ>
__global__ void __launch_bounds__(256) k_residuals(const int32_t* __restrict__ ptr,
                                                   const int32_t* __restrict__ col,
                                                   const int8_t* __restrict__ sgn, int64_t nn,
                                                   const Real* __restrict__ dG,
                                                   const RealQ* __restrict__ Qn,
                                                   const RealQ* __restrict__ Qo,
                                                   const uint8_t* __restrict__ wall,
                                                   const int4* __restrict__ tet_faces, int64_t nt,
                                                   const double* __restrict__ b, int nb_cont,
                                                   double* out) {
    __shared__ unsigned long long sh[32];
    if ((int)blockIdx.x < nb_cont) {
        const int64_t stride = (int64_t)nb_cont * blockDim.x;
        unsigned long long rmax = 0, imax = 0;
        float smax = 0.f, ismax = 0.f;
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += stride) {
            double r = 0.0;
            float sc = 0.f;
            if (dG) {
                const int j0 = __ldg(ptr + i), j1 = __ldg(ptr + i + 1);
                for (int j = j0; j < j1; ++j) {
                    const Real x = __ldg(dG + __ldg(col + j));
                    const double xd = as_f64(x);
                    const long long flip = __ldg(sgn + j) > 0 ? 0ll : (long long)0x8000000000000000ull;
                    r += __longlong_as_double(__double_as_longlong(xd) ^ flip);
                    sc += fabsf(as_f32(x));
                }
            }
            if (Qn) {
                r -= as_f64(Qn[i]);
                sc += fabsf(as_f32(Qn[i]));
            }
            if (Qo) {
                r += as_f64(Qo[i]);
                sc += fabsf(as_f32(Qo[i]));
            }
            const unsigned long long ar = abs_bits(r);
            rmax = ar > rmax ? ar : rmax;
            smax = fmaxf(smax, sc);
            if (!wall[i]) {
                imax = ar > imax ? ar : imax;
                ismax = fmaxf(ismax, sc);
            }
        }
        rmax = block_max_u64(rmax, sh);
        imax = block_max_u64(imax, sh);
        unsigned long long s1 = block_max_u64(__float_as_uint(smax), sh);
        unsigned long long s2 = block_max_u64(__float_as_uint(ismax), sh);
        if (threadIdx.x == 0) {
            atomicMax(reinterpret_cast<unsigned long long*>(out + 0), rmax);
            atomicMax(reinterpret_cast<unsigned long long*>(out + 4), imax);
            atomic_max_nonneg(out + 1, f2d(__uint_as_float((unsigned)s1)));
            atomic_max_nonneg(out + 5, f2d(__uint_as_float((unsigned)s2)));
        }
    } else {
        unsigned long long rmax = 0, smax = 0;
        if (b) {
            const int64_t nbk = (int64_t)gridDim.x - nb_cont;
            const int64_t stride = nbk * blockDim.x;
            for (int64_t t = (int64_t)(blockIdx.x - nb_cont) * blockDim.x + threadIdx.x; t < nt; t += stride) {
                const int4 f = __ldg(tet_faces + t);
                const double b0 = __ldg(b + f.x), b1 = __ldg(b + f.y), b2 = __ldg(b + f.z), b3 = __ldg(b + f.w);
                // D2 row: s_t (+b0 - b1 + b2 - b3); the sign s_t does not change |r|
                const unsigned long long ar = abs_bits(((b0 - b1) + b2) - b3);
                rmax = ar > rmax ? ar : rmax;
                unsigned long long m01 = abs_bits(b0) > abs_bits(b1) ? abs_bits(b0) : abs_bits(b1);
                unsigned long long m23 = abs_bits(b2) > abs_bits(b3) ? abs_bits(b2) : abs_bits(b3);
                unsigned long long m = m01 > m23 ? m01 : m23;
                smax = m > smax ? m : smax;
            }
        }
        rmax = block_max_u64(rmax, sh);
        smax = block_max_u64(smax, sh);
        if (threadIdx.x == 0) {
            atomicMax(reinterpret_cast<unsigned long long*>(out + 2), rmax);
            atomicMax(reinterpret_cast<unsigned long long*>(out + 3), smax);
        }
    }
}

template <typename Real>
void scatter(fem_pic* ctx, const fp_particles* src, fp_particles* dst, const void* cs, void* cd, int ncols,
             cudaStream_t s) {
    k_sort_scatter<Real><<<grid_cap(src->n, 256, 8, ctx->sm_count), 256, 0, s>>>(
        src->cell, (const Real*)src->off, (const Real*)src->vel, src->n, (int32_t)ctx->hc.nt,
        ctx->d_sort_count, ctx->d_sort_rank, dst->cell, (Real*)dst->off, (Real*)dst->vel);
    if (ncols > 0)
        k_sort_scatter_cols<Real><<<grid_cap(src->n, 256, 8, ctx->sm_count), 256, 0, s>>>(
            src->cell, src->n, (int32_t)ctx->hc.nt, ctx->d_sort_count, ctx->d_sort_rank, (const Real*)cs,
            (Real*)cd, ncols);
}

}  // namespace

fp_status launch_sort(fem_pic* ctx, const fp_particles* src, fp_particles* dst, cudaStream_t s,
                      const void* cols_src, void* cols_dst, int ncols) {
    const int64_t n = src->n, m = ctx->hc.nt + 1;
    const int64_t tiles = (m + kScanTile - 1) / kScanTile;
    if (n == 0) return FP_OK;
    if (n > INT32_MAX) {
        ctx->err = "fem_pic_sort: more than 2^31-1 particles";
        return FP_EINVAL;
    }
    if (!ctx->d_sort_count) {
        FP_CUDA_TRY(ctx, cudaMalloc((void**)&ctx->d_sort_count, (m + 1) * sizeof(int32_t)));
        FP_CUDA_TRY(ctx, cudaMalloc((void**)&ctx->d_sort_block, (tiles + 1) * sizeof(int32_t)));
    }
    if (ctx->sort_cap < n) {
        if (ctx->d_sort_rank) FP_CUDA_TRY(ctx, cudaFree(ctx->d_sort_rank));
        ctx->d_sort_rank = nullptr;
        ctx->sort_cap = 0;
        FP_CUDA_TRY(ctx, cudaMalloc((void**)&ctx->d_sort_rank, n * sizeof(int32_t)));
        ctx->sort_cap = n;
    }
    PhaseTimer pt(ctx, PH_SORT, s);
    FP_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_sort_count, 0, (m + 1) * sizeof(int32_t), s));
    k_sort_count<<<grid_cap(n, 256, 8, ctx->sm_count), 256, 0, s>>>(src->cell, n, (int32_t)ctx->hc.nt,
                                                     ctx->d_sort_count, ctx->d_sort_rank);
    k_scan_tiles<<<(unsigned)tiles, kScanTile, 0, s>>>(ctx->d_sort_count, m, ctx->d_sort_block);
    k_scan_sums<<<1, kScanTile, 0, s>>>(ctx->d_sort_block, tiles);
    k_scan_add<<<(unsigned)tiles, kScanTile, 0, s>>>(ctx->d_sort_count, m, ctx->d_sort_block);
    if (ctx->precision == FP_FP32)
        scatter<float>(ctx, src, dst, cols_src, cols_dst, ncols, s);
    else
        scatter<double>(ctx, src, dst, cols_src, cols_dst, ncols, s);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}

template <typename DG, typename DQ>
void residuals_t(fem_pic* ctx, const void* dG, const void* Qn, const void* Qo, const double* b, int nb_cont,
                 int grid, double* out, cudaStream_t s) {
    k_residuals<DG, DQ><<<grid, 256, 0, s>>>(ctx->d_n2e_ptr, ctx->d_n2e_col, ctx->d_n2e_sgn, ctx->hc.nn,
                                             (const DG*)dG, (const DQ*)Qn, (const DQ*)Qo, ctx->d_node_wall,
                                             ctx->d_tet_faces, ctx->hc.nt, b, nb_cont, out);
}

fp_status launch_residuals(fem_pic* ctx, const void* dG, const void* Qn, const void* Qo,
                           const double* b, double* out, cudaStream_t s) {
    PhaseTimer pt(ctx, PH_RESID, s);
    FP_CUDA_TRY(ctx, cudaMemsetAsync(out, 0, 6 * sizeof(double), s));
    const int64_t nn = ctx->hc.nn, nt = ctx->hc.nt;
    const int nb_cont = grid_cap(nn, 256, 4, ctx->sm_count);
    const int nb_div = grid_cap(nt, 256, 4, ctx->sm_count);
    const int grid = nb_cont + nb_div;
    if (dG_f32(ctx) && Q_f32(ctx))
        residuals_t<float, float>(ctx, dG, Qn, Qo, b, nb_cont, grid, out, s);
    else if (dG_f32(ctx))
        residuals_t<float, double>(ctx, dG, Qn, Qo, b, nb_cont, grid, out, s);
    else
        residuals_t<double, double>(ctx, dG, Qn, Qo, b, nb_cont, grid, out, s);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}

}  // namespace fempic
