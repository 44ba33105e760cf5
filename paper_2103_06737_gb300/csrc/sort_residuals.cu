// Periodic counting sort of the particle SoA by cell, and the FP64 invariant residuals.
#include "internal.cuh"

namespace fempic {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kScanTile = 1024;

int sm_count() {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

int grid_cap(int64_t n, int block, int per_sm) {
    int64_t g = (n + block - 1) / block, cap = (int64_t)sm_count() * per_sm;
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

__device__ __forceinline__ void atomic_max_nonneg(double* addr, double v) {
    // for non-negative doubles the IEEE bit pattern orders like the value
    atomicMax(reinterpret_cast<unsigned long long*>(addr), (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ double block_max(double v, double* sh) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(kFull, v, o));
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (wid == 0) {
        r = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) r = fmax(r, __shfl_xor_sync(kFull, r, o));
    }
    __syncthreads();
    return r;
}

// r_n = (D0^T dG)_n - (Q_new - Q_old)_n  (discrete continuity, FP64)
template <typename Real>
__global__ void __launch_bounds__(256) k_res_continuity(const int32_t* __restrict__ ptr,
                                                        const int32_t* __restrict__ col,
                                                        const int8_t* __restrict__ sgn, int64_t nn,
                                                        const Real* __restrict__ dG,
                                                        const Real* __restrict__ Qn,
                                                        const Real* __restrict__ Qo,
                                                        const uint8_t* __restrict__ wall, double* out) {
    __shared__ double sh[32];
    double rmax = 0.0, smax = 0.0, imax = 0.0, ismax = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nn; i += stride) {
        double r = 0.0, sc = 0.0;
        if (dG)
            for (int j = ptr[i]; j < ptr[i + 1]; ++j) {
                double t = (double)sgn[j] * (double)dG[col[j]];
                r += t;
                sc += fabs(t);
            }
        double qn = Qn ? (double)Qn[i] : 0.0, qo = Qo ? (double)Qo[i] : 0.0;
        r -= (qn - qo);
        sc += fabs(qn) + fabs(qo);
        rmax = fmax(rmax, fabs(r));
        smax = fmax(smax, sc);
        if (!wall[i]) {
            imax = fmax(imax, fabs(r));
            ismax = fmax(ismax, sc);
        }
    }
    rmax = block_max(rmax, sh);
    smax = block_max(smax, sh);
    imax = block_max(imax, sh);
    ismax = block_max(ismax, sh);
    if (threadIdx.x == 0) {
        atomic_max_nonneg(out + 0, rmax);
        atomic_max_nonneg(out + 1, smax);
        atomic_max_nonneg(out + 4, imax);
        atomic_max_nonneg(out + 5, ismax);
    }
}

// r_t = (D2 b)_t  (magnetic Gauss law, FP64)
__global__ void __launch_bounds__(256) k_res_divb(const TetTopo* __restrict__ topo,
                                                  const int8_t* __restrict__ orient, int64_t nt,
                                                  const double* __restrict__ b, double* out) {
    __shared__ double sh[32];
    double rmax = 0.0, smax = 0.0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
        const TetTopo& T = topo[t];
        const double s = (double)orient[t];
        double b0 = b[T.face[0]], b1 = b[T.face[1]], b2 = b[T.face[2]], b3 = b[T.face[3]];
        double r = s * (((b0 - b1) + b2) - b3);
        rmax = fmax(rmax, fabs(r));
        smax = fmax(smax, fabs(b0) + fabs(b1) + fabs(b2) + fabs(b3));
    }
    rmax = block_max(rmax, sh);
    smax = block_max(smax, sh);
    if (threadIdx.x == 0) {
        atomic_max_nonneg(out + 2, rmax);
        atomic_max_nonneg(out + 3, smax);
    }
}

template <typename Real>
void scatter(fem_pic* ctx, const fp_particles* src, fp_particles* dst, cudaStream_t s) {
    k_sort_scatter<Real><<<grid_cap(src->n, 256, 8), 256, 0, s>>>(
        src->cell, (const Real*)src->off, (const Real*)src->vel, src->n, (int32_t)ctx->hc.nt,
        ctx->d_sort_count, ctx->d_sort_rank, dst->cell, (Real*)dst->off, (Real*)dst->vel);
}

}  // namespace

fp_status launch_sort(fem_pic* ctx, const fp_particles* src, fp_particles* dst, cudaStream_t s) {
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
    FP_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_sort_count, 0, (m + 1) * sizeof(int32_t), s));
    k_sort_count<<<grid_cap(n, 256, 8), 256, 0, s>>>(src->cell, n, (int32_t)ctx->hc.nt,
                                                     ctx->d_sort_count, ctx->d_sort_rank);
    k_scan_tiles<<<(unsigned)tiles, kScanTile, 0, s>>>(ctx->d_sort_count, m, ctx->d_sort_block);
    k_scan_sums<<<1, kScanTile, 0, s>>>(ctx->d_sort_block, tiles);
    k_scan_add<<<(unsigned)tiles, kScanTile, 0, s>>>(ctx->d_sort_count, m, ctx->d_sort_block);
    if (ctx->precision == FP_FP32)
        scatter<float>(ctx, src, dst, s);
    else
        scatter<double>(ctx, src, dst, s);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}

fp_status launch_residuals(fem_pic* ctx, const void* dG, const void* Qn, const void* Qo,
                           const double* b, double* out, cudaStream_t s) {
    FP_CUDA_TRY(ctx, cudaMemsetAsync(out, 0, 6 * sizeof(double), s));
    const int64_t nn = ctx->hc.nn, nt = ctx->hc.nt;
    if (ctx->precision == FP_FP32)
        k_res_continuity<float><<<grid_cap(nn, 256, 4), 256, 0, s>>>(
            ctx->d_n2e_ptr, ctx->d_n2e_col, ctx->d_n2e_sgn, nn, (const float*)dG, (const float*)Qn,
            (const float*)Qo, ctx->d_node_wall, out);
    else
        k_res_continuity<double><<<grid_cap(nn, 256, 4), 256, 0, s>>>(
            ctx->d_n2e_ptr, ctx->d_n2e_col, ctx->d_n2e_sgn, nn, (const double*)dG, (const double*)Qn,
            (const double*)Qo, ctx->d_node_wall, out);
    if (b) k_res_divb<<<grid_cap(nt, 256, 4), 256, 0, s>>>(ctx->d_topo, ctx->d_orient, nt, b, out);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}

}  // namespace fempic
