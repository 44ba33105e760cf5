// The field solve's comparison systems and the Gauss-law residual (Sec. V, VI.A, VI.B):
//   fem_pic_mfem_step    first-order mixed FEM (MFEM) on Eq. maxwell_semi, advanced by
//                        Newmark (beta = 1/4, gamma = 1/2), which for a first-order system is
//                        the trapezoidal rule; no Gauss-law projection:
//                          (M + dt^2/4 S) E^{n+1} = (M - dt^2/4 S) E^n
//                                                   + dt [curl]^T [*mu^-1] b^n - dG^{n+1/2}
//                          b^{n+1} = b^n - dt [curl] (E^{n+1} + E^n) / 2
//   fem_pic_wave_step    Newmark on the wave equation (Eq. wave_cont) with no projection,
//                        i.e. steps 1 and 3 of fem_pic_field_step (the WE-FEM of Sec. V);
//   fem_pic_mfem_gauss_residual   D0^T [*eps] E + Q (Eq. discreteGauss) of any edge field.
// Without the projection the solves' errors stay in the fields' gradient modes: WE-FEM's
// grow linearly in time, MFEM's do not (Sec. V).  Both steps solve with the library's Newmark
// solver (fem_pic_field_solve); this file adds the right-hand sides, [*mu^-1] b and Faraday.
#include <algorithm>
#include <new>

#include "field.cuh"
#include "mfem.cuh"

using namespace fempic;

struct fem_pic_mfem {
    fem_pic* ctx = nullptr;
    const FieldDev* F = nullptr;  // the field setup the handle was made for
    double dt = 0, eps = 0, mu = 0;
    int bc = 0;
    int64_t ne = 0, nn = 0, nf = 0;
    HostMfem host;
    int32_t *f_rp = nullptr, *f_col = nullptr, *ef_rp = nullptr, *ef_col = nullptr;
    int8_t* ef_sgn = nullptr;
    double* f_val = nullptr;
    double *h = nullptr, *rhs = nullptr, *me = nullptr, *qsum = nullptr;
};

namespace {

constexpr int kThreads = 256;

int grid_for(const fem_pic* ctx, int64_t n) {
    const int64_t g = (n + kThreads - 1) / kThreads, cap = (int64_t)ctx->sm_count * 8;
    return (int)std::max<int64_t>(1, std::min(g, cap));
}

// h = [*mu^-1] b over every face (CSR)
__global__ void k_face_mass(const int32_t* __restrict__ rp, const int32_t* __restrict__ col,
                            const double* __restrict__ val, const double* __restrict__ b, int64_t nf,
                            double* __restrict__ h) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += stride) {
        double s = 0.0;
        for (int32_t j = rp[f]; j < rp[f + 1]; ++j) s = fma(val[j], b[col[j]], s);
        h[f] = s;
    }
}

// solver start a1 x + a2 y on free edges (y may be null), 0 on PEC edges
__global__ void k_guess(const uint8_t* __restrict__ fixed, const double* __restrict__ x,
                        const double* __restrict__ y, double a1, double a2, int64_t n, double* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] = fixed[i] ? 0.0 : a1 * x[i] + (y ? a2 * y[i] : 0.0);
}

// rhs_i = sum_j [ M_ij (a1 x_j + a2 y_j) + S_ij (b1 x_j + b2 y_j) ] + c ([curl]^T h)_i
//         - (gh_i - gp_i) on free edges, 0 on PEC edges.  M and S share the SELL-32 layout
// (padding entries point at their own row with value 0); y, h, gh, gp may be null.
template <typename Real>
__global__ void k_rhs(Sell Sl, const double* __restrict__ M, const double* __restrict__ S,
                      const uint8_t* __restrict__ fixed, const double* __restrict__ x,
                      const double* __restrict__ y, double a1, double a2, double b1, double b2,
                      const int32_t* __restrict__ ef_rp, const int32_t* __restrict__ ef_col,
                      const int8_t* __restrict__ ef_sgn, const double* __restrict__ h, double c,
                      const Real* __restrict__ gh, const Real* __restrict__ gp, int64_t n,
                      double* __restrict__ rhs) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        if (fixed[i]) {
            rhs[i] = 0.0;
            continue;
        }
        const int64_t sl = i >> 5;
        const int64_t base = Sl.ptr[sl] + (i & 31);
        const int w = Sl.w[sl];
        double s = 0.0;
        for (int j = 0; j < w; ++j) {
            const int64_t k = base + 32 * (int64_t)j;
            const int32_t cj = Sl.col[k];
            const double xv = x[cj], yv = y ? y[cj] : 0.0;
            s = fma(M[k], a1 * xv + a2 * yv, s);
            s = fma(S[k], b1 * xv + b2 * yv, s);
        }
        if (h) {
            double t = 0.0;
            for (int32_t j = ef_rp[i]; j < ef_rp[i + 1]; ++j) t += ef_sgn[j] > 0 ? h[ef_col[j]] : -h[ef_col[j]];
            s = fma(c, t, s);
        }
        const double g1 = gh ? (double)gh[i] : 0.0, g0 = gp ? (double)gp[i] : 0.0;
        rhs[i] = s - (g1 - g0);
    }
}

// b <- b - dt [curl] (E1 + E0) / 2, face (i<j<k): +(i,j) +(j,k) -(i,k)
__global__ void k_faraday_trap(const int32_t* __restrict__ fe, const double* __restrict__ E1,
                               const double* __restrict__ E0, double half_dt, int64_t nf, double* __restrict__ b) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < nf; f += stride) {
        const int32_t ij = fe[3 * f], jk = fe[3 * f + 1], ik = fe[3 * f + 2];
        b[f] -= half_dt * ((E1[ij] + E0[ij]) + (E1[jk] + E0[jk]) - (E1[ik] + E0[ik]));
    }
}

// me = [*eps] E (SELL rows)
__global__ void k_mass(Sell Sl, const double* __restrict__ M, const double* __restrict__ E, int64_t n,
                       double* __restrict__ me) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        me[i] = sell_row<double, double>(Sl, M, E, i);
}

// sum of Q over all nodes, one block of 1024 threads, fixed summation order
template <typename Real>
__global__ void __launch_bounds__(1024) k_qsum(const Real* __restrict__ Q, int64_t nn, double* __restrict__ out) {
    __shared__ double part[1024];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < nn; i += blockDim.x) s += (double)Q[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = part[0];
}

// Gauss-law residual on free nodes: g_n = (D0^T me)_n + Q_n, less (sum Q / sum alpha) alpha_n
// under the natural boundary (the net charge the zero-mean constraint spreads); out[0] = max |g|,
// out[1] = max of |Q_n| + sum over incident edges of |me_e| (the scale).  Non-negative doubles
// order like their bit patterns, so the maxima are atomicMax on those (order independent).
template <typename Real>
__global__ void k_gauss_res(const int32_t* __restrict__ ptr, const int32_t* __restrict__ col,
                            const int8_t* __restrict__ sgn, const uint8_t* __restrict__ fixed,
                            const double* __restrict__ me, const Real* __restrict__ Q,
                            const double* __restrict__ alpha, const double* __restrict__ qsum,
                            double inv_alpha_sum, int64_t nn, unsigned long long* __restrict__ out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    double worst = 0.0, scale = 0.0;
    for (int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; n < nn; n += stride) {
        if (fixed[n]) continue;
        const double q = Q ? (double)Q[n] : 0.0;
        double s = q, a = fabs(q);
        for (int32_t j = ptr[n]; j < ptr[n + 1]; ++j) {
            const double t = sgn[j] > 0 ? me[col[j]] : -me[col[j]];
            s += t;
            a += fabs(t);
        }
        if (alpha) s -= qsum[0] * inv_alpha_sum * alpha[n];
        worst = fmax(worst, fabs(s));
        scale = fmax(scale, a);
    }
    atomicMax(out, (unsigned long long)__double_as_longlong(worst));
    atomicMax(out + 1, (unsigned long long)__double_as_longlong(scale));
}

template <typename T>
fp_status upload(fem_pic* ctx, T** d, const std::vector<T>& v) {
    FP_CUDA_TRY(ctx, cudaMalloc((void**)d, v.size() * sizeof(T) + 16));
    if (!v.empty()) FP_CUDA_TRY(ctx, cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
    return FP_OK;
}

fp_status scratch(fem_pic* ctx, double** d, int64_t n) {
    FP_CUDA_TRY(ctx, cudaMalloc((void**)d, (size_t)n * sizeof(double) + 16));
    FP_CUDA_TRY(ctx, cudaMemset(*d, 0, (size_t)n * sizeof(double)));
    return FP_OK;
}

fp_status check(fem_pic_mfem* m, const char* who) {
    if (!m) return FP_EINVAL;
    const FieldDev* F = m->ctx->field;
    if (!F || F != m->F || F->dt != m->dt || F->eps != m->eps || F->mu != m->mu || F->bc != m->bc) {
        m->ctx->err = std::string(who) + ": the field setup changed since fem_pic_mfem_create";
        return FP_EINVAL;
    }
    return FP_OK;
}

// rhs of either step into m->rhs (dG in the context's particle precision)
fp_status launch_rhs(fem_pic_mfem* m, const double* x, const double* y, double a1, double a2, double b1,
                     double b2, const double* h, double c, const void* gh, const void* gp, cudaStream_t s) {
    fem_pic* ctx = m->ctx;
    const FieldDev* F = ctx->field;
    const Sell Sl{F->se_ptr, F->se_w, F->se_col};
    const int g = grid_for(ctx, m->ne);
    if (dG_f32(ctx))
        k_rhs<float><<<g, kThreads, 0, s>>>(Sl, F->se_M, F->se_S, F->edge_fixed, x, y, a1, a2, b1, b2, m->ef_rp,
                                            m->ef_col, m->ef_sgn, h, c, (const float*)gh, (const float*)gp, m->ne,
                                            m->rhs);
    else
        k_rhs<double><<<g, kThreads, 0, s>>>(Sl, F->se_M, F->se_S, F->edge_fixed, x, y, a1, a2, b1, b2, m->ef_rp,
                                             m->ef_col, m->ef_sgn, h, c, (const double*)gh, (const double*)gp,
                                             m->ne, m->rhs);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}

}  // namespace

extern "C" {

void fem_pic_mfem_destroy(fem_pic_mfem_t* m) {
    if (!m) return;
    cudaFree(m->f_rp);
    cudaFree(m->f_col);
    cudaFree(m->f_val);
    cudaFree(m->ef_rp);
    cudaFree(m->ef_col);
    cudaFree(m->ef_sgn);
    cudaFree(m->h);
    cudaFree(m->rhs);
    cudaFree(m->me);
    cudaFree(m->qsum);
    delete m;
}

fp_status fem_pic_mfem_create(fem_pic_t* ctx, fem_pic_mfem_t** out) {
    if (out) *out = nullptr;
    if (!ctx || !out || !ctx->field) {
        if (ctx) ctx->err = "fem_pic_mfem_create: bad argument (or fem_pic_field_setup not called)";
        return FP_EINVAL;
    }
    fem_pic_mfem* m = new (std::nothrow) fem_pic_mfem();
    if (!m) {
        ctx->err = "fem_pic_mfem_create: out of host memory";
        return FP_EINVAL;
    }
    const FieldDev* F = ctx->field;
    m->ctx = ctx;
    m->F = F;
    m->dt = F->dt, m->eps = F->eps, m->mu = F->mu, m->bc = F->bc;
    m->ne = F->ne, m->nn = F->nn, m->nf = F->nf;
    try {
        assemble_mfem(ctx->hc, F->mu, &m->host);
    } catch (const std::bad_alloc&) {   // no exception crosses the C ABI
        delete m;
        ctx->err = "fem_pic_mfem_create: out of host memory";
        return FP_EINVAL;
    }
    fp_status st = upload(ctx, &m->f_rp, m->host.f_rp);
    if (st == FP_OK) st = upload(ctx, &m->f_col, m->host.f_col);
    if (st == FP_OK) st = upload(ctx, &m->f_val, m->host.Fm);
    if (st == FP_OK) st = upload(ctx, &m->ef_rp, m->host.ef_rp);
    if (st == FP_OK) st = upload(ctx, &m->ef_col, m->host.ef_col);
    if (st == FP_OK) st = upload(ctx, &m->ef_sgn, m->host.ef_sgn);
    if (st == FP_OK) st = scratch(ctx, &m->h, m->nf);
    if (st == FP_OK) st = scratch(ctx, &m->rhs, m->ne);
    if (st == FP_OK) st = scratch(ctx, &m->me, m->ne);
    if (st == FP_OK) st = scratch(ctx, &m->qsum, 1);
    if (st != FP_OK) {
        fem_pic_mfem_destroy(m);
        return st;
    }
    *out = m;
    return FP_OK;
}

fp_status fem_pic_mfem_face_mass(const fem_pic_mfem_t* m, int64_t* nnz, int32_t* row_ptr, int32_t* col,
                                 double* val) {
    if (!m) return FP_EINVAL;
    if (nnz) *nnz = (int64_t)m->host.f_col.size();
    if (row_ptr) std::copy(m->host.f_rp.begin(), m->host.f_rp.end(), row_ptr);
    if (col) std::copy(m->host.f_col.begin(), m->host.f_col.end(), col);
    if (val) std::copy(m->host.Fm.begin(), m->host.Fm.end(), val);
    return FP_OK;
}

fp_status fem_pic_mfem_step(fem_pic_mfem_t* m, const double* E_cur, double* E_next, double* b,
                            const void* dG_half, double tol, int max_iter, int precond, fp_solve_info* info,
                            void* stream) {
    fp_status st = check(m, "fem_pic_mfem_step");
    if (st != FP_OK) return st;
    fem_pic* ctx = m->ctx;
    if (!E_cur || !E_next || !b || E_next == E_cur || !(tol > 0.0) || max_iter < 0) {
        ctx->err = "fem_pic_mfem_step: bad argument";
        return FP_EINVAL;
    }
    const FieldDev* F = ctx->field;
    cudaStream_t s = (cudaStream_t)stream;
    const double dt = F->dt;
    k_face_mass<<<grid_for(ctx, m->nf), kThreads, 0, s>>>(m->f_rp, m->f_col, m->f_val, b, m->nf, m->h);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    st = launch_rhs(m, E_cur, nullptr, 1.0, 0.0, -0.25 * dt * dt, 0.0, m->h, dt, dG_half, nullptr, s);
    if (st != FP_OK) return st;
    k_guess<<<grid_for(ctx, m->ne), kThreads, 0, s>>>(F->edge_fixed, E_cur, nullptr, 1.0, 0.0, m->ne, E_next);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    st = fem_pic_field_solve(ctx, FP_SYS_NEWMARK, m->rhs, E_next, tol, max_iter, precond, info, stream);
    if (st != FP_OK && st != FP_ENOCONV) return st;
    k_faraday_trap<<<grid_for(ctx, m->nf), kThreads, 0, s>>>(F->face_edges, E_next, E_cur, 0.5 * dt, m->nf, b);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return st;
}

fp_status fem_pic_wave_step(fem_pic_mfem_t* m, const double* E_prev, const double* E_cur, double* E_next,
                            double* b, const void* dG_half, const void* dG_prev, double tol, int max_iter,
                            int precond, fp_solve_info* info, void* stream) {
    fp_status st = check(m, "fem_pic_wave_step");
    if (st != FP_OK) return st;
    fem_pic* ctx = m->ctx;
    if (!E_prev || !E_cur || !E_next || E_next == E_cur || E_next == E_prev || !(tol > 0.0) || max_iter < 0) {
        ctx->err = "fem_pic_wave_step: bad argument";
        return FP_EINVAL;
    }
    const FieldDev* F = ctx->field;
    cudaStream_t s = (cudaStream_t)stream;
    const double dt2 = F->dt * F->dt;
    st = launch_rhs(m, E_cur, E_prev, 2.0, -1.0, -0.5 * dt2, -0.25 * dt2, nullptr, 0.0, dG_half, dG_prev, s);
    if (st != FP_OK) return st;
    k_guess<<<grid_for(ctx, m->ne), kThreads, 0, s>>>(F->edge_fixed, E_cur, E_prev, 2.0, -1.0, m->ne, E_next);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    st = fem_pic_field_solve(ctx, FP_SYS_NEWMARK, m->rhs, E_next, tol, max_iter, precond, info, stream);
    if (st != FP_OK && st != FP_ENOCONV) return st;
    if (b) {
        k_faraday_trap<<<grid_for(ctx, m->nf), kThreads, 0, s>>>(F->face_edges, E_next, E_cur, 0.5 * F->dt, m->nf,
                                                                  b);
        FP_CUDA_TRY(ctx, cudaGetLastError());
    }
    return st;
}

fp_status fem_pic_mfem_gauss_residual(fem_pic_mfem_t* m, const double* E, const void* Q, double* out,
                                      void* stream) {
    fp_status st = check(m, "fem_pic_mfem_gauss_residual");
    if (st != FP_OK) return st;
    fem_pic* ctx = m->ctx;
    if (!E || !out) {
        ctx->err = "fem_pic_mfem_gauss_residual: bad argument";
        return FP_EINVAL;
    }
    const FieldDev* F = ctx->field;
    cudaStream_t s = (cudaStream_t)stream;
    const bool f32 = Q_f32(ctx);   // Q is a float array
    const bool natural = F->bc == FP_BC_NEUMANN && Q != nullptr;
    k_mass<<<grid_for(ctx, m->ne), kThreads, 0, s>>>(Sell{F->se_ptr, F->se_w, F->se_col}, F->se_M, E, m->ne, m->me);
    if (natural) {
        if (f32)
            k_qsum<float><<<1, 1024, 0, s>>>((const float*)Q, m->nn, m->qsum);
        else
            k_qsum<double><<<1, 1024, 0, s>>>((const double*)Q, m->nn, m->qsum);
    }
    FP_CUDA_TRY(ctx, cudaMemsetAsync(out, 0, 2 * sizeof(double), s));
    const double inv_a = natural ? 1.0 / F->alpha_sum : 0.0;
    const double* alpha = natural ? F->alpha : nullptr;
    const int g = grid_for(ctx, m->nn);
    if (f32)
        k_gauss_res<float><<<g, kThreads, 0, s>>>(ctx->d_n2e_ptr, ctx->d_n2e_col, ctx->d_n2e_sgn, F->node_fixed, m->me,
                                                   (const float*)Q, alpha, m->qsum, inv_a, m->nn,
                                                   (unsigned long long*)out);
    else
        k_gauss_res<double><<<g, kThreads, 0, s>>>(ctx->d_n2e_ptr, ctx->d_n2e_col, ctx->d_n2e_sgn, F->node_fixed,
                                                    m->me, (const double*)Q, alpha, m->qsum, inv_a, m->nn,
                                                    (unsigned long long*)out);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}

}  // extern "C"
