// C ABI entry points: handle lifetime, mesh tables, conversions, status.
#include <cstdio>
#include <cstring>
#include <new>

#include "internal.cuh"

using namespace fempic;

namespace {

thread_local std::string g_create_err;

template <typename T>
fp_status upload(fem_pic* ctx, T** dst, const T* src, size_t n) {
    FP_CUDA_TRY(ctx, cudaMalloc((void**)dst, n * sizeof(T) + 16));
    FP_CUDA_TRY(ctx, cudaMemcpy(*dst, src, n * sizeof(T), cudaMemcpyHostToDevice));
    return FP_OK;
}

fp_status check_csr(const HostComplex& hc, int which, const fp_csr_i8* m, std::string* err) {
    if (!m) return FP_OK;
    std::vector<int32_t> rp, col;
    std::vector<int8_t> val;
    incidence_csr(hc, which, &rp, &col, &val);
    const int64_t rows = (int64_t)rp.size() - 1;
    const int64_t cols = which == 0 ? hc.nn : (which == 1 ? hc.ne : hc.nf);
    const char* name = which == 0 ? "D0" : (which == 1 ? "D1" : "D2");
    if (m->n_rows != rows || m->n_cols != cols || m->nnz != (int64_t)col.size() || !m->row_ptr ||
        !m->col || !m->val) {
        *err = std::string("fem_pic_create: ") + name + " has the wrong shape or nnz";
        return FP_EINVAL;
    }
    if (std::memcmp(m->row_ptr, rp.data(), rp.size() * 4) != 0 ||
        std::memcmp(m->col, col.data(), col.size() * 4) != 0 ||
        std::memcmp(m->val, val.data(), val.size()) != 0) {
        *err = std::string("fem_pic_create: ") + name +
               " differs from the incidence derived from the mesh (numbering or signs)";
        return FP_EINVAL;
    }
    return FP_OK;
}

__global__ void k_project_edges(const double* __restrict__ xyz, const int32_t* __restrict__ edges,
                                int64_t ne, double E0x, double E0y, double E0z, double* __restrict__ e) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ne;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double* a = xyz + 3 * (int64_t)edges[2 * i];
        const double* b = xyz + 3 * (int64_t)edges[2 * i + 1];
        e[i] = E0x * (b[0] - a[0]) + E0y * (b[1] - a[1]) + E0z * (b[2] - a[2]);
    }
}

__global__ void k_project_faces(const double* __restrict__ xyz, const int32_t* __restrict__ faces,
                                int64_t nf, double Bx, double By, double Bz, double* __restrict__ b) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nf;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double* p = xyz + 3 * (int64_t)faces[3 * i];
        const double* q = xyz + 3 * (int64_t)faces[3 * i + 1];
        const double* r = xyz + 3 * (int64_t)faces[3 * i + 2];
        double u[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
        double v[3] = {r[0] - p[0], r[1] - p[1], r[2] - p[2]};
        double n0 = u[1] * v[2] - u[2] * v[1], n1 = u[2] * v[0] - u[0] * v[2],
               n2 = u[0] * v[1] - u[1] * v[0];
        b[i] = 0.5 * (Bx * n0 + By * n1 + Bz * n2);
    }
}

template <typename Real>
__global__ void k_from_global(const fempic::TetGeo* __restrict__ geo, int64_t nt, int64_t n,
                              const int32_t* __restrict__ cell, const double* __restrict__ X,
                              Real* __restrict__ off, int32_t* status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = cell[i];
        if (c < 0) continue;
        if (c >= nt) {
            atomicOr(status, ST_INVAL);
            continue;
        }
        for (int d = 0; d < 3; ++d) off[d * n + i] = (Real)(X[3 * i + d] - geo[c].o[d]);
    }
}

template <typename Real>
__global__ void k_to_global(const fempic::TetGeo* __restrict__ geo, int64_t nt, int64_t n,
                            const int32_t* __restrict__ cell, const Real* __restrict__ off,
                            double* __restrict__ X, int32_t* status) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        int32_t c = cell[i];
        if (c < 0 || c >= nt) {
            if (c >= nt) atomicOr(status, ST_INVAL);
            for (int d = 0; d < 3; ++d) X[3 * i + d] = 0.0;
            continue;
        }
        for (int d = 0; d < 3; ++d) X[3 * i + d] = geo[c].o[d] + (double)off[d * n + i];
    }
}

int grid_for(int64_t n, int block) {
    int64_t g = (n + block - 1) / block;
    if (g > 152 * 32) g = 152 * 32;
    return g < 1 ? 1 : (int)g;
}

}  // namespace

extern "C" {

fp_status fem_pic_create(const fp_mesh* mesh, const fp_csr_i8* D0, const fp_csr_i8* D1,
                         const fp_csr_i8* D2, int precision, fem_pic_t** out) {
    if (!out) return FP_EINVAL;
    *out = nullptr;
    g_create_err.clear();
    if (!mesh || (precision != FP_FP64 && precision != FP_FP32)) {
        g_create_err = "fem_pic_create: NULL mesh or unknown precision";
        return FP_EINVAL;
    }
    fem_pic* ctx = new (std::nothrow) fem_pic();
    if (!ctx) return FP_EINVAL;
    ctx->precision = precision;
    fp_status st = build_complex(mesh, &ctx->hc, &ctx->err);
    if (st == FP_OK) st = check_csr(ctx->hc, 0, D0, &ctx->err);
    if (st == FP_OK) st = check_csr(ctx->hc, 1, D1, &ctx->err);
    if (st == FP_OK) st = check_csr(ctx->hc, 2, D2, &ctx->err);
    if (st != FP_OK) {
        g_create_err = ctx->err;
        delete ctx;
        return st;
    }
    const HostComplex& hc = ctx->hc;
    std::vector<TetTopo> topo(hc.nt);
    for (int64_t t = 0; t < hc.nt; ++t) {
        TetTopo& T = topo[t];
        for (int k = 0; k < 4; ++k) {
            T.node[k] = hc.tv[4 * t + k];
            T.face[k] = hc.tf[4 * t + k];
            T.nb[k] = hc.nb[4 * t + k];
        }
        for (int k = 0; k < 6; ++k) T.edge[k] = hc.te[6 * t + k];
        T.pad[0] = T.pad[1] = 0;
    }
    std::vector<TetHot> hot(hc.nt);
    for (int64_t t = 0; t < hc.nt; ++t) {
        TetHot& H = hot[t];
        std::memset(&H, 0, sizeof H);
        for (int k = 0; k < 4; ++k) H.node[k] = hc.tv[4 * t + k];
        for (int k = 0; k < 6; ++k) H.edge[k] = hc.te[6 * t + k];
        for (int k = 0; k < 9; ++k) H.g[k] = (float)hc.geo[t].g[k];
    }
    // node -> incident edges with the sign of D0^T
    std::vector<int32_t> n2e_ptr(hc.nn + 1, 0), n2e_col(2 * hc.ne);
    std::vector<int8_t> n2e_sgn(2 * hc.ne);
    for (int64_t e = 0; e < hc.ne; ++e) {
        n2e_ptr[hc.edges[2 * e] + 1]++;
        n2e_ptr[hc.edges[2 * e + 1] + 1]++;
    }
    for (int64_t i = 0; i < hc.nn; ++i) n2e_ptr[i + 1] += n2e_ptr[i];
    {
        std::vector<int32_t> fill(n2e_ptr.begin(), n2e_ptr.end() - 1);
        for (int64_t e = 0; e < hc.ne; ++e) {
            int32_t i = hc.edges[2 * e], j = hc.edges[2 * e + 1];
            n2e_col[fill[i]] = (int32_t)e;
            n2e_sgn[fill[i]++] = -1;
            n2e_col[fill[j]] = (int32_t)e;
            n2e_sgn[fill[j]++] = 1;
        }
    }
    cudaError_t ce = cudaGetDevice(&ctx->device);
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, ctx->device);
    if (ce == cudaSuccess) {
        fp_status s2 = FP_OK;
        if (s2 == FP_OK) s2 = upload(ctx, &ctx->d_geo, hc.geo.data(), hc.nt);
        if (s2 == FP_OK) s2 = upload(ctx, &ctx->d_topo, topo.data(), hc.nt);
        if (s2 == FP_OK) s2 = upload(ctx, &ctx->d_xyz, hc.xyz.data(), 3 * hc.nn);
        if (s2 == FP_OK) s2 = upload(ctx, &ctx->d_edges, hc.edges.data(), 2 * hc.ne);
        if (s2 == FP_OK) s2 = upload(ctx, &ctx->d_faces, hc.faces.data(), 3 * hc.nf);
        if (s2 == FP_OK) s2 = upload(ctx, &ctx->d_n2e_ptr, n2e_ptr.data(), n2e_ptr.size());
        if (s2 == FP_OK) s2 = upload(ctx, &ctx->d_n2e_col, n2e_col.data(), n2e_col.size());
        if (s2 == FP_OK) s2 = upload(ctx, &ctx->d_n2e_sgn, n2e_sgn.data(), n2e_sgn.size());
        if (s2 == FP_OK) s2 = upload(ctx, &ctx->d_orient, hc.orient.data(), hc.orient.size());
        if (s2 == FP_OK) s2 = upload(ctx, &ctx->d_hot, hot.data(), hot.size());
        if (s2 == FP_OK && precision == FP_FP64) {   // the FP64 path's per-tet field records
            ce = cudaMalloc((void**)&ctx->d_field64, (size_t)10 * hc.nt * sizeof(double));
            if (ce != cudaSuccess) {
                ctx->err = std::string("cudaMalloc: ") + cudaGetErrorString(ce);
                s2 = FP_ECUDA;
            }
        }
        if (s2 == FP_OK) s2 = upload(ctx, &ctx->d_tet_faces, reinterpret_cast<const int4*>(hc.tf.data()), hc.nt);
        if (s2 == FP_OK) {
            int32_t z4[4] = {0, 0, 0, 0};
            s2 = upload(ctx, &ctx->d_slow_count, z4, 4);
        }
        if (s2 == FP_OK) {
            // boundary flags of nodes (1 = on a PEC face), for the interior residuals
            std::vector<uint8_t> bn(hc.nn, 0);
            for (int64_t f = 0; f < hc.nf; ++f)
                if (hc.bface[f])
                    for (int k = 0; k < 3; ++k) bn[hc.faces[3 * f + k]] = 1;
            s2 = upload(ctx, &ctx->d_node_wall, bn.data(), bn.size());
        }
        if (s2 == FP_OK) {
            int32_t zero = 0;
            s2 = upload(ctx, &ctx->d_status, &zero, 1);
        }
        if (s2 == FP_OK && precision == FP_FP32) s2 = static_queue_lookup(ctx);
        if (s2 != FP_OK) {
            g_create_err = ctx->err;
            fem_pic_destroy(ctx);
            return s2;
        }
    } else {
        g_create_err = std::string("cudaGetDevice: ") + cudaGetErrorString(ce);
        delete ctx;
        return FP_ECUDA;
    }
    *out = ctx;
    return FP_OK;
}

void fem_pic_destroy(fem_pic_t* ctx) {
    if (!ctx) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    field_free(ctx);
    void* ptrs[] = {ctx->d_geo,     ctx->d_topo,    ctx->d_xyz,     ctx->d_edges,
                    ctx->d_faces,   ctx->d_n2e_ptr, ctx->d_n2e_col, ctx->d_n2e_sgn,
                    ctx->d_orient,  ctx->d_status,  ctx->d_sort_count, ctx->d_sort_block,
                    ctx->d_sort_rank, ctx->d_hot, ctx->d_field64, ctx->d_slow_idx, ctx->d_slow_count,
                    ctx->d_node_wall, ctx->d_tet_faces};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (auto& r : ctx->prof_pending) {
        cudaEventDestroy(r.a);
        cudaEventDestroy(r.b);
    }
    for (auto e : ctx->prof_pool) cudaEventDestroy(e);
    cudaSetDevice(prev);
    delete ctx;
}

const char* fem_pic_last_error(const fem_pic_t* ctx) {
    return ctx ? ctx->err.c_str() : g_create_err.c_str();
}

fp_status fem_pic_sizes(const fem_pic_t* ctx, int64_t sizes[5]) {
    if (!ctx || !sizes) return FP_EINVAL;
    sizes[0] = ctx->hc.nn;
    sizes[1] = ctx->hc.ne;
    sizes[2] = ctx->hc.nf;
    sizes[3] = ctx->hc.nt;
    sizes[4] = ctx->precision;
    return FP_OK;
}

fp_status fem_pic_set_deposit_precision(fem_pic_t* ctx, int precision) {
    if (!ctx) return FP_EINVAL;
    if (precision != FP_FP32 && precision != FP_FP64) {
        ctx->err = "fem_pic_set_deposit_precision: precision must be FP_FP32 or FP_FP64";
        return FP_EINVAL;
    }
    if (ctx->precision == FP_FP64) {
        if (precision != FP_FP64) {
            ctx->err = "fem_pic_set_deposit_precision: an FP64 context deposits in FP64";
            return FP_EINVAL;
        }
        return FP_OK;
    }
    ctx->dG64 = ctx->Q64 = precision == FP_FP64 ? 1 : 0;
    return FP_OK;
}

int fem_pic_deposit_precision(const fem_pic_t* ctx) {
    if (!ctx) return -1;
    return ctx->precision == FP_FP64 || ctx->dG64 ? FP_FP64 : FP_FP32;
}

fp_status fem_pic_set_charge_precision(fem_pic_t* ctx, int precision) {
    if (!ctx) return FP_EINVAL;
    if (precision != FP_FP32 && precision != FP_FP64) {
        ctx->err = "fem_pic_set_charge_precision: precision must be FP_FP32 or FP_FP64";
        return FP_EINVAL;
    }
    if (precision == FP_FP32 && (ctx->precision == FP_FP64 || ctx->dG64)) {
        ctx->err = "fem_pic_set_charge_precision: with double dG arrays Q is double too";
        return FP_EINVAL;
    }
    if (ctx->precision == FP_FP32) ctx->Q64 = precision == FP_FP64 ? 1 : 0;
    return FP_OK;
}

int fem_pic_charge_precision(const fem_pic_t* ctx) {
    if (!ctx) return -1;
    return ctx->precision == FP_FP64 || ctx->Q64 ? FP_FP64 : FP_FP32;
}

fp_status fem_pic_incidence(const fem_pic_t* ctx, int which, int32_t* row_ptr, int32_t* col,
                            int8_t* val) {
    if (!ctx || which < 0 || which > 2 || !row_ptr || !col || !val) return FP_EINVAL;
    std::vector<int32_t> rp, c;
    std::vector<int8_t> v;
    incidence_csr(ctx->hc, which, &rp, &c, &v);
    std::memcpy(row_ptr, rp.data(), rp.size() * 4);
    std::memcpy(col, c.data(), c.size() * 4);
    std::memcpy(val, v.data(), v.size());
    return FP_OK;
}

fp_status fem_pic_topology(const fem_pic_t* ctx, int32_t* tet_nodes, int32_t* tet_edges,
                           int32_t* tet_faces, int32_t* tet_neigh) {
    if (!ctx) return FP_EINVAL;
    const HostComplex& hc = ctx->hc;
    if (tet_nodes) std::memcpy(tet_nodes, hc.tv.data(), hc.tv.size() * 4);
    if (tet_edges) std::memcpy(tet_edges, hc.te.data(), hc.te.size() * 4);
    if (tet_faces) std::memcpy(tet_faces, hc.tf.data(), hc.tf.size() * 4);
    if (tet_neigh) std::memcpy(tet_neigh, hc.nb.data(), hc.nb.size() * 4);
    return FP_OK;
}

fp_status fem_pic_project_uniform(fem_pic_t* ctx, const double E0[3], const double B0[3], double* e,
                                  double* b, void* stream) {
    if (!ctx || !E0 || !B0) return FP_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    if (e) {
        k_project_edges<<<grid_for(ctx->hc.ne, 256), 256, 0, s>>>(ctx->d_xyz, ctx->d_edges, ctx->hc.ne,
                                                                  E0[0], E0[1], E0[2], e);
        FP_CUDA_TRY(ctx, cudaGetLastError());
    }
    if (b) {
        k_project_faces<<<grid_for(ctx->hc.nf, 256), 256, 0, s>>>(ctx->d_xyz, ctx->d_faces, ctx->hc.nf,
                                                                  B0[0], B0[1], B0[2], b);
        FP_CUDA_TRY(ctx, cudaGetLastError());
    }
    return FP_OK;
}

fp_status fem_pic_particles_from_global(fem_pic_t* ctx, int64_t n, const int32_t* cell,
                                        const double* X, void* off, void* stream) {
    if (!ctx || n < 0 || (n > 0 && (!cell || !X || !off))) return FP_EINVAL;
    if (n == 0) return FP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->precision == FP_FP32)
        k_from_global<float><<<grid_for(n, 256), 256, 0, s>>>(ctx->d_geo, ctx->hc.nt, n, cell, X,
                                                              (float*)off, ctx->d_status);
    else
        k_from_global<double><<<grid_for(n, 256), 256, 0, s>>>(ctx->d_geo, ctx->hc.nt, n, cell, X,
                                                               (double*)off, ctx->d_status);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}

fp_status fem_pic_particles_to_global(fem_pic_t* ctx, int64_t n, const int32_t* cell,
                                      const void* off, double* X, void* stream) {
    if (!ctx || n < 0 || (n > 0 && (!cell || !X || !off))) return FP_EINVAL;
    if (n == 0) return FP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->precision == FP_FP32)
        k_to_global<float><<<grid_for(n, 256), 256, 0, s>>>(ctx->d_geo, ctx->hc.nt, n, cell,
                                                            (const float*)off, X, ctx->d_status);
    else
        k_to_global<double><<<grid_for(n, 256), 256, 0, s>>>(ctx->d_geo, ctx->hc.nt, n, cell,
                                                             (const double*)off, X, ctx->d_status);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}

fp_status fem_pic_push_deposit(fem_pic_t* ctx, const double* e, const double* b,
                               const fp_particles* p, double dt, int max_cross, void* dG, void* Q,
                               int flags, void* stream) {
    if (!ctx || !p || !e || !b || !dG || !Q || p->n < 0 || max_cross < 0 || !(p->m > 0.0)) {
        if (ctx) ctx->err = "fem_pic_push_deposit: NULL pointer or bad argument";
        return FP_EINVAL;
    }
    if (p->n > 0 && (!p->cell || !p->off || !p->vel)) {
        ctx->err = "fem_pic_push_deposit: NULL particle array";
        return FP_EINVAL;
    }
    return launch_push_deposit(ctx, e, b, p, dt, max_cross, dG, Q, flags, (cudaStream_t)stream);
}

fp_status fem_pic_push_deposit_adams(fem_pic_t* ctx, const double* e, const double* b, const fp_particles* p,
                                     void* hist, int64_t step, double dt, int max_cross, void* dG, void* Q,
                                     int flags, void* stream) {
    if (!ctx || !p || !e || !b || !dG || !Q || p->n < 0 || max_cross < 0 || step < 0 || !(p->m > 0.0)) {
        if (ctx) ctx->err = "fem_pic_push_deposit_adams: NULL pointer or bad argument";
        return FP_EINVAL;
    }
    if (p->n > 0 && (!p->cell || !p->off || !p->vel || !hist)) {
        ctx->err = "fem_pic_push_deposit_adams: NULL particle or history array";
        return FP_EINVAL;
    }
    return launch_push_adams(ctx, e, b, p, hist, step, dt, max_cross, dG, Q, flags, (cudaStream_t)stream);
}

fp_status fem_pic_deposit_charge(fem_pic_t* ctx, const fp_particles* p, void* Q, int flags,
                                 void* stream) {
    if (!ctx || !p || !Q || p->n < 0) return FP_EINVAL;
    if (p->n > 0 && (!p->cell || !p->off)) return FP_EINVAL;
    return launch_deposit_charge(ctx, p, Q, flags, (cudaStream_t)stream);
}

fp_status fem_pic_sort(fem_pic_t* ctx, const fp_particles* src, fp_particles* dst, void* stream) {
    if (!ctx || !src || !dst || src->n != dst->n || src->n < 0) return FP_EINVAL;
    if (src->n > 0 && (!src->cell || !src->off || !src->vel || !dst->cell || !dst->off || !dst->vel ||
                       src->cell == dst->cell || src->off == dst->off || src->vel == dst->vel)) {
        ctx->err = "fem_pic_sort: NULL or aliased particle arrays";
        return FP_EINVAL;
    }
    return launch_sort(ctx, src, dst, (cudaStream_t)stream);
}

fp_status fem_pic_sort_columns(fem_pic_t* ctx, const fp_particles* src, fp_particles* dst, const void* cols_src,
                               void* cols_dst, int ncols, void* stream) {
    if (!ctx || !src || !dst || src->n != dst->n || src->n < 0 || ncols < 0) return FP_EINVAL;
    if (src->n > 0 && (!src->cell || !src->off || !src->vel || !dst->cell || !dst->off || !dst->vel ||
                       src->cell == dst->cell || src->off == dst->off || src->vel == dst->vel ||
                       (ncols > 0 && (!cols_src || !cols_dst || cols_src == cols_dst)))) {
        ctx->err = "fem_pic_sort_columns: NULL or aliased arrays";
        return FP_EINVAL;
    }
    return launch_sort(ctx, src, dst, (cudaStream_t)stream, cols_src, cols_dst, ncols);
}

fp_status fem_pic_residuals(fem_pic_t* ctx, const void* dG, const void* Q_new, const void* Q_old,
                            const double* b, double* out, void* stream) {
    if (!ctx || !out) return FP_EINVAL;
    return launch_residuals(ctx, dG, Q_new, Q_old, b, out, (cudaStream_t)stream);
}

fp_status fem_pic_profile_enable(fem_pic_t* ctx, int on) {
    if (!ctx) return FP_EINVAL;
    ctx->prof_on = on != 0;
    return FP_OK;
}

fp_status fem_pic_profile_read(fem_pic_t* ctx, double ms[16], int64_t count[16], int reset) {
    if (!ctx) return FP_EINVAL;
    for (auto& r : ctx->prof_pending) {
        FP_CUDA_TRY(ctx, cudaEventSynchronize(r.b));
        float t = 0.f;
        FP_CUDA_TRY(ctx, cudaEventElapsedTime(&t, r.a, r.b));
        ctx->prof_ms[r.phase] += t;
        ctx->prof_n[r.phase] += 1;
        ctx->prof_pool.push_back(r.a);
        ctx->prof_pool.push_back(r.b);
    }
    ctx->prof_pending.clear();
    for (int i = 0; i < PH_COUNT; ++i) {
        if (ms) ms[i] = ctx->prof_ms[i];
        if (count) count[i] = ctx->prof_n[i];
        if (reset) {
            ctx->prof_ms[i] = 0.0;
            ctx->prof_n[i] = 0;
        }
    }
    return FP_OK;
}

fp_status fem_pic_selftest_wait(fem_pic_t* ctx, double limit_s, void* stream) {
    if (!ctx || !(limit_s > 0.0) || limit_s > 10.0) {
        if (ctx) ctx->err = "fem_pic_selftest_wait: limit outside (0, 10] s";
        return FP_EINVAL;
    }
    return launch_wait_selftest(ctx, limit_s, (cudaStream_t)stream);
}

fp_status fem_pic_status(fem_pic_t* ctx, void* stream) {
    if (!ctx) return FP_EINVAL;
    int32_t h = 0;
    cudaStream_t s = (cudaStream_t)stream;
    FP_CUDA_TRY(ctx, cudaMemcpyAsync(&h, ctx->d_status, 4, cudaMemcpyDeviceToHost, s));
    FP_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    FP_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_status, 0, 4, s));
    FP_CUDA_TRY(ctx, cudaStreamSynchronize(s));
    if (h & ST_TIMEOUT) {
        ctx->err = "a kernel gave up waiting for its asynchronous copies";
        return FP_ECUDA;
    }
    if (h & ST_NONFINITE) {
        ctx->err = "a particle's position or velocity was not finite (NaN or Inf): it was removed "
                   "(cell -1) with nothing deposited";
        return FP_EINVAL;
    }
    if (h & ST_INVAL) {
        ctx->err = "a kernel saw a cell id outside [0, N_t)";
        return FP_EINVAL;
    }
    if (h & ST_WALK) {
        ctx->err = "a particle reached the crossing bound of the tet walk";
        return FP_EWALK;
    }
    if (h & ST_NOCONV) {
        ctx->err = "an iterative field solve reached its iteration cap";
        return FP_ENOCONV;
    }
    return FP_OK;
}

}  // extern "C"
