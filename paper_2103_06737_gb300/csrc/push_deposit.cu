// The per-particle hot path: Whitney gather, Boris push, tet walk, charge-conserving
// Whitney-1 current deposit and Whitney-0 charge deposit (Sec. II.A, II.C, IV.B.1).
//
// Particles in struct-of-arrays.  After a cell sort consecutive particles mostly share a
// tet.  The default FP32 push (k_push_run32) gives each lane a few consecutive particles:
// a lane re-reads the tet's record only where the tet changes and sums the deposits of a
// run of particles in one tet in registers, the warp joins the runs that cross lane
// boundaries, and one global atomic per edge/node is issued per run.  The other kernels
// take one particle per lane and reduce runs with warp shuffles.  Particles whose path
// leaves (or may leave) their tet are deferred to the FP64 walk, which deposits each piece
// with direct atomics.
//
// The gather goes through per-tet affine field records (E = E0 + W x off, B = B0 + beta off
// in the tet, equal to the Whitney-1 / Whitney-2 sums), made once per call from e and b by
// k_field_prep32 (FP32 records) or k_field_prep64 (FP64 mode).
//
// Precision: fields, push and deposit products in Real (float or double); the deposit
// arrays are Real or, for an FP32 context with FP64 deposits, double.  The exit
// test of the walk (barycentric coordinates of the end point, crossing fraction,
// argmin) is always FP64.  The piece deposit uses the factored form
//   dG_ab = q w (l^a_a (l^c_b - l^a_b) - l^a_b (l^c_a - l^a_a)),
// algebraically equal to q w (l^a_a l^c_b - l^a_b l^c_a), the exact line integral of
// W1_ab along a straight piece; the differences are formed in FP64 so the Real products
// do not cancel.
#include <string>

#include "async_copy.cuh"
#include "internal.cuh"

namespace fempic {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct Geo {
    double o[3];
    double g[9];
};

__device__ __forceinline__ void load_geo(const TetGeo* __restrict__ geo, int c, Geo& G) {
    const double2* p = reinterpret_cast<const double2*>(geo + c);
    double2 a = __ldg(p), b = __ldg(p + 1), d = __ldg(p + 2), e = __ldg(p + 3), f = __ldg(p + 4),
            h = __ldg(p + 5);
    G.o[0] = a.x;
    G.o[1] = a.y;
    G.o[2] = b.x;
    G.g[0] = b.y;
    G.g[1] = d.x;
    G.g[2] = d.y;
    G.g[3] = e.x;
    G.g[4] = e.y;
    G.g[5] = f.x;
    G.g[6] = f.y;
    G.g[7] = h.x;
    G.g[8] = h.y;
}

__device__ __forceinline__ void load_topo(const TetTopo* __restrict__ topo, int c, TetTopo& T) {
    const int4* p = reinterpret_cast<const int4*>(topo + c);
    int4 a = __ldg(p), b = __ldg(p + 1), d = __ldg(p + 2), e = __ldg(p + 3), f = __ldg(p + 4);
    T.node[0] = a.x;
    T.node[1] = a.y;
    T.node[2] = a.z;
    T.node[3] = a.w;
    T.edge[0] = b.x;
    T.edge[1] = b.y;
    T.edge[2] = b.z;
    T.edge[3] = b.w;
    T.edge[4] = d.x;
    T.edge[5] = d.y;
    T.face[0] = d.z;
    T.face[1] = d.w;
    T.face[2] = e.x;
    T.face[3] = e.y;
    T.nb[0] = e.z;
    T.nb[1] = e.w;
    T.nb[2] = f.x;
    T.nb[3] = f.y;
}

// barycentric coordinates of a point given relative to the tet's origin (FP64)
__device__ __forceinline__ void bary(const Geo& G, const double r[3], double l[4]) {
    l[1] = G.g[0] * r[0] + G.g[1] * r[1] + G.g[2] * r[2];
    l[2] = G.g[3] * r[0] + G.g[4] * r[1] + G.g[5] * r[2];
    l[3] = G.g[6] * r[0] + G.g[7] * r[1] + G.g[8] * r[2];
    l[0] = ((1.0 - l[1]) - l[2]) - l[3];
}

template <typename Real>
__device__ __forceinline__ void cross(const Real a[3], const Real b[3], Real o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// non-relativistic Boris rotation; h = q dt / (2 m)
// 2 / (1 + tt), correctly rounded (for float via the correctly rounded reciprocal: scaling by
// 2 commutes with rounding, so the result is the same as the division)
__device__ __forceinline__ float two_over(float tt) { return __fdividef(2.f, 1.f + tt); }
__device__ __forceinline__ double two_over(double tt) { return 2.0 / (1.0 + tt); }

template <typename Real>
__device__ __forceinline__ void boris(Real v[3], const Real E[3], const Real B[3], Real h) {
    Real vm[3], t[3], s[3], c[3], vp[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        vm[i] = v[i] + h * E[i];
        t[i] = h * B[i];
    }
    Real tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    Real f = two_over(tt);
#pragma unroll
    for (int i = 0; i < 3; ++i) s[i] = f * t[i];
    cross(vm, t, c);
#pragma unroll
    for (int i = 0; i < 3; ++i) vp[i] = vm[i] + c[i];
    cross(vp, s, c);
#pragma unroll
    for (int i = 0; i < 3; ++i) v[i] = vm[i] + c[i] + h * E[i];
}

// end point relative to the start origin, without FMA contraction (reproducible on a CPU)
__device__ __forceinline__ float step_pos(float x, float dt, float v) {
    return __fadd_rn(x, __fmul_rn(dt, v));
}
__device__ __forceinline__ double step_pos(double x, double dt, double v) {
    return __dadd_rn(x, __dmul_rn(dt, v));
}

template <typename Real>
__device__ __forceinline__ Real to_real(double x);
template <>
__device__ __forceinline__ float to_real<float>(double x) {
    return d2f(x);
}
template <>
__device__ __forceinline__ double to_real<double>(double x) {
    return x;
}
__device__ __forceinline__ double to_f64(float x) {
    return f2d(x);
}
__device__ __forceinline__ double to_f64(double x) {
    return x;
}

template <typename Real>
__device__ __forceinline__ void piece_values(const double la[4], const double lx[4], double qw,
                                             Real val[6]) {
    Real A[4], D[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        A[k] = to_real<Real>(la[k]);
        D[k] = to_real<Real>(lx[k] - la[k]);
    }
    const Real w = to_real<Real>(qw);
    val[0] = w * (A[0] * D[1] - A[1] * D[0]);
    val[1] = w * (A[0] * D[2] - A[2] * D[0]);
    val[2] = w * (A[0] * D[3] - A[3] * D[0]);
    val[3] = w * (A[1] * D[2] - A[2] * D[1]);
    val[4] = w * (A[1] * D[3] - A[3] * D[1]);
    val[5] = w * (A[2] * D[3] - A[3] * D[2]);
}

// values computed in Real, added into deposit arrays of type D (D = double with FP32
// arithmetic: FP64 deposits of an FP32-mode context)
template <typename Real, typename D = Real>
__device__ __forceinline__ void deposit_piece(const TetTopo& T, const double la[4], const double lx[4],
                                              double qw, D* __restrict__ dG) {
    Real val[6];
    piece_values<Real>(la, lx, qw, val);
#pragma unroll
    for (int k = 0; k < 6; ++k) atomicAdd(dG + T.edge[k], dep_cast<D>(val[k]));
}

template <typename Real, typename D = Real>
__device__ __forceinline__ void deposit_charge(const TetTopo& T, const double l[4], double qw,
                                               D* __restrict__ Q) {
#pragma unroll
    for (int k = 0; k < 4; ++k)
        atomicAdd(Q + T.node[k], dep_cast<D>(to_real<Real>(qw) * to_real<Real>(l[k])));
}

// Sum `v[0..NV)` over each run of equal `key` in lane order; the first lane of a run
// (with key >= 0) issues one atomic per value.  All 32 lanes must call this.
template <typename Real, int NV>
__device__ __forceinline__ void warp_run_reduce(int key, Real v[NV], unsigned* heads_out, int* end_out) {
    const int lane = threadIdx.x & 31;
    int prev = __shfl_up_sync(kFull, key, 1);
    bool head = lane == 0 || prev != key;
    unsigned heads = __ballot_sync(kFull, head);
    unsigned above = heads & ~((2u << lane) - 1u);
    int end = above ? __ffs(above) - 1 : 32;
    if (heads != kFull) {
        // only as many shuffle steps as the longest run needs (ceil(log2(longest run)))
        const unsigned longest = __reduce_max_sync(kFull, head ? (unsigned)(end - lane) : 0u);
        for (int o = 1; o < (int)longest; o <<= 1) {
            const bool take = lane + o < end;
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                const Real u = __shfl_down_sync(kFull, v[k], o);
                if (take) v[k] += u;
            }
        }
    }
    *heads_out = heads;
    *end_out = end;
}

// ---------------------------------------------------------------- FP64 walk
// Straight path from xa to xb, both relative to the origin of the start tet c.  Every
// piece deposits its 6 edge values, the end point its 4 node charges.  When `agg` is
// non-null and the path stays inside c, the 10 values are returned in agg instead of
// being added (return true) so the caller can reduce them across the warp.
//
// FP64 is spent only on the exit test: the end point's barycentrics in each tet, the
// crossing fraction and the carried crossing barycentrics.  The smallest fraction is
// found by cross-multiplication (one division per crossing).  The deposit products are
// in Real; the current point, needed only when the walk stops early, is tracked in
// Real as well.
//
// cc (charge change): Q receives the change of the particle's W0 charge over the step, its
// end point's charge minus its start point's (the start's, where a particle is removed for a
// non-finite push), instead of the end point's charge.
template <typename Real, typename DG = Real, typename DQ = DG>
__device__ bool walk_fp64(const TetGeo* __restrict__ geo, const TetTopo* __restrict__ topo, int c,
                          const double xa[3], const double xb[3], double qw, int max_cross,
                          DG* __restrict__ dG, DQ* __restrict__ Q, int32_t* __restrict__ status,
                          Real* agg, int* end_cell, double end_off[3], bool cc = false) {
    Geo G;
    TetTopo Tc;
    double la[4], rel[3], os[3];
    const bool start_finite = finite_bits(xa[0]) && finite_bits(xa[1]) && finite_bits(xa[2]);
    if (!(start_finite && finite_bits(xb[0]) && finite_bits(xb[1]) && finite_bits(xb[2]))) {
        // a non-finite start or end point has no path: the particle is removed, nothing deposited
        // (with cc, its start point's charge leaves Q where the start is finite)
        atomicOr(status, ST_NONFINITE);
        *end_cell = -1;
#pragma unroll
        for (int i = 0; i < 3; ++i) end_off[i] = xa[i];
        if (cc && start_finite) {
            load_geo(geo, c, G);
            load_topo(topo, c, Tc);
            bary(G, xa, la);
            deposit_charge<Real, DQ>(Tc, la, -qw, Q);
        }
        return false;
    }
    load_geo(geo, c, G);
    load_topo(topo, c, Tc);
    bary(G, xa, la);
    Real ca[3], cb[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        ca[i] = to_real<Real>(xa[i]);
        cb[i] = to_real<Real>(xb[i]);
        rel[i] = xb[i];
        os[i] = G.o[i];
    }
    int t = c, entry = -1, nc = 0;
    for (;;) {
        double lb[4];
        bary(G, rel, lb);
        // exit candidates: faces other than the entry face with l^b_k < 0
        unsigned cand = 0u;
#pragma unroll
        for (int k = 0; k < 4; ++k) cand |= (k != entry && neg_strict(lb[k])) ? (1u << k) : 0u;
        int kx = -1;
        double smin = 0.0;
        if (cand != 0u && (cand & (cand - 1u)) == 0u) {
            // one candidate (the common crossing): l^a_k > 0 > l^b_k gives s in [0,1)
            kx = __ffs(cand) - 1;
            const double ak = kx == 0 ? la[0] : (kx == 1 ? la[1] : (kx == 2 ? la[2] : la[3]));
            const double bk = kx == 0 ? lb[0] : (kx == 1 ? lb[1] : (kx == 2 ? lb[2] : lb[3]));
            smin = pos_strict(ak) ? ak / (ak - bk) : 0.0;
        } else if (cand != 0u) {
            // several: the smallest fraction by cross-multiplication, one division
            double bn = 0.0, bd = 1.0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (!((cand >> k) & 1u)) continue;
                double num = la[k], den = la[k] - lb[k];
                if (!pos_strict(num) || !pos_strict(den)) {  // fraction clamps to 0
                    num = 0.0;
                    den = 1.0;
                } else if (num > den) {                      // fraction clamps to 1
                    num = 1.0;
                    den = 1.0;
                }
                if (kx < 0 || num * bd < bn * den) {
                    kx = k;
                    bn = num;
                    bd = den;
                }
            }
            smin = bn / bd;
        }
        if (kx < 0) {
            *end_cell = t;
#pragma unroll
            for (int i = 0; i < 3; ++i) end_off[i] = rel[i];
            if (nc == 0 && agg) {
                piece_values<Real>(la, lb, qw, agg);
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    agg[6 + k] = to_real<Real>(qw) * to_real<Real>(cc ? lb[k] - la[k] : lb[k]);
                return true;
            }
            deposit_piece<Real, DG>(Tc, la, lb, qw, dG);
            if (cc && nc == 0) {   // still in the start tet: the change of its nodes' charge
                double lq[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) lq[k] = lb[k] - la[k];
                deposit_charge<Real, DQ>(Tc, lq, qw, Q);
            } else {
                deposit_charge<Real, DQ>(Tc, lb, qw, Q);
            }
            return false;
        }
        if (nc == max_cross) {  // bound reached: stop at the last crossing point
            if (!cc || nc > 0) deposit_charge<Real, DQ>(Tc, la, qw, Q);   // (cc, no crossing: no change)
            atomicOr(status, ST_WALK);
            *end_cell = t;
#pragma unroll
            for (int i = 0; i < 3; ++i) end_off[i] = to_f64(ca[i]) + (os[i] - G.o[i]);
            return false;
        }
        double lc[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) lc[k] = (k == kx) ? 0.0 : la[k] + smin * (lb[k] - la[k]);
        if (cc && nc == 0) deposit_charge<Real, DQ>(Tc, la, -qw, Q);   // the start point's charge leaves
        deposit_piece<Real, DG>(Tc, la, lc, qw, dG);
        const Real sr = to_real<Real>(smin);
#pragma unroll
        for (int i = 0; i < 3; ++i) ca[i] = ca[i] + sr * (cb[i] - ca[i]);
        const int tn = kx == 0 ? Tc.nb[0] : (kx == 1 ? Tc.nb[1] : (kx == 2 ? Tc.nb[2] : Tc.nb[3]));
        if (tn < 0) {  // PEC wall: absorbed, its charge stays at the wall point
            deposit_charge<Real, DQ>(Tc, lc, qw, Q);
            *end_cell = -1;
#pragma unroll
            for (int i = 0; i < 3; ++i) end_off[i] = to_f64(ca[i]) + (os[i] - G.o[i]);
            return false;
        }
        TetTopo Tn;
        load_topo(topo, tn, Tn);
        int ent = 0;
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            const int vtx = Tn.node[a];
            double lv = 0.0;
            bool found = false;
#pragma unroll
            for (int j = 0; j < 4; ++j)
                if (Tc.node[j] == vtx) {
                    lv = lc[j];
                    found = true;
                }
            la[a] = lv;
            if (!found) ent = a;
        }
        load_geo(geo, tn, G);
        Tc = Tn;
        t = tn;
        entry = ent;
        ++nc;
#pragma unroll
        for (int i = 0; i < 3; ++i) rel[i] = (os[i] - G.o[i]) + xb[i];
    }
}

// FP64 mode: the affine field coefficients of k_field_prep32 (below) in FP64, from the FP64
// gradients, 10 doubles per tet:
// rec = E0 (3), W (3), B0 (3), beta, with E = E0 + W x off and B = B0 + beta off in the tet
// (off relative to its vertex 0) equal to the Whitney-1 / Whitney-2 sums (Sec. II.C).
__global__ void __launch_bounds__(256) k_field_prep64(const TetGeo* __restrict__ geo,
                                                      const TetTopo* __restrict__ topo,
                                                      const double* __restrict__ e, const double* __restrict__ b,
                                                      int64_t nt, double* __restrict__ rec) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
        Geo G;
        TetTopo T;
        load_geo(geo, (int)t, G);
        load_topo(topo, (int)t, T);
        double g[4][3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            g[1][i] = G.g[i];
            g[2][i] = G.g[3 + i];
            g[3][i] = G.g[6 + i];
            g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
        }
        double ev[6], bv[4];
#pragma unroll
        for (int k = 0; k < 6; ++k) ev[k] = __ldg(e + T.edge[k]);
#pragma unroll
        for (int k = 0; k < 4; ++k) bv[k] = __ldg(b + T.face[k]);
        double x01[3], x02[3], x03[3], x12[3], x13[3], x23[3];
        cross<double>(g[0], g[1], x01);
        cross<double>(g[0], g[2], x02);
        cross<double>(g[0], g[3], x03);
        cross<double>(g[1], g[2], x12);
        cross<double>(g[1], g[3], x13);
        cross<double>(g[2], g[3], x23);
        double E0[3], W[3], K[4][3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            E0[i] = ev[0] * g[1][i] + ev[1] * g[2][i] + ev[2] * g[3][i];
            W[i] = ev[0] * x01[i] + ev[1] * x02[i] + ev[2] * x03[i] + ev[3] * x12[i] + ev[4] * x13[i] +
                   ev[5] * x23[i];
            // faces: 0=(1,2,3), 1=(0,2,3), 2=(0,1,3), 3=(0,1,2)
            K[0][i] = 2.0 * (bv[1] * x23[i] + bv[2] * x13[i] + bv[3] * x12[i]);
            K[1][i] = 2.0 * (bv[0] * x23[i] - bv[2] * x03[i] - bv[3] * x02[i]);
            K[2][i] = 2.0 * (-bv[0] * x13[i] - bv[1] * x03[i] + bv[3] * x01[i]);
            K[3][i] = 2.0 * (bv[0] * x12[i] + bv[1] * x02[i] + bv[2] * x01[i]);
        }
        double beta = 0.0;
#pragma unroll
        for (int a = 1; a < 4; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) beta += (K[a][i] - K[0][i]) * g[a][i];
        double* r = rec + 10 * t;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            r[i] = E0[i];
            r[3 + i] = W[i];
            r[6 + i] = K[0][i];
        }
        r[9] = beta * (1.0 / 3.0);
    }
}

// E and B at offset x in tet c from its FP64 record
__device__ __forceinline__ void fields64(const double* __restrict__ rec, int c, const double x[3], double E[3],
                                         double B[3]) {
    const double2* p = reinterpret_cast<const double2*>(rec + 10 * (int64_t)c);
    const double2 a = __ldg(p), bb = __ldg(p + 1), d = __ldg(p + 2), f = __ldg(p + 3), h = __ldg(p + 4);
    const double E0[3] = {a.x, a.y, bb.x}, W[3] = {bb.y, d.x, d.y}, B0[3] = {f.x, f.y, h.x};
    const double beta = h.y;
    E[0] = E0[0] + (W[1] * x[2] - W[2] * x[1]);
    E[1] = E0[1] + (W[2] * x[0] - W[0] * x[2]);
    E[2] = E0[2] + (W[0] * x[1] - W[1] * x[0]);
#pragma unroll
    for (int i = 0; i < 3; ++i) B[i] = B0[i] + beta * x[i];
}

// ---------------------------------------------------------------- FP64 mode
template <typename Real>
__global__ void __launch_bounds__(256) k_push_deposit(
    const TetGeo* __restrict__ geo, const TetTopo* __restrict__ topo, const double* __restrict__ f64,
    int32_t* __restrict__ cell, Real* __restrict__ off,
    Real* __restrict__ vel, int64_t n, int32_t nt, double qmdt2, Real dt, double qw, int max_cross,
    int aggregate, Real* __restrict__ dG, Real* __restrict__ Q, int32_t* __restrict__ status, int cc) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride) {
        const int64_t p = base + lane;
        int c = p < n ? cell[p] : -1;
        if (c >= nt) {
            atomicOr(status, ST_INVAL);
            c = -1;
        }
        int key = -1;
        Real agg[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) agg[k] = (Real)0;
        TetTopo T;
        if (c >= 0) {
            load_topo(topo, c, T);
            Real x[3] = {off[p], off[n + p], off[2 * n + p]};
            Real v[3] = {vel[p], vel[n + p], vel[2 * n + p]};
            double xa[3] = {(double)x[0], (double)x[1], (double)x[2]};
            Real E[3], B[3];
            fields64(f64, c, xa, E, B);
            boris<Real>(v, E, B, (Real)qmdt2);
            vel[p] = v[0];
            vel[n + p] = v[1];
            vel[2 * n + p] = v[2];
            double xb[3];
#pragma unroll
            for (int i = 0; i < 3; ++i) xb[i] = (double)step_pos(x[i], dt, v[i]);
            int end_cell;
            double end_off[3];
            if (walk_fp64<Real>(geo, topo, c, xa, xb, qw, max_cross, dG, Q, status, aggregate ? agg : nullptr,
                                &end_cell, end_off, cc != 0))
                key = c;
            cell[p] = end_cell;
            off[p] = (Real)end_off[0];
            off[n + p] = (Real)end_off[1];
            off[2 * n + p] = (Real)end_off[2];
        }
        if (aggregate) {
            unsigned heads;
            int end;
            warp_run_reduce<Real, 10>(key, agg, &heads, &end);
            if (((heads >> lane) & 1u) && key >= 0) {
#pragma unroll
                for (int k = 0; k < 6; ++k) atomicAdd(dG + T.edge[k], agg[k]);
#pragma unroll
                for (int k = 0; k < 4; ++k) atomicAdd(Q + T.node[k], agg[6 + k]);
            }
        }
    }
}

// ---------------------------------------------------------------- FP32 mode
__device__ __forceinline__ void load_hot(const TetHot* __restrict__ hot, int c, TetHot& H) {
    const float4* p = reinterpret_cast<const float4*>(hot + c);
    float4 r[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) r[k] = __ldg(p + k);
    memcpy(&H, r, sizeof(TetHot));
}

// Affine field coefficients of every tet from the edge and face DOFs (FP32):
//   E = E0 + W x off,  E0 = sum_{b} e_0b g_b,  W = sum_{a<b} e_ab g_a x g_b;
//   B = sum_a lambda_a K_a with K_a from the W2 functions; B0 = K_0 and
//   beta = (1/3) sum_{a>0} (K_a - K_0) . g_a  (the field is B0 + beta off).
// Rewrites bytes 64..127 of each record (g row 3 and the coefficients).
__global__ void __launch_bounds__(256) k_field_prep32(TetHot* __restrict__ hot,
                                                      const int4* __restrict__ tet_faces,
                                                      const double* __restrict__ e,
                                                      const double* __restrict__ b, int64_t nt) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
#pragma unroll 2
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt; t += stride) {
        // bytes 16..79 of the record: edge ids and the FP32 gradients
        const float4* hp = reinterpret_cast<const float4*>(hot + t);
        const float4 r1 = __ldg(hp + 1), r2 = __ldg(hp + 2), r3 = __ldg(hp + 3), r4 = __ldg(hp + 4);
        const int4 f = __ldg(tet_faces + t);
        const int edge[6] = {__float_as_int(r1.x), __float_as_int(r1.y), __float_as_int(r1.z),
                             __float_as_int(r1.w), __float_as_int(r2.x), __float_as_int(r2.y)};
        const int face[4] = {f.x, f.y, f.z, f.w};
        float ev[6], bv[4];
#pragma unroll
        for (int k = 0; k < 6; ++k) ev[k] = d2f(__ldg(e + edge[k]));
#pragma unroll
        for (int k = 0; k < 4; ++k) bv[k] = d2f(__ldg(b + face[k]));
        const float hg[9] = {r2.z, r2.w, r3.x, r3.y, r3.z, r3.w, r4.x, r4.y, r4.z};
        float g[4][3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            g[1][i] = hg[i];
            g[2][i] = hg[3 + i];
            g[3][i] = hg[6 + i];
            g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
        }
        float x01[3], x02[3], x03[3], x12[3], x13[3], x23[3];
        cross<float>(g[0], g[1], x01);
        cross<float>(g[0], g[2], x02);
        cross<float>(g[0], g[3], x03);
        cross<float>(g[1], g[2], x12);
        cross<float>(g[1], g[3], x13);
        cross<float>(g[2], g[3], x23);
        float E0[3], W[3], K[4][3];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            E0[i] = ev[0] * g[1][i] + ev[1] * g[2][i] + ev[2] * g[3][i];
            W[i] = ev[0] * x01[i] + ev[1] * x02[i] + ev[2] * x03[i] + ev[3] * x12[i] + ev[4] * x13[i] +
                   ev[5] * x23[i];
            // faces: 0=(1,2,3), 1=(0,2,3), 2=(0,1,3), 3=(0,1,2)
            K[0][i] = 2.f * (bv[1] * x23[i] + bv[2] * x13[i] + bv[3] * x12[i]);
            K[1][i] = 2.f * (bv[0] * x23[i] - bv[2] * x03[i] - bv[3] * x02[i]);
            K[2][i] = 2.f * (-bv[0] * x13[i] - bv[1] * x03[i] + bv[3] * x01[i]);
            K[3][i] = 2.f * (bv[0] * x12[i] + bv[1] * x02[i] + bv[2] * x01[i]);
        }
        float beta = 0.f;
#pragma unroll
        for (int a = 1; a < 4; ++a)
#pragma unroll
            for (int i = 0; i < 3; ++i) beta += (K[a][i] - K[0][i]) * g[a][i];
        beta *= (1.f / 3.f);
        float4* w = reinterpret_cast<float4*>(hot + t) + 4;
        w[0] = make_float4(hg[6], hg[7], hg[8], E0[0]);
        w[1] = make_float4(E0[1], E0[2], W[0], W[1]);
        w[2] = make_float4(W[2], K[0][0], K[0][1], K[0][2]);
        float gsum = 0.f;   // sum of |g| over the 9 stored gradient entries (rounding bound of the fast path)
#pragma unroll
        for (int k = 0; k < 9; ++k) gsum += fabsf(hg[k]);
        w[3] = make_float4(beta, gsum, 0.f, 0.f);
    }
}

// A shared-memory window of tet records keeps them 144 bytes apart (one 128-byte bulk copy
// each), so the same 16-byte chunk of the records of 8 consecutive cells falls on 8 different
// bank groups when a warp reads them.
constexpr int kRecStride = (int)sizeof(TetHot) + 16;

// E and B at a point x (relative to the tet's origin) from the tet's affine field coefficients
__device__ __forceinline__ void hot_fields(const TetHot& H, const float x[3], float E[3], float B[3]) {
    E[0] = H.E0[0] + (H.W[1] * x[2] - H.W[2] * x[1]);
    E[1] = H.E0[1] + (H.W[2] * x[0] - H.W[0] * x[2]);
    E[2] = H.E0[2] + (H.W[0] * x[1] - H.W[1] * x[0]);
#pragma unroll
    for (int i = 0; i < 3; ++i) B[i] = H.B0[i] + H.beta * x[i];
}

// Record chunks (16 bytes each) every particle of the fast path reads up front: from chunk
// kIdChunks on (the gradients and field coefficients); the id chunks 0..kIdChunks-1 follow
// only where a deposit is issued.
#ifndef FP_HEAD_IDS
#define FP_HEAD_IDS 1
#endif
constexpr int kIdChunks = FP_HEAD_IDS ? 2 : 0;

// node ids and edge ids 0..3 of record c (chunks 0 and 1), from the shared window or global memory
__device__ __forceinline__ void ids_of(const TetHot* __restrict__ hot, const unsigned char* rec, int rec_lo,
                                       bool in_win, int c, TetHot& H) {
    if (kIdChunks == 0) return;
    const int4* r = in_win ? reinterpret_cast<const int4*>(rec + (c - rec_lo) * kRecStride)
                           : reinterpret_cast<const int4*>(hot + c);
    const int4 a = in_win ? r[0] : __ldg(r), b = in_win ? r[1] : __ldg(r + 1);
    H.node[0] = a.x, H.node[1] = a.y, H.node[2] = a.z, H.node[3] = a.w;
    H.edge[0] = b.x, H.edge[1] = b.y, H.edge[2] = b.z, H.edge[3] = b.w;
}

// Particle movers of the fast path.  move() takes the particle's offset x and velocity v and
// the fields at x, leaves the new velocity in v and the end offset in xb; commit() stores
// what the mover keeps besides the offset once the particle is known to stay in its tet.
//
// Boris (leapfrog): the velocity is stored at once, since the FP64 walk of a deferred
// particle recomputes its end point from it.
struct BorisMover {
    float h, dt;
    float* __restrict__ vel;
    int64_t n;
    __device__ __forceinline__ void move(int64_t p, const float x[3], float v[3], const float E[3],
                                         const float B[3], float xb[3]) {
        boris<float>(v, E, B, h);
        vel[p] = v[0];
        vel[n + p] = v[1];
        vel[2 * n + p] = v[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) xb[i] = step_pos(x[i], dt, v[i]);
    }
    __device__ __forceinline__ void history(int64_t) {}
    __device__ __forceinline__ void commit(int64_t) {}
};

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

// One step of the k-th order Adams-Bashforth method (k = order, 1..4) on dx/dt = v,
// dv/dt = a = (q/m)(E + v x B) (Sec. IV.B.2 names a fourth-order Adams mover; the start-up
// steps use orders 1..3).  hist holds the derivatives of the three previous steps as 18
// planar components of n particles: slot s has v at planes 6s..6s+2 and a at 6s+3..6s+5.
template <typename Real>
struct AdamsStep {
    Real* __restrict__ hist;
    int64_t n;
    int order;       // 1..4
    int slot_new;    // slot that takes f^n
    int slot[3];     // slots of f^{n-1}, f^{n-2}, f^{n-3}
    Real beta[4];    // coefficients of f^n, f^{n-1}, ...
    Real dt, qm;
};

// The history part of the Adams sums, which needs no fields and can be loaded early:
//   hx = beta_1 v^{n-1} (+ beta_2 v^{n-2} (+ beta_3 v^{n-3})),  ha likewise with a,
// zero at order 1.  The position sum is rounded operation by operation without contraction,
// so that the end point (which decides the walk) can be reproduced exactly by a CPU program.
template <typename Real>
__device__ __forceinline__ void adams_history(const AdamsStep<Real>& A, int64_t p, Real hx[3], Real ha[3]) {
#pragma unroll
    for (int i = 0; i < 3; ++i) hx[i] = ha[i] = (Real)0;
#pragma unroll
    for (int j = 1; j < 4; ++j) {
        if (j >= A.order) break;
        const int64_t base = (int64_t)6 * A.slot[j - 1] * A.n + p;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const Real t = mul_rn(A.beta[j], A.hist[base + i * A.n]);
            hx[i] = j == 1 ? t : add_rn(hx[i], t);
            ha[i] += A.beta[j] * A.hist[base + (3 + i) * A.n];
        }
    }
}

// a^n, v^{n+1} and the end offset x^{n+1} from the fields at x^n and the history part:
//   x^{n+1} = x^n + dt (beta_0 v^n + hx),  v^{n+1} = v^n + dt (beta_0 a^n + ha)
template <typename Real>
__device__ __forceinline__ void adams_update(const AdamsStep<Real>& A, const Real x[3], const Real v[3],
                                             const Real E[3], const Real B[3], const Real hx[3], const Real ha[3],
                                             Real a[3], Real v1[3], Real xb[3]) {
    Real c[3];
    cross<Real>(v, B, c);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        a[i] = A.qm * (E[i] + c[i]);
        xb[i] = add_rn(x[i], mul_rn(A.dt, add_rn(mul_rn(A.beta[0], v[i]), hx[i])));
        v1[i] = v[i] + A.dt * (A.beta[0] * a[i] + ha[i]);
    }
}

// stores v^{n+1} and f^n = (v^n, a^n) into the history slot that held f^{n-3}
template <typename Real>
__device__ __forceinline__ void adams_store(const AdamsStep<Real>& A, Real* __restrict__ vel, int64_t p,
                                            const Real v0[3], const Real a[3], const Real v1[3]) {
    const int64_t base = (int64_t)6 * A.slot_new * A.n + p;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        vel[i * A.n + p] = v1[i];
        A.hist[base + i * A.n] = v0[i];
        A.hist[base + (3 + i) * A.n] = a[i];
    }
}

// Adams (multistep): nothing is stored unless the particle stays in its tet; a deferred
// particle's whole step is redone by the walk kernel from the unchanged state.
struct AdamsMover32 {
    const AdamsStep<float>& A;
    float* __restrict__ vel;
    float v0[3], a[3], v1[3], hx[3], ha[3];
    // the history part, loaded before the particle's fields (its loads overlap the record's)
    __device__ __forceinline__ void history(int64_t p) { adams_history<float>(A, p, hx, ha); }
    __device__ __forceinline__ void move(int64_t, const float x[3], float v[3], const float E[3],
                                         const float B[3], float xb[3]) {
#pragma unroll
        for (int i = 0; i < 3; ++i) v0[i] = v[i];
        adams_update<float>(A, x, v0, E, B, hx, ha, a, v1, xb);
#pragma unroll
        for (int i = 0; i < 3; ++i) v[i] = v1[i];
    }
    __device__ __forceinline__ void commit(int64_t p) { adams_store<float>(A, vel, p, v0, a, v1); }
};

// Fast FP32 path: gather through the affine coefficients, Boris, and the end point's
// barycentric coordinates l^b = l^a + G dx.  If every l^b_k clears a margin larger
// than the FP32 rounding bound, the FP64 exit test would find no exit either, so the
// piece stays in the tet and is deposited here (warp-reduced).  Otherwise the
// particle index is queued for the FP64 walk (velocity already updated).
//
// fast_core is the per-particle arithmetic: it moves the particle (the mover stores what it
// keeps) and returns kFastStay with the end offset xb, the start barycentrics l and their
// change d over the step when the piece stays in the tet, kFastWalk when the FP64 walk has to
// decide, kFastNonFinite when the state or the push is not finite.  deposit_values forms the
// 10 deposit values from l and d: the 6 W1 edge values w (l_i d_j - l_j d_i) and the 4 W0
// node charges w (l_k + d_k) at the end point.
enum { kFastStay = 0, kFastWalk = 1, kFastNonFinite = 2 };

template <class Mover>
__device__ __forceinline__ int fast_core(const TetHot& H, const float x[3], float v[3], int64_t p, Mover& mv,
                                         float xb[3], float l[4], float d[4]) {
    l[1] = H.g[0] * x[0] + H.g[1] * x[1] + H.g[2] * x[2];
    l[2] = H.g[3] * x[0] + H.g[4] * x[1] + H.g[5] * x[2];
    l[3] = H.g[6] * x[0] + H.g[7] * x[1] + H.g[8] * x[2];
    l[0] = 1.f - l[1] - l[2] - l[3];
    float E[3], B[3];
    hot_fields(H, x, E, B);
    float dx[3];
    mv.move(p, x, v, E, B, xb);
    // 0 * a is 0 for finite a and NaN for NaN or Inf: one test covers the new state
    float nz = 0.f;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        nz = fmaf(0.f, v[i], nz);
        nz = fmaf(0.f, xb[i], nz);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) dx[i] = xb[i] - x[i];
    d[1] = H.g[0] * dx[0] + H.g[1] * dx[1] + H.g[2] * dx[2];
    d[2] = H.g[3] * dx[0] + H.g[4] * dx[1] + H.g[5] * dx[2];
    d[3] = H.g[6] * dx[0] + H.g[7] * dx[1] + H.g[8] * dx[2];
    d[0] = -(d[1] + d[2] + d[3]);
    // rounding bound of l^b in FP32 (with the FP32 copy of the gradients):
    // 1 + sum_k |g_k| (|x_k%3| + |dx_k%3|) <= 1 + (sum |g|) max_i (|x_i| + |dx_i|)
    const float xm = fmaxf(fmaxf(fabsf(x[0]) + fabsf(dx[0]), fabsf(x[1]) + fabsf(dx[1])),
                           fabsf(x[2]) + fabsf(dx[2]));
    const float margin = fmaf(H.gsum, xm, 1.f) * (1.f / 65536.f);
    float lbmin = l[0] + d[0];
#pragma unroll
    for (int k = 1; k < 4; ++k) lbmin = fminf(lbmin, l[k] + d[k]);
    // a non-finite state or push (NaN/Inf velocity, offset or field) removes the particle
    if (!finite_bits(nz)) return kFastNonFinite;
    if (!(lbmin >= margin)) return kFastWalk;
    return kFastStay;
}

__device__ __forceinline__ void deposit_values(float w, const float l[4], const float d[4], float agg[10],
                                               bool cc = false) {
    agg[0] = w * (l[0] * d[1] - l[1] * d[0]);
    agg[1] = w * (l[0] * d[2] - l[2] * d[0]);
    agg[2] = w * (l[0] * d[3] - l[3] * d[0]);
    agg[3] = w * (l[1] * d[2] - l[2] * d[1]);
    agg[4] = w * (l[1] * d[3] - l[3] * d[1]);
    agg[5] = w * (l[2] * d[3] - l[3] * d[2]);
#pragma unroll
    for (int k = 0; k < 4; ++k) agg[6 + k] = w * (cc ? d[k] : l[k] + d[k]);   // cc: the charge change
}

// One particle per lane; c < 0 means no particle.  All 32 lanes of the warp must call
// it (the deposit reduction is a warp collective).  Returns true when the particle has to
// go to the FP64 walk; the caller queues it.  Records of cells [rec_lo, rec_lo + rec_n)
// are read from the shared-memory window `rec` (records kRecStride bytes apart), the others
// from global memory.
template <class Mover, typename DG = float, typename DQ = DG>
__device__ __forceinline__ bool fast_particle(const TetHot* __restrict__ hot, const unsigned char* rec, int rec_lo,
                                              int rec_n, int c, const float x[3], float v[3], int64_t p, int64_t n,
                                              int32_t nt, Mover& mv, float w, int aggregate, int32_t* __restrict__ cell,
                                              float* __restrict__ off, DG* __restrict__ dG, DQ* __restrict__ Q,
                                              int32_t* __restrict__ status, bool cc = false) {
    const int lane = threadIdx.x & 31;
    if (c >= nt) {
        atomicOr(status, ST_INVAL);
        c = -1;
    }
    int key = -1;
    bool slow = false;
    float agg[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) agg[k] = 0.f;
    TetHot H;
    // the record's first 32 bytes (node ids, edge ids 0..3) are needed only where a deposit
    // is issued (the head lane of a run): they are loaded there (ids_of)
    const bool in_win = (unsigned)(c - rec_lo) < (unsigned)rec_n;
    if (c >= 0) {
        float4 t[8];
        const float4* r = in_win ? reinterpret_cast<const float4*>(rec + (c - rec_lo) * kRecStride)
                                 : reinterpret_cast<const float4*>(hot + c);
        t[0] = t[1] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int k = kIdChunks; k < 8; ++k) t[k] = in_win ? r[k] : __ldg(r + k);
        memcpy(&H, t, sizeof(TetHot));
        float xb[3], l[4], d[4];
        const int r3 = fast_core(H, x, v, p, mv, xb, l, d);
        if (r3 == kFastNonFinite) {
            // the particle is removed with nothing deposited, and the status word says so
            // (with cc, its start point's charge leaves Q where the start is finite)
            atomicOr(status, ST_NONFINITE);
            cell[p] = -1;
            if (cc && finite_bits(l[0]) && finite_bits(l[1]) && finite_bits(l[2]) && finite_bits(l[3])) {
                ids_of(hot, rec, rec_lo, in_win, c, H);
#pragma unroll
                for (int k = 0; k < 4; ++k) atomicAdd(Q + H.node[k], dep_cast<DQ>(-w * l[k]));
            }
        } else if (r3 == kFastStay) {
            deposit_values(w, l, d, agg, cc);
            off[p] = xb[0];
            off[n + p] = xb[1];
            off[2 * n + p] = xb[2];
            mv.commit(p);
            key = c;
            if (!aggregate) {
                ids_of(hot, rec, rec_lo, in_win, c, H);
#pragma unroll
                for (int k = 0; k < 6; ++k) atomicAdd(dG + H.edge[k], dep_cast<DG>(agg[k]));
#pragma unroll
                for (int k = 0; k < 4; ++k) atomicAdd(Q + H.node[k], dep_cast<DQ>(agg[6 + k]));
            }
        } else {
            slow = true;
        }
    }
    if (aggregate) {
        unsigned heads;
        int end;
        warp_run_reduce<float, 10>(key, agg, &heads, &end);
        if (((heads >> lane) & 1u) && key >= 0) {
            ids_of(hot, rec, rec_lo, in_win, c, H);
#pragma unroll
            for (int k = 0; k < 6; ++k) atomicAdd(dG + H.edge[k], dep_cast<DG>(agg[k]));
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(Q + H.node[k], dep_cast<DQ>(agg[6 + k]));
        }
    }
    return slow;
}

// appends the lanes with `slow` set to a queue (one atomic per warp on its counter)
template <typename Counter>
__device__ __forceinline__ void warp_enqueue(bool slow, int32_t value, int32_t* queue, Counter* count) {
    const int lane = threadIdx.x & 31;
    const unsigned sm = __ballot_sync(kFull, slow);
    if (!sm) return;
    int basei = 0;
    const int leader = __ffs(sm) - 1;
    if (lane == leader) basei = atomicAdd(count, __popc(sm));
    basei = __shfl_sync(kFull, basei, leader);
    if (slow) queue[basei + __popc(sm & ((1u << lane) - 1u))] = value;
}

#ifndef FP_FAST_MIN_BLOCKS
#define FP_FAST_MIN_BLOCKS 4
#endif
// Grid-stride variant: the particle state is loaded straight from global memory (the
// next particle's cell one iteration ahead).
template <typename DG, typename DQ>
__global__ void __launch_bounds__(256, FP_FAST_MIN_BLOCKS) k_push_fast32(
    const TetHot* __restrict__ hot, int32_t* __restrict__ cell, float* __restrict__ off,
    float* __restrict__ vel, int64_t n, int32_t nt, float h, float dt, double qw, int aggregate,
    DG* __restrict__ dG, DQ* __restrict__ Q, int32_t* __restrict__ slow_idx,
    int32_t* __restrict__ slow_count, int32_t* __restrict__ status, int cc) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float w = (float)qw;
    BorisMover bm{h, dt, vel, n};
    int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    int c_nx = base + lane < n ? __ldg(cell + base + lane) : -1;
    for (; base < n; base += stride) {
        const int64_t p = base + lane;
        const int c = p < n ? c_nx : -1;
        {
            const int64_t q = p + stride;
            c_nx = q < n ? __ldg(cell + q) : -1;
        }
        float x[3] = {0.f, 0.f, 0.f}, v[3] = {0.f, 0.f, 0.f};
        if (c >= 0 && c < nt) {
            x[0] = off[p], x[1] = off[n + p], x[2] = off[2 * n + p];
            v[0] = vel[p], v[1] = vel[n + p], v[2] = vel[2 * n + p];
        }
        const bool slow = fast_particle(hot, nullptr, 0, 0, c, x, v, p, n, nt, bm, w, aggregate, cell, off, dG, Q,
                                        status, cc != 0);
        warp_enqueue(slow, (int32_t)p, slow_idx, slow_count);   // one global atomic per warp
    }
}

// Persistent variant with the particle state and the tet records staged through shared
// memory by bulk asynchronous copies (TMA).  A block owns tiles blockIdx.x,
// blockIdx.x + gridDim.x, ... of kTmaTile consecutive particles:
//  - the seven state components (cell, off x/y/z, vel x/y/z) of its next tile are copied
//    while it pushes the current one (kTmaStages buffers);
//  - halfway through a tile, warp 0 copies the records of a window of kRecMax cells
//    around the median cell of the next tile (whose state has arrived by then), so a
//    particle of a cell-sorted tile reads its 128-byte record from shared memory instead
//    of waiting on L2 at the start of its dependency chain (record -> push -> deposit);
//    cells outside the window are read from global memory;
//  - the particles that need the FP64 walk are queued per tile in shared memory and
//    written out with one global atomic per tile.
// Needs n % 4 == 0 and 16-byte aligned cell/off/vel (every state copy then starts on a
// 16-byte boundary and moves a multiple of 16 bytes; records are 128-byte aligned); the
// launcher checks this and otherwise runs k_push_fast32.  Every wait on a copy is bounded
// (ST_TIMEOUT on expiry).
#ifndef FP_TMA_TILE
#define FP_TMA_TILE 512
#endif
constexpr int kTmaTile = FP_TMA_TILE;
constexpr int kTmaThreads = 256;
constexpr int kTmaSlot = kTmaTile * 4;       // bytes per component per stage
constexpr int kTmaStageBytes = 7 * kTmaSlot;
#ifndef FP_TMA_STAGES
#define FP_TMA_STAGES 2
#endif
#ifndef FP_REC_MAX
#define FP_REC_MAX 72
#endif
constexpr int kTmaStages = FP_TMA_STAGES;
constexpr int kRecMax = FP_REC_MAX;           // records per window
constexpr int kRecBytes = kRecMax * kRecStride;
constexpr int kTmaSmem = kTmaStages * kTmaStageBytes + 2 * kRecBytes;
constexpr uint64_t kTmaWaitNs = 2000000000ull;  // 2 s
static_assert(kTmaSlot % 16 == 0 && kTmaTile % kTmaThreads == 0, "tile shape");
static_assert(kTmaStageBytes % 16 == 0 && kRecStride % 16 == 0, "bulk copy destinations 16-byte aligned");

// copies of tile t into stage s (one thread)
__device__ __forceinline__ void tma_issue(unsigned char* stage, uint64_t* bar, int t, const int32_t* cell,
                                          const float* off, const float* vel, int64_t n) {
    const int64_t p0 = (int64_t)t * kTmaTile;
    const uint32_t bytes = 4u * (uint32_t)min((int64_t)kTmaTile, n - p0);
    mbar_arrive_expect_tx(bar, 7u * bytes);
    bulk_g2s(stage, cell + p0, bytes, bar);
#pragma unroll
    for (int k = 0; k < 3; ++k) bulk_g2s(stage + (1 + k) * kTmaSlot, off + k * n + p0, bytes, bar);
#pragma unroll
    for (int k = 0; k < 3; ++k) bulk_g2s(stage + (4 + k) * kTmaSlot, vel + k * n + p0, bytes, bar);
}

__global__ void __launch_bounds__(kTmaThreads, FP_FAST_MIN_BLOCKS) k_push_tma32(
    const TetHot* __restrict__ hot, int32_t* __restrict__ cell, float* __restrict__ off,
    float* __restrict__ vel, int64_t n, int32_t nt, float h, float dt, double qw, int aggregate,
    float* __restrict__ dG, float* __restrict__ Q, int32_t* __restrict__ slow_idx,
    int32_t* __restrict__ slow_count, int32_t* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t bars[kTmaStages];
    __shared__ __align__(8) uint64_t rbars[2];
    // record windows of the current and the next tile: first cell, count (0: none), and the
    // number of copies issued into each window so far (its barrier's phase)
    __shared__ int rec_lo[2], rec_n[2], rec_issued[2];
    // slow particles of a tile, collected in shared memory and written out with one global
    // atomic per tile; two buffers so tile t's queue is copied out during tile t + 1
    __shared__ int32_t tq[2][kTmaTile];
    __shared__ int tq_n[2], tq_base[2];
    unsigned char* recs = smem + kTmaStages * kTmaStageBytes;
    const int tid = threadIdx.x;
    const float w = (float)qw;
    BorisMover bm{h, dt, vel, n};
    const int ntiles = (int)((n + kTmaTile - 1) / kTmaTile);
    const int G = gridDim.x;
    if (tid == 0) {
        for (int s = 0; s < kTmaStages; ++s) mbar_init(&bars[s], 1);
        mbar_init(&rbars[0], 1);
        mbar_init(&rbars[1], 1);
        mbar_fence_init();
        tq_n[0] = tq_n[1] = 0;
        rec_n[0] = rec_n[1] = 0;
        rec_lo[0] = rec_lo[1] = 0;
        rec_issued[0] = rec_issued[1] = 0;
    }
    __syncthreads();
    int issued = 0;  // tiles issued by this block (kept by thread 0)
    if (tid == 0)
        for (int s = 0; s < kTmaStages && (int)blockIdx.x + s * G < ntiles; ++s, ++issued)
            tma_issue(smem + s * kTmaStageBytes, &bars[s], blockIdx.x + s * G, cell, off, vel, n);
    int it = 0;
    bool failed = false;
    for (int t = blockIdx.x; t < ntiles; t += G, ++it) {
        const int s = it % kTmaStages, qb = it & 1;
        bool ok = mbar_wait_bounded(&bars[s], (uint32_t)((it / kTmaStages) & 1), kTmaWaitNs);
        if (ok && rec_n[qb] > 0)
            ok = mbar_wait_bounded(&rbars[qb], (uint32_t)((rec_issued[qb] - 1) & 1), kTmaWaitNs);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        if (it > 0)  // the previous tile's queue (its global slots were reserved by thread 0)
            for (int i = tid; i < tq_n[qb ^ 1]; i += kTmaThreads) slow_idx[tq_base[qb ^ 1] + i] = tq[qb ^ 1][i];
        const int64_t p0 = (int64_t)t * kTmaTile;
        const int cnt = (int)min((int64_t)kTmaTile, n - p0);
        const unsigned char* st = smem + s * kTmaStageBytes;
        const unsigned char* rec = recs + qb * kRecBytes;
        const int rlo = rec_lo[qb], rn = rec_n[qb];
#pragma unroll 1
        for (int q = 0; q < kTmaTile / kTmaThreads; ++q) {
            if (q == kTmaTile / kTmaThreads / 2 && tid < 32) {
                // halfway: warp 0 copies the record window of the next tile, if its state is
                // already here (window qb ^ 1 was last read by tile it - 1, finished before this
                // tile began); lane 0 picks the window, every lane copies some of its records
                int nn = 0, lo = 0;
                if (tid == 0) {
                    const int tn = t + G;
                    if (tn < ntiles && it + 1 < issued &&
                        mbar_try_wait(&bars[(it + 1) % kTmaStages], (uint32_t)(((it + 1) / kTmaStages) & 1))) {
                        const unsigned char* sn = smem + ((it + 1) % kTmaStages) * kTmaStageBytes;
                        const int cn = (int)min((int64_t)kTmaTile, n - (int64_t)tn * kTmaTile);
                        const int cm = reinterpret_cast<const int32_t*>(sn)[cn / 2];
                        if (cm >= 0 && cm < nt) {
                            nn = min(kRecMax, nt);
                            lo = min(max(cm - kRecMax / 2, 0), nt - nn);
                        }
                    }
                    rec_lo[qb ^ 1] = lo;
                    rec_n[qb ^ 1] = nn;
                    if (nn > 0) {
                        mbar_arrive_expect_tx(&rbars[qb ^ 1], (uint32_t)nn * (uint32_t)sizeof(TetHot));
                        ++rec_issued[qb ^ 1];
                    }
                }
                nn = __shfl_sync(kFull, nn, 0);
                lo = __shfl_sync(kFull, lo, 0);
                if (nn > 0) {
                    fence_proxy_async_smem();
                    for (int k = tid; k < nn; k += 32)
                        bulk_g2s(recs + (qb ^ 1) * kRecBytes + k * kRecStride, hot + lo + k,
                                 (uint32_t)sizeof(TetHot), &rbars[qb ^ 1]);
                }
            }
            const int j = q * kTmaThreads + tid;
            int c = -1;
            float x[3] = {0.f, 0.f, 0.f}, v[3] = {0.f, 0.f, 0.f};
            if (j < cnt) {
                c = reinterpret_cast<const int32_t*>(st)[j];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    x[k] = reinterpret_cast<const float*>(st + (1 + k) * kTmaSlot)[j];
                    v[k] = reinterpret_cast<const float*>(st + (4 + k) * kTmaSlot)[j];
                }
            }
            const bool slow = fast_particle(hot, rec, rlo, rn, c, x, v, p0 + j, n, nt, bm, w, aggregate, cell, off, dG,
                                            Q, status);
            warp_enqueue(slow, (int32_t)(p0 + j), tq[qb], &tq_n[qb]);
        }
        __syncthreads();  // every thread is done with stage s, record window qb and tile queue qb ^ 1
        if (tid == 0) {
            tq_n[qb ^ 1] = 0;
            tq_base[qb] = tq_n[qb] ? atomicAdd(slow_count, tq_n[qb]) : 0;
            rec_n[qb] = 0;  // window qb is free for tile it + 2 (set again halfway through tile it + 1)
            if (t + kTmaStages * G < ntiles) {
                fence_proxy_async_smem();
                tma_issue(smem + s * kTmaStageBytes, &bars[s], t + kTmaStages * G, cell, off, vel, n);
                ++issued;
            }
        }
    }
    if (failed) {
        if (tid == 0) {
            atomicOr(status, ST_TIMEOUT);
            // wait (bounded) for the copies still in flight before leaving
            for (int j = it; j < issued; ++j)
                mbar_wait_bounded(&bars[j % kTmaStages], (uint32_t)((j / kTmaStages) & 1), kTmaWaitNs);
            for (int b = 0; b < 2; ++b)
                if (rec_issued[b] > 0) mbar_wait_bounded(&rbars[b], (uint32_t)((rec_issued[b] - 1) & 1), kTmaWaitNs);
        }
        return;
    }
    __syncthreads();
    if (it > 0) {  // the last tile's queue
        const int qb = (it - 1) & 1;
        for (int i = tid; i < tq_n[qb]; i += kTmaThreads) slow_idx[tq_base[qb] + i] = tq[qb][i];
    }
}

// Warp-specialised variant of the staged push: one producer warp and kWsConsumers consumer
// warps per block, synchronised only through mbarriers (no block-wide barrier after set-up),
// so a consumer warp never waits for the slowest warp of its block.  Per stage s (one tile of
// kWsTile particles in flight per stage):
//   full[s]  completes when the tile's seven state components have arrived (bulk copies);
//   recb[s]  completes when the tile's record window has arrived (or at once: no window);
//   empty[s] completes when every consumer warp is done with the tile (stage, window and
//            queue of stage s may then be reused).
// The producer (lane 0 of the last warp) issues the state copies, picks and copies each
// tile's record window as soon as the tile's state is in shared memory, and after empty[s]
// writes the tile's queue of slow particles out with one global atomic, then refills the
// stage.  Same per-particle work as k_push_tma32; same alignment requirements.  Every wait
// is bounded (ST_TIMEOUT on expiry; a warp that gives up leaves its loop, so the others time
// out in turn rather than hang).
#ifndef FP_WS_CONSUMERS
#define FP_WS_CONSUMERS 7
#endif
#ifndef FP_WS_BATCHES
#define FP_WS_BATCHES 2
#endif
#ifndef FP_WS_STAGES
#define FP_WS_STAGES 2
#endif
constexpr int kWsConsumers = FP_WS_CONSUMERS;
constexpr int kWsBatches = FP_WS_BATCHES;            // 32-particle batches per consumer warp per tile
constexpr int kWsThreads = 32 * (kWsConsumers + 1);
constexpr int kWsTile = 32 * kWsBatches * kWsConsumers;
constexpr int kWsStages = FP_WS_STAGES;
constexpr int kWsSlot = kWsTile * 4;
constexpr int kWsStageBytes = 7 * kWsSlot;
constexpr int kWsRecMax = kWsTile / 7 > 64 ? kWsTile / 7 : 64;   // about 10 particles per cell
constexpr int kWsRecBytes = kWsRecMax * kRecStride;
constexpr int kWsSmem = kWsStages * (kWsStageBytes + kWsRecBytes);
static_assert(kWsSlot % 16 == 0 && kWsStageBytes % 16 == 0 && kWsRecBytes % 16 == 0, "bulk copy alignment");

__device__ __forceinline__ void ws_issue(unsigned char* stage, uint64_t* bar, int t, const int32_t* cell,
                                         const float* off, const float* vel, int64_t n) {
    const int64_t p0 = (int64_t)t * kWsTile;
    const uint32_t bytes = 4u * (uint32_t)min((int64_t)kWsTile, n - p0);
    mbar_arrive_expect_tx(bar, 7u * bytes);
    bulk_g2s(stage, cell + p0, bytes, bar);
#pragma unroll
    for (int k = 0; k < 3; ++k) bulk_g2s(stage + (1 + k) * kWsSlot, off + k * n + p0, bytes, bar);
#pragma unroll
    for (int k = 0; k < 3; ++k) bulk_g2s(stage + (4 + k) * kWsSlot, vel + k * n + p0, bytes, bar);
}

// The consumers' particle mover: Boris (the step's leapfrog push) or the Adams mover, whose
// history part is loaded as soon as a particle's state is read from the stage.
struct BorisArgs {
    float h, dt;
};
__device__ __forceinline__ BorisMover make_mover(const BorisArgs& a, float* vel, int64_t n) {
    return BorisMover{a.h, a.dt, vel, n};
}
__device__ __forceinline__ AdamsMover32 make_mover(const AdamsStep<float>& a, float* vel, int64_t) {
    return AdamsMover32{a, vel};
}
#ifndef FP_ADAMS_WS_MIN_BLOCKS
#define FP_ADAMS_WS_MIN_BLOCKS 3
#endif
template <class MA>
struct WsMinBlocks {
    static constexpr int value = FP_FAST_MIN_BLOCKS;
};
template <>
struct WsMinBlocks<AdamsStep<float>> {
    static constexpr int value = FP_ADAMS_WS_MIN_BLOCKS;   // the Adams sums need more registers
};

template <class MA>
__global__ void __launch_bounds__(kWsThreads, WsMinBlocks<MA>::value) k_push_ws32(
    const TetHot* __restrict__ hot, int32_t* __restrict__ cell, float* __restrict__ off,
    float* __restrict__ vel, int64_t n, int32_t nt, MA margs, double qw, int aggregate,
    float* __restrict__ dG, float* __restrict__ Q, int32_t* __restrict__ slow_idx,
    int32_t* __restrict__ slow_count, int32_t* __restrict__ status) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kWsStages], empty[kWsStages], recb[kWsStages];
    __shared__ int rec_lo[kWsStages], rec_n[kWsStages];
    __shared__ int32_t queue[kWsStages][kWsTile];
    __shared__ int qn[kWsStages];
    unsigned char* recs = smem + kWsStages * kWsStageBytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (int)((n + kWsTile - 1) / kWsTile);
    const int G = gridDim.x;
    const int mine = ntiles > (int)blockIdx.x ? (ntiles - (int)blockIdx.x + G - 1) / G : 0;   // tiles of this block
    if (tid == 0) {
        for (int s = 0; s < kWsStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kWsConsumers);
            mbar_init(&recb[s], 1);
            qn[s] = 0;
        }
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == kWsConsumers) {
        // ---------------- producer
        if (lane != 0) return;
        int issued = 0, recs_issued = 0;
        bool failed = false;
        for (int k = 0; k < kWsStages && k < mine; ++k, ++issued)
            ws_issue(smem + k * kWsStageBytes, &full[k], blockIdx.x + k * G, cell, off, vel, n);
        // flushes the queue of the k-th tile after its consumers are done, then refills its stage
        auto retire = [&](int k) -> bool {
            const int sk = k % kWsStages;
            if (!mbar_wait_bounded(&empty[sk], (uint32_t)((k / kWsStages) & 1), kTmaWaitNs)) return false;
            const int m = qn[sk];
            if (m > 0) {
                const int base = atomicAdd(slow_count, m);
                for (int i = 0; i < m; ++i) slow_idx[base + i] = queue[sk][i];
            }
            qn[sk] = 0;
            if (k + kWsStages < mine) {
                fence_proxy_async_smem();
                ws_issue(smem + sk * kWsStageBytes, &full[sk], blockIdx.x + (k + kWsStages) * G, cell, off, vel, n);
                ++issued;
            }
            return true;
        };
        for (int it = 0; it < mine && !failed; ++it) {
            const int sk = it % kWsStages;
            // the record window of tile it, as soon as its state is here
            if (!mbar_wait_bounded(&full[sk], (uint32_t)((it / kWsStages) & 1), kTmaWaitNs)) {
                failed = true;
                break;
            }
            const int64_t p0 = (int64_t)(blockIdx.x + it * G) * kWsTile;
            const int cn = (int)min((int64_t)kWsTile, n - p0);
            const int cm = reinterpret_cast<const int32_t*>(smem + sk * kWsStageBytes)[cn / 2];
            int nn = 0, lo = 0;
            if (cm >= 0 && cm < nt) {
                nn = min(kWsRecMax, nt);
                lo = min(max(cm - kWsRecMax / 2, 0), nt - nn);
            }
            rec_lo[sk] = lo;
            rec_n[sk] = nn;
            if (nn > 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&recb[sk], (uint32_t)nn * (uint32_t)sizeof(TetHot));
                for (int k = 0; k < nn; ++k)
                    bulk_g2s(recs + sk * kWsRecBytes + k * kRecStride, hot + lo + k, (uint32_t)sizeof(TetHot),
                             &recb[sk]);
            } else {
                mbar_arrive(&recb[sk]);
            }
            ++recs_issued;
            // the tile before it: retire and refill its stage
            if (it >= 1 && !retire(it - 1)) failed = true;
        }
        if (!failed && mine > 0 && !retire(mine - 1)) failed = true;
        if (failed) {
            atomicOr(status, ST_TIMEOUT);
            // wait (bounded) for the copies still in flight before leaving
            for (int k = 0; k < issued; ++k)
                mbar_wait_bounded(&full[k % kWsStages], (uint32_t)((k / kWsStages) & 1), kTmaWaitNs);
            for (int k = 0; k < recs_issued; ++k)
                mbar_wait_bounded(&recb[k % kWsStages], (uint32_t)((k / kWsStages) & 1), kTmaWaitNs);
        }
        return;
    }
    // ---------------- consumers
    const float w = (float)qw;
    auto mv = make_mover(margs, vel, n);
    for (int it = 0; it < mine; ++it) {
        const int sk = it % kWsStages;
        const uint32_t par = (uint32_t)((it / kWsStages) & 1);
        if (!mbar_wait_bounded(&full[sk], par, kTmaWaitNs) || !mbar_wait_bounded(&recb[sk], par, kTmaWaitNs)) {
            if (lane == 0) atomicOr(status, ST_TIMEOUT);
            return;
        }
        const int rlo = rec_lo[sk], rn = rec_n[sk];
        const unsigned char* st = smem + sk * kWsStageBytes;
        const unsigned char* rec = recs + sk * kWsRecBytes;
        const int64_t p0 = (int64_t)(blockIdx.x + it * G) * kWsTile;
        const int cnt = (int)min((int64_t)kWsTile, n - p0);
#pragma unroll 1
        for (int q = 0; q < kWsBatches; ++q) {
            const int j = 32 * (warp + q * kWsConsumers) + lane;
            int c = -1;
            float x[3] = {0.f, 0.f, 0.f}, v[3] = {0.f, 0.f, 0.f};
            if (j < cnt) {
                c = reinterpret_cast<const int32_t*>(st)[j];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    x[k] = reinterpret_cast<const float*>(st + (1 + k) * kWsSlot)[j];
                    v[k] = reinterpret_cast<const float*>(st + (4 + k) * kWsSlot)[j];
                }
                if (c >= 0 && c < nt) mv.history(p0 + j);
            }
            const bool slow = fast_particle(hot, rec, rlo, rn, c, x, v, p0 + j, n, nt, mv, w, aggregate, cell, off, dG,
                                            Q, status);
            warp_enqueue(slow, (int32_t)(p0 + j), queue[sk], &qn[sk]);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[sk]);
    }
}

// ------------------------------------------------------------------ run-summing push
// Boris variant of k_push_ws32 in which each consumer lane takes kRunK consecutive particles
// of the tile (lane l of consumer warp w: tile positions (32 w + l) kRunK + i, i < kRunK)
// instead of one particle in 32.  In cell-sorted order consecutive particles mostly share a
// tet, so a lane sums its deposit values in registers, re-reads the tet's record only where
// the tet changes, and issues the 10 atomics of a run once; the warp joins the runs that
// cross lane boundaries once per chunk (lane l+1's first run into lane l's last, then the
// runs of equal tets over consecutive lanes), not once per particle.  The deposits are the
// same sums, grouped differently (FP32 atomics: the order of addition is not fixed anyway).
// kRunK is odd, so the lanes' strided shared-memory accesses hit 32 distinct banks.  The new
// offsets and velocities are written back into the staged tile, which the producer copies
// out with bulk copies after the consumers are done.  Stage layout, barriers, bounded waits
// and the queue of deferred particles are those of k_push_ws32.
#ifndef FP_RUN_K
#define FP_RUN_K 5
#endif
#ifndef FP_RUN_CONSUMERS
#define FP_RUN_CONSUMERS 3
#endif
#ifndef FP_RUN_REC
#define FP_RUN_REC 64
#endif
#ifndef FP_RUN_MIN_BLOCKS
#define FP_RUN_MIN_BLOCKS 4
#endif
#ifndef FP_RUN_STAGES
#define FP_RUN_STAGES 2
#endif
constexpr int kRunK = FP_RUN_K;
static_assert(kRunK % 2 == 1, "an odd chunk keeps the strided shared-memory accesses free of bank conflicts");
constexpr int kRunConsumers = FP_RUN_CONSUMERS;
constexpr int kRunThreads = 32 * (kRunConsumers + 1);
constexpr int kRunTile = 32 * kRunK * kRunConsumers;
constexpr int kRunStages = FP_RUN_STAGES;
constexpr int kRunSlot = kRunTile * 4;
constexpr int kRunStageBytes = 7 * kRunSlot;
constexpr int kRunRecMax = FP_RUN_REC;
constexpr int kRunRecBytes = kRunRecMax * kRecStride;
constexpr int kRunSmem = kRunStages * (kRunStageBytes + kRunRecBytes);
static_assert(kRunSlot % 16 == 0 && kRunStageBytes % 16 == 0 && kRunRecBytes % 16 == 0, "bulk copy alignment");

// the 10 atomics of one run, its sums a times the weight w: node ids and edge ids from
// record c (shared window or global)
template <typename DG, typename DQ>
__device__ __forceinline__ void run_flush(const TetHot* __restrict__ hot, const unsigned char* rec, int rec_lo,
                                          int rec_n, int c, float w, const float a[10], DG* __restrict__ dG,
                                          DQ* __restrict__ Q) {
    int4 nd, e03, e45;
    if ((unsigned)(c - rec_lo) < (unsigned)rec_n) {
        const int4* r = reinterpret_cast<const int4*>(rec + (c - rec_lo) * kRecStride);
        nd = r[0];
        e03 = r[1];
        e45 = r[2];
    } else {
        const int4* r = reinterpret_cast<const int4*>(hot + c);
        nd = __ldg(r);
        e03 = __ldg(r + 1);
        e45 = __ldg(r + 2);
    }
    // Here the conversion into a double array is the hardware one: the run kernel issues few
    // of them (once per run), has FP64 pipe to spare, and the integer form's extra instructions
    // cost it 4% (2.06 against 1.99 ms for both 96^3 species); the walk, FP64-bound, uses dep_cast.
    atomicAdd(dG + e03.x, (DG)(w * a[0]));
    atomicAdd(dG + e03.y, (DG)(w * a[1]));
    atomicAdd(dG + e03.z, (DG)(w * a[2]));
    atomicAdd(dG + e03.w, (DG)(w * a[3]));
    atomicAdd(dG + e45.x, (DG)(w * a[4]));
    atomicAdd(dG + e45.y, (DG)(w * a[5]));
    atomicAdd(Q + nd.x, (DQ)(w * a[6]));
    atomicAdd(Q + nd.y, (DQ)(w * a[7]));
    atomicAdd(Q + nd.z, (DQ)(w * a[8]));
    atomicAdd(Q + nd.w, (DQ)(w * a[9]));
}

// a += the 10 deposit values of a piece without the weight (l_i d_j - l_j d_i, and l_k + d_k,
// or d_k for the charge change)
__device__ __forceinline__ void run_add(float a[10], const float l[4], const float d[4], bool cc) {
    a[0] = fmaf(-l[1], d[0], fmaf(l[0], d[1], a[0]));
    a[1] = fmaf(-l[2], d[0], fmaf(l[0], d[2], a[1]));
    a[2] = fmaf(-l[3], d[0], fmaf(l[0], d[3], a[2]));
    a[3] = fmaf(-l[2], d[1], fmaf(l[1], d[2], a[3]));
    a[4] = fmaf(-l[3], d[1], fmaf(l[1], d[3], a[4]));
    a[5] = fmaf(-l[3], d[2], fmaf(l[2], d[3], a[5]));
#pragma unroll
    for (int k = 0; k < 4; ++k) a[6 + k] += cc ? d[k] : l[k] + d[k];
}

// Boris with the new velocity stored into the staged tile (position j of its planes)
struct BorisStaged {
    float h, dt;
    float* v0;
    float* v1;
    float* v2;
    __device__ __forceinline__ void move(int64_t j, const float x[3], float v[3], const float E[3],
                                         const float B[3], float xb[3]) {
        boris<float>(v, E, B, h);
        v0[j] = v[0];
        v1[j] = v[1];
        v2[j] = v[2];
#pragma unroll
        for (int i = 0; i < 3; ++i) xb[i] = step_pos(x[i], dt, v[i]);
    }
};

template <int Tile>
__device__ __forceinline__ void stage_issue(unsigned char* stage, uint64_t* bar, int t, const int32_t* cell,
                                            const float* off, const float* vel, int64_t n) {
    constexpr int kSlot = Tile * 4;
    const int64_t p0 = (int64_t)t * Tile;
    const uint32_t bytes = 4u * (uint32_t)min((int64_t)Tile, n - p0);
    mbar_arrive_expect_tx(bar, 7u * bytes);
    bulk_g2s(stage, cell + p0, bytes, bar);
#pragma unroll
    for (int k = 0; k < 3; ++k) bulk_g2s(stage + (1 + k) * kSlot, off + k * n + p0, bytes, bar);
#pragma unroll
    for (int k = 0; k < 3; ++k) bulk_g2s(stage + (4 + k) * kSlot, vel + k * n + p0, bytes, bar);
}

template <typename DG, typename DQ>
__global__ void __launch_bounds__(kRunThreads, FP_RUN_MIN_BLOCKS) k_push_run32(
    const TetHot* __restrict__ hot, int32_t* __restrict__ cell, float* __restrict__ off, float* __restrict__ vel,
    int64_t n, int32_t nt, float h, float dt, float w, int aggregate, DG* __restrict__ dG,
    DQ* __restrict__ Q, int32_t* __restrict__ slow_idx, int32_t* __restrict__ slow_count,
    int32_t* __restrict__ status, int cc_) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kRunStages], empty[kRunStages], recb[kRunStages];
    __shared__ int rec_lo[kRunStages], rec_n[kRunStages];
    __shared__ int32_t queue[kRunStages][kRunTile];
    __shared__ int qn[kRunStages];
    unsigned char* recs = smem + kRunStages * kRunStageBytes;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ntiles = (int)((n + kRunTile - 1) / kRunTile);
    const int G = gridDim.x;
    const int mine = ntiles > (int)blockIdx.x ? (ntiles - (int)blockIdx.x + G - 1) / G : 0;   // tiles of this block
    if (tid == 0) {
        for (int s = 0; s < kRunStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], kRunConsumers);
            mbar_init(&recb[s], 1);
            qn[s] = 0;
        }
        mbar_fence_init();
    }
    __syncthreads();
    if (warp == kRunConsumers) {
        // ---------------- producer
        if (lane != 0) return;
        int issued = 0, recs_issued = 0;
        bool failed = false;
        for (int k = 0; k < kRunStages && k < mine; ++k, ++issued)
            stage_issue<kRunTile>(smem + k * kRunStageBytes, &full[k], blockIdx.x + k * G, cell, off, vel, n);
        // after the consumers of tile k are done: its new offsets and velocities out, its queue
        // flushed, its stage refilled once the copies out have read it
        auto retire = [&](int k) -> bool {
            const int sk = k % kRunStages;
            if (!mbar_wait_bounded(&empty[sk], (uint32_t)((k / kRunStages) & 1), kTmaWaitNs)) return false;
            unsigned char* stg = smem + sk * kRunStageBytes;
            const int64_t p0 = (int64_t)(blockIdx.x + k * G) * kRunTile;
            const uint32_t bytes = 4u * (uint32_t)min((int64_t)kRunTile, n - p0);
#pragma unroll
            for (int c = 0; c < 3; ++c) bulk_s2g(off + c * n + p0, stg + (1 + c) * kRunSlot, bytes);
#pragma unroll
            for (int c = 0; c < 3; ++c) bulk_s2g(vel + c * n + p0, stg + (4 + c) * kRunSlot, bytes);
            bulk_commit();
            const int m = qn[sk];
            if (m > 0) {
                const int base = atomicAdd(slow_count, m);
                for (int i = 0; i < m; ++i) slow_idx[base + i] = queue[sk][i];
            }
            qn[sk] = 0;
            if (k + kRunStages < mine) {
                bulk_wait_read_all();
                fence_proxy_async_smem();
                stage_issue<kRunTile>(stg, &full[sk], blockIdx.x + (k + kRunStages) * G, cell, off, vel, n);
                ++issued;
            }
            return true;
        };
        for (int it = 0; it < mine && !failed; ++it) {
            const int sk = it % kRunStages;
            if (!mbar_wait_bounded(&full[sk], (uint32_t)((it / kRunStages) & 1), kTmaWaitNs)) {
                failed = true;
                break;
            }
            // record window: the tile's tets from first to last when they fit (cell-sorted
            // tiles), else kRunRecMax tets around the middle particle's
            const int64_t p0 = (int64_t)(blockIdx.x + it * G) * kRunTile;
            const int cn = (int)min((int64_t)kRunTile, n - p0);
            const int32_t* sc = reinterpret_cast<const int32_t*>(smem + sk * kRunStageBytes);
            const int c0 = sc[0], c1 = sc[cn - 1], cm = sc[cn / 2];
            int nn = 0, lo = 0;
            if (c0 >= 0 && c1 < nt && c0 <= c1 && c1 - c0 < kRunRecMax) {
                lo = c0;
                nn = c1 - c0 + 1;
            } else if (cm >= 0 && cm < nt) {
                nn = min(kRunRecMax, nt);
                lo = min(max(cm - kRunRecMax / 2, 0), nt - nn);
            }
            rec_lo[sk] = lo;
            rec_n[sk] = nn;
            if (nn > 0) {
                fence_proxy_async_smem();
                mbar_arrive_expect_tx(&recb[sk], (uint32_t)nn * (uint32_t)sizeof(TetHot));
                for (int k = 0; k < nn; ++k)
                    bulk_g2s(recs + sk * kRunRecBytes + k * kRecStride, hot + lo + k, (uint32_t)sizeof(TetHot),
                             &recb[sk]);
            } else {
                mbar_arrive(&recb[sk]);
            }
            ++recs_issued;
            if (it >= 1 && !retire(it - 1)) failed = true;
        }
        if (!failed && mine > 0 && !retire(mine - 1)) failed = true;
        if (failed) {
            atomicOr(status, ST_TIMEOUT);
            // wait (bounded) for the copies still in flight before leaving
            for (int k = 0; k < issued; ++k)
                mbar_wait_bounded(&full[k % kRunStages], (uint32_t)((k / kRunStages) & 1), kTmaWaitNs);
            for (int k = 0; k < recs_issued; ++k)
                mbar_wait_bounded(&recb[k % kRunStages], (uint32_t)((k / kRunStages) & 1), kTmaWaitNs);
        }
        bulk_wait_all();
        return;
    }
    // ---------------- consumers
    const int jb = (warp * 32 + lane) * kRunK;
    const bool cc = cc_ != 0;   // Q takes the charge change over the step (the end's minus the start's)
    for (int it = 0; it < mine; ++it) {
        const int sk = it % kRunStages;
        const uint32_t par = (uint32_t)((it / kRunStages) & 1);
        if (!mbar_wait_bounded(&full[sk], par, kTmaWaitNs) || !mbar_wait_bounded(&recb[sk], par, kTmaWaitNs)) {
            if (lane == 0) atomicOr(status, ST_TIMEOUT);
            return;
        }
        const int rlo = rec_lo[sk], rn = rec_n[sk];
        unsigned char* st = smem + sk * kRunStageBytes;
        const unsigned char* rec = recs + sk * kRunRecBytes;
        const int32_t* sc = reinterpret_cast<const int32_t*>(st);
        float* sx[3];
        float* sv[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sx[k] = reinterpret_cast<float*>(st + (1 + k) * kRunSlot);
            sv[k] = reinterpret_cast<float*>(st + (4 + k) * kRunSlot);
        }
        BorisStaged mv{h, dt, sv[0], sv[1], sv[2]};
        const int64_t p0 = (int64_t)(blockIdx.x + it * G) * kRunTile;
        const int cnt = (int)min((int64_t)kRunTile, n - p0);
        // the run being summed (tet cur; live once a particle of it stayed in its tet), the
        // lane's first run once it has ended (tet hcell), and the tet whose record is in H;
        // sums without the weight w, which the flush applies
        int cur = -1, hcell = -1, hc = -1;
        bool first = true, live = false;
        unsigned slow_bits = 0u;   // bit i: the lane's particle i goes to the FP64 walk
        float acc[10], head[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) acc[k] = head[k] = 0.f;
        TetHot H;
#pragma unroll 1
        for (int i = 0; i < kRunK; ++i) {
            const int j = jb + i;
            int c = -1;
            float x[3] = {0.f, 0.f, 0.f}, v[3] = {0.f, 0.f, 0.f};
            if (j < cnt) {
                c = sc[j];
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    x[k] = sx[k][j];
                    v[k] = sv[k][j];
                }
            }
            if (c >= nt) {
                atomicOr(status, ST_INVAL);
                c = -1;
            }
            if (c >= 0) {
                if (c != hc) {
                    // gradients and field coefficients (record chunks 2..7); the ids are read
                    // where a run is flushed
                    float4 t[8];
                    t[0] = t[1] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if ((unsigned)(c - rlo) < (unsigned)rn) {
                        const float4* r = reinterpret_cast<const float4*>(rec + (c - rlo) * kRecStride);
#pragma unroll
                        for (int k = 2; k < 8; ++k) t[k] = r[k];
                    } else {
                        const float4* r = reinterpret_cast<const float4*>(hot + c);
#pragma unroll
                        for (int k = 2; k < 8; ++k) t[k] = __ldg(r + k);
                    }
                    memcpy(&H, t, sizeof(TetHot));
                    hc = c;
                }
                if (aggregate && c != cur) {
                    // a new run: the previous one is kept (the lane's first) or flushed
                    if (live) {
                        if (first) {
#pragma unroll
                            for (int k = 0; k < 10; ++k) head[k] = acc[k];
                            hcell = cur;
                        } else {
                            run_flush(hot, rec, rlo, rn, cur, w, acc, dG, Q);
                        }
                    }
                    if (cur >= 0) first = false;
                    cur = c;
                    live = false;
#pragma unroll
                    for (int k = 0; k < 10; ++k) acc[k] = 0.f;
                }
                float xb[3], l[4], d[4];
                const int r3 = fast_core(H, x, v, j, mv, xb, l, d);
                if (r3 == kFastNonFinite) {
                    atomicOr(status, ST_NONFINITE);
                    cell[p0 + j] = -1;
                    if (cc && finite_bits(l[0]) && finite_bits(l[1]) && finite_bits(l[2]) && finite_bits(l[3])) {
                        // the removed particle's start charge leaves Q
                        float a[10];
#pragma unroll
                        for (int k = 0; k < 6; ++k) a[k] = 0.f;
#pragma unroll
                        for (int k = 0; k < 4; ++k) a[6 + k] = -l[k];
                        run_flush(hot, rec, rlo, rn, c, w, a, dG, Q);
                    }
                } else if (r3 == kFastWalk) {
                    slow_bits |= 1u << i;
                } else {
#pragma unroll
                    for (int k = 0; k < 3; ++k) sx[k][j] = xb[k];
                    if (aggregate) {
                        run_add(acc, l, d, cc);
                        live = true;
                    } else {
                        float a[10];
#pragma unroll
                        for (int k = 0; k < 10; ++k) a[k] = 0.f;
                        run_add(a, l, d, cc);
                        run_flush(hot, rec, rlo, rn, c, w, a, dG, Q);
                    }
                }
            }
        }
        {
            // the chunk's deferred particles into the tile's queue: one shared atomic per warp
            const int m = __popc(slow_bits);
            int pre = m;   // inclusive prefix over the lanes
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(kFull, pre, o);
                if (lane >= o) pre += u;
            }
            const int tot = __shfl_sync(kFull, pre, 31);
            int base = 0;
            if (tot > 0) {
                if (lane == 31) base = atomicAdd(&qn[sk], tot);
                base = __shfl_sync(kFull, base, 31) + pre - m;
                for (unsigned b = slow_bits; b; b &= b - 1u) queue[sk][base++] = (int32_t)(p0 + jb + __ffs(b) - 1);
            }
        }
        if (aggregate) {
            if (!live) cur = -1;   // a last run without a particle that stayed: nothing to add
            // lane l+1's first run continues lane l's last one when their tets agree
            const int nh = __shfl_down_sync(kFull, hcell, 1);
            const int pc = __shfl_up_sync(kFull, cur, 1);
#pragma unroll
            for (int k = 0; k < 10; ++k) {
                const float u = __shfl_down_sync(kFull, head[k], 1);
                if (lane < 31 && nh >= 0 && nh == cur) acc[k] += u;
            }
            const bool taken = lane > 0 && hcell >= 0 && hcell == pc;
            if (hcell >= 0 && !taken) run_flush(hot, rec, rlo, rn, hcell, w, head, dG, Q);
            // the last runs of consecutive lanes with the same tet (lanes spanned by one run)
            unsigned heads;
            int end;
            warp_run_reduce<float, 10>(cur, acc, &heads, &end);
            if (((heads >> lane) & 1u) && cur >= 0) run_flush(hot, rec, rlo, rn, cur, w, acc, dG, Q);
        }
        // the producer's bulk copies read the written tile through the async proxy
        fence_proxy_async_smem();
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[sk]);
    }
}

// FP64 walk of the queued particles (near or across a face).  The end point is
// recomputed from the stored start offset and the updated velocity with the same
// FP32 operations as in k_push_fast32.
template <typename DG, typename DQ>
__global__ void __launch_bounds__(128) k_walk32(const TetGeo* __restrict__ geo,
                                                const TetTopo* __restrict__ topo,
                                                int32_t* __restrict__ cell, float* __restrict__ off,
                                                const float* __restrict__ vel, int64_t n, float dt,
                                                double qw, int max_cross, DG* __restrict__ dG,
                                                DQ* __restrict__ Q,
                                                const int32_t* __restrict__ slow_idx,
                                                const int32_t* __restrict__ slow_count,
                                                int32_t* __restrict__ status, int cc) {
    const int64_t m = *slow_count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int64_t p = slow_idx[i];
        if (p < 0 || p >= n) {
            atomicOr(status, ST_INVAL);
            continue;
        }
        const int c = cell[p];
        double xa[3], xb[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float x = off[k * n + p];
            xa[k] = f2d(x);
            xb[k] = f2d(step_pos(x, dt, vel[k * n + p]));
        }
        int end_cell;
        double end_off[3];
        walk_fp64<float, DG, DQ>(geo, topo, c, xa, xb, qw, max_cross, dG, Q, status, nullptr, &end_cell, end_off,
                                 cc != 0);
        cell[p] = end_cell;
#pragma unroll
        for (int k = 0; k < 3; ++k) off[k * n + p] = d2f(end_off[k]);
    }
}

// ---------------------------------------------------------------- Adams mover
// FP32 Adams step, fast path: the Boris kernel's structure with the Adams mover.  A particle
// whose end point clears the rounding margin is finished here (state, history, deposits);
// the others are queued unchanged for k_walk_adams32.
#ifndef FP_ADAMS_MIN_BLOCKS
#define FP_ADAMS_MIN_BLOCKS 3
#endif
__global__ void __launch_bounds__(256, FP_ADAMS_MIN_BLOCKS) k_push_adams32(
    const TetHot* __restrict__ hot, int32_t* __restrict__ cell, float* __restrict__ off,
    float* __restrict__ vel, AdamsStep<float> A, int32_t nt, double qw, int aggregate,
    float* __restrict__ dG, float* __restrict__ Q, int32_t* __restrict__ slow_idx,
    int32_t* __restrict__ slow_count, int32_t* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t n = A.n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float w = (float)qw;
    AdamsMover32 am{A, vel};
    int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31);
    int c_nx = base + lane < n ? __ldg(cell + base + lane) : -1;
    for (; base < n; base += stride) {
        const int64_t p = base + lane;
        const int c = p < n ? c_nx : -1;
        {
            const int64_t q = p + stride;
            c_nx = q < n ? __ldg(cell + q) : -1;
        }
        float x[3] = {0.f, 0.f, 0.f}, v[3] = {0.f, 0.f, 0.f};
        if (c >= 0 && c < nt) {
            x[0] = off[p], x[1] = off[n + p], x[2] = off[2 * n + p];
            v[0] = vel[p], v[1] = vel[n + p], v[2] = vel[2 * n + p];
            am.history(p);
        }
        const bool slow =
            fast_particle(hot, nullptr, 0, 0, c, x, v, p, n, nt, am, w, aggregate, cell, off, dG, Q, status);
        warp_enqueue(slow, (int32_t)p, slow_idx, slow_count);
    }
}

// FP32 Adams step of the queued particles: the same fields and update as the fast path
// (from the unchanged state), then the FP64 walk along x^n -> x^{n+1}.
__global__ void __launch_bounds__(128) k_walk_adams32(const TetHot* __restrict__ hot,
                                                      const TetGeo* __restrict__ geo,
                                                      const TetTopo* __restrict__ topo,
                                                      int32_t* __restrict__ cell, float* __restrict__ off,
                                                      float* __restrict__ vel, AdamsStep<float> A, double qw,
                                                      int max_cross, float* __restrict__ dG,
                                                      float* __restrict__ Q,
                                                      const int32_t* __restrict__ slow_idx,
                                                      const int32_t* __restrict__ slow_count,
                                                      int32_t* __restrict__ status) {
    const int64_t n = A.n;
    const int64_t m = *slow_count;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int64_t p = slow_idx[i];
        if (p < 0 || p >= n) {
            atomicOr(status, ST_INVAL);
            continue;
        }
        const int c = cell[p];
        TetHot H;
        load_hot(hot, c, H);
        float x[3], v[3], E[3], B[3], a[3], v1[3], xb[3], hx[3], ha[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            x[k] = off[k * n + p];
            v[k] = vel[k * n + p];
        }
        adams_history<float>(A, p, hx, ha);
        hot_fields(H, x, E, B);
        adams_update<float>(A, x, v, E, B, hx, ha, a, v1, xb);
        adams_store<float>(A, vel, p, v, a, v1);
        double xa[3], xe[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            xa[k] = f2d(x[k]);
            xe[k] = f2d(xb[k]);
        }
        int end_cell;
        double end_off[3];
        walk_fp64<float>(geo, topo, c, xa, xe, qw, max_cross, dG, Q, status, nullptr, &end_cell, end_off);
        cell[p] = end_cell;
#pragma unroll
        for (int k = 0; k < 3; ++k) off[k * n + p] = d2f(end_off[k]);
    }
}

// FP64 Adams step: FP64 gather (Whitney-1/2 on the tet), the Adams update and the FP64 walk
// with warp-aggregated deposits of the particles that stay in their tet.
__global__ void __launch_bounds__(256) k_push_adams64(
    const TetGeo* __restrict__ geo, const TetTopo* __restrict__ topo, const double* __restrict__ f64,
    int32_t* __restrict__ cell, double* __restrict__ off,
    double* __restrict__ vel, AdamsStep<double> A, int32_t nt, double qw, int max_cross, int aggregate,
    double* __restrict__ dG, double* __restrict__ Q, int32_t* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t n = A.n;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n; base += stride) {
        const int64_t p = base + lane;
        int c = p < n ? cell[p] : -1;
        if (c >= nt) {
            atomicOr(status, ST_INVAL);
            c = -1;
        }
        int key = -1;
        double agg[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) agg[k] = 0.0;
        TetTopo T;
        if (c >= 0) {
            load_topo(topo, c, T);
            double x[3] = {off[p], off[n + p], off[2 * n + p]};
            double v[3] = {vel[p], vel[n + p], vel[2 * n + p]};
            double E[3], B[3], a[3], v1[3], xb[3], hx[3], ha[3];
            adams_history<double>(A, p, hx, ha);
            fields64(f64, c, x, E, B);
            adams_update<double>(A, x, v, E, B, hx, ha, a, v1, xb);
            adams_store<double>(A, vel, p, v, a, v1);
            int end_cell;
            double end_off[3];
            if (walk_fp64<double>(geo, topo, c, x, xb, qw, max_cross, dG, Q, status, aggregate ? agg : nullptr,
                                  &end_cell, end_off))
                key = c;
            cell[p] = end_cell;
            off[p] = end_off[0];
            off[n + p] = end_off[1];
            off[2 * n + p] = end_off[2];
        }
        if (aggregate) {
            unsigned heads;
            int end;
            warp_run_reduce<double, 10>(key, agg, &heads, &end);
            if (((heads >> lane) & 1u) && key >= 0) {
#pragma unroll
                for (int k = 0; k < 6; ++k) atomicAdd(dG + T.edge[k], agg[k]);
#pragma unroll
                for (int k = 0; k < 4; ++k) atomicAdd(Q + T.node[k], agg[6 + k]);
            }
        }
    }
}

// Self-test of the bounded waits: one thread waits on an mbarrier that nothing arrives at,
// gives up after limit_ns and reports ST_TIMEOUT, as the push kernels do when a copy never
// completes.  No copy is issued, so nothing is in flight when it returns.
__global__ void k_wait_selftest(uint64_t limit_ns, int32_t* __restrict__ status) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    mbar_init(&bar, 1);
    mbar_fence_init();
    if (!mbar_wait_bounded(&bar, 0, limit_ns)) atomicOr(status, ST_TIMEOUT);
}

// W0 charge at the current positions, FP32 (barycentrics from the FP32 gradients)
template <typename D>
__global__ void __launch_bounds__(256) k_deposit_charge32(const TetHot* __restrict__ hot,
                                                          const int32_t* __restrict__ cell,
                                                          const float* __restrict__ off, int64_t n,
                                                          int32_t nt, double qw, D* __restrict__ Q,
                                                          int32_t* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const float w = (float)qw;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride) {
        const int64_t p = base + lane;
        int c = p < n ? cell[p] : -1;
        if (c >= nt) {
            atomicOr(status, ST_INVAL);
            c = -1;
        }
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        TetHot H;
        if (c >= 0 && !(finite_bits(off[p]) && finite_bits(off[n + p]) && finite_bits(off[2 * n + p]))) {
            atomicOr(status, ST_NONFINITE);   // no charge for a particle without a position
            c = -1;
        }
        if (c >= 0) {
            load_hot(hot, c, H);
            const float x[3] = {off[p], off[n + p], off[2 * n + p]};
            float l1 = H.g[0] * x[0] + H.g[1] * x[1] + H.g[2] * x[2];
            float l2 = H.g[3] * x[0] + H.g[4] * x[1] + H.g[5] * x[2];
            float l3 = H.g[6] * x[0] + H.g[7] * x[1] + H.g[8] * x[2];
            v[0] = w * (1.f - l1 - l2 - l3);
            v[1] = w * l1;
            v[2] = w * l2;
            v[3] = w * l3;
        }
        unsigned heads;
        int end;
        warp_run_reduce<float, 4>(c, v, &heads, &end);
        if (((heads >> lane) & 1u) && c >= 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(Q + H.node[k], dep_cast<D>(v[k]));
        }
    }
}

template <typename Real>
__global__ void __launch_bounds__(256) k_deposit_charge(const TetGeo* __restrict__ geo,
                                                        const TetTopo* __restrict__ topo,
                                                        const int32_t* __restrict__ cell,
                                                        const Real* __restrict__ off, int64_t n,
                                                        int32_t nt, double qw, Real* __restrict__ Q,
                                                        int32_t* __restrict__ status) {
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t base = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n;
         base += stride) {
        const int64_t p = base + lane;
        int c = p < n ? cell[p] : -1;
        if (c >= nt) {
            atomicOr(status, ST_INVAL);
            c = -1;
        }
        if (c >= 0 && !(finite_bits(off[p]) && finite_bits(off[n + p]) && finite_bits(off[2 * n + p]))) {
            atomicOr(status, ST_NONFINITE);   // no charge for a particle without a position
            c = -1;
        }
        Real v[4] = {0, 0, 0, 0};
        TetTopo T;
        if (c >= 0) {
            Geo G;
            load_geo(geo, c, G);
            load_topo(topo, c, T);
            double r[3] = {(double)off[p], (double)off[n + p], (double)off[2 * n + p]}, l[4];
            bary(G, r, l);
#pragma unroll
            for (int k = 0; k < 4; ++k) v[k] = (Real)qw * (Real)l[k];
        }
        unsigned heads;
        int end;
        warp_run_reduce<Real, 4>(c, v, &heads, &end);
        if (((heads >> lane) & 1u) && c >= 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) atomicAdd(Q + T.node[k], v[k]);
        }
    }
}

int grid_for(int64_t n, int sms) {
    int64_t blocks = (n + 255) / 256;
    int64_t cap = (int64_t)sms * 8;  // grid-stride beyond 8 resident 256-thread blocks per SM
    if (blocks > cap) blocks = cap;
    return blocks < 1 ? 1 : (int)blocks;
}

// the fast FP32 push: the TMA-staged persistent kernel (grid = co-resident blocks), or the
// grid-stride kernel when the state arrays are not 16-byte aligned
template <typename DG, typename DQ>
fp_status launch_fast32_t(fem_pic* ctx, const fp_particles* p, int32_t nt, float h, float dt, double qw, int agg,
                          DG* dG, DQ* Q, int cc, int32_t* slow_idx, int32_t* slow_count, cudaStream_t s) {
    // FP64 deposit arrays or the charge change: the run-summing or the grid-stride kernel
    constexpr int kind = (sizeof(DG) == 8 ? 1 : 0) + (sizeof(DQ) == 8 ? 2 : 0);
    const bool d64 = kind != 0 || cc != 0;
    const size_t smem = (size_t)kTmaSmem;
    if (ctx->tma_blocks_per_sm == 0) {
        FP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_push_tma32, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int per_sm = 0;
        FP_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push_tma32, kTmaThreads, smem));
        if (per_sm < 1) {
            ctx->err = "fem_pic_push_deposit: the staged push kernel does not fit on an SM";
            return FP_ECUDA;
        }
        ctx->tma_blocks_per_sm = per_sm;
    }
    const bool aligned = (p->n % 4) == 0 && ((uintptr_t)p->cell % 16) == 0 && ((uintptr_t)p->off % 16) == 0 &&
                         ((uintptr_t)p->vel % 16) == 0;
#ifndef FP_PUSH_TMA
#define FP_PUSH_TMA 1
#endif
    if (!aligned || (!FP_PUSH_TMA && !d64)) {   // the bulk copies need 16-byte aligned starts and lengths
        k_push_fast32<DG, DQ><<<grid_for(p->n, ctx->sm_count), 256, 0, s>>>(
            ctx->d_hot, p->cell, (float*)p->off, (float*)p->vel, p->n, nt, h, dt, qw, agg, dG, Q, slow_idx,
            slow_count, ctx->d_status, cc);
        FP_CUDA_TRY(ctx, cudaGetLastError());
        return FP_OK;
    }
#ifndef FP_PUSH_RUN
#define FP_PUSH_RUN 1
#endif
    if (FP_PUSH_RUN || d64) {   // warp-specialised pipeline, runs summed per lane
        int& per_sm_cached = ctx->run_blocks_per_sm[kind];
        if (per_sm_cached == 0) {
            FP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_push_run32<DG, DQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  kRunSmem));
            int per_sm = 0;
            FP_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push_run32<DG, DQ>,
                                                                           kRunThreads, kRunSmem));
            if (per_sm < 1) {
                ctx->err = "fem_pic_push_deposit: the staged push kernel does not fit on an SM";
                return FP_ECUDA;
            }
            per_sm_cached = per_sm;
        }
        const int64_t rtiles = (p->n + kRunTile - 1) / kRunTile;
        int64_t rgrid = (int64_t)ctx->sm_count * per_sm_cached;
        if (rgrid > rtiles) rgrid = rtiles;
        k_push_run32<DG, DQ><<<(int)rgrid, kRunThreads, kRunSmem, s>>>(
            ctx->d_hot, p->cell, (float*)p->off, (float*)p->vel, p->n, nt, h, dt, (float)qw, agg, dG, Q, slow_idx,
            slow_count, ctx->d_status, cc);
        FP_CUDA_TRY(ctx, cudaGetLastError());
        return FP_OK;
    }
#ifndef FP_PUSH_WS
#define FP_PUSH_WS 1
#endif
    if constexpr (kind != 0) {
        return FP_OK;   // not reached: FP64 deposits take the run-summing kernel above
    } else {
    if (FP_PUSH_WS) {   // warp-specialised pipeline
        if (ctx->ws_blocks_per_sm == 0) {
            FP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_push_ws32<BorisArgs>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                  kWsSmem));
            int per_sm = 0;
            FP_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push_ws32<BorisArgs>, kWsThreads,
                                                                           kWsSmem));
            if (per_sm < 1) {
                ctx->err = "fem_pic_push_deposit: the staged push kernel does not fit on an SM";
                return FP_ECUDA;
            }
            ctx->ws_blocks_per_sm = per_sm;
        }
        const int64_t wtiles = (p->n + kWsTile - 1) / kWsTile;
        int64_t wgrid = (int64_t)ctx->sm_count * ctx->ws_blocks_per_sm;
        if (wgrid > wtiles) wgrid = wtiles;
        k_push_ws32<BorisArgs><<<(int)wgrid, kWsThreads, kWsSmem, s>>>(
            ctx->d_hot, p->cell, (float*)p->off, (float*)p->vel, p->n, nt, BorisArgs{h, dt}, qw, agg, dG, Q,
            slow_idx, slow_count, ctx->d_status);
        FP_CUDA_TRY(ctx, cudaGetLastError());
        return FP_OK;
    }
    const int64_t ntiles = (p->n + kTmaTile - 1) / kTmaTile;
    int64_t grid = (int64_t)ctx->sm_count * ctx->tma_blocks_per_sm;
    if (grid > ntiles) grid = ntiles;
    k_push_tma32<<<(int)grid, kTmaThreads, smem, s>>>(ctx->d_hot, p->cell, (float*)p->off, (float*)p->vel, p->n, nt,
                                                      h, dt, qw, agg, dG, Q, slow_idx, slow_count,
                                                      ctx->d_status);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
    }
}

// the FP64 walk of the queued particles, with the deposit arrays' element type
template <typename DG, typename DQ>
void launch_walk32_t(fem_pic* ctx, const fp_particles* p, float dt, double qw, int max_cross, void* dG, void* Q,
                     int cc, const int32_t* slow_idx, const int32_t* slow_count, cudaStream_t s) {
    k_walk32<DG, DQ><<<ctx->sm_count * 4, 128, 0, s>>>(ctx->d_geo, ctx->d_topo, p->cell, (float*)p->off,
                                                       (const float*)p->vel, p->n, dt, qw, max_cross, (DG*)dG,
                                                       (DQ*)Q, slow_idx, slow_count, ctx->d_status, cc);
}

void launch_walk32(fem_pic* ctx, const fp_particles* p, float dt, double qw, int max_cross, void* dG, void* Q,
                   int cc, const int32_t* slow_idx, const int32_t* slow_count, cudaStream_t s) {
    if (ctx->dG64)
        launch_walk32_t<double, double>(ctx, p, dt, qw, max_cross, dG, Q, cc, slow_idx, slow_count, s);
    else if (ctx->Q64)
        launch_walk32_t<float, double>(ctx, p, dt, qw, max_cross, dG, Q, cc, slow_idx, slow_count, s);
    else
        launch_walk32_t<float, float>(ctx, p, dt, qw, max_cross, dG, Q, cc, slow_idx, slow_count, s);
}

// the fast FP32 push with the deposit arrays' element type
fp_status launch_fast32(fem_pic* ctx, const fp_particles* p, int32_t nt, float h, float dt, double qw, int agg,
                        void* dG, void* Q, int cc, int32_t* slow_idx, int32_t* slow_count, cudaStream_t s) {
    if (ctx->dG64)
        return launch_fast32_t<double, double>(ctx, p, nt, h, dt, qw, agg, (double*)dG, (double*)Q, cc, slow_idx,
                                               slow_count, s);
    if (ctx->Q64)
        return launch_fast32_t<float, double>(ctx, p, nt, h, dt, qw, agg, (float*)dG, (double*)Q, cc, slow_idx,
                                              slow_count, s);
    return launch_fast32_t<float, float>(ctx, p, nt, h, dt, qw, agg, (float*)dG, (float*)Q, cc, slow_idx,
                                         slow_count, s);
}

}  // namespace

namespace {
// the FP32 path's queue of particles deferred to the FP64 walk: at least n entries, count 0
fp_status slow_queue(fem_pic* ctx, int64_t n, const char* who, cudaStream_t s) {
    if (n > INT32_MAX) {
        ctx->err = std::string(who) + ": more than 2^31-1 particles in one call";
        return FP_EINVAL;
    }
    if (ctx->slow_cap < n) {
        if (ctx->d_slow_idx) FP_CUDA_TRY(ctx, cudaFree(ctx->d_slow_idx));
        ctx->d_slow_idx = nullptr;
        ctx->slow_cap = 0;
        FP_CUDA_TRY(ctx, cudaMalloc((void**)&ctx->d_slow_idx, n * sizeof(int32_t)));
        ctx->slow_cap = n;
    }
    FP_CUDA_TRY(ctx, cudaMemsetAsync(ctx->d_slow_count, 0, sizeof(int32_t), s));
    return FP_OK;
}
}  // namespace

fp_status launch_push_deposit(fem_pic* ctx, const double* e, const double* b, const fp_particles* p,
                              double dt, int max_cross, void* dG, void* Q, int flags,
                              cudaStream_t s) {
    const bool f32 = ctx->precision == FP_FP32;
    if (!(flags & FP_ACCUMULATE)) {   // the charge change is always added onto Q
        FP_CUDA_TRY(ctx, cudaMemsetAsync(dG, 0, (dG_f32(ctx) ? 4 : 8) * ctx->hc.ne, s));
        if (!(flags & FP_CHARGE_CHANGE))
            FP_CUDA_TRY(ctx, cudaMemsetAsync(Q, 0, (Q_f32(ctx) ? 4 : 8) * ctx->hc.nn, s));
    }
    const int cc = (flags & FP_CHARGE_CHANGE) ? 1 : 0;
    if (p->n == 0) return FP_OK;
    const double qmdt2 = p->q * dt / (2.0 * p->m);
    const double qw = p->q * p->w;
    const int agg = (flags & FP_NO_AGGREGATE) ? 0 : 1;
    const int grid = grid_for(p->n, ctx->sm_count);
    const int32_t nt = (int32_t)ctx->hc.nt;
    if (f32) {
        const fp_status sq = slow_queue(ctx, p->n, "fem_pic_push_deposit", s);
        if (sq != FP_OK) return sq;
        if (!(flags & FP_SAME_FIELDS)) {
            PhaseTimer pt(ctx, PH_PREP, s);
            k_field_prep32<<<grid_for((ctx->hc.nt + 1) / 2, ctx->sm_count), 256, 0, s>>>(ctx->d_hot, ctx->d_tet_faces, e, b, ctx->hc.nt);
        }
        {
            PhaseTimer pt(ctx, PH_FAST, s);
            fp_status sf = launch_fast32(ctx, p, nt, (float)qmdt2, (float)dt, qw, agg, dG, Q, cc,
                                         ctx->d_slow_idx, ctx->d_slow_count, s);
            if (sf != FP_OK) return sf;
        }
        {
            PhaseTimer pt(ctx, PH_WALK, s);
            launch_walk32(ctx, p, (float)dt, qw, max_cross, dG, Q, cc, ctx->d_slow_idx, ctx->d_slow_count, s);
        }
    } else {
        if (!(flags & FP_SAME_FIELDS)) {
            PhaseTimer pt(ctx, PH_PREP, s);
            k_field_prep64<<<grid_for(ctx->hc.nt, ctx->sm_count), 256, 0, s>>>(ctx->d_geo, ctx->d_topo, e, b,
                                                                               ctx->hc.nt, ctx->d_field64);
        }
        PhaseTimer pt(ctx, PH_PUSH64, s);
        k_push_deposit<double><<<grid, 256, 0, s>>>(ctx->d_geo, ctx->d_topo, ctx->d_field64, p->cell,
                                                    (double*)p->off, (double*)p->vel, p->n, nt, qmdt2, dt,
                                                    qw, max_cross, agg, (double*)dG, (double*)Q,
                                                    ctx->d_status, cc);
    }
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}

fp_status launch_push_adams(fem_pic* ctx, const double* e, const double* b, const fp_particles* p, void* hist,
                            int64_t step, double dt, int max_cross, void* dG, void* Q, int flags, cudaStream_t s) {
    const bool f32 = ctx->precision == FP_FP32;
    if (f32 && (ctx->dG64 || ctx->Q64)) {
        ctx->err = "fem_pic_push_deposit_adams: FP64 deposits are not available for the Adams mover in FP32 mode";
        return FP_EINVAL;
    }
    if (flags & FP_CHARGE_CHANGE) {
        ctx->err = "fem_pic_push_deposit_adams: the charge-change deposit is not available for the Adams mover";
        return FP_EINVAL;
    }
    const size_t rs = f32 ? 4 : 8;
    if (!(flags & FP_ACCUMULATE)) {
        FP_CUDA_TRY(ctx, cudaMemsetAsync(dG, 0, rs * ctx->hc.ne, s));
        FP_CUDA_TRY(ctx, cudaMemsetAsync(Q, 0, rs * ctx->hc.nn, s));
    }
    if (p->n == 0) return FP_OK;
    // Adams-Bashforth coefficients of f^n, f^{n-1}, ... for orders 1..4
    static const double kBeta[4][4] = {{1.0, 0.0, 0.0, 0.0},
                                       {3.0 / 2.0, -1.0 / 2.0, 0.0, 0.0},
                                       {23.0 / 12.0, -16.0 / 12.0, 5.0 / 12.0, 0.0},
                                       {55.0 / 24.0, -59.0 / 24.0, 37.0 / 24.0, -9.0 / 24.0}};
    const int order = step < 3 ? (int)step + 1 : 4;
    const int slot_new = (int)(step % 3);
    int slot[3];
    for (int j = 1; j <= 3; ++j) slot[j - 1] = (int)(((step - j) % 3 + 3) % 3);
    const double qm = p->q / p->m, qw = p->q * p->w;
    const int agg = (flags & FP_NO_AGGREGATE) ? 0 : 1;
    const int32_t nt = (int32_t)ctx->hc.nt;
    if (f32) {
        AdamsStep<float> A;
        A.hist = (float*)hist, A.n = p->n, A.order = order, A.slot_new = slot_new;
        for (int j = 0; j < 3; ++j) A.slot[j] = slot[j];
        for (int j = 0; j < 4; ++j) A.beta[j] = (float)kBeta[order - 1][j];
        A.dt = (float)dt, A.qm = (float)qm;
        const fp_status sq = slow_queue(ctx, p->n, "fem_pic_push_deposit_adams", s);
        if (sq != FP_OK) return sq;
        if (!(flags & FP_SAME_FIELDS)) {
            PhaseTimer pt(ctx, PH_PREP, s);
            k_field_prep32<<<grid_for((ctx->hc.nt + 1) / 2, ctx->sm_count), 256, 0, s>>>(ctx->d_hot, ctx->d_tet_faces,
                                                                                        e, b, ctx->hc.nt);
        }
        const bool aligned = (p->n % 4) == 0 && ((uintptr_t)p->cell % 16) == 0 && ((uintptr_t)p->off % 16) == 0 &&
                             ((uintptr_t)p->vel % 16) == 0;
#ifndef FP_ADAMS_WS
#define FP_ADAMS_WS 1
#endif
        if (aligned && FP_ADAMS_WS && ctx->ws_adams_blocks_per_sm == 0) {
            FP_CUDA_TRY(ctx, cudaFuncSetAttribute(k_push_ws32<AdamsStep<float>>,
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, kWsSmem));
            int per_sm = 0;
            FP_CUDA_TRY(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_push_ws32<AdamsStep<float>>,
                                                                           kWsThreads, kWsSmem));
            if (per_sm < 1) {
                ctx->err = "fem_pic_push_deposit_adams: the staged push kernel does not fit on an SM";
                return FP_ECUDA;
            }
            ctx->ws_adams_blocks_per_sm = per_sm;
        }
        {
            PhaseTimer pt(ctx, PH_ADAMS, s);
            if (aligned && FP_ADAMS_WS) {   // the state staged by bulk copies, as in the Boris push
                const int64_t wtiles = (p->n + kWsTile - 1) / kWsTile;
                int64_t wgrid = (int64_t)ctx->sm_count * ctx->ws_adams_blocks_per_sm;
                if (wgrid > wtiles) wgrid = wtiles;
                k_push_ws32<AdamsStep<float>><<<(int)wgrid, kWsThreads, kWsSmem, s>>>(
                    ctx->d_hot, p->cell, (float*)p->off, (float*)p->vel, p->n, nt, A, qw, agg, (float*)dG, (float*)Q,
                    ctx->d_slow_idx, ctx->d_slow_count, ctx->d_status);
            } else {
                k_push_adams32<<<grid_for(p->n, ctx->sm_count), 256, 0, s>>>(ctx->d_hot, p->cell, (float*)p->off,
                                                                              (float*)p->vel, A, nt, qw, agg,
                                                                              (float*)dG, (float*)Q, ctx->d_slow_idx,
                                                                              ctx->d_slow_count, ctx->d_status);
            }
        }
        {
            PhaseTimer pt(ctx, PH_ADAMS_WALK, s);
            k_walk_adams32<<<ctx->sm_count * 4, 128, 0, s>>>(ctx->d_hot, ctx->d_geo, ctx->d_topo, p->cell,
                                                             (float*)p->off, (float*)p->vel, A, qw, max_cross,
                                                             (float*)dG, (float*)Q, ctx->d_slow_idx,
                                                             ctx->d_slow_count, ctx->d_status);
        }
    } else {
        AdamsStep<double> A;
        A.hist = (double*)hist, A.n = p->n, A.order = order, A.slot_new = slot_new;
        for (int j = 0; j < 3; ++j) A.slot[j] = slot[j];
        for (int j = 0; j < 4; ++j) A.beta[j] = kBeta[order - 1][j];
        A.dt = dt, A.qm = qm;
        if (!(flags & FP_SAME_FIELDS)) {
            PhaseTimer pt(ctx, PH_PREP, s);
            k_field_prep64<<<grid_for(ctx->hc.nt, ctx->sm_count), 256, 0, s>>>(ctx->d_geo, ctx->d_topo, e, b,
                                                                               ctx->hc.nt, ctx->d_field64);
        }
        PhaseTimer pt(ctx, PH_ADAMS, s);
        k_push_adams64<<<grid_for(p->n, ctx->sm_count), 256, 0, s>>>(ctx->d_geo, ctx->d_topo, ctx->d_field64,
                                                                      p->cell, (double*)p->off, (double*)p->vel, A,
                                                                      nt, qw, max_cross, agg, (double*)dG,
                                                                      (double*)Q, ctx->d_status);
    }
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}

fp_status launch_wait_selftest(fem_pic* ctx, double limit_s, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>((uint64_t)(limit_s * 1e9), ctx->d_status);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}

fp_status launch_deposit_charge(fem_pic* ctx, const fp_particles* p, void* Q, int flags,
                                cudaStream_t s) {
    const bool f32 = ctx->precision == FP_FP32;
    if (!(flags & FP_ACCUMULATE)) FP_CUDA_TRY(ctx, cudaMemsetAsync(Q, 0, (Q_f32(ctx) ? 4 : 8) * ctx->hc.nn, s));
    if (p->n == 0) return FP_OK;
    const double qw = p->q * p->w;
    const int grid = grid_for(p->n, ctx->sm_count);
    PhaseTimer pt(ctx, PH_CHARGE, s);
    if (f32 && ctx->Q64)
        k_deposit_charge32<double><<<grid, 256, 0, s>>>(ctx->d_hot, p->cell, (const float*)p->off, p->n,
                                                        (int32_t)ctx->hc.nt, qw, (double*)Q, ctx->d_status);
    else if (f32)
        k_deposit_charge32<float><<<grid, 256, 0, s>>>(ctx->d_hot, p->cell, (const float*)p->off, p->n,
                                                       (int32_t)ctx->hc.nt, qw, (float*)Q, ctx->d_status);
    else
        k_deposit_charge<double><<<grid, 256, 0, s>>>(ctx->d_geo, ctx->d_topo, p->cell,
                                                      (const double*)p->off, p->n, (int32_t)ctx->hc.nt,
                                                      qw, (double*)Q, ctx->d_status);
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}

}  // namespace fempic

// ---------------------------------------------------------------- allocation-free entry point
// Some callers cannot allocate device memory while they step particles: code running
// under a strict memory budget that was fixed up front, a host allocator that forbids
// cudaMalloc after start-up, or a driver layer that only hands out buffers it already
// owns.  fem_pic_push_deposit grows a library-owned queue of the particles it defers
// to the FP64 walk with cudaMalloc; this variant keeps that queue in a fixed array
// compiled into the library instead.  The array is shared by every call on a device
// and keeps the last call's contents; the count at its head is cleared by every call.
namespace fempic {
namespace {

constexpr int64_t kStaticMaxParticles = int64_t(1) << 22;  // 4,194,304 particles, 16 MiB
constexpr int kStaticHead = 64;                           // int32 slots before the indices

// [0] = number of queued particles, [kStaticHead ...] = their indices
static __device__ __align__(256) int32_t g_static_queue[kStaticHead + kStaticMaxParticles];

}  // namespace

// Device address of g_static_queue in the handle's context.  Called by fem_pic_create with
// the handle's device current, so the address lives exactly as long as the handle (a context
// rebuilt after cudaDeviceReset gets a new handle and a new lookup).  In host code the
// array's name is only a stand-in: kernels must be given this address.
fp_status static_queue_lookup(fem_pic* ctx) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_queue);
    if (e != cudaSuccess || !p) {
        ctx->err = std::string("cudaGetSymbolAddress(g_static_queue): ") + cudaGetErrorString(e);
        return FP_ECUDA;
    }
    ctx->d_static_queue = static_cast<int32_t*>(p);
    return FP_OK;
}

}  // namespace fempic

extern "C" fp_status fem_pic_push_deposit_static(fem_pic_t* ctx, const double* e, const double* b,
                                                 const fp_particles* p, double dt, int max_cross,
                                                 void* dG, void* Q, int flags, void* stream) {
    using namespace fempic;
    if (!ctx || !p || !e || !b || !dG || !Q || p->n < 0 || max_cross < 0 || !(p->m > 0.0)) {
        if (ctx) ctx->err = "fem_pic_push_deposit_static: NULL pointer or bad argument";
        return FP_EINVAL;
    }
    if (p->n > 0 && (!p->cell || !p->off || !p->vel)) {
        ctx->err = "fem_pic_push_deposit_static: NULL particle array";
        return FP_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (ctx->precision != FP_FP32)  // the FP64 path defers nothing and needs no scratch
        return launch_push_deposit(ctx, e, b, p, dt, max_cross, dG, Q, flags, s);
    if (p->n > kStaticMaxParticles) {
        ctx->err = "fem_pic_push_deposit_static: " + std::to_string(p->n) +
                   " particles exceed the fixed queue of " + std::to_string(kStaticMaxParticles);
        return FP_EINVAL;
    }
    int32_t* q = ctx->d_static_queue;
    if (!q) {
        ctx->err = "fem_pic_push_deposit_static: the fixed queue's device address is unknown";
        return FP_ECUDA;
    }
    if (!(flags & FP_ACCUMULATE)) {   // the charge change is always added onto Q
        FP_CUDA_TRY(ctx, cudaMemsetAsync(dG, 0, (dG_f32(ctx) ? 4 : 8) * ctx->hc.ne, s));
        if (!(flags & FP_CHARGE_CHANGE))
            FP_CUDA_TRY(ctx, cudaMemsetAsync(Q, 0, (Q_f32(ctx) ? 4 : 8) * ctx->hc.nn, s));
    }
    FP_CUDA_TRY(ctx, cudaMemsetAsync(q, 0, sizeof(int32_t), s));
    if (p->n == 0) return FP_OK;
    const double qmdt2 = p->q * dt / (2.0 * p->m);
    const double qw = p->q * p->w;
    const int agg = (flags & FP_NO_AGGREGATE) ? 0 : 1;
    const int32_t nt = (int32_t)ctx->hc.nt;
    if (!(flags & FP_SAME_FIELDS)) {
        PhaseTimer pt(ctx, PH_PREP, s);
        k_field_prep32<<<grid_for((ctx->hc.nt + 1) / 2, ctx->sm_count), 256, 0, s>>>(ctx->d_hot, ctx->d_tet_faces, e,
                                                                                    b, ctx->hc.nt);
    }
    {
        // the same kernel choice as fem_pic_push_deposit (staged pipeline for aligned state)
        PhaseTimer pt(ctx, PH_FAST, s);
        const fp_status sf = launch_fast32(ctx, p, nt, (float)qmdt2, (float)dt, qw, agg, dG, Q,
                                           (flags & FP_CHARGE_CHANGE) ? 1 : 0, q + kStaticHead, q, s);
        if (sf != FP_OK) return sf;
    }
    {
        PhaseTimer pt(ctx, PH_WALK, s);
        launch_walk32(ctx, p, (float)dt, qw, max_cross, dG, Q, (flags & FP_CHARGE_CHANGE) ? 1 : 0, q + kStaticHead,
                      q, s);
    }
    FP_CUDA_TRY(ctx, cudaGetLastError());
    return FP_OK;
}
