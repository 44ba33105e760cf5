/*
 * FP64 CPU oracle of the per-particle FEM-PIC step.  TEST INFRASTRUCTURE ONLY:
 * used by tests/, the smoke check and the bench's CPU-baseline leg, never by the
 * product path.  Shares no code with the CUDA library.
 *
 * Everything here is the plain definition, evaluated at physical points:
 *   - barycentric coordinates by Cramer's rule on the tet's affine map;
 *   - E = sum_e e_e W1_e, B = sum_f b_f W2_f with lowest-order Whitney forms
 *     (Sec. II.C: E in span W1, B in span W2);
 *   - the textbook non-relativistic Boris rotation (Lorentz force, Sec. II.A);
 *   - the straight path split at tet faces, and on every piece the Whitney-1
 *     line integral  G_e += q w * int_path W1_e . dr  (Sec. IV.B.1, the path-integral
 *     form of the time-integrated current) evaluated with 2-point Gauss-Legendre,
 *     which is exact for the linear integrand;
 *   - the Whitney-0 charge  Q_n += q w * lambda_n(x_end).
 * Parity unpinned parts: none (see tests/test_oracle_*.py for the pins).
 *
 * Readings where the paper is silent (walk rules): an exit needs lambda_k(end) < 0
 * strictly; the entry face is not an exit candidate; the exit is the smallest
 * crossing fraction s_k = la_k/(la_k-lb_k) (0 if la_k-lb_k <= 0), clamped to [0,1],
 * ties to the lowest local face index; a face with no neighbour is a PEC wall and
 * absorbs the particle at the wall point (its charge stays on the wall nodes);
 * at most max_cross crossings, after which the particle stops at the last
 * crossing point and the call reports it.
 *
 * Local numbering: tet vertices sorted by global id (v0<v1<v2<v3); local edges
 * (01,02,03,12,13,23) in that order; face k is the face opposite local vertex k.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static const int LE[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
static const int LF[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};

typedef struct {
    const double* xyz;
    const int32_t* tv;
    const int32_t* te;
    const int32_t* tf;
    const int32_t* nb;
    const double* e;
    const double* b;
} mesh_t;

static double det3(const double a[3], const double b[3], const double c[3]) {
    return a[0] * (b[1] * c[2] - b[2] * c[1]) - a[1] * (b[0] * c[2] - b[2] * c[0]) +
           a[2] * (b[0] * c[1] - b[1] * c[0]);
}

static void cross3(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

static void vertex(const mesh_t* M, int t, int k, double x[3]) {
    const double* p = M->xyz + 3 * (int64_t)M->tv[4 * (int64_t)t + k];
    x[0] = p[0];
    x[1] = p[1];
    x[2] = p[2];
}

/* barycentric coordinates of X in tet t (Cramer's rule on x = x0 + J l) */
static void bary(const mesh_t* M, int t, const double X[3], double lam[4]) {
    double x0[3], x1[3], x2[3], x3[3], e1[3], e2[3], e3[3], d[3];
    vertex(M, t, 0, x0);
    vertex(M, t, 1, x1);
    vertex(M, t, 2, x2);
    vertex(M, t, 3, x3);
    for (int i = 0; i < 3; ++i) {
        e1[i] = x1[i] - x0[i];
        e2[i] = x2[i] - x0[i];
        e3[i] = x3[i] - x0[i];
        d[i] = X[i] - x0[i];
    }
    double D = det3(e1, e2, e3);
    lam[1] = det3(d, e2, e3) / D;
    lam[2] = det3(e1, d, e3) / D;
    lam[3] = det3(e1, e2, d) / D;
    lam[0] = 1.0 - lam[1] - lam[2] - lam[3];
}

/* gradients of the barycentric coordinates (rows of the inverse Jacobian) */
static void grads(const mesh_t* M, int t, double g[4][3]) {
    double x0[3], x1[3], x2[3], x3[3], e1[3], e2[3], e3[3];
    vertex(M, t, 0, x0);
    vertex(M, t, 1, x1);
    vertex(M, t, 2, x2);
    vertex(M, t, 3, x3);
    for (int i = 0; i < 3; ++i) {
        e1[i] = x1[i] - x0[i];
        e2[i] = x2[i] - x0[i];
        e3[i] = x3[i] - x0[i];
    }
    double D = det3(e1, e2, e3);
    cross3(e2, e3, g[1]);
    cross3(e3, e1, g[2]);
    cross3(e1, e2, g[3]);
    for (int i = 0; i < 3; ++i) {
        g[1][i] /= D;
        g[2][i] /= D;
        g[3][i] /= D;
        g[0][i] = -(g[1][i] + g[2][i] + g[3][i]);
    }
}

/* W1 of local edge (a,b): lam_a grad lam_b - lam_b grad lam_a */
static void whitney1(const double lam[4], double g[4][3], int a, int b, double w[3]) {
    for (int i = 0; i < 3; ++i) w[i] = lam[a] * g[b][i] - lam[b] * g[a][i];
}

/* W2 of local face (a,b,c): 2 (lam_a g_b x g_c + lam_b g_c x g_a + lam_c g_a x g_b) */
static void whitney2(const double lam[4], double g[4][3], int a, int b, int c, double w[3]) {
    double bc[3], ca[3], ab[3];
    cross3(g[b], g[c], bc);
    cross3(g[c], g[a], ca);
    cross3(g[a], g[b], ab);
    for (int i = 0; i < 3; ++i) w[i] = 2.0 * (lam[a] * bc[i] + lam[b] * ca[i] + lam[c] * ab[i]);
}

static void gather(const mesh_t* M, int t, const double X[3], double E[3], double B[3]) {
    double lam[4], g[4][3], w[3];
    bary(M, t, X, lam);
    grads(M, t, g);
    E[0] = E[1] = E[2] = 0.0;
    B[0] = B[1] = B[2] = 0.0;
    for (int k = 0; k < 6; ++k) {
        whitney1(lam, g, LE[k][0], LE[k][1], w);
        double ek = M->e[M->te[6 * (int64_t)t + k]];
        for (int i = 0; i < 3; ++i) E[i] += ek * w[i];
    }
    for (int k = 0; k < 4; ++k) {
        whitney2(lam, g, LF[k][0], LF[k][1], LF[k][2], w);
        double bk = M->b[M->tf[4 * (int64_t)t + k]];
        for (int i = 0; i < 3; ++i) B[i] += bk * w[i];
    }
}

/* textbook Boris rotation, non-relativistic */
static void boris(double v[3], const double E[3], const double B[3], double q, double m, double dt) {
    double h = q * dt / (2.0 * m);
    double vm[3], t[3], s[3], vp[3], c[3];
    for (int i = 0; i < 3; ++i) {
        vm[i] = v[i] + h * E[i];
        t[i] = h * B[i];
    }
    double tt = t[0] * t[0] + t[1] * t[1] + t[2] * t[2];
    for (int i = 0; i < 3; ++i) s[i] = 2.0 * t[i] / (1.0 + tt);
    cross3(vm, t, c);
    for (int i = 0; i < 3; ++i) vp[i] = vm[i] + c[i];
    cross3(vp, s, c);
    for (int i = 0; i < 3; ++i) v[i] = vm[i] + c[i] + h * E[i];
}

typedef struct {
    double* G;
    double* Gabs;
    double* Q;
    double* Qabs;
    /* optional (NULL: not kept): sum of |q w| over the pieces / end points touching each entry,
     * the scale of the rounding a deposit computed in a given precision can carry there */
    double* Gtouch;
    double* Qtouch;
} acc_t;

/* G_e += qw * int_P^R W1_e . dr on a straight piece inside tet t (2-pt Gauss-Legendre) */
static void deposit_segment(const mesh_t* M, int t, const double P[3], const double R[3], double qw,
                            acc_t* A) {
    static const double gl_s[2] = {0.21132486540518711775, 0.78867513459481288225};
    double g[4][3], d[3];
    grads(M, t, g);
    for (int i = 0; i < 3; ++i) d[i] = R[i] - P[i];
    double val[6] = {0, 0, 0, 0, 0, 0};
    for (int q = 0; q < 2; ++q) {
        double X[3], lam[4], w[3];
        for (int i = 0; i < 3; ++i) X[i] = P[i] + gl_s[q] * d[i];
        bary(M, t, X, lam);
        for (int k = 0; k < 6; ++k) {
            whitney1(lam, g, LE[k][0], LE[k][1], w);
            val[k] += 0.5 * (w[0] * d[0] + w[1] * d[1] + w[2] * d[2]);
        }
    }
    for (int k = 0; k < 6; ++k) {
        int64_t ed = M->te[6 * (int64_t)t + k];
        A->G[ed] += qw * val[k];
        A->Gabs[ed] += fabs(qw * val[k]);
        if (A->Gtouch) A->Gtouch[ed] += fabs(qw);
    }
}

static void deposit_charge(const mesh_t* M, int t, const double X[3], double qw, acc_t* A) {
    double lam[4];
    bary(M, t, X, lam);
    for (int k = 0; k < 4; ++k) {
        int64_t n = M->tv[4 * (int64_t)t + k];
        A->Q[n] += qw * lam[k];
        A->Qabs[n] += fabs(qw * lam[k]);
        if (A->Qtouch) A->Qtouch[n] += fabs(qw);
    }
}

/* optional record of the walk's pieces: the tet and start point of each piece */
typedef struct {
    int32_t* cell;
    double* start;
    int cap, n;
} trace_t;

static void trace_piece(trace_t* tr, int t, const double P[3]) {
    if (!tr) return;
    if (tr->n < tr->cap) {
        tr->cell[tr->n] = t;
        for (int i = 0; i < 3; ++i) tr->start[3 * tr->n + i] = P[i];
    }
    tr->n++;
}

/* walk X_a -> X_b from tet t; returns the final tet (-1 = absorbed), writes the stop point */
static int walk(const mesh_t* M, int t, const double Xa[3], const double Xb[3], double qw,
                int max_cross, acc_t* A, double Xstop[3], int* ncross, int* bound_hit, trace_t* tr) {
    double cur[3] = {Xa[0], Xa[1], Xa[2]};
    double la[4], lb[4];
    int entry = -1;
    bary(M, t, cur, la);
    *ncross = 0;
    *bound_hit = 0;
    for (int c = 0;; ++c) {
        bary(M, t, Xb, lb);
        int kx = -1;
        double smin = 0.0;
        for (int k = 0; k < 4; ++k) {
            if (k == entry || !(lb[k] < 0.0)) continue;
            double den = la[k] - lb[k];
            double s = den > 0.0 ? la[k] / den : 0.0;
            if (s < 0.0) s = 0.0;
            if (s > 1.0) s = 1.0;
            if (kx < 0 || s < smin) {
                kx = k;
                smin = s;
            }
        }
        if (kx < 0) {
            trace_piece(tr, t, cur);
            deposit_segment(M, t, cur, Xb, qw, A);
            deposit_charge(M, t, Xb, qw, A);
            Xstop[0] = Xb[0];
            Xstop[1] = Xb[1];
            Xstop[2] = Xb[2];
            return t;
        }
        if (c == max_cross) {
            /* bound reached: stop where the walk is */
            deposit_charge(M, t, cur, qw, A);
            Xstop[0] = cur[0];
            Xstop[1] = cur[1];
            Xstop[2] = cur[2];
            *bound_hit = 1;
            return t;
        }
        double Xc[3];
        for (int i = 0; i < 3; ++i) Xc[i] = cur[i] + smin * (Xb[i] - cur[i]);
        trace_piece(tr, t, cur);
        deposit_segment(M, t, cur, Xc, qw, A);
        int nt = M->nb[4 * (int64_t)t + kx];
        if (nt < 0) {
            deposit_charge(M, t, Xc, qw, A);
            Xstop[0] = Xc[0];
            Xstop[1] = Xc[1];
            Xstop[2] = Xc[2];
            *ncross = c + 1;
            return -1;
        }
        /* entry face of the neighbour = face opposite its vertex not shared with t */
        int ent = -1;
        for (int a = 0; a < 4; ++a) {
            int v = M->tv[4 * (int64_t)nt + a], shared = 0;
            for (int j = 0; j < 4; ++j) shared |= (M->tv[4 * (int64_t)t + j] == v);
            if (!shared) ent = a;
        }
        t = nt;
        entry = ent;
        cur[0] = Xc[0];
        cur[1] = Xc[1];
        cur[2] = Xc[2];
        bary(M, t, cur, la);
        *ncross = c + 1;
    }
}

typedef struct {
    int64_t ne, nn;
    double *G, *Gabs, *Q, *Qabs, *Gt, *Qt;
} thr_acc;

/*
 * One step for np particles of one species.  push=1: gather at X, Boris, X_b = X + dt v.
 * push=0: only walk from X to the given Xend (velocities untouched).
 * cell/X/V are updated in place; dG, dGabs, Q, Qabs are accumulated (dGtouch, Qtouch too
 * when not NULL).
 * Returns the number of particles that hit the crossing bound.
 */
int64_t oracle_step(int64_t ne, int64_t nn, const double* xyz, const int32_t* tv, const int32_t* te,
                    const int32_t* tf, const int32_t* nb, const double* e, const double* b, int64_t np,
                    int32_t* cell, double* X, double* V, double q, double m, double w, double dt,
                    int max_cross, int push, const double* Xend, double* dG, double* dGabs, double* Q,
                    double* Qabs, int32_t* ncross, int nthreads, double* dGtouch, double* Qtouch) {
    mesh_t M = {xyz, tv, te, tf, nb, e, b};
    double qw = q * w;
    int64_t nbound = 0;
    int T = 1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
    T = nthreads;
#endif
    thr_acc* acc = (thr_acc*)calloc((size_t)T, sizeof(thr_acc));
    for (int i = 0; i < T; ++i) {
        acc[i].G = (double*)calloc((size_t)ne, sizeof(double));
        acc[i].Gabs = (double*)calloc((size_t)ne, sizeof(double));
        acc[i].Q = (double*)calloc((size_t)nn, sizeof(double));
        acc[i].Qabs = (double*)calloc((size_t)nn, sizeof(double));
        acc[i].Gt = dGtouch ? (double*)calloc((size_t)ne, sizeof(double)) : NULL;
        acc[i].Qt = Qtouch ? (double*)calloc((size_t)nn, sizeof(double)) : NULL;
    }
#ifdef _OPENMP
#pragma omp parallel for num_threads(T) schedule(static) reduction(+ : nbound)
#endif
    for (int64_t p = 0; p < np; ++p) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        acc_t A = {acc[tid].G, acc[tid].Gabs, acc[tid].Q, acc[tid].Qabs, acc[tid].Gt, acc[tid].Qt};
        int t = cell[p];
        if (t < 0) {
            if (ncross) ncross[p] = 0;
            continue;
        }
        double Xa[3] = {X[3 * p], X[3 * p + 1], X[3 * p + 2]}, Xb[3];
        if (push) {
            double E[3], B[3], v[3] = {V[3 * p], V[3 * p + 1], V[3 * p + 2]};
            gather(&M, t, Xa, E, B);
            boris(v, E, B, q, m, dt);
            for (int i = 0; i < 3; ++i) {
                V[3 * p + i] = v[i];
                Xb[i] = Xa[i] + dt * v[i];
            }
        } else {
            for (int i = 0; i < 3; ++i) Xb[i] = Xend[3 * p + i];
        }
        double Xs[3];
        int nc = 0, hit = 0;
        int tn = walk(&M, t, Xa, Xb, qw, max_cross, &A, Xs, &nc, &hit, NULL);
        cell[p] = tn;
        for (int i = 0; i < 3; ++i) X[3 * p + i] = Xs[i];
        if (ncross) ncross[p] = nc;
        nbound += hit;
    }
    for (int i = 0; i < T; ++i) {
        for (int64_t k = 0; k < ne; ++k) {
            dG[k] += acc[i].G[k];
            dGabs[k] += acc[i].Gabs[k];
            if (dGtouch) dGtouch[k] += acc[i].Gt[k];
        }
        for (int64_t k = 0; k < nn; ++k) {
            Q[k] += acc[i].Q[k];
            Qabs[k] += acc[i].Qabs[k];
            if (Qtouch) Qtouch[k] += acc[i].Qt[k];
        }
        free(acc[i].G);
        free(acc[i].Gabs);
        free(acc[i].Q);
        free(acc[i].Qabs);
        free(acc[i].Gt);
        free(acc[i].Qt);
    }
    free(acc);
    return nbound;
}

/* E and B at particle positions (Whitney gather) */
void oracle_gather(const double* xyz, const int32_t* tv, const int32_t* te, const int32_t* tf,
                   const double* e, const double* b, int64_t np, const int32_t* cell, const double* X,
                   double* Eout, double* Bout) {
    mesh_t M = {xyz, tv, te, tf, NULL, e, b};
    for (int64_t p = 0; p < np; ++p) gather(&M, cell[p], X + 3 * p, Eout + 3 * p, Bout + 3 * p);
}

/* barycentric coordinates of points (for tests) */
void oracle_bary(const double* xyz, const int32_t* tv, int64_t np, const int32_t* cell, const double* X,
                 double* lam) {
    mesh_t M = {xyz, tv, NULL, NULL, NULL, NULL, NULL};
    for (int64_t p = 0; p < np; ++p) bary(&M, cell[p], X + 3 * p, lam + 4 * p);
}

/* Boris only (for the closed-form pins): E, B given per particle */
void oracle_boris(int64_t np, double* V, const double* E, const double* B, double q, double m, double dt) {
    for (int64_t p = 0; p < np; ++p) boris(V + 3 * p, E + 3 * p, B + 3 * p, q, m, dt);
}

/* W0 charge of particles at their positions */
void oracle_charge(const double* xyz, const int32_t* tv, int64_t nn, int64_t np, const int32_t* cell,
                   const double* X, double qw, double* Q, double* Qabs) {
    mesh_t M = {xyz, tv, NULL, NULL, NULL, NULL, NULL};
    acc_t A = {NULL, NULL, Q, Qabs, NULL, NULL};
    (void)nn;
    for (int64_t p = 0; p < np; ++p)
        if (cell[p] >= 0) deposit_charge(&M, cell[p], X + 3 * p, qw, &A);
}

/*
 * The pieces of one particle's walk from Xa (in tet t) to Xb, for tests: cells[k] and
 * start[3k..3k+2] are the tet and the start point of piece k (at most cap are stored);
 * the stop point (Xb, the wall point or the point where the crossing bound stopped the
 * walk) goes to stop[3] and the final tet (-1 = absorbed) to *end_cell.  Deposits go to
 * dG, dGabs, Q, Qabs as in oracle_step.  Returns the number of pieces.
 */
int oracle_walk_trace(int64_t ne, int64_t nn, const double* xyz, const int32_t* tv, const int32_t* te,
                      const int32_t* tf, const int32_t* nb, int t, const double* Xa, const double* Xb, double qw,
                      int max_cross, int cap, int32_t* cells, double* start, double* stop, int32_t* end_cell,
                      double* dG, double* dGabs, double* Q, double* Qabs) {
    mesh_t M = {xyz, tv, te, tf, nb, NULL, NULL};
    acc_t A = {dG, dGabs, Q, Qabs, NULL, NULL};
    trace_t tr = {cells, start, cap, 0};
    int nc = 0, hit = 0;
    (void)ne;
    (void)nn;
    *end_cell = walk(&M, t, Xa, Xb, qw, max_cross, &A, stop, &nc, &hit, &tr);
    return tr.n;
}
