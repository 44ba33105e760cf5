/*
 * fem_pic.h -- C ABI of the GB300 (sm_103a) charge-conserving FEM-PIC hot path.
 *
 * The method (arXiv 2103.06737, "Quasi-Helmholtz Decomposition, Gauss' Laws and
 * Charge Conservation for Finite Element Particle-in-Cell"):
 *   - fields on an unstructured tet mesh: E in span of Whitney-1 edge functions,
 *     B in span of Whitney-2 face functions (Sec. II.C);
 *   - point particles moved by the Lorentz force (Sec. II.A), non-relativistic;
 *   - the current deposit is the time-integrated current G_e = int W1_e . dr along
 *     each particle's path, and the node charge follows from it, so the discrete
 *     continuity equation D0^T dG = dQ holds analytically (Sec. IV.B.1);
 *   - [grad], [curl], [div] are the signed incidence matrices D0, D1, D2 (Sec. II.C).
 *
 * Conventions shared by every call:
 *   - Mesh numbering.  Tet vertices are taken in increasing global id
 *     (v0<v1<v2<v3); local edges are (01,02,03,12,13,23); local face k is opposite
 *     local vertex k.  Global edges are the sorted node pairs (i<j), global faces
 *     the sorted triples (i<j<k), each numbered in lexicographic order.  Edge DOF
 *     e_ij is the circulation of E along i->j; face DOF b_ijk the flux of B along
 *     (x_j-x_i)x(x_k-x_i).  D0[e,i]=-1, D0[e,j]=+1; D1[f,(i,j)]=D1[f,(j,k)]=+1,
 *     D1[f,(i,k)]=-1; D2[t,f_k]=s_t*(-1)^k with s_t the sign of the sorted tet's volume.
 *   - Boundary faces (one tet) are PEC walls: a particle reaching one is absorbed
 *     there and its charge stays on the wall nodes.
 *   - Particle state (caller-owned, device memory, struct-of-arrays): cell[n]
 *     (int32, the containing tet, -1 once absorbed), off[3*n] (planar x|y|z blocks:
 *     position minus the position of the cell's vertex v0), vel[3*n] (planar).
 *     off/vel are float in FP_FP32 mode and double in FP_FP64 mode.
 *   - Field DOFs e[N_e], b[N_f] are double (device).  Deposit outputs dG[N_e],
 *     Q[N_n] are float in FP_FP32 mode and double in FP_FP64 mode (device), or double in
 *     FP_FP32 mode after fem_pic_set_deposit_precision(ctx, FP_FP64).
 *   - All device work is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 *     stream) and is asynchronous unless stated.  Errors found by kernels (walk
 *     bound, invalid cell) are OR-ed into a device status word read by
 *     fem_pic_status().  No exception crosses the ABI; every call returns fp_status.
 *   - Ownership: the library owns the handle, its mesh tables and its scratch;
 *     the caller owns every pointer it passes.  Host pointers are read during the
 *     call only.
 */
#ifndef FEM_PIC_H
#define FEM_PIC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fem_pic fem_pic_t;

typedef enum {
    FP_OK = 0,
    FP_EINVAL = 1,   /* bad argument, size or pointer; invalid cell id; non-finite particle state */
    FP_ECUDA = 2,    /* a CUDA runtime call failed (text in fem_pic_last_error) */
    FP_EWALK = 3,    /* a particle hit the crossing bound of the tet walk */
    FP_ENOCONV = 4,  /* an iterative solve reached its iteration cap */
    FP_EGEOM = 5     /* a tet with zero volume, or a non-manifold face */
} fp_status;

enum { FP_FP64 = 0, FP_FP32 = 1 };

/* fem_pic_push_deposit flags */
enum {
    FP_ACCUMULATE = 1, /* add into dG and Q instead of overwriting them */
    FP_NO_AGGREGATE = 2, /* one global atomic per contribution (no warp aggregation) */
    FP_SAME_FIELDS = 4, /* e and b are those of this handle's previous push call, unchanged since:
                           its per-tet field records are reused (e.g. the second species of a step) */
    FP_CHARGE_CHANGE = 8 /* Q receives the change of the W0 charge over the step (see
                            fem_pic_push_deposit) instead of the charge at the end point */
};

typedef struct {
    int64_t n_nodes;
    int64_t n_tets;
    const double* xyz;   /* host [3*n_nodes], interleaved x,y,z per node */
    const int32_t* tet;  /* host [4*n_tets], node ids, any order */
} fp_mesh;

/* CSR matrix with int8 values (incidence), host memory */
typedef struct {
    int64_t n_rows, n_cols, nnz;
    const int32_t* row_ptr; /* [n_rows+1] */
    const int32_t* col;     /* [nnz], increasing within a row */
    const int8_t* val;      /* [nnz] */
} fp_csr_i8;

typedef struct {
    int64_t n;        /* number of particles */
    int32_t* cell;    /* device [n] */
    void* off;        /* device [3*n], float or double per precision */
    void* vel;        /* device [3*n], float or double per precision */
    double q;         /* charge of one physical particle (C) */
    double m;         /* mass of one physical particle (kg) */
    double w;         /* macro weight: physical particles per macro-particle */
} fp_particles;

/*
 * Build the discrete complex {N,E,F,T} of a tet mesh (Sec. II.C) and upload the
 * per-tet tables.  D0, D1, D2 may be NULL; when given they are checked entry by
 * entry against the library's own derivation (same numbering as above) and a
 * mismatch returns FP_EINVAL.  precision is FP_FP64 or FP_FP32 (particle path).
 * Uses the current CUDA device.  Synchronous.  *out is NULL on failure.
 */
fp_status fem_pic_create(const fp_mesh* mesh, const fp_csr_i8* D0, const fp_csr_i8* D1,
                         const fp_csr_i8* D2, int precision, fem_pic_t** out);

/* Free the handle and every device buffer it owns (synchronises the device). */
void fem_pic_destroy(fem_pic_t* ctx);

/* Text of the last error on this handle (or of the last failed create if ctx is NULL). */
const char* fem_pic_last_error(const fem_pic_t* ctx);

/* sizes[0..3] = N_n, N_e, N_f, N_t; sizes[4] = precision */
fp_status fem_pic_sizes(const fem_pic_t* ctx, int64_t sizes[5]);

/*
 * Element type of the deposit arrays of an FP32 context: the W1 current dG and the W0 charge Q
 * of Sec. IV.B.1 (Eq. for Gbar and rhobar) as fem_pic_push_deposit, fem_pic_push_deposit_static
 * and fem_pic_deposit_charge write them, and as fem_pic_field_step, fem_pic_field_initial,
 * fem_pic_residuals and the comparison steps (fem_pic_mfem_*, fem_pic_wave_step) read them.
 *   FP_FP32 (the default of an FP32 context): float arrays, accumulated with FP32 atomics.
 *   FP_FP64: double arrays.  The particle arithmetic stays FP32: each particle's
 *            contributions, and the fast push's sums over a run of particles in one tet, are
 *            formed in FP32 and added into the arrays with FP64 atomics.  The arrays then keep
 *            charge continuity (D0^T dG against the change of Q) about ten times closer than
 *            FP32 arrays, whose atomic sums round at the scale of each entry's total, and the
 *            Gauss-law projection of the field step, which corrects exactly that residual,
 *            needs fewer iterations.  (A float contribution below 1.2e-38 in magnitude, a
 *            subnormal, may add zero: some kernels widen floats through their bit patterns.)
 *            The charge change into a double Q (FP_CHARGE_CHANGE,
 *            fem_pic_set_charge_precision) keeps it closer still, with float dG.
 * An FP64 context always deposits in FP64 (FP_FP64 accepted, FP_FP32 -> FP_EINVAL).  The FP32
 * Adams mover (fem_pic_push_deposit_adams) takes FP32 deposits only (FP_EINVAL otherwise).
 * FP_FP32 sets Q back to float as well (see fem_pic_set_charge_precision).
 * The setting applies to calls made after it; arrays already passed keep their type.
 */
fp_status fem_pic_set_deposit_precision(fem_pic_t* ctx, int precision);

/* FP_FP32 or FP_FP64: the element type of this context's dG array, and of Q unless
 * fem_pic_set_charge_precision changed it (-1 for NULL). */
int fem_pic_deposit_precision(const fem_pic_t* ctx);

/*
 * Element type of the charge array Q alone (fem_pic_set_deposit_precision sets dG and Q
 * together).  FP_FP64 with float dG suits FP_CHARGE_CHANGE: the step's charge change
 * q w (lambda^end - lambda^start) is added onto the previous step's Q in FP64, so Q^{n+1}
 * keeps continuity with D0^T dG to the rounding of the FP32 per-particle terms instead of
 * the rounding of the FP32 sums of whole node charges.  FP_FP32 while dG is double, or in
 * an FP64 context, is FP_EINVAL.  Applies to calls made after it.  Q's element type is
 * what fem_pic_charge_precision returns, for every call that takes Q (the push calls,
 * fem_pic_deposit_charge, fem_pic_field_step, fem_pic_field_initial, fem_pic_residuals
 * and the comparison steps).
 */
fp_status fem_pic_set_charge_precision(fem_pic_t* ctx, int precision);

/* FP_FP32 or FP_FP64: the element type of this context's Q array (-1 for NULL). */
int fem_pic_charge_precision(const fem_pic_t* ctx);

/*
 * Copy incidence matrix `which` (0: D0, 1: D1, 2: D2) to caller host buffers.
 * row_ptr [n_rows+1], col [nnz], val [nnz]; nnz = 2 N_e, 3 N_f, 4 N_t.  Synchronous.
 */
fp_status fem_pic_incidence(const fem_pic_t* ctx, int which, int32_t* row_ptr, int32_t* col,
                            int8_t* val);

/*
 * Copy topology tables to host: tet_nodes [4 N_t] (sorted vertex ids), tet_edges
 * [6 N_t], tet_faces [4 N_t], tet_neigh [4 N_t] (-1 = wall).  Any may be NULL.
 */
fp_status fem_pic_topology(const fem_pic_t* ctx, int32_t* tet_nodes, int32_t* tet_edges,
                           int32_t* tet_faces, int32_t* tet_neigh);

/*
 * DOFs of uniform fields E0, B0 (host double[3] each): e_ij = E0.(x_j-x_i),
 * b_ijk = B0.(x_j-x_i)x(x_k-x_i)/2, written to device e[N_e], b[N_f] (either may
 * be NULL).  The W1/W2 interpolants of these DOFs reproduce E0 and B0 exactly.
 */
fp_status fem_pic_project_uniform(fem_pic_t* ctx, const double E0[3], const double B0[3], double* e,
                                  double* b, void* stream);

/*
 * Load particles: X (device double [3*n], interleaved x,y,z) with their containing
 * tets cell[n] (device) -> off (device [3*n] planar, float/double per precision).
 * A cell id outside [0,N_t) sets FP_EINVAL in the status word.
 */
fp_status fem_pic_particles_from_global(fem_pic_t* ctx, int64_t n, const int32_t* cell,
                                        const double* X, void* off, void* stream);

/* Positions back to global coordinates: X (device double [3*n], interleaved). */
fp_status fem_pic_particles_to_global(fem_pic_t* ctx, int64_t n, const int32_t* cell,
                                      const void* off, double* X, void* stream);

/*
 * THE HOT PATH: one particle step of one species (Sec. II.A, II.C, IV.B.1).
 * For each live particle: barycentric coordinates lambda in its tet; gather
 * E = sum e_k W1_k(lambda) from e and B = sum b_f W2_f(lambda) from b; Boris push
 * v <- v(E,B,q/m,dt); straight path x -> x + dt v walked tet to tet (exit tests in
 * FP64); on every piece inside tet T from lambda^a to lambda^c the Whitney-1 path
 * integral dG_ij += q w (lambda^a_i lambda^c_j - lambda^a_j lambda^c_i) on T's
 * 6 edges; at the end point Q_n += q w lambda_n on the end tet's 4 nodes
 * (Whitney-0 charge).  Reaching a wall absorbs the particle (cell = -1, charge at the
 * wall point); more than max_cross crossings stops it at its last crossing point and
 * sets FP_EWALK in the status word.  A particle whose position or velocity, given or
 * pushed, is not finite (NaN or Inf, e.g. from a non-finite field DOF) is removed
 * (cell = -1) with nothing deposited and sets FP_EINVAL in the status word, so dG and Q
 * stay finite.  dG and Q are zeroed first unless FP_ACCUMULATE.
 * With FP_CHARGE_CHANGE, Q is never zeroed and receives q w (lambda^end_n - lambda^start_n)
 * per particle instead (the start charge subtracted on the start tet's nodes, the end charge
 * added on the end tet's; a particle that stays in its tet adds the difference once; a
 * removed particle with a finite start subtracts its start charge): a Q that holds the
 * charge of the start positions (fem_pic_deposit_charge, or the previous step) becomes the
 * charge of the end positions.  dG is zeroed unless FP_ACCUMULATE, as without the flag.
 * (A particle absorbed by a PEC wall leaves its charge on the wall's nodes, in this step as
 * without the flag, and a carried Q keeps it there in later steps; wall nodes are fixed in
 * the Gauss-law solve, so the field step does not read it.)
 * The change equals D0^T dG exactly in real arithmetic (the continuity equation of
 * Sec. II.A), so FP32 rounding touches only the change, not the node charges.
 * Particle arrays are updated in place.  Asynchronous.
 */
fp_status fem_pic_push_deposit(fem_pic_t* ctx, const double* e, const double* b,
                               const fp_particles* p, double dt, int max_cross, void* dG, void* Q,
                               int flags, void* stream);

/*
 * Same step as fem_pic_push_deposit, for callers that must not allocate device
 * memory once they are running (a memory budget fixed at start-up, an allocator
 * that refuses new device allocations, a framework that only passes in buffers it
 * already owns).  The paper has no counterpart: this is a property of the library.
 * fem_pic_push_deposit keeps the particles it hands to the FP64 walk in a queue it
 * grows with cudaMalloc; here that queue is a fixed array inside the library
 * (4,194,304 entries, 16 MiB, held on every device that loads the library until the
 * process exits).  The call allocates nothing: p->n above 4,194,304 returns
 * FP_EINVAL with nothing launched.  fem_pic_create (FP_FP32) looks up the array's
 * device address in the handle's context (cudaGetSymbolAddress) and keeps it in the
 * handle.  All calls on a device share the array and it keeps the last call's contents
 * (each call clears the count it needs), so calls whose GPU work overlaps (other
 * streams, other threads, other handles) race on it: serialise them.  It runs the same
 * kernels as fem_pic_push_deposit (the staged pipeline when n is a multiple of 4 and the
 * state arrays are 16-byte aligned, the grid-stride kernel otherwise).  In FP_FP64 mode no
 * queue is used and the call behaves like fem_pic_push_deposit.
 */
fp_status fem_pic_push_deposit_static(fem_pic_t* ctx, const double* e, const double* b,
                                      const fp_particles* p, double dt, int max_cross, void* dG,
                                      void* Q, int flags, void* stream);

/*
 * One particle step of one species with the fourth-order Adams mover (Sec. IV.B.2 moves
 * the particles with a fourth-order Adams method and leaves its details to another paper;
 * read here as explicit Adams-Bashforth on dx/dt = v, dv/dt = (q/m)(E(x) + v x B(x))).
 * x and v are at the same time level (no leapfrog staggering).  Per live particle:
 * E, B gathered at x^n as in fem_pic_push_deposit; a^n = (q/m)(E + v^n x B);
 *   x^{n+1} = x^n + dt sum_{j<k} beta_{k,j} v^{n-j},  v^{n+1} = v^n + dt sum_{j<k} beta_{k,j} a^{n-j}
 * with the k-step Adams-Bashforth coefficients, k = min(step + 1, 4) (orders 1, 2, 3 start
 * the method); then the walk and the Whitney-1 / Whitney-0 deposits along the straight
 * segment x^n -> x^{n+1}, exactly as in fem_pic_push_deposit (continuity holds the same way).
 * The fields are those passed in (time level n) for the whole step.
 *   hist: device array of 18*n reals (float in FP_FP32 mode, double in FP_FP64 mode),
 *         caller-owned, planar: slot s (0..2) holds v at planes 6s..6s+2 and a at planes
 *         6s+3..6s+5 (plane c is hist[c*n .. c*n+n)).  Slot (step - j) mod 3 must hold
 *         f^{n-j} = (v^{n-j}, a^{n-j}) for j = 1..min(step, 3); the call writes f^n into slot
 *         step mod 3 of each live particle (other slots are left alone).  Contents are
 *         ignored on step 0 (nothing needs initialising).
 *   step: number of earlier Adams steps of these particles (>= 0); the caller counts.
 * The position sum is rounded operation by operation without fused multiply-adds, in
 * this order: h = beta_1 v^{n-1}, h += beta_2 v^{n-2}, h += beta_3 v^{n-3} (the terms the
 * order has), s = beta_0 v^n + h (s = beta_0 v^n at order 1), x^{n+1} = x^n + dt s.  Absorbed particles
 * (cell -1) are left alone.  A particle's history must move with it: sort with
 * fem_pic_sort_columns(..., hist, hist_sorted, 18, ...).  The explicit method is stable for
 * gyration only while omega_c dt stays below about 0.43.  dG and Q are zeroed first unless
 * FP_ACCUMULATE.  Errors and asynchrony as fem_pic_push_deposit; hist NULL with n > 0,
 * step < 0, FP_CHARGE_CHANGE, or double dG or Q in FP_FP32 mode return FP_EINVAL.
 */
fp_status fem_pic_push_deposit_adams(fem_pic_t* ctx, const double* e, const double* b,
                                     const fp_particles* p, void* hist, int64_t step, double dt,
                                     int max_cross, void* dG, void* Q, int flags, void* stream);

/*
 * Whitney-0 charge of the particles at their current positions:
 * Q_n (+)= q w lambda_n (Sec. IV.B.1, the node charge the continuity equation pairs
 * with dG).  Q is zeroed first unless FP_ACCUMULATE.  Asynchronous.
 */
fp_status fem_pic_deposit_charge(fem_pic_t* ctx, const fp_particles* p, void* Q, int flags,
                                 void* stream);

/*
 * Counting sort of one species by cell (dead particles last): src -> dst, both
 * caller-owned with the same n, q, m, w; src is not modified.  Keeps particles of a
 * cell together so the push reads each tet's tables once per run of particles and
 * aggregates deposits before its global atomics.  Uses library-owned scratch
 * (grown on demand, kept until destroy).  Asynchronous.
 */
fp_status fem_pic_sort(fem_pic_t* ctx, const fp_particles* src, fp_particles* dst, void* stream);

/*
 * fem_pic_sort that also moves ncols planar columns of per-particle data (device,
 * float in FP_FP32 mode and double in FP_FP64 mode, column k at cols[k*n .. k*n+n)) with
 * the same permutation: cols_src -> cols_dst (caller-owned, not aliased).  Used for the
 * Adams history (ncols = 18).  ncols = 0 is fem_pic_sort.  Asynchronous.
 */
fp_status fem_pic_sort_columns(fem_pic_t* ctx, const fp_particles* src, fp_particles* dst,
                               const void* cols_src, void* cols_dst, int ncols, void* stream);

/*
 * Invariant residuals, sums in FP64 (Sec. II.A continuity, Sec. IV.B.1, Sec. V item 5):
 *   out[0] = max_n |(D0^T dG)_n - (Q_new - Q_old)_n| over all nodes,  out[1] = max_n of
 *            the sum of the absolute values of those terms (scale, accumulated in FP32);
 *   out[2] = max_t |(D2 b)_t|,  out[3] = max_f |b_f| (scale; a row of D2 has 4 terms);
 *   out[4], out[5] = as out[0], out[1] over interior nodes only (charge absorbed by a
 *            PEC wall in an earlier step leaves the particle set, so over several
 *            steps continuity is checked where the field solve uses it).
 * dG has the deposit precision (fem_pic_deposit_precision), Q_new and Q_old the charge
 * precision (fem_pic_charge_precision); b is double.  Any
 * input may be NULL (its entries are then 0).  out is device double[6].  Asynchronous.
 */
fp_status fem_pic_residuals(fem_pic_t* ctx, const void* dG, const void* Q_new, const void* Q_old,
                            const double* b, double* out, void* stream);

/* ------------------------------------------------------------------ implicit field step */

enum { FP_SYS_NEWMARK = 0, FP_SYS_GAUSS = 1 };
/* FP_PC_JACOBI: Jacobi-PCG by mixed-precision iterative refinement (FP64 residual and dot
 * products, FP32 inner solves); FP_PC_JACOBI_FP64: plain Jacobi-PCG entirely in FP64;
 * FP_PC_LEARNED: learned correction of the Newmark solve's starting point with fallback,
 * FP_PC_LEARNED_GAUSS: the same for the Gauss-law projection (see fem_pic_learned_*).
 * fem_pic_field_step takes an OR of these bits (FP_PC_JACOBI = none of them). */
enum { FP_PC_JACOBI = 0, FP_PC_LEARNED = 1, FP_PC_JACOBI_FP64 = 2, FP_PC_LEARNED_GAUSS = 4 };

typedef struct {
    int32_t iters;     /* CG iterations taken (inner iterations for the mixed solver) */
    int32_t precond;   /* preconditioner used (FP_PC_*) */
    int32_t fell_back; /* 1 if a learned solve fell back to plain Jacobi-CG */
    int32_t outer;     /* refinement steps (mixed solver), 0 for plain FP64 PCG */
    double rel_res;    /* final ||r|| / ||reference|| (see each call) */
    double abs_res;    /* final ||r|| */
    double ms;         /* device time of the solve when measured, else 0 */
} fp_solve_info;

/*
 * Assemble the FP64 field operators of Sec. II.C for time step dt, permittivity eps,
 * permeability mu, and upload them as CSR matrices:
 *   M = [*eps] (edge mass, <W1_i, eps W1_j>), S = [*S] = [curl]^T [*mu^-1] [curl]
 *   (Eq. wave_cont), A = M + dt^2/4 S (Newmark beta = 1/4), L = D0^T M D0 (the discrete
 *   Laplacian of Eq. discreteGauss).
 * PEC walls: edges and nodes on boundary faces are fixed at zero (their rows keep a unit
 * diagonal, their columns are removed).  Replaces any earlier setup.  Synchronous.
 */
fp_status fem_pic_field_setup(fem_pic_t* ctx, double dt, double eps, double mu);

/* Field boundary conditions: FP_BC_PEC (the default of fem_pic_field_setup) fixes the
 * tangential E on boundary edges and the projection's correction on boundary nodes at zero;
 * FP_BC_NEUMANN is the natural boundary (nothing fixed).  Then the node Laplacian L is
 * singular (its null space the constants) and the Gauss-law projection takes the zero-mean
 * constraint of Eq. zero_mean_constraint (Sec. IV.B): d = C_z y with alpha^T d = 0 (alpha_n
 * the integral of W0_n), which solves L d = g - (sum g / sum alpha) alpha, i.e. a net charge
 * is spread as a uniform background, as the paper asks when the net charge is not zero.
 * The library solves that consistent system with the same CG and shifts d to alpha^T d = 0.
 * Particles are absorbed at the boundary under either condition. */
enum { FP_BC_PEC = 0, FP_BC_NEUMANN = 1 };

/* fem_pic_field_setup with a boundary condition bc (FP_BC_*); FP_EINVAL for another bc. */
fp_status fem_pic_field_setup_bc(fem_pic_t* ctx, double dt, double eps, double mu, int bc);

/* nnz[0] = entries of the edge operators (M, S, A), nnz[1] = entries of L. */
fp_status fem_pic_field_nnz(const fem_pic_t* ctx, int64_t nnz[2]);

/*
 * Copy operator `which` (0 M, 1 S, 2 A, 3 L) to host CSR buffers: row_ptr [rows+1],
 * col [nnz], val [nnz] (any may be NULL).  Rows = N_e for 0..2, N_n for 3.
 */
fp_status fem_pic_field_matrix(const fem_pic_t* ctx, int which, int32_t* row_ptr, int32_t* col,
                               double* val);

/*
 * Solve A x = rhs (FP_SYS_NEWMARK, edges) or L x = rhs (FP_SYS_GAUSS, nodes) with
 * Jacobi-preconditioned CG (precond, see FP_PC_*), starting from the x passed in (device, in/out),
 * until ||rhs - A x|| <= tol ||rhs|| or max_iter iterations.  rhs must be zero on PEC
 * rows.  info (host, may be NULL) is filled after a stream synchronisation; with info
 * a solve that stops at max_iter returns FP_ENOCONV, otherwise the status word records it.
 */
fp_status fem_pic_field_solve(fem_pic_t* ctx, int system, const double* rhs, double* x, double tol,
                              int max_iter, int precond, fp_solve_info* info, void* stream);

/*
 * One implicit field step (Sec. IV.B with Newmark-beta, beta = 1/4, gamma = 1/2):
 *   1. (M + dt^2/4 S) E^N = M(2E^n - E^{n-1}) - dt^2 S(E^n/2 + E^{n-1}/4)
 *                            - (dG^{n+1/2} - dG^{n-1/2}),
 *      CG from the guess 2E^n - E^{n-1}, to ||r|| <= tol ||rhs||;
 *   2. Gauss-law projection (Eq. discreteGauss, modified projector Eq. efld_mod_proj):
 *      L d = D0^T M E^N + Q^{n+1} on interior nodes, CG from 0 to ||r|| <= tol ||Q||
 *      (the residual of this solve is the Gauss-law residual D0^T M E^{n+1} + Q^{n+1});
 *      E^{n+1} = E^N - D0 d;
 *   3. Faraday: b <- b - dt D1 (E^{n+1} + E^n)/2 (skipped if b is NULL).
 * E_prev = E^{n-1}, E_cur = E^n (device double [N_e]); E_next receives E^{n+1} (distinct
 * buffer); dG_half = dG^{n+1/2} (the deposit of the push that used E^n), dG_prev =
 * dG^{n-1/2} (NULL = 0), Q_new = Q^{n+1} (charge precision).  info[2] (host, may be
 * NULL): the Newmark and Gauss solves; with info, FP_ENOCONV if either missed tol.
 */
fp_status fem_pic_field_step(fem_pic_t* ctx, const double* E_prev, const double* E_cur, double* E_next,
                             double* b, const void* dG_half, const void* dG_prev, const void* Q_new,
                             double tol, int max_iter, int precond, fp_solve_info info[2],
                             void* stream);

/*
 * Initial field: E (device double [N_e]) with D0^T M E + Q = 0 at interior nodes and no
 * solenoidal part (the Gauss-law projection of E = 0), CG to ||r|| <= tol ||Q||.  Q has the
 * charge precision (fem_pic_charge_precision).
 */
fp_status fem_pic_field_initial(fem_pic_t* ctx, const void* Q, double* E, double tol, int max_iter,
                                fp_solve_info* info, void* stream);

/* ------------------------------------------- comparison systems of the field solve (Sec. V, VI) */

/*
 * Handle for the systems the paper compares the quasi-Helmholtz step with, and for the
 * Gauss-law residual.  Made from the field setup of ctx (fem_pic_field_setup first); it
 * holds the face mass [*mu^-1]_fg = integral of W2_f . mu^-1 W2_g (Sec. II.C, every face
 * free), the transpose of [curl] = D1, and scratch.  Owned by the library: destroy it
 * before ctx.  Calls made after a new fem_pic_field_setup return FP_EINVAL.  Create returns
 * FP_EINVAL without a field setup or when host memory runs out, FP_ECUDA when a device
 * allocation fails (*out is then NULL).
 */
typedef struct fem_pic_mfem fem_pic_mfem_t;
fp_status fem_pic_mfem_create(fem_pic_t* ctx, fem_pic_mfem_t** out);
void fem_pic_mfem_destroy(fem_pic_mfem_t* m);

/* Host copy of the face mass in CSR (rows N_f, sorted columns): nnz, row_ptr [N_f+1], col
 * [nnz], val [nnz]; any may be NULL (call with NULL arrays first to size them). */
fp_status fem_pic_mfem_face_mass(const fem_pic_mfem_t* m, int64_t* nnz, int32_t* row_ptr, int32_t* col,
                                 double* val);

/*
 * One step of the first-order mixed FEM (MFEM) of Eq. maxwell_semi with Newmark (beta = 1/4,
 * gamma = 1/2), the trapezoidal rule for a first-order system, and NO Gauss-law projection:
 *   (M + dt^2/4 S) E^{n+1} = (M - dt^2/4 S) E^n + dt [curl]^T [*mu^-1] b^n - dG^{n+1/2}
 *   b^{n+1} = b^n - dt [curl] (E^{n+1} + E^n)/2
 * with M = [*eps], S = [*S] and dt of the field setup.  E_cur = E^n, E_next receives E^{n+1}
 * (device double [N_e], distinct buffers); b (device double [N_f], all faces) is updated in
 * place; dG_half (deposit precision [N_e], NULL = 0) is the step's deposit.  The Newmark
 * system is solved by fem_pic_field_solve from the start E^n (precond: FP_PC_JACOBI or
 * FP_PC_JACOBI_FP64; tol, max_iter and info as there, FP_ENOCONV after a finished step whose
 * solve missed tol).  With E^0 a gradient and the same deposits it gives the E of
 * fem_pic_wave_step; unlike it, a gradient error in E stays constant instead of growing (Sec. V).
 */
fp_status fem_pic_mfem_step(fem_pic_mfem_t* m, const double* E_cur, double* E_next, double* b,
                            const void* dG_half, double tol, int max_iter, int precond, fp_solve_info* info,
                            void* stream);

/*
 * Newmark on the wave equation (Eq. wave_cont) without the Gauss-law projection: steps 1 and 3
 * of fem_pic_field_step (the wave-equation FEM of Sec. V, whose gradient null space grows
 * linearly in time).  Arguments as there (b may be NULL: no Faraday update); solved by
 * fem_pic_field_solve from 2E^n - E^{n-1}, precond and errors as fem_pic_mfem_step.
 */
fp_status fem_pic_wave_step(fem_pic_mfem_t* m, const double* E_prev, const double* E_cur, double* E_next,
                            double* b, const void* dG_half, const void* dG_prev, double tol, int max_iter,
                            int precond, fp_solve_info* info, void* stream);

/*
 * Gauss-law residual g = D0^T [*eps] E + Q (Eq. discreteGauss) on the free nodes, in FP64:
 * out[0] = max |g_n|, out[1] = max over the same nodes of |Q_n| + sum over incident edges of
 * |([*eps] E)_e| (the scale).  Natural boundary: g less (sum Q / sum alpha) alpha, the net
 * charge the zero-mean constraint spreads.  E device double [N_e], Q charge precision [N_n]
 * (NULL = 0), out device double [2].  Asynchronous.
 */
fp_status fem_pic_mfem_gauss_residual(fem_pic_mfem_t* m, const double* E, const void* Q, double* out,
                                      void* stream);

/*
 * Solver per system, overriding the precond argument of the solve calls: newmark_solver
 * and gauss_solver are FP_PC_JACOBI (mixed-precision refinement), FP_PC_JACOBI_FP64, or
 * -1 (use the precond passed to each call).  inner_tol in (0,1): residual reduction of each
 * FP32 inner solve of the mixed solver (default 1e-5).
 */
fp_status fem_pic_field_options(fem_pic_t* ctx, int newmark_solver, int gauss_solver, double inner_tol);

/*
 * Preconditioner of the mixed solver's FP32 inner solves for one system (FP_SYS_NEWMARK or
 * FP_SYS_GAUSS): degree 1 is Jacobi (the default); degree 2..16 is the Chebyshev polynomial of
 * that degree in D^-1 A, on the interval [b / ratio, b] with b 5% above a Lanczos estimate of
 * the largest eigenvalue of D^-1 A (made at fem_pic_field_setup).  A degree-m polynomial costs
 * m - 1 products and grid barriers per CG iteration and no extra reductions.  Not from the
 * paper (it defers its solver); the stopping test is unchanged.  FP_EINVAL for a degree
 * outside [1, 16] or ratio <= 1.
 */
fp_status fem_pic_field_poly(fem_pic_t* ctx, int system, int degree, double ratio);

/* Iteration counts and residuals of the last Newmark (info[0]) and Gauss (info[1]) solves.
 * Synchronises the stream. */
fp_status fem_pic_field_last_info(fem_pic_t* ctx, fp_solve_info info[2], void* stream);

/*
 * alpha^0_n = integral over the domain of W0_n = sum over tets containing n of |T|/4
 * (the alpha of Sec. IV.B, used for zero-mean constraints and for a uniform background
 * charge Q_n = rho alpha^0_n).  alpha: host double [N_n].  Synchronous.
 */
fp_status fem_pic_whitney0_integrals(const fem_pic_t* ctx, double* alpha);

/* ------------------------------------------------------------------ learned correction
 * Not in the paper (it defers its solver details).  A message-passing network on the graph
 * of one system's operator (Newmark: graph nodes are the edge DOFs, graph edges the
 * nonzeros of A; Gauss-law projection: the node DOFs and the nonzeros of L), 3 layers of 64
 * features, BF16 weights with FP32 accumulation (tensor-core GEMMs), maps the Jacobi-scaled
 * residual of the solve's starting point (Newmark: 2E^n - E^{n-1}; projection: 0) to a
 * correction.  With FP_PC_LEARNED (Newmark) or FP_PC_LEARNED_GAUSS (projection) in the
 * precond bits of fem_pic_field_step the corrected start is used only when its FP64
 * residual is smaller than the plain one's (else fell_back = 1 in that system's info); the
 * CG then runs to the same tolerance either way.  Each system has its own network; the
 * fem_pic_learned_* calls address the system chosen by fem_pic_learned_select (Newmark
 * until then).  Requires fem_pic_field_setup; a new setup discards the networks.  Vectors
 * called [N] below have N_e entries for the Newmark system and N_n for the Gauss system. */

/* Choose the system (FP_SYS_NEWMARK or FP_SYS_GAUSS) later fem_pic_learned_* calls address. */
fp_status fem_pic_learned_select(fem_pic_t* ctx, int system);

/* Allocate and initialise the network (seeded) and a store for sample_capacity training
 * residuals.  Synchronous.  Same as fem_pic_learned_init_model(..., FP_LEARNED_GUESS). */
fp_status fem_pic_learned_init(fem_pic_t* ctx, uint64_t seed, int sample_capacity);

/*
 * The two uses of the network (the model of the selected system's network):
 *   FP_LEARNED_GUESS: the start correction described above.
 *   FP_LEARNED_PRECOND: a learned preconditioner inside the CG iteration.  The network runs
 *     on a static input (the Jacobi-scaled row sums of the operator) and its features h
 *     define, for every stored entry of the operator (Jacobi-scaled: A~ = D^-1/2 A D^-1/2),
 *       Delta~_ii = d0 + sum_f v_f h_if^2,   Delta~_ij = A~_ij (b0 + sum_f w_f h_if h_jf),
 *     symmetric by construction; the mixed solver's inner CG then uses
 *       z = D^-1 r + D^-1/2 Delta~ D^-1/2 r
 *     instead of z = D^-1 r (Delta~ = 0 is Jacobi; w = v = 0 a degree-1 polynomial in
 *     D^-1 A), one product on the operator's pattern per iteration.  Training minimises the
 *     mean over samples of ||A~ (r~ + Delta~ r~) - r~||^2 / ||r~||^2 (r~ = D^-1/2 r scaled to
 *     unit RMS), the residual one application leaves, over residuals the method produces,
 *     in mini-batches of 8.  fem_pic_learned_build makes the correction from the current
 *     weights; FP_PC_LEARNED / FP_PC_LEARNED_GAUSS (fem_pic_field_step) or FP_PC_LEARNED
 *     (fem_pic_field_solve, either system) then use it in the mixed solver (the FP64 solver
 *     ignores it).  If an inner iteration finds p.Ap <= 0 (the learned operator is not
 *     positive there) the solve falls back to Jacobi for the rest of the call
 *     (fell_back = 1).  The weights do not depend on the mesh size: weights trained on one
 *     mesh (fem_pic_learned_params) can be set on another of the same kind.
 */
enum { FP_LEARNED_GUESS = 0, FP_LEARNED_PRECOND = 1 };
fp_status fem_pic_learned_init_model(fem_pic_t* ctx, uint64_t seed, int sample_capacity, int model);

/* FP_LEARNED_PRECOND: the preconditioner's correction from the current weights, for the
 * solver (asynchronous).  Call after training or after setting the weights. */
fp_status fem_pic_learned_build(fem_pic_t* ctx, void* stream);

/* FP_LEARNED_PRECOND, for tests: Delta~ per entry of the system's operator in CSR order
 * (fem_pic_field_matrix's pattern; device float [nnz]) and the static input (device float
 * [N], may be NULL). */
fp_status fem_pic_learned_delta(fem_pic_t* ctx, float* delta_out, float* xin_out, void* stream);

/* collect != 0: every fem_pic_field_step stores the residual of the system's plain start
 * (ring buffer; eager launches only: a captured graph would replay one slot).
 * active != 0: use the network in fem_pic_field_solve-independent steps as with
 * FP_PC_LEARNED. */
fp_status fem_pic_learned_mode(fem_pic_t* ctx, int collect, int active);

/* Number of stored samples. */
fp_status fem_pic_learned_samples(fem_pic_t* ctx, int* count);

/* Train on stored samples [first, first+count) for `epochs` passes (Adam, cosine-decayed
 * learning rate lr, shuffled with seed).  loss (host [epochs], may be NULL): mean
 * ||A~ c~ - r~||^2 / ||r~||^2 per epoch.  Synchronous per epoch. */
fp_status fem_pic_learned_train(fem_pic_t* ctx, int first, int count, int epochs, double lr, uint64_t seed,
                                double* loss, void* stream);

/* ratio[k] = ||A~ c~ - r~||^2 / ||r~||^2 of stored sample first+k (held-out evaluation). */
fp_status fem_pic_learned_eval(fem_pic_t* ctx, int first, int count, double* ratio, void* stream);

/* Parameters (FP32 master copy): get and/or set host arrays of *n_params floats. */
fp_status fem_pic_learned_params(fem_pic_t* ctx, float* get, const float* set, int64_t* n_params);

/* FP_LEARNED_GUESS: forward pass on one residual r (device double [N]): writes c~ and r~
 * (device float [N]). */
fp_status fem_pic_learned_forward(fem_pic_t* ctx, const double* r, float* ct_out, float* rt_out,
                                  void* stream);

/* Loss gradient for one residual r (device float [N]) into grad_out (host float
 * [n_params], n_params of the network's model); the weights and optimizer state are left
 * unchanged.  Synchronous. */
fp_status fem_pic_learned_gradient(fem_pic_t* ctx, const float* r, float* grad_out, double* loss,
                                   void* stream);

/*
 * Optional per-phase timing (not part of the method).  When enabled, the library
 * records a pair of CUDA events on the launch stream around each of its kernels,
 * by phase: 0 field-coefficient prep, 1 FP32 push, 2 FP64 walk of deferred particles,
 * 3 FP64-mode push, 4 charge deposit, 5 sort, 6 residuals, 7 field-step kernels other than
 * the solvers, 8 Newmark CG, 9 Gauss-law CG, 10 learned correction, 11 Adams push (FP32 fast
 * path, or the whole FP64-mode step), 12 FP64 walk of deferred Adams particles.
 * fem_pic_profile_read waits for the recorded events, adds their durations to
 * per-phase totals and returns them: ms[16] (milliseconds), count[16] (event pairs);
 * reset != 0 clears the totals.  Either output may be NULL.
 */
fp_status fem_pic_profile_enable(fem_pic_t* ctx, int on);
fp_status fem_pic_profile_read(fem_pic_t* ctx, double ms[16], int64_t count[16], int reset);

/*
 * Self-test of the failure path of the library's bounded waits (not part of the method; the
 * paper has no counterpart): a one-thread kernel waits on a barrier that nothing completes,
 * gives up after limit_s seconds (0 < limit_s <= 10, else FP_EINVAL) and sets the time-out
 * bit of the status word, exactly as a push kernel does when a bulk copy never lands; the
 * next fem_pic_status returns FP_ECUDA and clears it, and the context stays usable.  Nothing
 * faults or hangs.  Asynchronous.
 */
fp_status fem_pic_selftest_wait(fem_pic_t* ctx, double limit_s, void* stream);

/*
 * Synchronise `stream`, return and clear the device status word: FP_OK, or the first
 * error class seen in this order: FP_ECUDA (a bounded wait gave up), FP_EINVAL (a
 * non-finite particle state, or a cell id outside [0, N_t)), FP_EWALK, FP_ENOCONV.
 * fem_pic_last_error names the cause.
 */
fp_status fem_pic_status(fem_pic_t* ctx, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* FEM_PIC_H */
