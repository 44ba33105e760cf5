"""Oracle: FP64 field operators and the implicit field step, plain numpy/scipy.  TEST INFRASTRUCTURE.

Sec. II.C defines the Hodge matrices by inner products of Whitney functions:
  [*eps]_ij  = <W1_i, eps W1_j>            (edge mass, M)
  [*mu^-1]_ij = <W2_i, mu^-1 W2_j>          (face mass)
and the wave-equation stiffness [*S] = [curl]^T [*mu^-1] [curl] (Eq. wave_cont), with
[curl] = D1 for Whitney forms.  The integrals are evaluated here with a 4-point
quadrature that is exact for the quadratic integrands of lowest-order Whitney forms.

The field step (the reading of Sec. IV.B with Newmark-beta, beta = 1/4, gamma = 1/2):
  1. Newmark on  M E'' + S E = -J' :
       (M + dt^2/4 S) E^N = M (2E^n - E^{n-1}) - dt^2 S (E^n/2 + E^{n-1}/4) - (dG^{n+1/2} - dG^{n-1/2})
  2. Gauss-law projection (Eq. discreteGauss with the modified projector, Eq. efld_mod_proj):
       L d = D0^T M E^N + Q^{n+1},  L = D0^T M D0  (interior nodes);   E^{n+1} = E^N - D0 d
  3. Faraday: b^{n+1} = b^n - dt D1 (E^{n+1} + E^n)/2.
Boundary conditions (bc):
  "pec"      PEC walls: edge DOFs on boundary edges and the correction d on boundary nodes
             are zero.
  "neumann"  natural boundary: no DOF is fixed.  L is then singular (constants), and the
             projection takes the zero-mean constraint of Eq. zero_mean_constraint: d = C_z y
             with C_z the identity on the first n-1 nodes and the last row -alpha_i/alpha_n
             (alpha_i the integral of W0_i), y from (C_z^T L C_z) y = C_z^T g.  Then
             alpha^T d = 0 and L d = g - (sum g / sum alpha) alpha: a net charge is spread as a
             uniform background (the modification the paper asks for when the net charge is
             not zero).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .mesh import Complex, LOCAL_EDGES, LOCAL_FACES

EPS0 = 8.854_187_8128e-12
MU0 = 1.256_637_062_12e-6

# symmetric 4-point rule on a tet, exact for polynomials of degree 2 (weights 1/4 each)
_QA = 0.5854101966249685
_QB = 0.1381966011250105
QUAD_LAMBDA = np.array([[_QA, _QB, _QB, _QB], [_QB, _QA, _QB, _QB], [_QB, _QB, _QA, _QB],
                        [_QB, _QB, _QB, _QA]])


def grads(cx: Complex) -> np.ndarray:
    """[nt, 4, 3] gradients of the barycentric coordinates (rows of the inverse Jacobian)."""
    x = cx.xyz[cx.tv]
    J = np.stack([x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]], axis=2)   # columns
    Ji = np.linalg.inv(J)                                                              # rows = grad l1..3
    g = np.empty((cx.n_tets, 4, 3))
    g[:, 1:] = Ji
    g[:, 0] = -Ji.sum(axis=1)
    return g


def _w1(lam, g):
    """[nt, 6, 3] Whitney-1 functions at barycentric point lam (lam_a g_b - lam_b g_a)."""
    return np.stack([lam[a] * g[:, b] - lam[b] * g[:, a] for a, b in LOCAL_EDGES], axis=1)


def _w2(lam, g):
    """[nt, 4, 3] Whitney-2 functions 2(l_a g_b x g_c + l_b g_c x g_a + l_c g_a x g_b)."""
    out = []
    for a, b, c in LOCAL_FACES:
        out.append(2.0 * (lam[a] * np.cross(g[:, b], g[:, c]) + lam[b] * np.cross(g[:, c], g[:, a]) +
                          lam[c] * np.cross(g[:, a], g[:, b])))
    return np.stack(out, axis=1)


def _assemble(cx, local, ids, n):
    nt, k = ids.shape
    rows = np.repeat(ids, k, axis=1).ravel()
    cols = np.tile(ids, (1, k)).ravel()
    return sp.csr_matrix((local.ravel(), (rows, cols)), shape=(n, n))


def edge_mass(cx: Complex, eps: float = EPS0) -> sp.csr_matrix:
    """[*eps]_ij = sum_T int_T W1_i . eps W1_j (4-point quadrature, exact here)."""
    g = grads(cx)
    loc = np.zeros((cx.n_tets, 6, 6))
    for lam in QUAD_LAMBDA:
        w = _w1(lam, g)
        loc += 0.25 * np.einsum("tid,tjd->tij", w, w)
    loc *= (eps * cx.vol)[:, None, None]
    return _assemble(cx, loc, cx.tet_edges, cx.n_edges)


def face_mass(cx: Complex, mu: float = MU0) -> sp.csr_matrix:
    """[*mu^-1]_ij = sum_T int_T W2_i . mu^-1 W2_j."""
    g = grads(cx)
    loc = np.zeros((cx.n_tets, 4, 4))
    for lam in QUAD_LAMBDA:
        w = _w2(lam, g)
        loc += 0.25 * np.einsum("tid,tjd->tij", w, w)
    loc *= (cx.vol / mu)[:, None, None]
    return _assemble(cx, loc, cx.tet_faces, cx.n_faces)


def curl_curl(cx: Complex, mu: float = MU0) -> sp.csr_matrix:
    """[*S] = [curl]^T [*mu^-1] [curl] with [curl] = D1 (Eq. wave_cont)."""
    D1 = cx.D1().astype(np.float64)
    return (D1.T @ face_mass(cx, mu) @ D1).tocsr()


def node_laplacian(cx: Complex, eps: float = EPS0) -> sp.csr_matrix:
    """[grad]^T [*eps] [grad] with [grad] = D0 (the left side of Eq. discreteGauss)."""
    D0 = cx.D0().astype(np.float64)
    return (D0.T @ edge_mass(cx, eps) @ D0).tocsr()


def _solve(Amat, rhs, tol=1e-13):
    if Amat.shape[0] == 0:
        return np.zeros(0)
    if Amat.shape[0] <= 60_000:
        return spla.spsolve(Amat.tocsc(), rhs)
    x, info = spla.cg(Amat, rhs, rtol=tol, atol=0.0, maxiter=20_000)
    assert info == 0, "oracle CG did not converge"
    return x


def zero_mean_constraint(alpha: np.ndarray) -> sp.csr_matrix:
    """C_z of Eq. zero_mean_constraint, n x (n-1): identity on the first n-1 rows, last row
    -alpha_i / alpha_n, so that alpha^T (C_z y) = 0 for every y."""
    n = alpha.shape[0]
    rows = np.concatenate([np.arange(n - 1), np.full(n - 1, n - 1)])
    cols = np.concatenate([np.arange(n - 1), np.arange(n - 1)])
    vals = np.concatenate([np.ones(n - 1), -alpha[:-1] / alpha[-1]])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n - 1))


class FieldOracle:
    """Implicit field step on one mesh for a fixed dt (bc: "pec" or "neumann")."""

    def __init__(self, cx: Complex, dt: float, eps: float = EPS0, mu: float = MU0, bc: str = "pec"):
        if bc not in ("pec", "neumann"):
            raise ValueError("bc is 'pec' or 'neumann'")
        self.bc = bc
        self.cx = cx
        self.dt = dt
        self.M = edge_mass(cx, eps)
        self.S = curl_curl(cx, mu)
        self.D0 = cx.D0().astype(np.float64).tocsr()
        self.D1 = cx.D1().astype(np.float64).tocsr()
        self.A = (self.M + 0.25 * dt * dt * self.S).tocsr()
        self.L = (self.D0.T @ self.M @ self.D0).tocsr()
        if bc == "pec":
            self.ie = np.nonzero(~cx.boundary_edge)[0]      # interior (free) edges
            self.inn = np.nonzero(~cx.boundary_node)[0]     # interior nodes
        else:
            self.ie = np.arange(cx.n_edges)
            self.inn = np.arange(cx.n_nodes)
        self.A_II = self.A[self.ie][:, self.ie].tocsr()
        self.L_II = self.L[self.inn][:, self.inn].tocsr()
        self.alpha = cx.node_volume()
        if bc == "neumann":
            self.Cz = zero_mean_constraint(self.alpha)
            self.L_z = (self.Cz.T @ self.L @ self.Cz).tocsr()

    def newmark_rhs(self, En, Enm1, dG_half, dG_prev):
        dt2 = self.dt * self.dt
        return self.M @ (2.0 * En - Enm1) - dt2 * (self.S @ (0.5 * En + 0.25 * Enm1)) - (dG_half - dG_prev)

    def newmark(self, En, Enm1, dG_half, dG_prev):
        rhs = self.newmark_rhs(En, Enm1, dG_half, dG_prev)
        E = np.zeros(self.cx.n_edges)
        E[self.ie] = _solve(self.A_II, rhs[self.ie])
        return E

    def gauss_rhs(self, E, Q):
        return self.D0.T @ (self.M @ E) + Q

    def gauss_project(self, E, Q):
        g = self.gauss_rhs(E, Q)
        d = np.zeros(self.cx.n_nodes)
        if self.bc == "pec":
            d[self.inn] = _solve(self.L_II, g[self.inn])
        else:
            d = self.Cz @ _solve(self.L_z, self.Cz.T @ g)
        return E - self.D0 @ d, d

    def faraday(self, b, E_new, E_old):
        return b - self.dt * (self.D1 @ (0.5 * (E_new + E_old)))

    def step(self, En, Enm1, b, dG_half, dG_prev, Q_new):
        EN = self.newmark(En, Enm1, dG_half, dG_prev)
        E1, _ = self.gauss_project(EN, Q_new)
        return E1, self.faraday(b, E1, En)

    def gauss_residual(self, E, Q):
        """Gauss residual D0^T M E + Q on the free nodes and its scale (Neumann: less the net
        charge spread as alpha, the part the zero-mean projection leaves by construction)."""
        r = self.gauss_rhs(E, Q)
        if self.bc == "neumann":
            r = r - (Q.sum() / self.alpha.sum()) * self.alpha
        sc = (np.abs(self.D0.T) @ np.abs(self.M @ E))[self.inn] + np.abs(Q[self.inn])
        return r[self.inn], sc

    def initial_field(self, Q):
        """E with D0^T M E + Q = 0 at interior nodes and no solenoidal part (the start state)."""
        E, _ = self.gauss_project(np.zeros(self.cx.n_edges), Q)
        return E

    def amplification_matrix(self):
        """Dense Newmark amplification of the homogeneous system on the interior edges."""
        M = self.M[self.ie][:, self.ie].toarray()
        S = self.S[self.ie][:, self.ie].toarray()
        dt2 = self.dt * self.dt
        A = M + 0.25 * dt2 * S
        Ai = np.linalg.inv(A)
        n = M.shape[0]
        G = np.zeros((2 * n, 2 * n))
        G[:n, :n] = Ai @ (2.0 * M - 0.5 * dt2 * S)
        G[:n, n:] = -Ai @ (M + 0.25 * dt2 * S)
        G[n:, :n] = np.eye(n)
        return G
