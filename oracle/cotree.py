"""Oracle: the tree / co-tree reduced field system and the first-order mixed FEM (MFEM), in
dense numpy (small meshes only).  TEST INFRASTRUCTURE.

The library advances E by Newmark on the full edge wave equation and then projects it onto
the discrete Gauss law.  This module builds the system the paper writes down for the same
fields (Sec. IV.B), so that the tests can hold the two against each other:

  * a minimum spanning tree of the node graph (edge lengths as weights), grounded on the PEC
    wall, whose complement among the free edges is the edge co-tree E_c; a minimum spanning
    tree of the dual graph (tets joined through free faces, centroid distances as weights)
    whose complement is the face co-tree F_c.
  * the selection matrices C_c^e and C_c^b (Eq. cotree_mat_e, cotree_mat_b), the zero-mean
    constraints C_z^e and C_z^b (Eq. zero_mean_constraint), the modified projectors
    P_e^Sigma and P_b^Sigma (Eq. efld_mod_proj) and their complements P_e^Lambda and
    P_b^Lambda (Eq. proj_el, bfld_projector).
  * Z11 .. Z23 as the paper defines them; the reduced first-order system (Eq. reduceMEs) and
    the reduced wave equation (Eq. reducedWaveEqn), both advanced by Newmark
    (beta = 1/4, gamma = 1/2), with E_ns from the discrete Gauss law (Eq. discreteGauss).
  * the full first-order mixed system (Eq. maxwell_semi) under the same Newmark rule, which
    for a first-order system is the trapezoidal rule: the MFEM of Sec. V and VI.A.

Readings (where the paper leaves the choice open):
  * Sigma = [*eps][grad] (stated in Sec. IV.B).  Sigma_m = [div]^T with [div] the tet-face
    incidence D2 on the free faces.  The reduced wave operator Z22 Z11^-1 Z12 does not depend
    on this choice: any Sigma_m that makes P_b^Lambda a projector onto divergence-free fluxes
    turns it into C_c^eT [*S] C_c^e.
  * alpha^3_t = integral of W3_t = 1 for every tet (W3_t is 1/|T| on T).
  * Free DOFs.  PEC fixes the boundary edges, the boundary nodes (the grounded root of the
    edge tree) and the boundary faces (their flux cannot change while n x E = 0 on the wall).
    Then C_z^e is the identity and C_z^b removes the constant of the tet potentials.  The
    natural boundary fixes nothing: the edge tree spans all nodes (C_z^e needed), and the dual
    graph gains an exterior vertex joined through the boundary faces (C_z^b the identity).
  * The source terms of Eq. reduceMEs / reducedWaveEqn over one step: dt * dG/dt is the
    deposit dG^{n+1/2} of that step (the path integral over the step, Sec. IV.B.1), and the
    E_ns term takes the same time difference as the E_s term it sits beside (first
    difference in Ampere's law, second difference in the wave equation).
  * Charge: E_ns solves [grad]^T [*eps] [grad] C_z^e E_ns = -Q on the free nodes (the
    library's sign, D0^T [*eps] E + Q = 0); under the natural boundary the net charge is
    spread as alpha^0, which C_z^eT removes.
"""
from __future__ import annotations

import numpy as np

from .fields import EPS0, MU0, edge_mass, face_mass, zero_mean_constraint


def spanning_tree(n_vertices: int, ends: np.ndarray, weights: np.ndarray) -> np.ndarray:
    """Kruskal's minimum spanning forest: a boolean mask over the graph's edges `ends`
    ([m, 2] vertex ids), ties broken by edge index.  Self-loops never enter the tree."""
    parent = np.arange(n_vertices)

    def root(a):
        while parent[a] != a:
            parent[a] = parent[parent[a]]
            a = parent[a]
        return a

    in_tree = np.zeros(len(weights), dtype=bool)
    for k in np.lexsort((np.arange(len(weights)), np.asarray(weights))):
        a, b = root(int(ends[k, 0])), root(int(ends[k, 1]))
        if a != b:
            parent[a] = b
            in_tree[k] = True
    return in_tree


class CoTree:
    """Tree / co-tree split and the Z-matrices of Sec. IV.B on one mesh (bc "pec" or "neumann").

    Index sets (positions into the full numbering): ie free edges, inn free nodes, jf free
    faces.  Within them: cot_e / tree_e (positions into ie), cot_f / tree_f (into jf)."""

    def __init__(self, cx, bc: str = "pec", eps: float = EPS0, mu: float = MU0):
        if bc not in ("pec", "neumann"):
            raise ValueError("bc is 'pec' or 'neumann'")
        self.cx, self.bc = cx, bc
        pec = bc == "pec"
        self.ie = np.nonzero(~cx.boundary_edge)[0] if pec else np.arange(cx.n_edges)
        self.inn = np.nonzero(~cx.boundary_node)[0] if pec else np.arange(cx.n_nodes)
        self.jf = np.nonzero(~cx.boundary_face)[0] if pec else np.arange(cx.n_faces)
        ne, nn, nf, nt = len(self.ie), len(self.inn), len(self.jf), cx.n_tets

        # edge tree: PEC merges every wall node into one grounded vertex
        vid = np.full(cx.n_nodes, -1, dtype=np.int64)
        vid[self.inn] = np.arange(nn)
        if pec:
            vid[cx.boundary_node] = nn
        ends = vid[cx.edges[self.ie]]
        x = cx.xyz
        length = np.linalg.norm(x[cx.edges[self.ie, 1]] - x[cx.edges[self.ie, 0]], axis=1)
        in_tree = spanning_tree(nn + (1 if pec else 0), ends, length)
        self.tree_e = np.nonzero(in_tree)[0]
        self.cot_e = np.nonzero(~in_tree)[0]

        # face tree on the dual graph: tets, plus the exterior under the natural boundary
        cent_t = x[cx.tv].mean(axis=1)
        ft = cx.face_tets[self.jf]
        ext = nt
        dual = np.where(ft >= 0, ft, ext)
        p0 = cent_t[dual[:, 0]]
        fc = x[cx.faces[self.jf]].mean(axis=1)
        p1 = np.where((dual[:, 1] == ext)[:, None], fc, cent_t[np.minimum(dual[:, 1], nt - 1)])
        in_tree = spanning_tree(nt + (0 if pec else 1), dual, np.linalg.norm(p1 - p0, axis=1))
        self.tree_f = np.nonzero(in_tree)[0]
        self.cot_f = np.nonzero(~in_tree)[0]

        # operators on the free DOFs (dense)
        D0 = cx.D0().astype(np.float64).toarray()
        D1 = cx.D1().astype(np.float64).toarray()
        D2 = cx.D2().astype(np.float64).toarray()
        self.M = edge_mass(cx, eps).toarray()[np.ix_(self.ie, self.ie)]
        self.Fm = face_mass(cx, mu).toarray()[np.ix_(self.jf, self.jf)]
        self.grad = D0[np.ix_(self.ie, self.inn)]              # [grad]: free nodes -> free edges
        self.curl = D1[np.ix_(self.jf, self.ie)]               # [curl]: free edges -> free faces
        self.div = D2[:, self.jf]                              # [div]: free faces -> tets
        self.Sigma = self.M @ self.grad                        # Sigma = [*eps][grad]
        self.Sigma_m = self.div.T                              # reading: [div]^T
        self.Cz_e = (zero_mean_constraint(cx.node_volume()).toarray() if not pec else np.eye(nn))
        self.Cz_b = (zero_mean_constraint(np.ones(nt)).toarray() if pec else np.eye(nt))
        self.Cc_e = np.zeros((ne, len(self.cot_e)))
        self.Cc_e[self.cot_e, np.arange(len(self.cot_e))] = 1.0
        self.Cc_b = np.zeros((nf, len(self.cot_f)))
        self.Cc_b[self.cot_f, np.arange(len(self.cot_f))] = 1.0

        # Eq. efld_mod_proj, proj_el, bfld_projector
        GtS = self.grad.T @ self.Sigma
        Cz = self.Cz_e
        self.P_sigma_e = self.Sigma @ Cz @ np.linalg.solve(Cz.T @ GtS @ Cz, Cz.T @ self.grad.T)
        self.P_lambda_e = np.eye(ne) - self.P_sigma_e
        Cb = self.Cz_b
        self.P_sigma_b = self.Sigma_m @ Cb @ np.linalg.solve(Cb.T @ self.div @ self.Sigma_m @ Cb, Cb.T @ self.div)
        self.P_lambda_b = np.eye(nf) - self.P_sigma_b

        # the Z-matrices of Eq. reduceMEs
        Minv = np.linalg.inv(self.M)
        Cce, Ccb = self.Cc_e, self.Cc_b
        self.Z11 = Ccb.T @ self.P_lambda_b @ Ccb
        self.Z12 = Ccb.T @ self.curl @ Minv @ self.P_lambda_e @ self.M @ Cce
        self.Z13 = Ccb.T @ self.curl @ Minv @ self.Sigma @ Cz
        self.Z21 = Cce.T @ self.P_lambda_e @ self.M @ Cce
        self.Z22 = Cce.T @ self.curl.T @ self.Fm @ self.P_lambda_b @ Ccb
        self.Z23 = Cce.T @ self.Sigma @ Cz
        self.K = self.Z22 @ np.linalg.solve(self.Z11, self.Z12)     # Eq. reducedWaveEqn's stiffness
        self.gauss = Cz.T @ GtS @ Cz                               # Eq. discreteGauss, constrained
        # E_s coefficients -> the solenoidal edge field, from D_s = P_e^Lambda [*eps] C_c^e E_s
        self.Lam_e = Minv @ self.P_lambda_e @ self.M @ Cce
        # B_s coefficients -> the divergence-free face fluxes of Eq. bfld_projected (B_ns = 0)
        self.Lam_b = self.P_lambda_b @ Ccb

    # ---- sizes -------------------------------------------------------------------------
    @property
    def n_cotree_edges(self) -> int:
        return len(self.cot_e)

    @property
    def n_cotree_faces(self) -> int:
        return len(self.cot_f)

    # ---- the decomposition of Eq. efld_decomp_flux ------------------------------------
    def e_ns(self, Q: np.ndarray) -> np.ndarray:
        """E_ns (the C_z^e-reduced potential coefficients) from Eq. discreteGauss for node charge Q."""
        return np.linalg.solve(self.gauss, self.Cz_e.T @ (-np.asarray(Q, np.float64)[self.inn]))

    def decompose(self, E: np.ndarray):
        """(E_ns, E_s) of a full edge vector E: the flux [*eps] E split as Sigma C_z E_ns +
        P_e^Lambda [*eps] E, and E_s the co-tree coefficients of that solenoidal flux."""
        Ef = np.asarray(E, np.float64)[self.ie]
        D = self.M @ Ef
        Cz = self.Cz_e
        y = np.linalg.solve(self.gauss, Cz.T @ (self.grad.T @ D))
        s = np.linalg.solve(self.Z21, self.Cc_e.T @ (self.P_lambda_e @ D))
        return y, s

    def compose(self, y: np.ndarray, s: np.ndarray) -> np.ndarray:
        """Full edge vector (zeros on fixed edges) from E_ns and E_s."""
        E = np.zeros(self.cx.n_edges)
        E[self.ie] = self.grad @ (self.Cz_e @ y) + self.Lam_e @ s
        return E

    # ---- Newmark on the reduced wave equation (Eq. reducedWaveEqn) ---------------------
    def wave_step(self, s, s_prev, y_new, y, y_prev, dG_half, dG_prev, dt):
        """E_s^{n+1} from E_s^n, E_s^{n-1}, the E_ns of levels n+1, n, n-1 and the deposits."""
        dt2 = dt * dt
        ddG = (np.asarray(dG_half, np.float64) - np.asarray(dG_prev, np.float64))[self.ie]
        rhs = (self.Z21 @ (2.0 * s - s_prev) - dt2 * (self.K @ (0.5 * s + 0.25 * s_prev))
               - self.Cc_e.T @ ddG - self.Z23 @ (y_new - 2.0 * y + y_prev))
        return np.linalg.solve(self.Z21 + 0.25 * dt2 * self.K, rhs)

    # ---- Newmark (trapezoidal rule) on the reduced first-order system (Eq. reduceMEs) --
    def mfem_reduced_step(self, s, Bs, y_new, y, dG_half, dt):
        """(E_s, B_s) at n+1 from their values at n; Z13 E_ns is kept although it is zero."""
        nb = self.n_cotree_faces
        lhs = np.block([[self.Z11 / dt, 0.5 * self.Z12], [-0.5 * self.Z22, self.Z21 / dt]])
        rhs = np.concatenate([
            self.Z11 @ Bs / dt - 0.5 * self.Z12 @ s - self.Z13 @ (0.5 * (y_new + y)),
            self.Z21 @ s / dt + 0.5 * self.Z22 @ Bs
            - self.Cc_e.T @ np.asarray(dG_half, np.float64)[self.ie] / dt - self.Z23 @ (y_new - y) / dt])
        out = np.linalg.solve(lhs, rhs)
        return out[nb:], out[:nb]

    def reduced_amplification(self, dt):
        """Amplification matrix of the homogeneous reduced first-order system, state (B_s, E_s)."""
        lhs = np.block([[self.Z11 / dt, 0.5 * self.Z12], [-0.5 * self.Z22, self.Z21 / dt]])
        rhs = np.block([[self.Z11 / dt, -0.5 * self.Z12], [0.5 * self.Z22, self.Z21 / dt]])
        return np.linalg.solve(lhs, rhs)

    # ---- the full first-order mixed FEM (Eq. maxwell_semi) -----------------------------
    def mfem_step(self, E, b, dG_half, dt):
        """Trapezoidal (Newmark) step of Eq. maxwell_semi on the free DOFs:
             b^{n+1} = b^n - dt [curl] (E^{n+1} + E^n) / 2
             [*eps] (E^{n+1} - E^n) = dt [curl]^T [*mu^-1] (b^{n+1} + b^n) / 2 - dG^{n+1/2}
        b holds the free faces' fluxes only (fixed faces do not change)."""
        Ef = np.asarray(E, np.float64)[self.ie]
        bf = np.asarray(b, np.float64)
        CtF = self.curl.T @ self.Fm
        S = CtF @ self.curl
        A = self.M + 0.25 * dt * dt * S
        rhs = (self.M @ Ef - 0.25 * dt * dt * (S @ Ef) + dt * (CtF @ bf)
               - np.asarray(dG_half, np.float64)[self.ie])
        E1f = np.linalg.solve(A, rhs)
        b1 = bf - 0.5 * dt * (self.curl @ (E1f + Ef))
        E1 = np.zeros(self.cx.n_edges)
        E1[self.ie] = E1f
        return E1, b1

    def mfem_amplification(self, dt):
        """Amplification matrix of the homogeneous full MFEM, state (b on free faces, E on free edges)."""
        nf, ne = len(self.jf), len(self.ie)
        h = 0.5 * dt
        CtF = self.curl.T @ self.Fm
        lhs = np.block([[np.eye(nf), h * self.curl], [-h * CtF, self.M]])
        rhs = np.block([[np.eye(nf), -h * self.curl], [h * CtF, self.M]])
        assert lhs.shape == (nf + ne, nf + ne)
        return np.linalg.solve(lhs, rhs)
