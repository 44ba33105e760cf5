"""Pins of the oracle's field operators and implicit field step (Sec. II.C, IV.A-B, VI.A.1).

Each operator is computed by the oracle one way and checked here against an
independent form: the W1/W2 interpolants of uniform fields carry exactly the field
energy; [*S] = D1^T [*mu^-1] D1 (oracle) equals the element curl-curl integral of
curl W1_ab = 2 grad l_a x grad l_b (test); D0^T [*eps] D0 (oracle) equals the P1
stiffness eps |T| grad l_a . grad l_b (test); [*S] D0 = 0 (curl grad = 0); the
Newmark amplification matrix has its eigenvalues on the unit circle (Sec. VI.A.1);
the sparse Gauss-law projection equals the dense modified projector of Eq.
efld_mod_proj; Faraday keeps D2 b = 0.  Natural (Neumann) boundary: C_z annihilates alpha,
the constrained projection equals the pseudo-inverse route shifted to alpha-mean zero, and
the Gauss law holds at every node up to the net charge spread as alpha.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_2103_06737_gb300 import inputs as I
import oracle as O
from oracle import fields as OF


@pytest.fixture(scope="module")
def mesh4():
    m = I.cube_mesh(4, 1.0, 0.1, seed=1)
    return O.Complex(m.xyz, m.tets)


def _elem(cx, loc, ids, n):
    k = ids.shape[1]
    rows = np.repeat(ids, k, axis=1).ravel()
    cols = np.tile(ids, (1, k)).ravel()
    return sp.csr_matrix((loc.ravel(), (rows, cols)), shape=(n, n))


def test_uniform_field_energies(mesh4):
    cx = mesh4
    E0 = np.array([1.0, -2.0, 0.5])
    B0 = np.array([0.3, 0.1, -0.7])
    e, b = cx.project_uniform(E0, B0)
    M = OF.edge_mass(cx)
    Mf = OF.face_mass(cx)
    assert abs(e @ (M @ e) - OF.EPS0 * (E0 @ E0) * 1.0) <= 1e-12 * OF.EPS0 * (E0 @ E0)
    assert abs(b @ (Mf @ b) - (B0 @ B0) / OF.MU0) <= 1e-12 * (B0 @ B0) / OF.MU0
    assert abs(M - M.T).max() <= 1e-15 * abs(M).max()
    w = np.linalg.eigvalsh(M.toarray())
    assert w.min() > 0


def test_curl_curl_two_ways_and_gradient_null_space(mesh4):
    cx = mesh4
    S = OF.curl_curl(cx)                       # paper route: D1^T [*mu^-1] D1
    g = OF.grads(cx)
    cw = np.stack([2.0 * np.cross(g[:, a], g[:, b]) for a, b in O.LOCAL_EDGES], axis=1)
    loc = np.einsum("tid,tjd->tij", cw, cw) * (cx.vol / OF.MU0)[:, None, None]
    S2 = _elem(cx, loc, cx.tet_edges, cx.n_edges)
    assert abs(S - S2).max() <= 1e-12 * abs(S2).max()
    D0 = cx.D0().astype(float)
    assert abs(S @ D0).max() <= 1e-12 * abs(S).max()


def test_laplacian_two_ways(mesh4):
    cx = mesh4
    L = OF.node_laplacian(cx)                  # D0^T [*eps] D0
    g = OF.grads(cx)
    loc = np.einsum("tid,tjd->tij", g, g) * (OF.EPS0 * cx.vol)[:, None, None]
    L2 = _elem(cx, loc, cx.tv, cx.n_nodes)
    assert abs(L - L2).max() <= 1e-12 * abs(L2).max()


def test_newmark_eigenvalues_on_unit_circle():
    m = I.cube_mesh(3, 1.0, 0.0)
    cx = O.Complex(m.xyz, m.tets)
    # a step comparable to the cavity's light-crossing scale, where explicit schemes fail
    dt = 2.0 * (1.0 / 3.0) / I.C_LIGHT
    fo = OF.FieldOracle(cx, dt)
    mu = np.linalg.eigvals(fo.amplification_matrix())
    assert np.abs(np.abs(mu) - 1.0).max() < 1e-7
    # the gradient null space of the wave equation gives a double eigenvalue at 1
    n_grad = len(fo.inn)
    assert (np.abs(mu - 1.0) < 1e-6).sum() >= n_grad


def test_gauss_projection_matches_dense_modified_projector(mesh4):
    cx = mesh4
    fo = OF.FieldOracle(cx, 1e-10)
    rng = np.random.default_rng(0)
    EN = rng.uniform(-1, 1, cx.n_edges)
    EN[cx.boundary_edge] = 0.0
    Q = np.zeros(cx.n_nodes)
    E1, _ = fo.gauss_project(EN, Q)
    # dense Eq. efld_mod_proj: P = Sigma (grad^T Sigma)^-1 grad^T with Sigma = [*eps][grad]
    ie, inn = fo.ie, fo.inn
    M = fo.M.toarray()[np.ix_(ie, ie)]
    G = fo.D0.toarray()[np.ix_(ie, inn)]
    Sigma = M @ G
    P = Sigma @ np.linalg.solve(G.T @ Sigma, G.T)
    D = M @ EN[ie]
    lhs = M @ E1[ie]
    rhs = D - P @ D
    assert np.abs(lhs - rhs).max() <= 1e-9 * np.abs(D).max()
    # the projected flux is discretely divergence free at interior nodes
    assert np.abs(G.T @ lhs).max() <= 1e-10 * np.abs(G.T @ D).max()


def test_projection_with_charge_and_idempotence(mesh4):
    cx = mesh4
    fo = OF.FieldOracle(cx, 1e-10)
    rng = np.random.default_rng(1)
    Q = rng.uniform(-1e-12, 1e-12, cx.n_nodes)
    E = rng.uniform(-1, 1, cx.n_edges)
    E[cx.boundary_edge] = 0.0
    E1, _ = fo.gauss_project(E, Q)
    r, sc = fo.gauss_residual(E1, Q)
    assert np.abs(r).max() <= 1e-11 * sc.max()
    E2, d2 = fo.gauss_project(E1, Q)
    assert np.abs(E2 - E1).max() <= 1e-10 * np.abs(E1).max()
    assert (E1[cx.boundary_edge] == 0).all()


def test_faraday_keeps_div_b_zero(mesh4):
    cx = mesh4
    fo = OF.FieldOracle(cx, 1e-9)
    _, b = cx.project_uniform((0, 0, 0), (0.0, 0.0, 0.1))
    rng = np.random.default_rng(2)
    for _ in range(5):
        b = fo.faraday(b, rng.uniform(-1, 1, cx.n_edges), rng.uniform(-1, 1, cx.n_edges))
    assert np.abs(cx.D2() @ b).max() <= 1e-14 * np.abs(b).max()


def test_newmark_keeps_gauss_law_with_a_continuity_respecting_current(mesh4):
    """With dG and dQ from the same charge-conserving deposit, the Newmark update keeps
    D0^T M E + Q = 0 (the reason the decomposition removes the t grad(phi) growth)."""
    cx = mesh4
    orc = O.Oracle(cx.xyz, cx.tv)
    dt = 2e-10
    fo = OF.FieldOracle(cx, dt)
    m = I.cube_mesh(4, 1.0, 0.1, seed=1)
    sp_ = I.uniform_species(m, 400, 9, 2e6, -I.Q_E, I.M_E, 1e5)
    e0, b = cx.project_uniform((0, 0, 0), (0, 0, 0.05))
    Q0, _ = orc.charge(sp_.cell, sp_.X, sp_.q, sp_.w)
    E_prev = E = fo.initial_field(Q0)
    dG_prev = np.zeros(cx.n_edges)
    cell, X, V, Qo = sp_.cell, sp_.X, sp_.V, Q0
    for _ in range(4):
        r = orc.step(cell, X, V, E, b, sp_.q, sp_.m, sp_.w, dt)
        cell, X, V = r["cell"], r["X"], r["V"]
        EN = fo.newmark(E, E_prev, r["dG"], dG_prev)
        g, sc = fo.gauss_residual(EN, r["Q"])
        assert np.abs(g).max() <= 1e-8 * sc.max()      # before any projection
        E_new, b = fo.step(E, E_prev, b, r["dG"], dG_prev, r["Q"])
        g, sc = fo.gauss_residual(E_new, r["Q"])
        assert np.abs(g).max() <= 1e-11 * sc.max()
        E_prev, E, dG_prev = E, E_new, r["dG"]


# ---------------------------------------------------------------- natural (Neumann) boundary
def test_zero_mean_constraint_matrix(mesh4):
    """C_z of Eq. zero_mean_constraint: alpha^T C_z = 0, identity on the first n-1 rows, rank n-1."""
    a = mesh4.node_volume()
    assert abs(a.sum() - 1.0) < 1e-13                     # the W0 integrals add up to |Omega| = 1 m^3
    Cz = OF.zero_mean_constraint(a).toarray()
    n = a.size
    assert Cz.shape == (n, n - 1)
    assert np.array_equal(Cz[:-1], np.eye(n - 1))
    assert np.abs(a @ Cz).max() <= 1e-15
    assert np.linalg.matrix_rank(Cz) == n - 1


def test_neumann_laplacian_null_space_and_newmark_stability():
    m = I.cube_mesh(3, 1.0, 0.1, seed=1)
    cx = O.Complex(m.xyz, m.tets)
    dt = 2.0 * (1.0 / 3.0) / I.C_LIGHT
    fo = OF.FieldOracle(cx, dt, bc="neumann")
    assert np.abs(fo.L @ np.ones(cx.n_nodes)).max() <= 1e-12 * abs(fo.L).max()
    assert len(fo.ie) == cx.n_edges and len(fo.inn) == cx.n_nodes
    mu = np.linalg.eigvals(fo.amplification_matrix())
    assert np.abs(np.abs(mu) - 1.0).max() < 1e-7


def test_neumann_projection_against_pseudo_inverse(mesh4):
    """The C_z-reduced solve against an independent route: the pseudo-inverse of the singular
    L applied to the consistent part of g, shifted to alpha-mean zero."""
    cx = mesh4
    fo = OF.FieldOracle(cx, 1e-10, bc="neumann")
    rng = np.random.default_rng(3)
    EN = rng.uniform(-1, 1, cx.n_edges)
    Q = rng.uniform(-1e-12, 1e-12, cx.n_nodes) + 2e-13          # a net charge
    E1, d = fo.gauss_project(EN, Q)
    a = fo.alpha
    g = fo.gauss_rhs(EN, Q)
    L = fo.L.toarray()
    dp = np.linalg.pinv(L) @ (g - g.sum() / a.sum() * a)
    d_ref = dp - (a @ dp) / a.sum()
    assert np.abs(d - d_ref).max() <= 1e-9 * np.abs(d_ref).max()
    assert np.abs(E1 - (EN - fo.D0 @ d_ref)).max() <= 1e-9 * np.abs(EN).max()


def test_neumann_gauss_law_and_zero_mean(mesh4):
    cx = mesh4
    fo = OF.FieldOracle(cx, 1e-10, bc="neumann")
    rng = np.random.default_rng(4)
    EN = rng.uniform(-1, 1, cx.n_edges)
    Q = rng.uniform(-1e-12, 1e-12, cx.n_nodes)
    E1, d = fo.gauss_project(EN, Q)
    a = fo.alpha
    assert abs(a @ d) <= 1e-12 * (a @ np.abs(d))                 # zero mean (the constraint)
    # Gauss law at every node, less the net charge spread as alpha
    lhs = fo.D0.T @ (fo.M @ E1) + Q
    scale = (np.abs(fo.D0.T) @ np.abs(fo.M @ E1) + np.abs(Q)).max()
    assert np.abs(lhs - Q.sum() / a.sum() * a).max() <= 1e-11 * scale
    r, sc = fo.gauss_residual(E1, Q)
    assert np.abs(r).max() <= 1e-11 * sc.max()
    # a neutral charge satisfies the Gauss law exactly, boundary nodes included
    Qn = Q - Q.sum() / a.sum() * a
    E2, _ = fo.gauss_project(EN, Qn)
    assert np.abs(fo.D0.T @ (fo.M @ E2) + Qn).max() <= 1e-11 * scale
    # boundary edges are free under the natural boundary
    assert np.abs(E1[cx.boundary_edge]).max() > 0
