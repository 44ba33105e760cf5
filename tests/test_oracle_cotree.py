"""Pins of the tree / co-tree reduced system and the first-order MFEM (Sec. IV.B, V, VI.A.1).

The co-tree oracle builds the paper's matrices literally (trees, C_c, C_z, projectors,
Z11..Z23) and is held here against facts the paper and the algebra fix:
  * the trees: spanning, grounded as the boundary condition asks, of minimum total length
    (checked against scipy's minimum_spanning_tree), and as many co-tree edges as co-tree
    faces on a simply connected domain (Sec. V, item 7, by Euler's relation);
  * the projectors: Sigma^T Lambda = 0 and [div] P_b^Lambda = 0, both idempotent; Z13 = 0
    (stated in Sec. IV.B); the reduced wave stiffness Z22 Z11^-1 Z12 equals the co-tree block
    of [*S] (a consequence of D2 D1 = 0 that any transposed or misplaced factor breaks);
  * the reduced wave equation (Eq. reducedWaveEqn) with E_ns from Eq. discreteGauss gives the
    same fields, step by step, as the projected Newmark step the library computes (the
    algebraic equivalence the library's design rests on), for PEC and natural boundaries;
  * MFEM with the trapezoidal rule and the reduced first-order system (Eq. reduceMEs) give
    the same E and b as well;
  * eigenvalues (Sec. VI.A.1): every amplification eigenvalue on the unit circle; the
    reduced system's spectrum is MFEM's with its static modes (eigenvalue 1) removed; the
    wave-equation FEM's gradient modes carry a Jordan chain, the t grad(phi) growth of Sec. V,
    while MFEM's do not; an injected gradient error grows linearly in WE-FEM, stays constant in
    MFEM and is removed by the projection (the behaviour Sec. VI.B reports for the Gauss law).
"""
import numpy as np
import pytest
from scipy.sparse.csgraph import minimum_spanning_tree

from paper_2103_06737_gb300 import inputs as I
import oracle as O
from oracle import cotree as OC
from oracle import fields as OF

from helpers import continuity_run


@pytest.fixture(scope="module")
def mesh4():
    m = I.cube_mesh(4, 1.0, 0.1, seed=1)
    return m, O.Complex(m.xyz, m.tets)


@pytest.fixture(scope="module")
def mesh3():
    m = I.cube_mesh(3, 1.0, 0.1, seed=1)
    return O.Complex(m.xyz, m.tets)


@pytest.fixture(scope="module")
def trees4(mesh4):
    _, cx = mesh4
    return {bc: OC.CoTree(cx, bc) for bc in ("pec", "neumann")}


def _mst_weight(n_vertices, ends, w):
    """Total weight of a minimum spanning tree by scipy (parallel edges keep the lightest)."""
    W = np.full((n_vertices, n_vertices), np.inf)
    for (a, b), x in zip(ends, w):
        if a != b:
            W[a, b] = W[b, a] = min(W[a, b], x)
    W[~np.isfinite(W)] = 0.0
    return minimum_spanning_tree(W).sum()


@pytest.mark.parametrize("bc", ["pec", "neumann"])
def test_trees_span_ground_and_are_minimal(mesh4, trees4, bc):
    _, cx = mesh4
    ct = trees4[bc]
    nn, nt = len(ct.inn), cx.n_tets
    # edge tree: PEC grounds every interior node to the wall, so the tree's incidence
    # block is square and unimodular; the natural boundary spans the nodes with one root
    G_tree = ct.grad[ct.tree_e]
    if bc == "pec":
        assert len(ct.tree_e) == nn
        assert abs(abs(np.linalg.det(G_tree)) - 1.0) < 1e-9
    else:
        assert len(ct.tree_e) == nn - 1
        assert np.linalg.matrix_rank(G_tree) == nn - 1
    # face tree on the dual graph: PEC leaves the tet potentials' constant (C_z^b), the
    # natural boundary grounds them on the exterior
    Dv_tree = ct.div[:, ct.tree_f]
    assert len(ct.tree_f) == (nt - 1 if bc == "pec" else nt)
    assert np.linalg.matrix_rank(Dv_tree) == nt - 1 if bc == "pec" else nt
    # Euler (Sec. V item 7): as many co-tree edges as co-tree faces on a simply connected domain
    assert ct.n_cotree_edges == ct.n_cotree_faces
    assert ct.n_cotree_edges == len(ct.ie) - len(ct.tree_e)
    # minimum total length against scipy's minimum spanning tree of the same graph
    vid = np.full(cx.n_nodes, -1)
    vid[ct.inn] = np.arange(nn)
    if bc == "pec":
        vid[cx.boundary_node] = nn
    ends = vid[cx.edges[ct.ie]]
    lengths = np.linalg.norm(cx.xyz[cx.edges[ct.ie, 1]] - cx.xyz[cx.edges[ct.ie, 0]], axis=1)
    ref = _mst_weight(nn + (bc == "pec"), ends, lengths)
    assert abs(lengths[ct.tree_e].sum() - ref) <= 1e-12 * ref


@pytest.mark.parametrize("bc", ["pec", "neumann"])
def test_projectors_and_z_matrices(mesh4, trees4, bc):
    _, cx = mesh4
    ct = trees4[bc]
    Pe, Pb = ct.P_lambda_e, ct.P_lambda_b
    # Sigma^T Lambda = 0: the co-tree flux carries no charge; idempotent projectors
    assert np.abs(ct.grad.T @ Pe).max() <= 1e-12
    assert np.abs(Pe @ Pe - Pe).max() <= 1e-10
    assert np.abs(ct.div @ Pb).max() <= 1e-12
    assert np.abs(Pb @ Pb - Pb).max() <= 1e-12
    # the pseudo-inverse projector of Eq. proj_es has the same range (the gradient fluxes) but
    # projects along ker(Sigma^T), so its complement is not divergence-free: the projector of
    # Eq. efld_mod_proj is the one that imposes the discrete Gauss law
    S = ct.Sigma
    P_pinv = S @ np.linalg.pinv(S.T @ S, rcond=1e-10, hermitian=True) @ S.T
    assert np.abs(P_pinv @ ct.P_sigma_e - ct.P_sigma_e).max() <= 1e-12
    assert np.abs(S.T @ (np.eye(len(ct.ie)) - P_pinv)).max() <= 1e-12 * np.abs(S).max()
    assert np.abs(ct.grad.T @ (np.eye(len(ct.ie)) - P_pinv)).max() > 0.1
    # Z13 = 0 (Sec. IV.B)
    assert np.abs(ct.Z13).max() <= 1e-10 * np.abs(ct.Z12).max()
    # Z21 and the reduced stiffness are symmetric positive definite: no null space in the
    # reduced wave equation on a simply connected domain
    for Z in (ct.Z21, ct.K):
        assert np.abs(Z - Z.T).max() <= 1e-9 * np.abs(Z).max()
        assert np.linalg.eigvalsh(0.5 * (Z + Z.T)).min() > 0
    # Z22 Z11^-1 Z12 = C_c^eT [*S] C_c^e with [*S] from the field oracle
    S = OF.curl_curl(cx).toarray()[np.ix_(ct.ie, ct.ie)]
    ref = ct.Cc_e.T @ S @ ct.Cc_e
    assert np.abs(ct.K - ref).max() <= 1e-9 * np.abs(ref).max()


@pytest.mark.parametrize("bc", ["pec", "neumann"])
def test_decomposition_round_trip(mesh4, trees4, bc):
    _, cx = mesh4
    ct = trees4[bc]
    rng = np.random.default_rng(5)
    E = np.zeros(cx.n_edges)
    E[ct.ie] = rng.uniform(-1, 1, len(ct.ie))
    y, s = ct.decompose(E)
    assert np.abs(ct.compose(y, s) - E).max() <= 1e-10
    phi = np.zeros(cx.n_nodes)
    phi[ct.inn] = rng.uniform(-1, 1, len(ct.inn))
    if bc == "neumann":
        phi -= (cx.node_volume() @ phi) / cx.node_volume().sum()
    Eg = np.zeros(cx.n_edges)
    Eg[ct.ie] = (cx.D0() @ phi)[ct.ie]
    y, s = ct.decompose(Eg)
    assert np.abs(s).max() <= 1e-10 * np.abs(y).max()          # a gradient has no E_s
    assert np.abs(ct.Cz_e @ y - phi[ct.inn]).max() <= 1e-10 * np.abs(phi).max()
    _, s2 = ct.decompose(ct.compose(np.zeros_like(y), s + 1.0))
    assert np.abs(s2 - (s + 1.0)).max() <= 1e-10 * np.abs(s + 1.0).max()


@pytest.mark.parametrize("bc", ["pec", "neumann"])
def test_reduced_systems_reproduce_the_projected_step(mesh4, trees4, bc):
    """Eq. reducedWaveEqn (Newmark) with Eq. discreteGauss, the reduced first-order system
    (Eq. reduceMEs) and the full MFEM give the fields of the projected Newmark step."""
    m, cx = mesh4
    ct = trees4[bc]
    dt = 0.2 * I.gyro_period(0.1)
    fo = OF.FieldOracle(cx, dt, bc=bc)
    Q0, E0, b0, run = continuity_run(m, cx, fo, dt, 5, 11)
    y_prev = y = ct.e_ns(Q0)
    y0, s0 = ct.decompose(E0)
    assert np.abs(s0).max() <= 1e-10 * np.abs(y0).max()       # the start has no solenoidal part
    assert np.abs(ct.Cz_e @ (y0 - y)).max() <= 1e-9 * np.abs(y).max()
    s_prev = s = s0
    s1, Bs = s0.copy(), np.zeros(ct.n_cotree_faces)           # reduced first-order state
    Em, bm = E0.copy(), np.zeros(len(ct.jf))                  # MFEM state (b: change since start)
    Escale = max(np.abs(r["E"]).max() for r in run)
    for k, r in enumerate(run):
        y_new = ct.e_ns(r["Q"])
        s_new = ct.wave_step(s, s_prev, y_new, y, y_prev, r["dG"], r["dG_prev"], dt)
        s1, Bs = ct.mfem_reduced_step(s1, Bs, y_new, y, r["dG"], dt)
        Em, bm = ct.mfem_step(Em, bm, r["dG"], dt)
        E_ref = r["E"]
        db_ref = (r["b"] - b0)[ct.jf]
        tol = 1e-9 * Escale
        assert np.abs(ct.compose(y_new, s_new) - E_ref).max() <= tol, k
        assert np.abs(ct.compose(y_new, s1) - E_ref).max() <= tol, k
        assert np.abs(Em - E_ref).max() <= tol, k
        # Sec. VI.A.2's comparison by components: MFEM's E split by Eq. efld_decomp_flux
        # against the E_ns of Eq. discreteGauss and the E_s of Eq. reducedWaveEqn
        y_m, s_m = ct.decompose(Em)
        assert np.abs(y_m - y_new).max() <= 1e-9 * np.abs(y_new).max(), k
        assert np.abs(s_m - s_new).max() <= 1e-9 * Escale, k
        # db_ref = b - b0 carries the rounding of the 0.1 T background flux b0
        btol = 1e-8 * np.abs(db_ref).max() + (k + 2) * 2.3e-16 * np.abs(b0).max()
        assert np.abs(ct.Lam_b @ Bs - db_ref).max() <= btol, k
        assert np.abs(bm - db_ref).max() <= btol, k
        assert np.abs(ct.Lam_b @ Bs - bm).max() <= 1e-9 * np.abs(bm).max(), k
        s_prev, s, y_prev, y = s, s_new, y, y_new
    # the run excited the solenoidal part (the comparison is not only of E_ns)
    assert np.abs(ct.Lam_e @ s).max() > 1e-4 * Escale


@pytest.mark.parametrize("bc", ["pec", "neumann"])
def test_eigenvalues_and_null_spaces(mesh3, bc):
    """Sec. VI.A.1 and Sec. V on a box with PEC or natural walls (units with eps = mu = 1,
    dt = 2 h).  Static modes of MFEM: the gradients of node potentials (PEC: one per interior
    node; natural: N_n - 1, constants map to zero) and the non-solenoidal fluxes (PEC: N_t - 1
    over the interior faces; natural: N_t), by Euler's relation."""
    cx = mesh3
    h = 1.0 / 3.0
    dt = 2.0 * h
    ct = OC.CoTree(cx, bc, eps=1.0, mu=1.0)
    fo = OF.FieldOracle(cx, dt, eps=1.0, mu=1.0, bc=bc)
    nn, nt = len(ct.inn), cx.n_tets
    n_grad = nn if bc == "pec" else nn - 1
    n_div = nt - 1 if bc == "pec" else nt
    G_m = ct.mfem_amplification(dt)
    G_r = ct.reduced_amplification(dt)
    mu_m = np.linalg.eigvals(G_m)
    mu_r = np.linalg.eigvals(G_r)
    assert np.abs(np.abs(mu_m) - 1.0).max() < 1e-8
    assert np.abs(np.abs(mu_r) - 1.0).max() < 1e-8
    static = np.abs(mu_m - 1.0) < 1e-6
    assert static.sum() == n_grad + n_div
    assert not (np.abs(mu_r - 1.0) < 1e-6).any()
    # the reduced system keeps exactly MFEM's dynamic spectrum
    ang_m = np.sort(np.angle(mu_m[~static]))
    ang_r = np.sort(np.angle(mu_r))
    assert ang_m.shape == ang_r.shape
    assert np.abs(ang_m - ang_r).max() < 1e-8
    # MFEM: a gradient E is a fixed point with no Jordan chain (rank(G-I) = rank((G-I)^2))
    nf = len(ct.jf)
    rng = np.random.default_rng(2)
    gphi = ct.grad @ rng.uniform(-1, 1, nn)
    v = np.concatenate([np.zeros(nf), gphi])
    assert np.abs(G_m @ v - v).max() <= 1e-10 * np.abs(v).max()
    Im = np.eye(G_m.shape[0])
    r1 = np.linalg.matrix_rank(G_m - Im, tol=1e-8)
    r2 = np.linalg.matrix_rank((G_m - Im) @ (G_m - Im), tol=1e-8)
    assert r1 == r2 == G_m.shape[0] - (n_grad + n_div)
    # WE-FEM (state E^n, E^{n-1}): the gradient modes form Jordan chains, E^n = (n+1) grad phi
    G_w = fo.amplification_matrix()
    assert np.abs(np.abs(np.linalg.eigvals(G_w)) - 1.0).max() < 1e-6
    v1 = np.concatenate([gphi, gphi])
    v2 = np.concatenate([2.0 * gphi, gphi])
    assert np.abs(G_w @ v1 - v1).max() <= 1e-9 * np.abs(v1).max()
    assert np.abs(G_w @ v2 - v2 - v1).max() <= 1e-9 * np.abs(v1).max()
    Iw = np.eye(G_w.shape[0])
    rw1 = np.linalg.matrix_rank(G_w - Iw, tol=1e-8)
    rw2 = np.linalg.matrix_rank((G_w - Iw) @ (G_w - Iw), tol=1e-8)
    assert rw1 == G_w.shape[0] - n_grad and rw2 == G_w.shape[0] - 2 * n_grad


def test_eigenvalue_experiment_at_the_papers_resolution():
    """Sec. VI.A.1: a PEC box of side 1 m, average edge about 0.214 m (here the jittered 6^3
    cube, 0.209 m), Newmark far beyond any explicit limit (dt = 10 h / c): every eigenvalue of
    the full MFEM and of the reduced first-order system lies on the unit circle, and the reduced
    system keeps exactly MFEM's dynamic spectrum (units with eps = mu = 1)."""
    m = I.cube_mesh(6, 1.0, 0.1, seed=1)
    cx = O.Complex(m.xyz, m.tets)
    edge = np.linalg.norm(cx.xyz[cx.edges[:, 1]] - cx.xyz[cx.edges[:, 0]], axis=1).mean()
    assert 0.2 < edge < 0.22
    ct = OC.CoTree(cx, "pec", eps=1.0, mu=1.0)
    dt = 10.0 / 6.0
    mu_m = np.linalg.eigvals(ct.mfem_amplification(dt))
    mu_r = np.linalg.eigvals(ct.reduced_amplification(dt))
    assert np.abs(np.abs(mu_m) - 1.0).max() < 1e-10
    assert np.abs(np.abs(mu_r) - 1.0).max() < 1e-10
    static = np.abs(mu_m - 1.0) < 1e-6
    assert static.sum() == len(ct.inn) + cx.n_tets - 1
    assert not (np.abs(mu_r - 1.0) < 1e-6).any()
    assert np.abs(np.sort(np.angle(mu_m[~static])) - np.sort(np.angle(mu_r))).max() < 1e-8


def test_gauss_error_grows_in_we_fem_only(mesh4, trees4):
    """A gradient error left by one inexact solve: WE-FEM's Gauss residual grows linearly,
    MFEM's stays where it was, and the projection removes it."""
    m, cx = mesh4
    ct = trees4["pec"]
    dt = 0.2 * I.gyro_period(0.1)
    fo = OF.FieldOracle(cx, dt)
    rng = np.random.default_rng(9)
    phi = np.zeros(cx.n_nodes)
    phi[fo.inn] = rng.uniform(-1, 1, len(fo.inn))
    delta = cx.D0() @ phi
    zero_e, zero_q = np.zeros(cx.n_edges), np.zeros(cx.n_nodes)
    r0 = np.abs(fo.gauss_residual(delta, zero_q)[0]).max()
    # WE-FEM without projection: E^{-1} = 0, E^0 = delta (the erroneous solve)
    Ep, Ec = zero_e.copy(), delta.copy()
    Em, bm = delta.copy(), np.zeros(len(ct.jf))
    Eq_p, Eq = zero_e.copy(), delta.copy()
    for n in range(1, 9):
        Ep, Ec = Ec, fo.newmark(Ec, Ep, zero_e, zero_e)
        Em, bm = ct.mfem_step(Em, bm, zero_e, dt)
        En = fo.newmark(Eq, Eq_p, zero_e, zero_e)
        Eq_p, Eq = Eq, fo.gauss_project(En, zero_q)[0]
        rw = np.abs(fo.gauss_residual(Ec, zero_q)[0]).max()
        rm = np.abs(fo.gauss_residual(Em, zero_q)[0]).max()
        rq = np.abs(fo.gauss_residual(Eq, zero_q)[0]).max()
        assert abs(rw / r0 - (n + 1)) < 1e-6 * (n + 1), n
        assert abs(rm / r0 - 1.0) < 1e-6, n
        assert rq <= 1e-10 * r0, n
