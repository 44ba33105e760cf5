"""Pins of the oracle's Whitney gather (Sec. II.C: E in span W1, B in span W2).

The incidence matrices are tied to the Whitney functions by the identities that
define [grad], [curl], [div] for Whitney forms: grad of sum phi_n W0_n is the W1
field with DOFs D0 phi, curl of the W1 field with DOFs e is the W2 field with
DOFs D1 e, and the divergence of the W2 field with DOFs b is (D2 b)_t / |T|.
Each is checked with finite differences of the oracle's own point evaluation,
so a wrong sign or index in W1, W2, D0, D1 or D2 fails here.
"""
import numpy as np

from paper_2103_06737_gb300 import inputs as I
import oracle as O


def _mesh(n=4, jit=0.1, seed=1):
    m = I.cube_mesh(n, 1.0, jit, seed=seed)
    return m, O.Oracle(m.xyz, m.tets)


def _interior_points(orc, m, n, seed):
    sp = I.uniform_species(m, n, seed, 1.0, -1.0, 1.0)
    lam = orc.bary(sp.cell, sp.X)
    keep = lam.min(axis=1) > 1e-3
    return sp.cell[keep], sp.X[keep]


def test_uniform_field_reproduction():
    m, orc = _mesh()
    cell, X = _interior_points(orc, m, 2000, 4)
    E0 = np.array([1.5, -0.25, 2.0])
    B0 = np.array([-0.3, 0.7, 0.1])
    e, b = orc.project_uniform(E0, B0)
    E, B = orc.gather(cell, X, e, b)
    assert np.abs(E - E0).max() < 1e-12
    assert np.abs(B - B0).max() < 1e-12


def _fd(fn, cell, X, h=1e-6):
    """Jacobian of a field linear in each tet by central differences: J[p,i,j] = d F_i / d x_j."""
    J = np.empty((X.shape[0], 3, 3))
    for j in range(3):
        d = np.zeros(3)
        d[j] = h
        J[:, :, j] = (fn(cell, X + d) - fn(cell, X - d)) / (2 * h)
    return J


def test_grad_curl_div_match_incidence():
    m, orc = _mesh()
    cx = orc.cx
    cell, X = _interior_points(orc, m, 500, 5)
    rng = np.random.default_rng(0)
    phi = rng.uniform(-1, 1, cx.n_nodes)
    e = rng.uniform(-1, 1, cx.n_edges)
    b = rng.uniform(-1, 1, cx.n_faces)
    D0, D1, D2 = cx.D0(), cx.D1(), cx.D2()
    zf = np.zeros(cx.n_faces)
    ze = np.zeros(cx.n_edges)

    # grad: field of D0 phi equals grad(sum phi_n lambda_n)
    E_grad, _ = orc.gather(cell, X, D0 @ phi, zf)
    lam_phi = lambda c, x: (orc.bary(c, x) * phi[cx.tv[c]]).sum(axis=1)[:, None] * np.ones(3)
    g = np.stack([(lam_phi(cell, X + d)[:, 0] - lam_phi(cell, X - d)[:, 0]) / 2e-6
                  for d in np.eye(3) * 1e-6], axis=1)
    assert np.abs(E_grad - g).max() < 1e-6 * np.abs(g).max()

    # curl: curl of the W1 field of e equals the W2 field of D1 e
    J = _fd(lambda c, x: orc.gather(c, x, e, zf)[0], cell, X)
    curl = np.stack([J[:, 2, 1] - J[:, 1, 2], J[:, 0, 2] - J[:, 2, 0], J[:, 1, 0] - J[:, 0, 1]], axis=1)
    _, B_curl = orc.gather(cell, X, ze, D1 @ e)
    assert np.abs(curl - B_curl).max() < 1e-6 * np.abs(B_curl).max()

    # div: divergence of the W2 field of b is (D2 b)_t / |T|
    Jb = _fd(lambda c, x: orc.gather(c, x, ze, b)[1], cell, X)
    div = Jb[:, 0, 0] + Jb[:, 1, 1] + Jb[:, 2, 2]
    ref = (D2 @ b)[cell] / cx.vol[cell]
    assert np.abs(div - ref).max() < 1e-6 * np.abs(ref).max()


def test_w1_tangential_and_w2_normal_continuity():
    """Across an interior face the W1 field keeps its tangential part and W2 its normal part."""
    m, orc = _mesh(4, 0.1, 2)
    cx = orc.cx
    rng = np.random.default_rng(1)
    e = rng.uniform(-1, 1, cx.n_edges)
    b = rng.uniform(-1, 1, cx.n_faces)
    inner = np.nonzero(~cx.boundary_face)[0][:200]
    f = cx.faces[inner]
    x = cx.xyz[f]                                    # [n,3,3]
    w = rng.dirichlet([1, 1, 1], size=inner.size)
    P = np.einsum("nk,nkd->nd", w, x)
    nrm = np.cross(x[:, 1] - x[:, 0], x[:, 2] - x[:, 0])
    nrm /= np.linalg.norm(nrm, axis=1)[:, None]
    t0, t1 = cx.face_tets[inner, 0], cx.face_tets[inner, 1]
    E0, B0 = orc.gather(t0, P, e, b)
    E1, B1 = orc.gather(t1, P, e, b)
    tang = lambda v: v - (v * nrm).sum(1)[:, None] * nrm
    assert np.abs(tang(E0) - tang(E1)).max() < 1e-11
    assert np.abs((B0 * nrm).sum(1) - (B1 * nrm).sum(1)).max() < 1e-11
    # and the normal part of W1 does jump for generic e (the test can see a jump)
    assert np.abs((E0 * nrm).sum(1) - (E1 * nrm).sum(1)).max() > 1e-3


def test_divergence_free_b_gives_zero_D2b():
    m, orc = _mesh(4, 0.1, 3)
    cx = orc.cx
    e = np.random.default_rng(2).uniform(-1, 1, cx.n_edges)
    b = cx.D1() @ e      # a curl
    assert np.abs(cx.D2() @ b).max() < 1e-14
