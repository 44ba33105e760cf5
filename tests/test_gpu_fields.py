"""Parity of the GPU field operators and implicit field step with the FP64 oracle.

The library assembles [*eps], [*S] and L from closed-form element matrices; the oracle
uses quadrature and the paper's products D1^T [*mu^-1] D1 and D0^T [*eps] D0.  Solves stop
at a relative residual of 1e-10, so solutions are compared within the error that
residual allows (1e-8 relative, a condition-number margin of 100 on these meshes).
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from paper_2103_06737_gb300 import inputs as I
import oracle as O
from oracle import fields as OF

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_2103_06737_gb300.fem_pic")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2103_06737_gb300 import build
    build.build()


def _csr(h, which, n):
    rp, col, val = F.fem_pic_field_matrix(h, which)
    return sp.csr_matrix((val, col, rp), shape=(n, n))


@pytest.fixture(scope="module")
def setup6():
    m = I.cube_mesh(6, 1.0, 0.1, seed=1)
    cx = O.Complex(m.xyz, m.tets)
    dt = 0.2 * I.gyro_period(0.1)
    fo = OF.FieldOracle(cx, dt)
    return m, cx, dt, fo


@pytest.mark.parametrize("prec", [F.FP_FP64])
def test_operators_match_oracle(setup6, prec):
    m, cx, dt, fo = setup6
    lib = F.FemPic(m.xyz, m.tets, prec)
    F.fem_pic_field_setup(lib.h, dt)
    ie, inn = fo.ie, fo.inn
    for which, ref, n, free in ((0, fo.M, cx.n_edges, ie), (1, fo.S, cx.n_edges, ie), (2, fo.A, cx.n_edges, ie),
                                (3, fo.L, cx.n_nodes, inn)):
        got = _csr(lib.h, which, n)
        a = got[free][:, free].toarray()
        r = ref[free][:, free].toarray()
        assert np.abs(a - r).max() <= 1e-12 * np.abs(r).max(), which
        fixed = np.setdiff1d(np.arange(n), free)
        blk = got[fixed]
        if which == 1:
            assert blk.count_nonzero() == 0
        else:
            assert np.array_equal(blk.toarray()[np.arange(fixed.size), fixed], np.ones(fixed.size))
            assert abs(blk).sum() == fixed.size
    lib.close()


@pytest.mark.parametrize("precond", [F.FP_PC_JACOBI, F.FP_PC_JACOBI_FP64])
def test_newmark_solve_matches_direct(setup6, precond):
    m, cx, dt, fo = setup6
    lib = F.FemPic(m.xyz, m.tets, F.FP_FP64)
    F.fem_pic_field_setup(lib.h, dt)
    rng = np.random.default_rng(3)
    rhs = rng.uniform(-1, 1, cx.n_edges) * 1e-12
    rhs[cx.boundary_edge] = 0.0
    x_ref = np.zeros(cx.n_edges)
    x_ref[fo.ie] = OF._solve(fo.A_II, rhs[fo.ie])
    x = torch.zeros(cx.n_edges, dtype=torch.float64, device="cuda")
    st, info = F.fem_pic_field_solve(lib.h, F.FP_SYS_NEWMARK, torch.as_tensor(rhs, device="cuda"), x, tol=1e-10,
                                     precond=precond)
    assert st == F.FP_OK and info["rel_res"] <= 1e-10 and info["iters"] > 1
    assert np.abs(x.cpu().numpy() - x_ref).max() <= 1e-8 * np.abs(x_ref).max()
    # an iteration cap of 1 reports non-convergence, and the status word records it
    x.zero_()
    st, info = F.fem_pic_field_solve(lib.h, F.FP_SYS_NEWMARK, torch.as_tensor(rhs, device="cuda"), x, tol=1e-10,
                                     max_iter=1, precond=precond)
    assert st == F.FP_ENOCONV and info["iters"] == 1
    assert lib.status() == F.FP_ENOCONV
    # the Gauss-law (node Laplacian) system
    g = rng.uniform(-1, 1, cx.n_nodes) * 1e-20
    g[cx.boundary_node] = 0.0
    d_ref = np.zeros(cx.n_nodes)
    d_ref[fo.inn] = OF._solve(fo.L_II, g[fo.inn])
    d = torch.zeros(cx.n_nodes, dtype=torch.float64, device="cuda")
    st, info = F.fem_pic_field_solve(lib.h, F.FP_SYS_GAUSS, torch.as_tensor(g, device="cuda"), d, tol=1e-10,
                                     precond=precond)
    assert st == F.FP_OK and info["rel_res"] <= 1e-10
    assert np.abs(d.cpu().numpy() - d_ref).max() <= 1e-7 * np.abs(d_ref).max()
    lib.close()


def test_chebyshev_inner_preconditioner(setup6):
    """Mixed solver with Chebyshev-Jacobi inner preconditioning: same tolerance and solution,
    fewer CG iterations on the node Laplacian than plain Jacobi."""
    m, cx, dt, fo = setup6
    lib = F.FemPic(m.xyz, m.tets, F.FP_FP64)
    F.fem_pic_field_setup(lib.h, dt)
    rng = np.random.default_rng(4)
    g = rng.uniform(-1, 1, cx.n_nodes) * 1e-20
    g[cx.boundary_node] = 0.0
    d_ref = np.zeros(cx.n_nodes)
    d_ref[fo.inn] = OF._solve(fo.L_II, g[fo.inn])
    rhs = rng.uniform(-1, 1, cx.n_edges) * 1e-12
    rhs[cx.boundary_edge] = 0.0
    x_ref = np.zeros(cx.n_edges)
    x_ref[fo.ie] = OF._solve(fo.A_II, rhs[fo.ie])
    iters = {}
    for deg in (1, 4):
        F.fem_pic_field_poly(lib.h, F.FP_SYS_GAUSS, deg, 30.0)
        F.fem_pic_field_poly(lib.h, F.FP_SYS_NEWMARK, deg, 30.0)
        d = torch.zeros(cx.n_nodes, dtype=torch.float64, device="cuda")
        st, info = F.fem_pic_field_solve(lib.h, F.FP_SYS_GAUSS, torch.as_tensor(g, device="cuda"), d, tol=1e-10,
                                         precond=F.FP_PC_JACOBI)
        assert st == F.FP_OK and info["rel_res"] <= 1e-10
        assert np.abs(d.cpu().numpy() - d_ref).max() <= 1e-7 * np.abs(d_ref).max()
        iters[deg] = info["iters"]
        x = torch.zeros(cx.n_edges, dtype=torch.float64, device="cuda")
        st, info = F.fem_pic_field_solve(lib.h, F.FP_SYS_NEWMARK, torch.as_tensor(rhs, device="cuda"), x,
                                         tol=1e-10, precond=F.FP_PC_JACOBI)
        assert st == F.FP_OK and info["rel_res"] <= 1e-10
        assert np.abs(x.cpu().numpy() - x_ref).max() <= 1e-8 * np.abs(x_ref).max()
    assert iters[4] < iters[1]
    with pytest.raises(F.FemPicError):
        F.fem_pic_field_poly(lib.h, F.FP_SYS_GAUSS, 0, 30.0)
    lib.close()


@pytest.mark.parametrize("prec", [F.FP_FP64, F.FP_FP32])
def test_field_steps_match_oracle(setup6, prec):
    """Particles and fields together for a few steps; the GPU field step is fed the
    oracle's own deposits, so the comparison isolates the field solve."""
    m, cx, dt, fo = setup6
    orc = O.Oracle(m.xyz, m.tets)
    lib = F.FemPic(m.xyz, m.tets, prec)
    F.fem_pic_field_setup(lib.h, dt)
    R = torch.float32 if prec == F.FP_FP32 else torch.float64
    sp_ = I.uniform_species(m, 3000, 4, 0.01 * I.C_LIGHT, -I.Q_E, I.M_E, 1e6)
    _, b0 = cx.project_uniform((0, 0, 0), (0, 0, 0.1))
    Q0, _ = orc.charge(sp_.cell, sp_.X, sp_.q, sp_.w)
    E_ref = fo.initial_field(Q0)
    Ed = torch.empty(cx.n_edges, dtype=torch.float64, device="cuda")
    st, info = F.fem_pic_field_initial(lib.h, torch.as_tensor(Q0, device="cuda").to(R), Ed, tol=1e-10)
    assert st == F.FP_OK
    tol_e = 1e-8 if prec == F.FP_FP64 else 1e-5     # FP32 deposits feed the FP32 path
    assert np.abs(Ed.cpu().numpy() - E_ref).max() <= tol_e * np.abs(E_ref).max()
    E_prev_r, E_r, b_r = E_ref.copy(), E_ref.copy(), b0.copy()
    dGp_r = np.zeros(cx.n_edges)
    Ep = torch.as_tensor(E_ref, device="cuda")
    Ec = Ep.clone()
    En = torch.empty_like(Ec)
    bd = torch.as_tensor(b0, device="cuda")
    dGp = torch.zeros(cx.n_edges, dtype=R, device="cuda")
    cell, X, V = sp_.cell, sp_.X, sp_.V
    for step in range(3):
        r = orc.step(cell, X, V, E_r, b_r, sp_.q, sp_.m, sp_.w, dt)
        cell, X, V = r["cell"], r["X"], r["V"]
        E1_r, b1_r = fo.step(E_r, E_prev_r, b_r, r["dG"], dGp_r, r["Q"])
        dGh = torch.as_tensor(r["dG"], device="cuda").to(R)
        Qn = torch.as_tensor(r["Q"], device="cuda").to(R)
        st, info = F.fem_pic_field_step(lib.h, Ep, Ec, En, bd, dGh, dGp, Qn, tol=1e-10)
        assert st == F.FP_OK, info
        assert info[0]["rel_res"] <= 1e-10 and info[1]["rel_res"] <= 1e-10
        if prec == F.FP_FP64:
            E1 = En.cpu().numpy()
            assert np.abs(E1 - E1_r).max() <= 1e-8 * np.abs(E1_r).max(), step
            assert np.abs(bd.cpu().numpy() - b1_r).max() <= 1e-8 * np.abs(b1_r).max() + 1e-14
            g, sc = fo.gauss_residual(E1, r["Q"])
            assert np.abs(g).max() <= 1e-9 * sc.max()
        # feed the GPU its own field from now on only in FP64; in FP32 reset to the oracle's
        Ep, Ec, En = Ec, En, Ep
        if prec == F.FP_FP32:
            Ec.copy_(torch.as_tensor(E1_r, device="cuda"))
            bd.copy_(torch.as_tensor(b1_r, device="cuda"))
        dGp = dGh
        E_prev_r, E_r, b_r, dGp_r = E_r, E1_r, b1_r, r["dG"]
    # magnetic Gauss law is kept by the Faraday update (D2 D1 = 0)
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    lib.residuals(None, None, None, bd, out)
    o = out.cpu().numpy()
    assert o[2] <= 1e-13 * o[3]
    lib.close()
