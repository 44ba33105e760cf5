"""The natural (Neumann) field boundary on the GPU against the oracle's zero-mean constrained
projection (Eq. zero_mean_constraint, Sec. IV.B): operators over all DOFs, the initial field
and implicit field steps with a net charge (spread as alpha by the constraint), the Gauss law
at every node, and the mixed-precision solver on the singular node Laplacian.
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


@pytest.fixture(scope="module")
def setup6():
    m = I.cube_mesh(6, 1.0, 0.1, seed=1)
    cx = O.Complex(m.xyz, m.tets)
    dt = 0.2 * I.gyro_period(0.1)
    fo = OF.FieldOracle(cx, dt, bc="neumann")
    return m, cx, dt, fo


def _csr(h, which, n):
    rp, col, val = F.fem_pic_field_matrix(h, which)
    return sp.csr_matrix((val, col, rp), shape=(n, n))


def test_neumann_operators_cover_every_dof(setup6):
    m, cx, dt, fo = setup6
    lib = F.FemPic(m.xyz, m.tets, F.FP_FP64)
    F.fem_pic_field_setup(lib.h, dt, bc=F.FP_BC_NEUMANN)
    A = _csr(lib.h, 2, cx.n_edges)
    L = _csr(lib.h, 3, cx.n_nodes)
    assert abs(A - fo.A).max() <= 1e-12 * abs(fo.A).max()
    assert abs(L - fo.L).max() <= 1e-12 * abs(fo.L).max()
    assert np.abs(L @ np.ones(cx.n_nodes)).max() <= 1e-12 * abs(fo.L).max()   # singular: constants
    with pytest.raises(F.FemPicError):
        F.fem_pic_field_setup(lib.h, dt, bc=7)
    lib.close()


@pytest.mark.parametrize("solver", [F.FP_PC_JACOBI, F.FP_PC_JACOBI_FP64])
def test_neumann_field_steps_match_oracle(setup6, solver):
    """Electrons only (a net charge), FP64 deposits from the oracle's own particle steps."""
    m, cx, dt, fo = setup6
    orc = O.Oracle(m.xyz, m.tets)
    lib = F.FemPic(m.xyz, m.tets, F.FP_FP64)
    F.fem_pic_field_setup(lib.h, dt, bc=F.FP_BC_NEUMANN)
    F.fem_pic_field_options(lib.h, solver, solver, 1e-5)
    sp_ = I.uniform_species(m, 3000, 4, 0.01 * I.C_LIGHT, -I.Q_E, I.M_E, 1e6)
    _, b0 = cx.project_uniform((0, 0, 0), (0, 0, 0.1))
    Q0, _ = orc.charge(sp_.cell, sp_.X, sp_.q, sp_.w)
    E_ref = fo.initial_field(Q0)
    Ed = torch.empty(cx.n_edges, dtype=torch.float64, device="cuda")
    st, info = F.fem_pic_field_initial(lib.h, torch.as_tensor(Q0, device="cuda"), Ed, tol=1e-10)
    assert st == F.FP_OK and info["rel_res"] <= 1e-10
    assert np.abs(Ed.cpu().numpy() - E_ref).max() <= 1e-8 * np.abs(E_ref).max()
    assert np.abs(E_ref[cx.boundary_edge]).max() > 0          # boundary edges are free
    E_prev_r, E_r, b_r = E_ref.copy(), E_ref.copy(), b0.copy()
    dGp_r = np.zeros(cx.n_edges)
    Ep = torch.as_tensor(E_ref, device="cuda")
    Ec = Ep.clone()
    En = torch.empty_like(Ec)
    bd = torch.as_tensor(b0, device="cuda")
    dGp = torch.zeros(cx.n_edges, dtype=torch.float64, device="cuda")
    cell, X, V = sp_.cell, sp_.X, sp_.V
    a = fo.alpha
    for step in range(3):
        r = orc.step(cell, X, V, E_r, b_r, sp_.q, sp_.m, sp_.w, dt)
        cell, X, V = r["cell"], r["X"], r["V"]
        E1_r, b1_r = fo.step(E_r, E_prev_r, b_r, r["dG"], dGp_r, r["Q"])
        dGh = torch.as_tensor(r["dG"], device="cuda")
        Qn = torch.as_tensor(r["Q"], device="cuda")
        st, info = F.fem_pic_field_step(lib.h, Ep, Ec, En, bd, dGh, dGp, Qn, tol=1e-10)
        assert st == F.FP_OK, info
        assert info[0]["rel_res"] <= 1e-10 and info[1]["rel_res"] <= 1e-10
        E1 = En.cpu().numpy()
        assert np.abs(E1 - E1_r).max() <= 1e-8 * np.abs(E1_r).max(), step
        assert np.abs(bd.cpu().numpy() - b1_r).max() <= 1e-8 * np.abs(b1_r).max() + 1e-14
        # Gauss law at every node, less the net charge spread as alpha
        g = fo.D0.T @ (fo.M @ E1) + r["Q"] - r["Q"].sum() / a.sum() * a
        sc = (np.abs(fo.D0.T) @ np.abs(fo.M @ E1) + np.abs(r["Q"])).max()
        assert np.abs(g).max() <= 1e-9 * sc
        Ep, Ec, En = Ec, En, Ep
        dGp = dGh
        E_prev_r, E_r, b_r, dGp_r = E_r, E1_r, b1_r, r["dG"]
    lib.close()


def test_neumann_neutral_charge_full_gauss_law(setup6):
    """A neutral charge (electrons + the alpha-weighted ion background): the projection
    satisfies the Gauss law exactly at every node, boundary nodes included."""
    m, cx, dt, fo = setup6
    orc = O.Oracle(m.xyz, m.tets)
    lib = F.FemPic(m.xyz, m.tets, F.FP_FP32)
    F.fem_pic_field_setup(lib.h, dt, bc=F.FP_BC_NEUMANN)
    sp_ = I.uniform_species(m, 20_000, 6, 0.01 * I.C_LIGHT, -I.Q_E, I.M_E, 1e6)
    Qe, _ = orc.charge(sp_.cell, sp_.X, sp_.q, sp_.w)
    a = fo.alpha
    Q = Qe - Qe.sum() / a.sum() * a
    Ed = torch.empty(cx.n_edges, dtype=torch.float64, device="cuda")
    Qd = torch.as_tensor(Q, device="cuda").float()
    st, info = F.fem_pic_field_initial(lib.h, Qd, Ed, tol=1e-10)
    assert st == F.FP_OK
    E = Ed.cpu().numpy()
    Qf = Qd.double().cpu().numpy()
    g = fo.D0.T @ (fo.M @ E) + Qf - Qf.sum() / a.sum() * a
    sc = (np.abs(fo.D0.T) @ np.abs(fo.M @ E) + np.abs(Qf)).max()
    assert np.abs(g).max() <= 1e-9 * sc
    E_ref = fo.initial_field(Qf)
    assert np.abs(E - E_ref).max() <= 1e-8 * np.abs(E_ref).max()
    lib.close()
