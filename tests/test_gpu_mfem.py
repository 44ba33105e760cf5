"""The comparison systems on the GPU (Sec. V, VI): the first-order mixed FEM, the wave-equation
FEM without the Gauss-law projection, and the Gauss-law residual, against the oracle.

* The face mass [*mu^-1] equals the oracle's quadrature, and [curl]^T [*mu^-1] [curl] equals
  the library's own [*S].
* From a solenoidal start (E = the co-tree field of random coefficients, b = 0) the MFEM step
  follows the oracle's MFEM step by step; the unprojected wave step started from MFEM's first
  two levels reproduces MFEM's later levels (the two are one recursion, Sec. V).
* The Gauss-law residual equals the oracle's, under both boundaries and both precisions.
* A gradient error left in E grows linearly under the wave step, stays constant under MFEM and
  is removed by the projected step: the null-space behaviour of Sec. V and Sec. VI.B.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from paper_2103_06737_gb300 import inputs as I
import oracle as O
from oracle import cotree as OC
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
def mesh4():
    m = I.cube_mesh(4, 1.0, 0.1, seed=1)
    return m, O.Complex(m.xyz, m.tets)


def _setup(m, prec, dt, bc):
    lib = F.FemPic(m.xyz, m.tets, prec)
    F.fem_pic_field_setup(lib.h, dt, bc=F.FP_BC_NEUMANN if bc == "neumann" else F.FP_BC_PEC)
    return lib, F.fem_pic_mfem_create(lib.h)


def test_face_mass_and_curl_curl(mesh4):
    m, cx = mesh4
    lib, mh = _setup(m, F.FP_FP64, 1e-10, "pec")
    rp, col, val = F.fem_pic_mfem_face_mass(lib.h, mh)
    Fg = sp.csr_matrix((val, col, rp), shape=(cx.n_faces, cx.n_faces))
    Fo = OF.face_mass(cx)
    assert abs(Fg - Fo).max() <= 1e-12 * abs(Fo).max()
    D1 = cx.D1().astype(np.float64)
    rp, col, val = F.fem_pic_field_matrix(lib.h, 1)
    S_lib = sp.csr_matrix((val, col, rp), shape=(cx.n_edges, cx.n_edges))
    free = np.nonzero(~cx.boundary_edge)[0]
    S_mf = (D1.T @ Fg @ D1)[free][:, free]
    assert abs(S_mf - S_lib[free][:, free]).max() <= 1e-12 * abs(S_lib).max()
    F.fem_pic_mfem_destroy(mh)
    # a new field setup retires the handle
    mh = F.fem_pic_mfem_create(lib.h)
    F.fem_pic_field_setup(lib.h, 2e-10)
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    E = torch.zeros(cx.n_edges, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FemPicError):
        F.fem_pic_mfem_gauss_residual(lib.h, mh, E, None, out)
    F.fem_pic_mfem_destroy(mh)
    lib.close()


@pytest.mark.parametrize("bc", ["pec", "neumann"])
def test_mfem_and_wave_steps_match_oracle(mesh4, bc):
    m, cx = mesh4
    dt = 2.0 * 0.25 / I.C_LIGHT                      # two cells per step at c: strong dynamics
    ct = OC.CoTree(cx, bc)
    lib, mh = _setup(m, F.FP_FP64, dt, bc)
    rng = np.random.default_rng(21)
    E0 = ct.compose(np.zeros(ct.gauss.shape[0]), rng.uniform(-1, 1, ct.n_cotree_edges))
    zero_g = np.zeros(cx.n_edges)
    Em, bm = E0.copy(), np.zeros(len(ct.jf))
    Ed = [torch.as_tensor(E0, device="cuda"), torch.empty(cx.n_edges, dtype=torch.float64, device="cuda")]
    bd = torch.zeros(cx.n_faces, dtype=torch.float64, device="cuda")
    hist_E, hist_b = [E0.copy()], [np.zeros(cx.n_faces)]
    for k in range(6):
        Em, bm = ct.mfem_step(Em, bm, zero_g, dt)
        st, info = F.fem_pic_mfem_step(lib.h, mh, Ed[0], Ed[1], bd, None, tol=1e-12, precond=F.FP_PC_JACOBI_FP64)
        assert st == F.FP_OK and info["rel_res"] <= 1e-12, info
        E_gpu, b_gpu = Ed[1].cpu().numpy(), bd.cpu().numpy()
        escale, bscale = np.abs(Em).max(), np.abs(bm).max()
        assert np.abs(E_gpu - Em).max() <= 1e-8 * escale, k
        assert np.abs(b_gpu[ct.jf] - bm).max() <= 1e-8 * bscale, k
        if bc == "pec":
            assert np.abs(b_gpu[cx.boundary_face]).max() <= 1e-12 * bscale
        hist_E.append(E_gpu.copy())
        hist_b.append(b_gpu.copy())
        Ed = [Ed[1], Ed[0]]
    # the solenoidal start made the fields move
    assert np.abs(hist_E[-1] - hist_E[0]).max() > 0.1 * np.abs(E0).max()
    # the unprojected wave step from MFEM's levels 0 and 1 gives MFEM's levels 2..6
    Ep = torch.as_tensor(hist_E[0], device="cuda")
    Ec = torch.as_tensor(hist_E[1], device="cuda")
    En = torch.empty_like(Ec)
    bw = torch.as_tensor(hist_b[1], device="cuda")
    for k in range(2, 7):
        st, info = F.fem_pic_wave_step(lib.h, mh, Ep, Ec, En, bw, None, None, tol=1e-12,
                                       precond=F.FP_PC_JACOBI_FP64)
        assert st == F.FP_OK, info
        ref = hist_E[k]
        assert np.abs(En.cpu().numpy() - ref).max() <= 1e-7 * np.abs(ref).max(), k
        assert np.abs(bw.cpu().numpy() - hist_b[k]).max() <= 1e-7 * np.abs(hist_b[k]).max(), k
        Ep, Ec, En = Ec, En, Ep
    F.fem_pic_mfem_destroy(mh)
    lib.close()


@pytest.mark.parametrize("bc", ["pec", "neumann"])
@pytest.mark.parametrize("prec", [F.FP_FP64, F.FP_FP32])
def test_gauss_residual_matches_oracle(mesh4, bc, prec):
    m, cx = mesh4
    fo = OF.FieldOracle(cx, 1e-10, bc=bc)
    lib, mh = _setup(m, prec, 1e-10, bc)
    rng = np.random.default_rng(4)
    E = rng.uniform(-1, 1, cx.n_edges)
    if bc == "pec":
        E[cx.boundary_edge] = 0.0
    Q = rng.uniform(-1e-11, 1e-11, cx.n_nodes) + 3e-12
    R = torch.float32 if prec == F.FP_FP32 else torch.float64
    Qd = torch.as_tensor(Q, device="cuda").to(R)
    Qr = Qd.double().cpu().numpy()                    # the charge the library sees
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    F.fem_pic_mfem_gauss_residual(lib.h, mh, torch.as_tensor(E, device="cuda"), Qd, out)
    r, sc = fo.gauss_residual(E, Qr)
    o = out.cpu().numpy()
    assert abs(o[0] - np.abs(r).max()) <= 1e-11 * sc.max()
    assert abs(o[1] - sc.max()) <= 1e-11 * sc.max()
    F.fem_pic_mfem_destroy(mh)
    lib.close()


def test_gradient_error_growth(mesh4):
    """E = E_Q + delta with delta a gradient (the error an inexact solve leaves) and no current:
    the wave step's Gauss residual after n steps is (n+1) times delta's, MFEM's stays at delta's,
    and the projected step removes it."""
    m, cx = mesh4
    dt = 0.2 * I.gyro_period(0.1)
    lib, mh = _setup(m, F.FP_FP64, dt, "pec")
    rng = np.random.default_rng(8)
    Q = np.zeros(cx.n_nodes)
    Q[~cx.boundary_node] = rng.uniform(-1e-12, 1e-12, (~cx.boundary_node).sum())
    Qd = torch.as_tensor(Q, device="cuda")
    EQ = torch.empty(cx.n_edges, dtype=torch.float64, device="cuda")
    st, _ = F.fem_pic_field_initial(lib.h, Qd, EQ, tol=1e-12)
    assert st == F.FP_OK
    phi = np.zeros(cx.n_nodes)
    phi[~cx.boundary_node] = rng.uniform(-1, 1, (~cx.boundary_node).sum()) * np.abs(EQ.cpu().numpy()).max()
    delta = torch.as_tensor(cx.D0() @ phi, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")

    def res(E):
        F.fem_pic_mfem_gauss_residual(lib.h, mh, E, Qd, out)
        return out[0].item()

    r0 = res(EQ + delta)
    assert r0 > 1e3 * res(EQ)
    Ew = [EQ.clone(), EQ + delta, torch.empty_like(EQ)]        # wave step: E^{-1}, E^0
    Em = [EQ + delta, torch.empty_like(EQ)]                     # MFEM
    bm = torch.zeros(cx.n_faces, dtype=torch.float64, device="cuda")
    Eq = [EQ.clone(), EQ + delta, torch.empty_like(EQ)]        # projected step
    for n in range(1, 7):
        st, _ = F.fem_pic_wave_step(lib.h, mh, Ew[0], Ew[1], Ew[2], None, None, None, tol=1e-11)
        assert st == F.FP_OK
        Ew = [Ew[1], Ew[2], Ew[0]]
        st, _ = F.fem_pic_mfem_step(lib.h, mh, Em[0], Em[1], bm, None, tol=1e-11)
        assert st == F.FP_OK
        Em = [Em[1], Em[0]]
        st, _ = F.fem_pic_field_step(lib.h, Eq[0], Eq[1], Eq[2], None, None, None, Qd, tol=1e-10)
        assert st == F.FP_OK
        Eq = [Eq[1], Eq[2], Eq[0]]
        assert abs(res(Ew[1]) / r0 - (n + 1)) <= 1e-6 * (n + 1), n
        assert abs(res(Em[0]) / r0 - 1.0) <= 1e-6, n
        assert res(Eq[1]) <= 1e-9 * r0, n
    F.fem_pic_mfem_destroy(mh)
    lib.close()
