"""The library's field step against the paper's tree / co-tree reduced system (Sec. IV.B).

The library advances E by Newmark on the full edge wave equation followed by the Gauss-law
projection.  Here its FP64 field steps, fed the oracle's charge-conserving deposits, are
split into E_ns and the co-tree coefficients E_s (Eq. efld_decomp_flux) and compared with
the oracle's Newmark solution of the reduced wave equation (Eq. reducedWaveEqn, E_ns from
Eq. discreteGauss); the library's Faraday update is compared with the reduced first-order
system's B_s (Eq. reduceMEs) and with the first-order mixed FEM.  Both field boundaries.

Solves stop at a relative residual of 1e-10, so fields are compared at 1e-8 of their scale
(as in the other field tests); b depends on the solenoidal part only, a few per cent of E
here, and is compared at the error that E's tolerance allows through one Faraday update.
"""
import numpy as np
import pytest
import torch

from paper_2103_06737_gb300 import inputs as I
import oracle as O
from oracle import cotree as OC
from oracle import fields as OF

from helpers import continuity_run

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_2103_06737_gb300.fem_pic")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2103_06737_gb300 import build
    build.build()


@pytest.mark.parametrize("bc", ["pec", "neumann"])
def test_field_steps_match_the_reduced_system(bc):
    m = I.cube_mesh(4, 1.0, 0.1, seed=1)
    cx = O.Complex(m.xyz, m.tets)
    dt = 0.2 * I.gyro_period(0.1)
    fo = OF.FieldOracle(cx, dt, bc=bc)
    ct = OC.CoTree(cx, bc)
    Q0, E0, b0, run = continuity_run(m, cx, fo, dt, 6, 11)

    lib = F.FemPic(m.xyz, m.tets, F.FP_FP64)
    F.fem_pic_field_setup(lib.h, dt, bc=F.FP_BC_NEUMANN if bc == "neumann" else F.FP_BC_PEC)
    Ed = torch.empty(cx.n_edges, dtype=torch.float64, device="cuda")
    st, info = F.fem_pic_field_initial(lib.h, torch.as_tensor(Q0, device="cuda"), Ed, tol=1e-10)
    assert st == F.FP_OK and info["rel_res"] <= 1e-10
    Ep, Ec = Ed.clone(), Ed.clone()
    En = torch.empty_like(Ec)
    bd = torch.as_tensor(b0, device="cuda").clone()
    dGp = torch.zeros(cx.n_edges, dtype=torch.float64, device="cuda")

    # E_s and E_ns are linear in E; their tolerances are E's times the gain of that map
    # (the co-tree coefficients are circulations around fundamental cycles)
    Ms = np.linalg.solve(ct.Z21, ct.Cc_e.T @ ct.P_lambda_e @ ct.M)
    My = np.linalg.solve(ct.gauss, ct.Cz_e.T @ ct.grad.T @ ct.M)
    gain_s = np.abs(Ms).sum(axis=1).max()
    gain_y = np.abs(My).sum(axis=1).max()
    # the reduced systems' start: E_s = 0 (the initial field is a gradient), B_s = 0
    y_prev = y = ct.e_ns(Q0)
    y_lib, s_lib = ct.decompose(Ed.cpu().numpy())
    Escale = max(np.abs(r["E"]).max() for r in run)
    assert np.abs(s_lib).max() <= gain_s * 1e-8 * Escale
    assert np.abs(y_lib - y).max() <= gain_y * 1e-8 * Escale
    s_prev = s = np.zeros(ct.n_cotree_edges)
    s1, Bs = s.copy(), np.zeros(ct.n_cotree_faces)
    Em, bm = E0.copy(), np.zeros(len(ct.jf))
    for k, r in enumerate(run):
        dGh = torch.as_tensor(r["dG"], device="cuda")
        Qn = torch.as_tensor(r["Q"], device="cuda")
        st, info = F.fem_pic_field_step(lib.h, Ep, Ec, En, bd, dGh, dGp, Qn, tol=1e-10)
        assert st == F.FP_OK, info
        assert info[0]["rel_res"] <= 1e-10 and info[1]["rel_res"] <= 1e-10
        y_new = ct.e_ns(r["Q"])
        s_new = ct.wave_step(s, s_prev, y_new, y, y_prev, r["dG"], r["dG_prev"], dt)
        s1, Bs = ct.mfem_reduced_step(s1, Bs, y_new, y, r["dG"], dt)
        Em, bm = ct.mfem_step(Em, bm, r["dG"], dt)

        E_gpu = En.cpu().numpy()
        y_gpu, s_gpu = ct.decompose(E_gpu)
        assert np.abs(E_gpu - ct.compose(y_new, s_new)).max() <= 1e-8 * Escale, k
        assert np.abs(y_gpu - y_new).max() <= gain_y * 1e-8 * Escale, k
        assert np.abs(s_gpu - s_new).max() <= gain_s * 1e-8 * Escale, k
        assert np.abs(s_gpu - s1).max() <= gain_s * 1e-8 * Escale, k
        assert np.abs(E_gpu - Em).max() <= 1e-8 * Escale, k
        db_gpu = (bd.cpu().numpy() - b0)[ct.jf]
        btol = 2.0 * dt * 3.0 * 1e-8 * Escale * (k + 1) + (k + 2) * 2.3e-16 * np.abs(b0).max()
        assert np.abs(db_gpu - ct.Lam_b @ Bs).max() <= btol, k
        assert np.abs(db_gpu - bm).max() <= btol, k

        Ep, Ec, En = Ec, En, Ep
        dGp = dGh
        s_prev, s, y_prev, y = s, s_new, y, y_new
    # the comparison covered a solenoidal part well above its tolerance
    assert np.abs(ct.Lam_e @ s).max() > 1e3 * 1e-8 * Escale
    assert np.abs(s).max() > 1e2 * gain_s * 1e-8 * Escale
    assert np.abs(ct.Lam_b @ Bs).max() > 1e3 * btol
    lib.close()
