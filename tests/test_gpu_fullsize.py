"""Parity at the full size of the benchmark workload: the 32^3 x 6 jittered mesh with 2M
electrons (dt = 0.2 gyro-periods at B0 = 0.1 T), FP32 particle path, in the configuration
bench.py times: cell-sorted state (the staged bulk-copy push kernel with its shared-memory
record windows), the mixed-precision field solver.

The FP64 oracle steps all 2M particles (C, OpenMP), so the comparison is element by element:
velocities against the oracle push from the same FP32 start state, cells bit-exact against
the oracle walk on the GPU's own FP32 end points, deposits within the FP32 tolerance.  One
implicit field step on the oracle's deposits is compared with the oracle's field step.
"""
import numpy as np
import pytest
import torch

from paper_2103_06737_gb300 import inputs as I
import oracle as O
from oracle import fields as OF
from helpers import TOL, assert_deposit_close, fp32_continuity_tol

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_2103_06737_gb300.fem_pic")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2103_06737_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def workload():
    wl = I.config(2)
    orc = O.Oracle(wl.mesh.xyz, wl.mesh.tets)
    return wl, orc


def test_push_deposit_full_size(workload):
    wl, orc = workload
    sp = wl.species[0]
    lib = F.FemPic(wl.mesh.xyz, wl.mesh.tets, F.FP_FP32)
    d0 = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    d = d0.empty_like()
    lib.sort(d0, d)
    assert d.n == 2_000_000 and d.n % 4 == 0
    # fields: the uniform B0 plus a seeded random E of 1e3 V/m times the edge length
    cx = orc.cx
    rng = np.random.default_rng(11)
    ev = cx.xyz[cx.edges[:, 1]] - cx.xyz[cx.edges[:, 0]]
    e = 1e3 * np.linalg.norm(ev, axis=1) * rng.uniform(-1.0, 1.0, cx.n_edges)
    e[cx.boundary_edge] = 0.0
    _, b = cx.project_uniform((0.0, 0.0, 0.0), wl.B0)
    cell0 = d.cell.cpu().numpy().copy()
    off0 = d.off.cpu().numpy().copy()
    v0 = d.vel.cpu().numpy().copy()
    ed = torch.as_tensor(e, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    dG = torch.empty(cx.n_edges, dtype=torch.float32, device="cuda")
    Q = torch.empty(cx.n_nodes, dtype=torch.float32, device="cuda")
    Q0 = torch.empty_like(Q)
    lib.deposit_charge(d, Q0)
    lib.push_deposit(ed, bd, d, wl.dt, dG, Q)
    assert lib.status() == F.FP_OK
    res = torch.zeros(6, dtype=torch.float64, device="cuda")
    lib.residuals(dG, Q, Q0, bd, res)
    o = orc.origin(cell0)
    Xa = o + off0.T.astype(np.float64)
    Va = v0.T.astype(np.float64)
    ref_push = orc.step(cell0, Xa, Va, e, b, sp.q, sp.m, sp.w, wl.dt)
    V1 = d.vel.double().cpu().numpy().T
    assert np.abs(V1 - ref_push["V"]).max() <= TOL["fp32"] * np.abs(ref_push["V"]).max()
    v1f = d.vel.cpu().numpy()
    end = (off0 + np.float32(wl.dt) * v1f).astype(np.float32)   # two roundings, as on the GPU
    ref = orc.step(cell0, Xa, Va, e, b, sp.q, sp.m, sp.w, wl.dt, Xend=o + end.T.astype(np.float64))
    cell1 = d.cell.cpu().numpy()
    assert np.array_equal(cell1, ref["cell"])
    alive = cell1 >= 0
    X1 = lib.positions(d).cpu().numpy()
    assert np.abs(X1[alive] - ref["X"][alive]).max() <= 1e-6
    assert_deposit_close(dG.cpu().numpy(), ref["dG"], ref["dG_abs"], TOL["fp32"], "dG")
    assert_deposit_close(Q.cpu().numpy(), ref["Q"], ref["Q_abs"], TOL["fp32"], "Q")
    r = res.cpu().numpy()
    assert r[0] <= fp32_continuity_tol(d.n, cx.n_nodes, cx.n_edges) * r[1]
    assert r[2] <= 1e-13 * r[3]
    lib.close()


def test_field_step_full_size(workload):
    """One implicit field step (mixed solver, FP32 deposits) on the oracle's own deposits."""
    wl, orc = workload
    cx = orc.cx
    fo = OF.FieldOracle(cx, wl.dt)
    sp = wl.species[0]
    lib = F.FemPic(wl.mesh.xyz, wl.mesh.tets, F.FP_FP32)
    F.fem_pic_field_setup(lib.h, wl.dt)
    _, b0 = cx.project_uniform((0.0, 0.0, 0.0), wl.B0)
    Q0, _ = orc.charge(sp.cell, sp.X, sp.q, sp.w)
    alpha = F.fem_pic_whitney0_integrals(lib.h)
    Q_ion = -alpha * Q0.sum() / alpha.sum()          # immobile ions, node charge proportional to the W0 integrals
    E0 = fo.initial_field(Q0 + Q_ion)
    r = orc.step(sp.cell, sp.X, sp.V, E0, b0, sp.q, sp.m, sp.w, wl.dt)
    Q1 = r["Q"] + Q_ion
    E1_r, b1_r = fo.step(E0, E0, b0, r["dG"], np.zeros(cx.n_edges), Q1)
    Ep = torch.as_tensor(E0, device="cuda")
    Ec = Ep.clone()
    En = torch.empty_like(Ec)
    bd = torch.as_tensor(b0, device="cuda")
    dGh = torch.as_tensor(r["dG"], device="cuda").float()
    dGp = torch.zeros_like(dGh)
    Qn = torch.as_tensor(Q1, device="cuda").float()
    st, info = F.fem_pic_field_step(lib.h, Ep, Ec, En, bd, dGh, dGp, Qn, tol=1e-10)
    assert st == F.FP_OK, info
    assert info[0]["rel_res"] <= 1e-10 and info[1]["rel_res"] <= 1e-10
    E1 = En.cpu().numpy()
    assert np.abs(E1 - E1_r).max() <= 1e-5 * np.abs(E1_r).max()   # FP32 deposits on the GPU side
    assert np.abs(bd.cpu().numpy() - b1_r).max() <= 1e-5 * np.abs(b1_r).max() + 1e-14
    g, sc = fo.gauss_residual(E1, Qn.double().cpu().numpy())
    assert np.abs(g).max() <= 1e-9 * sc.max()
    lib.close()


def test_adams_step_full_size(workload):
    """The fourth-order Adams particle step (order 4, history from earlier steps' shape) on all
    2M sorted electrons, in the launch configuration the benchmark times it in."""
    from oracle import adams as AD
    wl, orc = workload
    sp = wl.species[0]
    lib = F.FemPic(wl.mesh.xyz, wl.mesh.tets, F.FP_FP32)
    d0 = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    n = d0.n
    rng = np.random.default_rng(12)
    dt = wl.dt / 4
    # history: the current velocities with a small seeded perturbation, accelerations of the
    # size the uniform B0 gives (|q/m| v B0)
    v = sp.V.T
    wc = abs(sp.q / sp.m) * np.linalg.norm(wl.B0)
    h = np.empty((18, n))
    for s in range(3):
        h[6 * s:6 * s + 3] = v * (1.0 + 0.01 * rng.standard_normal((3, n)))
        h[6 * s + 3:6 * s + 6] = wc * v[[1, 0, 2]] * rng.uniform(-1, 1, (3, n))
    hist0 = torch.as_tensor(h, device="cuda").float().contiguous()
    d = d0.empty_like()
    hist = torch.empty_like(hist0)
    lib.sort_columns(d0, d, hist0, hist, 18)
    cx = orc.cx
    e = 1e3 * np.linalg.norm(cx.xyz[cx.edges[:, 1]] - cx.xyz[cx.edges[:, 0]], axis=1) * \
        np.random.default_rng(11).uniform(-1.0, 1.0, cx.n_edges)
    e[cx.boundary_edge] = 0.0
    _, b = cx.project_uniform((0.0, 0.0, 0.0), wl.B0)
    cell0 = d.cell.cpu().numpy().copy()
    off0 = d.off.cpu().numpy().copy()
    v0 = d.vel.cpu().numpy().copy()
    h_in = hist.cpu().numpy().copy()
    ed = torch.as_tensor(e, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    dG = torch.empty(cx.n_edges, dtype=torch.float32, device="cuda")
    Q = torch.empty(cx.n_nodes, dtype=torch.float32, device="cuda")
    step = 3
    lib.push_deposit_adams(ed, bd, d, hist, step, dt, dG, Q)
    assert lib.status() == F.FP_OK
    # end points as the library rounds them (FP32, operation by operation)
    beta = [np.float32(x) for x in AD.ab_coefficients(4)]
    hs = None
    for j in range(1, 4):
        sl = (step - j) % 3
        t = (beta[j] * h_in[6 * sl:6 * sl + 3]).astype(np.float32)
        hs = t if hs is None else (hs + t).astype(np.float32)
    acc = ((beta[0] * v0).astype(np.float32) + hs).astype(np.float32)
    end = (off0 + (np.float32(dt) * acc).astype(np.float32)).astype(np.float32)
    o = orc.origin(cell0)
    Xa = o + off0.T.astype(np.float64)
    hv = np.stack([h_in[6 * s:6 * s + 3].T for s in range(3)]).astype(np.float64)
    ha = np.stack([h_in[6 * s + 3:6 * s + 6].T for s in range(3)]).astype(np.float64)
    ref = AD.adams_step(orc, cell0, Xa, v0.T.astype(np.float64), hv, ha, step, e, b, sp.q, sp.m, sp.w, dt,
                        Xend=o + end.T.astype(np.float64))
    V1 = d.vel.double().cpu().numpy().T
    assert np.abs(V1 - ref["V"]).max() <= TOL["fp32"] * np.abs(ref["V"]).max()
    hs = hist.cpu().numpy()
    assert np.array_equal(hs[0:3], v0)                       # slot 3 % 3 = 0 takes v^n
    assert np.array_equal(hs[6:18], h_in[6:18])
    cell1 = d.cell.cpu().numpy()
    assert np.array_equal(cell1, ref["cell"])
    alive = cell1 >= 0
    X1 = lib.positions(d).cpu().numpy()
    assert np.abs(X1[alive] - ref["X"][alive]).max() <= 1e-6
    assert_deposit_close(dG.cpu().numpy(), ref["dG"], ref["dG_abs"], TOL["fp32"], "dG")
    assert_deposit_close(Q.cpu().numpy(), ref["Q"], ref["Q_abs"], TOL["fp32"], "Q")
    lib.close()
