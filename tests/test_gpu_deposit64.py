"""FP64 deposit arrays in an FP32 context (fem_pic_set_deposit_precision).

The FP32 push still forms each particle's W1 current and W0 charge contributions (Sec. IV.B.1)
and the fast push's run sums in FP32, but adds them into double dG and Q.  The deposits then
meet the FP32 tolerance of the parity tests against the FP64 oracle, the continuity residual
D0^T dG - (Q_new - Q_old) shrinks by well over an order of magnitude against float arrays
(whose atomic sums round at the scale of each entry's total), and the field step's Gauss-law
projection, whose right-hand side is that residual, needs fewer iterations to the same 1e-10.
"""
import numpy as np
import pytest
import torch

from paper_2103_06737_gb300 import inputs as I
import oracle as O
from helpers import TOL, assert_deposit_close

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_2103_06737_gb300.fem_pic")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2103_06737_gb300 import build
    build.build()


def _state(lib, sp, sort):
    d = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    if sort:
        s = d.empty_like()
        lib.sort(d, s)
        d = s
    return d


def _push(lib, orc, d0, e, b, dtype):
    """One push of a copy of the state d0 into deposit arrays of the given dtype."""
    d = d0.empty_like()
    d.cell.copy_(d0.cell)
    d.off.copy_(d0.off)
    d.vel.copy_(d0.vel)
    cell0 = d.cell.cpu().numpy().copy()
    off0 = d.off.cpu().numpy().copy()
    v0 = d.vel.cpu().numpy().copy()
    ed = torch.as_tensor(e, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    dG = torch.empty(orc.n_edges, dtype=dtype, device="cuda")
    Q = torch.empty(orc.n_nodes, dtype=dtype, device="cuda")
    Q0 = torch.empty_like(Q)
    lib.deposit_charge(d, Q0)
    lib.push_deposit(ed, bd, d, 1.0, dG, Q)
    assert lib.status() == F.FP_OK
    res = torch.zeros(6, dtype=torch.float64, device="cuda")
    lib.residuals(dG, Q, Q0, bd, res)
    return d, cell0, off0, v0, dG.double().cpu().numpy(), Q.double().cpu().numpy(), Q0.double().cpu().numpy(), \
        res.cpu().numpy()


# 1,200,000 sorted: the run-summing staged kernel; 50,001: the grid-stride kernel
@pytest.mark.parametrize("npart,sort", [(1_200_000, True), (50_001, False)])
def test_fp64_deposits_match_oracle_and_tighten_continuity(npart, sort):
    m = I.cube_mesh(8, 1.0, 0.1, seed=1)
    orc = O.Oracle(m.xyz, m.tets)
    sp = I.uniform_species(m, npart, 3, 0.15, -1.0, 1.0, 0.7)
    rng = np.random.default_rng(7)
    e = rng.uniform(-0.2, 0.2, orc.n_edges)
    b = rng.uniform(-0.5, 0.5, orc.n_faces)
    lib = F.FemPic(m.xyz, m.tets, F.FP_FP32)
    assert F.fem_pic_deposit_precision(lib.h) == F.FP_FP32
    d0 = _state(lib, sp, sort)      # one state (the sort orders equal cells arbitrarily)
    r32 = _push(lib, orc, d0, e, b, torch.float32)
    lib.set_deposit_precision(F.FP_FP64)
    assert lib.deposit_dtype == torch.float64
    d, cell0, off0, v0, dG, Q, Q0, res = _push(lib, orc, d0, e, b, torch.float64)
    # the particles are those of the FP32-deposit push, bit for bit
    assert torch.equal(d.cell, r32[0].cell) and torch.equal(d.off, r32[0].off) and torch.equal(d.vel, r32[0].vel)
    # deposits against the oracle walk on the GPU's own end points
    o = orc.origin(cell0)
    Xa = o + off0.T.astype(np.float64)
    Va = v0.T.astype(np.float64)
    end = (off0 + np.float32(1.0) * d.vel.cpu().numpy()).astype(np.float32)
    Xb = o + end.T.astype(np.float64)
    ref = orc.step(cell0, Xa, Va, e, b, sp.q, sp.m, sp.w, 1.0, Xend=Xb)
    assert_deposit_close(dG, ref["dG"], ref["dG_abs"], TOL["fp32"], "dG")
    assert_deposit_close(Q, ref["Q"], ref["Q_abs"], TOL["fp32"], "Q")
    Q0r, Q0a = orc.charge(cell0, Xa, sp.q, sp.w)
    assert_deposit_close(Q0, Q0r, Q0a, TOL["fp32"], "Q0")
    # continuity: FP32 contributions summed in FP64 against the same sums in FP32
    assert res[0] <= 1e-6 * res[1]
    assert res[0] * 10.0 <= r32[7][0]
    with pytest.raises(F.FemPicError):
        lib.set_deposit_precision(3)
    lib.close()


def test_fp64_deposits_shorten_the_projection_and_adams_refuses_them():
    wl = I.config(2, 1.0, mesh_n=16)        # 16^3 x 6, 10 electrons per tet
    its = {}
    for dep, R in ((F.FP_FP32, torch.float32), (F.FP_FP64, torch.float64)):
        lib = F.FemPic(wl.mesh.xyz, wl.mesh.tets, F.FP_FP32)
        lib.set_deposit_precision(dep)
        F.fem_pic_field_setup(lib.h, wl.dt)
        s0 = wl.species[0]
        d = lib.species(s0.cell, s0.X, s0.V, s0.q, s0.m, s0.w)
        e, b = lib.fields_uniform((0, 0, 0), wl.B0)
        Q0 = torch.zeros(lib.n_nodes, dtype=R, device="cuda")
        lib.deposit_charge(d, Q0)
        st, _ = F.fem_pic_field_initial(lib.h, Q0, e, tol=1e-10)
        assert st == F.FP_OK
        E_prev, E_next = e.clone(), torch.empty_like(e)
        dG = torch.zeros(lib.n_edges, dtype=R, device="cuda")
        dGp = torch.zeros_like(dG)
        Q = torch.zeros_like(Q0)
        g = []
        for _ in range(4):
            lib.push_deposit(e, b, d, wl.dt, dG, Q)
            st, info = F.fem_pic_field_step(lib.h, E_prev, e, E_next, b, dG, dGp, Q, tol=1e-10)
            assert st == F.FP_OK and info[1]["rel_res"] <= 1e-10
            g.append(info[1]["iters"])
            E_prev, e, E_next = e, E_next, E_prev
            dGp, dG = dG, dGp
        assert lib.status() == F.FP_OK
        its[dep] = np.mean(g[1:])
        if dep == F.FP_FP64:
            hist = torch.zeros(18 * d.n, dtype=torch.float32, device="cuda")
            st = lib_adams_status(lib, e, b, d, hist, wl.dt)
            assert st == F.FP_EINVAL
        lib.close()
    assert its[F.FP_FP64] < 0.8 * its[F.FP_FP32], its


def lib_adams_status(lib, e, b, d, hist, dt):
    import ctypes
    f = F.lib().fem_pic_push_deposit_adams
    dG = torch.zeros(lib.n_edges, dtype=torch.float64, device="cuda")
    Q = torch.zeros(lib.n_nodes, dtype=torch.float64, device="cuda")
    p = d.abi()
    return int(f(lib.h, ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(b.data_ptr()), ctypes.byref(p),
                 ctypes.c_void_p(hist.data_ptr()), 0, ctypes.c_double(dt), 64, ctypes.c_void_p(dG.data_ptr()),
                 ctypes.c_void_p(Q.data_ptr()), 0, None))
