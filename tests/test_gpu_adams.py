"""Parity of the Adams particle step (fem_pic_push_deposit_adams, through the C ABI) with the
FP64 oracle's Adams mover (oracle/adams.py) on the same seeded inputs.

Per step s (orders 1..4 and every history-slot pattern of the ring): v^{n+1} and a^n within
the precision's tolerance of the oracle; the new history slot holds v^n bit-exact; the other
slots are untouched; the end points x^{n+1} are reproduced exactly on the host (the library
rounds the position sum operation by operation), and the oracle walk on them gives the cells
bit-exact and the deposits within the per-entry tolerance.  Also: a multi-step FP64 run
against the oracle, the sort moving the history with the particles, absorbed particles left
alone, and the argument errors.
"""
import numpy as np
import pytest
import torch

from paper_2103_06737_gb300 import inputs as I
import oracle as O
from oracle import adams as AD
from helpers import TOL, assert_deposit_close, fp32_continuity_tol

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_2103_06737_gb300.fem_pic")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2103_06737_gb300 import build
    build.build()


def _setup(n_hex=8, jit=0.1, npart=50_001, seed=3, speed=0.15, prec=F.FP_FP64, field_seed=7):
    m = I.cube_mesh(n_hex, 1.0, jit, seed=1)
    orc = O.Oracle(m.xyz, m.tets)
    lib = F.FemPic(m.xyz, m.tets, prec)
    sp = I.uniform_species(m, npart, seed, speed, -1.0, 1.0, 0.7)
    rng = np.random.default_rng(field_seed)
    e = rng.uniform(-0.2, 0.2, orc.n_edges)
    b = rng.uniform(-0.5, 0.5, orc.n_faces)
    return m, orc, lib, sp, e, b


def _history(n, seed, vscale, ascale):
    """Seeded history [18, n]: slot s has v at rows 6s..6s+2 and a at rows 6s+3..6s+5."""
    rng = np.random.default_rng(seed)
    h = np.empty((18, n))
    for s in range(3):
        h[6 * s:6 * s + 3] = rng.normal(0.0, vscale, (3, n))
        h[6 * s + 3:6 * s + 6] = rng.normal(0.0, ascale, (3, n))
    return h


def _split(h):
    """[18, n] -> oracle layout hist_v, hist_a [3, n, 3]."""
    hv = np.stack([h[6 * s:6 * s + 3].T for s in range(3)])
    ha = np.stack([h[6 * s + 3:6 * s + 6].T for s in range(3)])
    return hv, ha


def _end_points(off0, v0, h, step, dt, real):
    """x^{n+1} offsets as the library rounds them: h = beta_1 v^{n-1}, h += beta_j v^{n-j}
    (j = 2, 3), s = beta_0 v^n + h, x + dt s, each operation rounded to `real` (no fused
    multiply-adds)."""
    k = AD.order_for(step)
    beta = [real(x) for x in AD.ab_coefficients(k)]
    s = (beta[0] * v0.astype(real)).astype(real)
    if k > 1:
        hs = None
        for j in range(1, k):
            sl = (step - j) % 3
            t = (beta[j] * h[6 * sl:6 * sl + 3].astype(real)).astype(real)
            hs = t if hs is None else (hs + t).astype(real)
        s = (s + hs).astype(real)
    return (off0.astype(real) + (real(dt) * s).astype(real)).astype(real)


def _adams_case(prec, step, npart=50_001, sort=False, speed=0.15, seed=3):
    real = np.float64 if prec == F.FP_FP64 else np.float32
    tdev = torch.float64 if prec == F.FP_FP64 else torch.float32
    m, orc, lib, sp, e, b = _setup(npart=npart, speed=speed, prec=prec, seed=seed)
    q, mass, w, dt = sp.q, sp.m, sp.w, 1.0
    d = lib.species(sp.cell, sp.X, sp.V, q, mass, w)
    h0 = _history(npart, 100 + step, speed / 4, 0.3)
    hist = torch.as_tensor(h0, device="cuda").to(tdev).contiguous()
    if sort:
        d2 = d.empty_like()
        hist2 = torch.empty_like(hist)
        lib.sort_columns(d, d2, hist, hist2, 18)
        d, hist = d2, hist2
    cell0 = d.cell.cpu().numpy().copy()
    off0 = d.off.cpu().numpy().copy()
    v0 = d.vel.cpu().numpy().copy()
    h_in = hist.cpu().numpy().copy()
    ed = torch.as_tensor(e, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    dG = torch.empty(orc.n_edges, dtype=tdev, device="cuda")
    Q = torch.empty(orc.n_nodes, dtype=tdev, device="cuda")
    Q0 = torch.empty_like(Q)
    lib.deposit_charge(d, Q0)
    lib.push_deposit_adams(ed, bd, d, hist, step, dt, dG, Q)
    assert lib.status() == F.FP_OK
    res = torch.zeros(6, dtype=torch.float64, device="cuda")
    lib.residuals(dG, Q, Q0, bd, res)
    # oracle from the same start state (promoted to FP64)
    o = orc.origin(cell0)
    Xa = o + off0.T.astype(np.float64)
    Va = v0.T.astype(np.float64)
    hv, ha = _split(h_in.astype(np.float64))
    end = _end_points(off0, v0, h_in, step, dt, real)
    Xb = o + end.T.astype(np.float64)
    ref = AD.adams_step(orc, cell0, Xa, Va, hv, ha, step, e, b, q, mass, w, dt, Xend=Xb)
    return dict(lib=lib, orc=orc, d=d, hist=hist.cpu().numpy(), h_in=h_in, ref=ref, cell0=cell0, Xa=Xa,
                dG=dG.cpu().numpy(), Q=Q.cpu().numpy(), Q0=Q0.cpu().numpy(), res=res.cpu().numpy(),
                end=end, off0=off0, v0=v0, npart=npart, q=q, w=w, step=step, real=real)


def _check(r, tol):
    lib, orc, d, ref = r["lib"], r["orc"], r["d"], r["ref"]
    step, cell0 = r["step"], r["cell0"]
    live0 = cell0 >= 0
    V1 = d.vel.double().cpu().numpy().T
    vs = np.abs(ref["V"]).max()
    assert np.abs(V1[live0] - ref["V"][live0]).max() <= tol * vs
    # the Adams end points themselves agree with the oracle's FP64 ones to the precision
    o = orc.origin(cell0)
    Xab_gpu = o + r["end"].T.astype(np.float64)
    assert np.abs(Xab_gpu[live0] - ref["Xab"][live0]).max() <= 4 * tol * (1.0 + np.abs(ref["Xab"]).max())
    # history: new slot = (v^n bit-exact, a^n within tol); the other slots untouched
    h, h_in = r["hist"], r["h_in"]
    s = step % 3
    assert np.array_equal(h[6 * s:6 * s + 3][:, live0], r["v0"][:, live0])
    a_ref = ref["A"][live0].T
    assert np.abs(h[6 * s + 3:6 * s + 6][:, live0] - a_ref).max() <= tol * np.abs(a_ref).max()
    for o_ in range(3):
        if o_ != s:
            assert np.array_equal(h[6 * o_:6 * o_ + 6], h_in[6 * o_:6 * o_ + 6])
    # walk and deposits on the same end points
    cell1 = d.cell.cpu().numpy()
    assert np.array_equal(cell1, ref["cell"])
    alive = cell1 >= 0
    X1 = lib.positions(d).cpu().numpy()
    assert np.abs(X1[alive] - ref["X"][alive]).max() <= (1e-12 if r["real"] == np.float64 else 1e-6)
    assert_deposit_close(r["dG"], ref["dG"], ref["dG_abs"], tol, "dG")
    assert_deposit_close(r["Q"], ref["Q"], ref["Q_abs"], tol, "Q")
    if r["real"] == np.float64:
        assert r["res"][0] <= 1e-14 * r["res"][1]
    else:
        assert r["res"][0] <= fp32_continuity_tol(r["npart"], orc.n_nodes, orc.n_edges) * r["res"][1]
    return ref


@pytest.mark.parametrize("step", [0, 1, 2, 3, 4, 5])
def test_adams_fp64_parity(step):
    r = _adams_case(F.FP_FP64, step)
    ref = _check(r, TOL["fp64"])
    assert ref["dG_abs"].any() and (ref["cell"] != r["cell0"]).sum() > r["npart"] // 20
    r["lib"].close()


@pytest.mark.parametrize("step,npart,sort", [(0, 50_001, False), (1, 50_000, True), (2, 50_001, False),
                                             (3, 50_000, False), (4, 200_000, True), (5, 50_001, True)])
def test_adams_fp32_parity(step, npart, sort):
    r = _adams_case(F.FP_FP32, step, npart=npart, sort=sort)
    ref = _check(r, TOL["fp32"])
    assert (ref["cell"] != r["cell0"]).sum() > npart // 20      # many particles take the FP64 walk
    r["lib"].close()


def test_adams_fp64_six_steps_against_oracle():
    """Steps 0..5 in a row on each side (start-up orders, then the ring wraps)."""
    npart = 20_000
    m, orc, lib, sp, _, _ = _setup(npart=npart, speed=0.05, prec=F.FP_FP64, seed=5)
    # weak fields: omega_c dt ~ 0.06, inside the explicit method's stability interval
    rng = np.random.default_rng(8)
    e = rng.uniform(-2e-3, 2e-3, orc.n_edges)
    b = rng.uniform(-1e-3, 1e-3, orc.n_faces)
    q, mass, w, dt = sp.q, sp.m, sp.w, 0.5
    d = lib.species(sp.cell, sp.X, sp.V, q, mass, w)
    hist = torch.zeros((18, npart), dtype=torch.float64, device="cuda")
    ed = torch.as_tensor(e, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    dG = torch.empty(orc.n_edges, dtype=torch.float64, device="cuda")
    Q = torch.empty(orc.n_nodes, dtype=torch.float64, device="cuda")
    cell, X, V = sp.cell.copy(), sp.X.copy(), sp.V.copy()
    hv = np.zeros((3, npart, 3))
    ha = np.zeros((3, npart, 3))
    for step in range(6):
        lib.push_deposit_adams(ed, bd, d, hist, step, dt, dG, Q)
        r = AD.adams_step(orc, cell, X, V, hv, ha, step, e, b, q, mass, w, dt)
        cell, X, V, hv, ha = r["cell"], r["X"], r["V"], r["hist_v"], r["hist_a"]
    assert lib.status() == F.FP_OK
    cg = d.cell.cpu().numpy()
    assert (cg == cell).mean() > 0.999            # a point within round-off of a face may differ
    same = (cg == cell) & (cell >= 0)
    Xg = lib.positions(d).cpu().numpy()
    assert np.abs(Xg[same] - X[same]).max() <= 1e-10
    Vg = d.vel.cpu().numpy().T
    assert np.abs(Vg[same] - V[same]).max() <= 1e-10 * np.abs(V).max()
    assert_deposit_close(dG.cpu().numpy(), r["dG"], r["dG_abs"], 1e-9, "dG (last step)")
    lib.close()


@pytest.mark.parametrize("prec", [F.FP_FP64, F.FP_FP32])
def test_sort_columns_moves_history(prec):
    tdev = torch.float64 if prec == F.FP_FP64 else torch.float32
    m, orc, lib, sp, e, b = _setup(npart=30_001, prec=prec, seed=9)
    d = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    cell = d.cell.clone()
    cell[::97] = -1                                          # absorbed particles sort last
    d.cell.copy_(cell)
    # columns = copies of the state, so the permutation can be checked against the state's
    cols = torch.cat([d.off, d.vel, d.off * 2, d.vel * 3, d.off + 1, d.vel - 1], dim=0).to(tdev).contiguous()
    d2 = d.empty_like()
    c2 = torch.empty_like(cols)
    lib.sort_columns(d, d2, cols, c2, 18)
    # a permutation of the state (the order inside a cell is not fixed) ...
    for a, b_ in ((d.off, d2.off), (d.vel, d2.vel)):
        assert torch.equal(torch.sort(a, dim=1).values, torch.sort(b_, dim=1).values)
    # ... and the columns went through the same one
    want = torch.cat([d2.off, d2.vel, d2.off * 2, d2.vel * 3, d2.off + 1, d2.vel - 1], dim=0)
    assert torch.equal(c2, want)
    c = d2.cell.cpu().numpy()
    alive = c >= 0
    assert np.all(np.diff(c[alive]) >= 0) and not alive[alive.sum():].any()
    lib.close()


def test_absorbed_and_empty_and_errors():
    m, orc, lib, sp, e, b = _setup(npart=1000, prec=F.FP_FP32, seed=11)
    d = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    d.cell[::3] = -1
    cell0, off0, vel0 = d.cell.clone(), d.off.clone(), d.vel.clone()
    hist = torch.full((18, d.n), 0.01, dtype=torch.float32, device="cuda")
    ed = torch.as_tensor(e, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    dG = torch.empty(orc.n_edges, dtype=torch.float32, device="cuda")
    Q = torch.empty(orc.n_nodes, dtype=torch.float32, device="cuda")
    lib.push_deposit_adams(ed, bd, d, hist, 4, 0.5, dG, Q)
    assert lib.status() == F.FP_OK
    dead = (cell0 < 0)
    assert torch.equal(d.cell[dead], cell0[dead])
    assert torch.equal(d.off[:, dead], off0[:, dead]) and torch.equal(d.vel[:, dead], vel0[:, dead])
    assert bool((hist[:, dead] == torch.tensor(0.01, dtype=torch.float32)).all())
    # the charge of the live particles only
    assert abs(float(Q.double().sum()) - (~dead).sum().item() * sp.q * sp.w) <= 1e-4 * d.n * abs(sp.w)
    # empty species: outputs zeroed, nothing else
    e0 = F.Species(torch.empty(0, dtype=torch.int32, device="cuda"), torch.empty((3, 0), device="cuda"),
                   torch.empty((3, 0), device="cuda"), sp.q, sp.m, sp.w)
    dG.fill_(1.0)
    lib.push_deposit_adams(ed, bd, e0, torch.empty((18, 0), device="cuda"), 0, 0.5, dG, Q)
    assert float(dG.abs().max()) == 0.0
    # argument errors from the C ABI: negative step, NULL history
    import ctypes
    p = d.abi()
    L = F.lib()
    rc = L.fem_pic_push_deposit_adams(lib.h, ed.data_ptr(), bd.data_ptr(), ctypes.byref(p), hist.data_ptr(), -1,
                                      0.5, 64, dG.data_ptr(), Q.data_ptr(), 0, None)
    assert rc == F.FP_EINVAL
    rc = L.fem_pic_push_deposit_adams(lib.h, ed.data_ptr(), bd.data_ptr(), ctypes.byref(p), None, 0,
                                      0.5, 64, dG.data_ptr(), Q.data_ptr(), 0, None)
    assert rc == F.FP_EINVAL
    lib.close()
