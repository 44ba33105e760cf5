"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same seeded inputs.

Cells and walk outcomes bit-exact; particle state and deposits within 1e-12 (FP64)
or 1e-5 (FP32) under the per-entry reading in tests/helpers.py.  In FP32 mode the
oracle walk is re-run from the GPU's own FP32 end points promoted to FP64.
"""
import numpy as np
import pytest
import torch

from paper_2103_06737_gb300 import inputs as I
import oracle as O
from helpers import TOL, assert_deposit_close, csr_tuple, fp32_continuity_tol

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


def _to_host(sp, lib):
    X = lib.positions(sp).cpu().numpy()
    return sp.cell.cpu().numpy(), X, sp.vel.double().cpu().numpy().T.copy(), sp.off.cpu().numpy()


@pytest.mark.parametrize("n_hex,jit", [(4, 0.0), (6, 0.1)])
def test_incidence_and_topology_bit_exact(n_hex, jit):
    m = I.cube_mesh(n_hex, 1.0, jit, seed=1)
    orc = O.Oracle(m.xyz, m.tets)
    cx = orc.cx
    lib = F.FemPic(m.xyz, m.tets, F.FP_FP64)
    assert (lib.n_nodes, lib.n_edges, lib.n_faces, lib.n_tets) == \
        (cx.n_nodes, cx.n_edges, cx.n_faces, cx.n_tets)
    for which, mat, ncols in ((0, cx.D0(), cx.n_nodes), (1, cx.D1(), cx.n_edges), (2, cx.D2(), cx.n_faces)):
        rp, col, val = F.fem_pic_incidence(lib.h, which)
        ref = csr_tuple(mat, ncols)
        assert np.array_equal(rp, ref[0]) and np.array_equal(col, ref[1]) and np.array_equal(val, ref[2])
    topo = F.fem_pic_topology(lib.h)
    assert np.array_equal(topo["tet_nodes"], cx.tv)
    assert np.array_equal(topo["tet_edges"], cx.tet_edges)
    assert np.array_equal(topo["tet_faces"], cx.tet_faces)
    assert np.array_equal(topo["tet_neigh"], cx.neigh)
    # the create call validates caller-supplied incidence, and rejects a flipped sign
    F.FemPic(m.xyz, m.tets, F.FP_FP64, D0=csr_tuple(cx.D0(), cx.n_nodes), D1=csr_tuple(cx.D1(), cx.n_edges),
             D2=csr_tuple(cx.D2(), cx.n_faces)).close()
    bad = csr_tuple(cx.D1(), cx.n_edges)
    bad[2][0] = -bad[2][0]
    with pytest.raises(F.FemPicError) as ei:
        F.FemPic(m.xyz, m.tets, F.FP_FP64, D1=bad)
    assert ei.value.code == F.FP_EINVAL
    lib.close()


def test_degenerate_tet_rejected():
    m = I.cube_mesh(2, 1.0, 0.0)
    tets = m.tets.copy()
    tets[0, 1] = tets[0, 0] if tets[0, 0] != tets[0, 2] else tets[0, 1]
    xyz = m.xyz.copy()
    with pytest.raises(F.FemPicError) as ei:
        F.FemPic(xyz, tets, F.FP_FP64)
    assert ei.value.code in (F.FP_EGEOM, F.FP_EINVAL)


def test_project_uniform_and_divb():
    m = I.cube_mesh(6, 1.0, 0.1, seed=1)
    orc = O.Oracle(m.xyz, m.tets)
    lib = F.FemPic(m.xyz, m.tets, F.FP_FP64)
    e, b = lib.fields_uniform((1.0, -2.0, 0.5), (0.1, 0.2, -0.3))
    er, br = orc.project_uniform((1.0, -2.0, 0.5), (0.1, 0.2, -0.3))
    assert np.abs(e.cpu().numpy() - er).max() <= 1e-15 * np.abs(er).max()
    assert np.abs(b.cpu().numpy() - br).max() <= 1e-15 * np.abs(br).max()
    out = torch.zeros(6, dtype=torch.float64, device="cuda")
    lib.residuals(None, None, None, b, out)
    r = out.cpu().numpy()
    assert r[2] <= 4e-15 * r[3]
    lib.close()


def _push_fp64(npart, speed, max_cross=64, agg=True):
    m, orc, lib, sp, e, b = _setup(npart=npart, speed=speed, prec=F.FP_FP64)
    dt = 1.0
    q, mass, w = sp.q, sp.m, sp.w
    d = lib.species(sp.cell, sp.X, sp.V, q, mass, w)
    ed = torch.as_tensor(e, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    dG = torch.empty(orc.n_edges, dtype=torch.float64, device="cuda")
    Q = torch.empty(orc.n_nodes, dtype=torch.float64, device="cuda")
    Q0 = torch.empty_like(Q)
    lib.deposit_charge(d, Q0)
    lib.push_deposit(ed, bd, d, dt, dG, Q, max_cross=max_cross, flags=0 if agg else F.FP_NO_AGGREGATE)
    st = lib.status()
    res = torch.zeros(6, dtype=torch.float64, device="cuda")
    lib.residuals(dG, Q, Q0, bd, res)
    ref = orc.step(sp.cell, sp.X, sp.V, e, b, q, mass, w, dt, max_cross=max_cross)
    Q0r, Q0a = orc.charge(sp.cell, sp.X, q, w)
    return dict(lib=lib, orc=orc, d=d, dG=dG.cpu().numpy(), Q=Q.cpu().numpy(), Q0=Q0.cpu().numpy(),
                ref=ref, Q0r=Q0r, Q0a=Q0a, st=st, res=res.cpu().numpy(), sp=sp)


@pytest.mark.parametrize("agg", [True, False])
def test_push_deposit_fp64_parity(agg):
    r = _push_fp64(50_001, 0.15, agg=agg)
    ref, lib, d = r["ref"], r["lib"], r["d"]
    cell, X, V, _ = _to_host(d, lib)
    assert r["st"] == F.FP_OK
    assert ref["ncross"].sum() > 5000 and (ref["cell"] < 0).sum() > 10
    assert np.array_equal(cell, ref["cell"])
    alive = cell >= 0
    assert np.abs(X[alive] - ref["X"][alive]).max() <= 1e-12
    assert np.abs(V - ref["V"]).max() <= 1e-12 * np.abs(ref["V"]).max()
    tol = TOL["fp64"]
    assert_deposit_close(r["dG"], ref["dG"], ref["dG_abs"], tol, "dG")
    assert_deposit_close(r["Q"], ref["Q"], ref["Q_abs"], tol, "Q")
    assert_deposit_close(r["Q0"], r["Q0r"], r["Q0a"], tol, "Q0")
    # discrete continuity on the GPU (FP64 residual kernel)
    assert r["res"][0] <= 1e-14 * r["res"][1]
    lib.close()


# 50,001 particles: the grid-stride fast kernel (length not a multiple of 4); 50,000 and
# 1,200,000: the staged (bulk-copy) kernel, the latter with several tiles per block so
# every pipeline stage and record window is reused; sorted by cell, most records come
# from the shared-memory windows, unsorted most come from global memory
@pytest.mark.parametrize("npart,sort", [(50_001, False), (50_000, False), (1_200_000, False), (1_200_000, True)])
def test_push_deposit_fp32_parity(npart, sort):
    m, orc, lib, sp, e, b = _setup(npart=npart, speed=0.15, prec=F.FP_FP32)
    q, mass, w, dt = sp.q, sp.m, sp.w, 1.0
    d = lib.species(sp.cell, sp.X, sp.V, q, mass, w)
    if sort:
        d2 = d.empty_like()
        lib.sort(d, d2)
        d = d2
    cell0 = d.cell.cpu().numpy().copy()
    off0 = d.off.cpu().numpy().copy()                 # [3,n] float32
    v0 = d.vel.cpu().numpy().copy()
    ed = torch.as_tensor(e, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    dG = torch.empty(orc.n_edges, dtype=torch.float32, device="cuda")
    Q = torch.empty(orc.n_nodes, dtype=torch.float32, device="cuda")
    Q0 = torch.empty_like(Q)
    lib.deposit_charge(d, Q0)
    lib.push_deposit(ed, bd, d, dt, dG, Q)
    assert lib.status() == F.FP_OK
    res = torch.zeros(6, dtype=torch.float64, device="cuda")
    lib.residuals(dG, Q, Q0, bd, res)
    cell1, X1, V1, off1 = _to_host(d, lib)
    # velocities vs the FP64 oracle push from the same (FP32) start state
    o = orc.origin(cell0)
    Xa = o + off0.T.astype(np.float64)
    Va = v0.T.astype(np.float64)
    ref_push = orc.step(cell0, Xa, Va, e, b, q, mass, w, dt)
    assert np.abs(V1 - ref_push["V"]).max() <= TOL["fp32"] * np.abs(ref_push["V"]).max()
    # walk + deposit vs the oracle walk on the GPU's own FP32 end points
    v1f = d.vel.cpu().numpy()
    end = (off0 + np.float32(dt) * v1f).astype(np.float32)   # two roundings, as on the GPU
    Xb = o + end.T.astype(np.float64)
    ref = orc.step(cell0, Xa, Va, e, b, q, mass, w, dt, Xend=Xb)
    assert ref["ncross"].sum() > npart // 10
    assert np.array_equal(cell1, ref["cell"])
    alive = cell1 >= 0
    assert np.abs(X1[alive] - ref["X"][alive]).max() <= 1e-6
    Q0r, Q0a = orc.charge(cell0, Xa, q, w)
    tol = TOL["fp32"]
    assert_deposit_close(dG.cpu().numpy(), ref["dG"], ref["dG_abs"], tol, "dG")
    assert_deposit_close(Q.cpu().numpy(), ref["Q"], ref["Q_abs"], tol, "Q")
    assert_deposit_close(Q0.cpu().numpy(), Q0r, Q0a, tol, "Q0")
    ctol = fp32_continuity_tol(npart, orc.n_nodes, orc.n_edges)
    assert res.cpu().numpy()[0] <= ctol * res.cpu().numpy()[1]
    lib.close()


def test_walk_bound_status_and_continuity():
    r = _push_fp64(5_000, 2.0, max_cross=1)
    assert r["st"] == F.FP_EWALK
    ref, lib, d = r["ref"], r["lib"], r["d"]
    assert ref["n_bound"] > 0
    cell, X, _, _ = _to_host(d, lib)
    assert np.array_equal(cell, ref["cell"])
    assert_deposit_close(r["dG"], ref["dG"], ref["dG_abs"], TOL["fp64"], "dG")
    assert r["res"][0] <= 1e-14 * r["res"][1]
    lib.close()


def test_invalid_cell_and_empty_input():
    m, orc, lib, sp, e, b = _setup(npart=100, prec=F.FP_FP64)
    d = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    d.cell[7] = orc.n_tets + 5            # corrupt one id: the kernel flags and skips it
    ed = torch.as_tensor(e, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    dG = torch.empty(orc.n_edges, dtype=torch.float64, device="cuda")
    Q = torch.empty(orc.n_nodes, dtype=torch.float64, device="cuda")
    lib.push_deposit(ed, bd, d, 0.1, dG, Q)
    assert lib.status() == F.FP_EINVAL
    assert lib.status() == F.FP_OK        # cleared
    empty = F.Species(torch.empty(0, dtype=torch.int32, device="cuda"),
                      torch.empty((3, 0), dtype=torch.float64, device="cuda"),
                      torch.empty((3, 0), dtype=torch.float64, device="cuda"), -1.0, 1.0, 1.0)
    dG.fill_(1.0)
    lib.push_deposit(ed, bd, empty, 0.1, dG, Q)
    assert float(dG.abs().max()) == 0.0
    lib.sort(empty, empty.empty_like())
    assert lib.status() == F.FP_OK
    lib.close()


def test_bounded_wait_runs_out_and_reports():
    """A wait that nothing completes gives up after its limit (1 ms) and sets the time-out
    status; fem_pic_status reports it once, and the context keeps working (a push follows)."""
    m, orc, lib, sp, e, b = _setup(npart=2000, prec=F.FP_FP32)
    F.fem_pic_selftest_wait(lib.h, 1e-3)
    assert lib.status() == F.FP_ECUDA
    assert "gave up waiting" in F.fem_pic_last_error(lib.h)
    assert lib.status() == F.FP_OK            # cleared
    with pytest.raises(F.FemPicError):
        F.fem_pic_selftest_wait(lib.h, 0.0)   # the limit must be positive
    d = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    dG = torch.empty(orc.n_edges, dtype=torch.float32, device="cuda")
    Q = torch.empty(orc.n_nodes, dtype=torch.float32, device="cuda")
    lib.push_deposit(torch.as_tensor(e, device="cuda"), torch.as_tensor(b, device="cuda"), d, 1.0, dG, Q)
    assert lib.status() == F.FP_OK
    assert abs(float(Q.double().sum()) - sp.n * sp.q * sp.w) <= 1e-4 * sp.n * abs(sp.w)
    lib.close()


@pytest.mark.parametrize("prec", [F.FP_FP32, F.FP_FP64])
def test_sort_is_a_permutation_by_cell(prec):
    m, orc, lib, sp, e, b = _setup(npart=30_001, prec=prec, speed=0.3)
    d = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    d.cell[::97] = -1                      # some absorbed particles: they go last
    out = d.empty_like()
    lib.sort(d, out)
    assert lib.status() == F.FP_OK
    c_in = d.cell.cpu().numpy()
    c_out = out.cell.cpu().numpy()
    alive = c_out[c_out >= 0]
    assert np.all(np.diff(alive) >= 0)
    assert np.all(c_out[len(alive):] == -1)

    def rows(s):
        a = np.concatenate([s.cell.cpu().numpy()[None].astype(np.float64), s.off.double().cpu().numpy(),
                            s.vel.double().cpu().numpy()], axis=0).T
        return a[np.lexsort(a.T[::-1])]
    assert np.array_equal(rows(d), rows(out))
    assert np.array_equal(np.sort(c_in), np.sort(c_out))
    lib.close()


def test_sorted_and_unsorted_push_agree():
    m, orc, lib, sp, e, b = _setup(npart=40_000, prec=F.FP_FP64, speed=0.1)
    d = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    s = d.empty_like()
    lib.sort(d, s)
    ed = torch.as_tensor(e, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    out = []
    for sp_ in (d, s):
        dG = torch.empty(orc.n_edges, dtype=torch.float64, device="cuda")
        Q = torch.empty(orc.n_nodes, dtype=torch.float64, device="cuda")
        lib.push_deposit(ed, bd, sp_, 1.0, dG, Q)
        out.append((dG.cpu().numpy(), Q.cpu().numpy()))
    ref = orc.step(sp.cell, sp.X, sp.V, e, b, sp.q, sp.m, sp.w, 1.0)
    for dG, Q in out:
        assert_deposit_close(dG, ref["dG"], ref["dG_abs"], TOL["fp64"], "dG")
        assert_deposit_close(Q, ref["Q"], ref["Q_abs"], TOL["fp64"], "Q")
    lib.close()


# n = 50,000 (staged pipeline), 50,001 (grid-stride kernel) in FP32; FP64 mode
@pytest.mark.parametrize("prec,npart", [(F.FP_FP32, 50_000), (F.FP_FP32, 50_001), (F.FP_FP64, 50_001)])
def test_nonfinite_state_is_flagged_and_not_deposited(prec, npart):
    """NaN and Inf written on the host into some velocities and offsets: those particles are
    removed (cell -1) with nothing deposited, the status word reports FP_EINVAL, and the other
    particles' steps and the deposits equal those of the same push with the bad particles
    already absent.  The charge call drops (and reports) the particles whose offsets are not
    finite."""
    m, orc, lib, sp, e, b = _setup(npart=npart, speed=0.15, prec=prec)
    ed = torch.as_tensor(e, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    bad = np.array([3, 1000, 20_001, 33_333, npart - 1])
    d = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    d.vel[0, 3] = float("nan")
    d.vel[1, 1000] = float("inf")
    d.off[2, 20_001] = float("nan")
    d.off[0, 33_333] = float("-inf")
    d.vel[2, npart - 1] = float("-inf")
    clean = F.Species(d.cell.clone(), d.off.clone(), d.vel.clone(), d.q, d.m, d.w)
    clean.cell[torch.as_tensor(bad, device="cuda")] = -1
    # the charge call needs only positions: it drops the two particles without one
    clean_pos = F.Species(d.cell.clone(), d.off.clone(), d.vel.clone(), d.q, d.m, d.w)
    clean_pos.cell[torch.as_tensor([20_001, 33_333], device="cuda")] = -1
    R = lib.real
    out = {}
    for name, sp_, sp_q in (("bad", d, d), ("clean", clean, clean_pos)):
        Q0 = torch.empty(lib.n_nodes, dtype=R, device="cuda")
        lib.deposit_charge(sp_q, Q0)
        st0 = lib.status()
        dG = torch.empty(lib.n_edges, dtype=R, device="cuda")
        Q = torch.empty(lib.n_nodes, dtype=R, device="cuda")
        lib.push_deposit(ed, bd, sp_, 1.0, dG, Q)
        st = lib.status()
        err = F.fem_pic_last_error(lib.h)
        out[name] = (st0, st, err, Q0.double().cpu().numpy(), dG.double().cpu().numpy(), Q.double().cpu().numpy())
    st0, st, err, Q0, dG, Q = out["bad"]
    assert st0 == F.FP_EINVAL                       # the charge call flags the non-finite offsets
    assert st == F.FP_EINVAL and "not finite" in err
    assert out["clean"][0] == F.FP_OK and out["clean"][1] == F.FP_OK
    assert np.isfinite(Q0).all() and np.isfinite(dG).all() and np.isfinite(Q).all()
    cb = d.cell.cpu().numpy()
    assert (cb[bad] == -1).all()
    assert np.array_equal(cb, clean.cell.cpu().numpy())
    good = np.ones(npart, bool)
    good[bad] = False
    for a, c in ((d.off, clean.off), (d.vel, clean.vel)):
        assert np.array_equal(a.cpu().numpy()[:, good], c.cpu().numpy()[:, good])
    tol = 1e-12 if prec == F.FP_FP64 else TOL["fp32"]
    for x, y in zip(out["bad"][3:], out["clean"][3:]):
        assert np.abs(x - y).max() <= tol * np.abs(y).max()
    if prec == F.FP_FP64:                           # and the clean step is the oracle's
        cell0 = sp.cell.copy()
        cell0[bad] = -1
        ref = orc.step(cell0, sp.X, sp.V, e, b, sp.q, sp.m, sp.w, 1.0)
        assert np.array_equal(cb, ref["cell"])
        assert_deposit_close(dG, ref["dG"], ref["dG_abs"], TOL["fp64"], "dG")
        assert_deposit_close(Q, ref["Q"], ref["Q_abs"], TOL["fp64"], "Q")
    lib.close()


def test_fp32_staged_push_without_aggregation_matches():
    """The staged FP32 push with FP_NO_AGGREGATE (one atomic per contribution) gives the same
    particles bit for bit and the same deposits within the FP32 tolerance as the run-summed
    push, on a cell-sorted state of 50,000 particles (the last tile partial)."""
    m, orc, lib, sp, e, b = _setup(npart=50_000, speed=0.15, prec=F.FP_FP32)
    d = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    s = d.empty_like()
    lib.sort(d, s)
    ed = torch.as_tensor(e, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    runs = []
    for flags in (0, F.FP_NO_AGGREGATE):
        t = s.empty_like()
        t.cell.copy_(s.cell)
        t.off.copy_(s.off)
        t.vel.copy_(s.vel)
        dG = torch.empty(orc.n_edges, dtype=torch.float32, device="cuda")
        Q = torch.empty(orc.n_nodes, dtype=torch.float32, device="cuda")
        lib.push_deposit(ed, bd, t, 1.0, dG, Q, flags=flags)
        assert lib.status() == F.FP_OK
        runs.append((t, dG.double().cpu().numpy(), Q.double().cpu().numpy()))
    (a, dGa, Qa), (c, dGc, Qc) = runs
    assert torch.equal(a.cell, c.cell) and torch.equal(a.off, c.off) and torch.equal(a.vel, c.vel)
    for x, y in ((dGa, dGc), (Qa, Qc)):
        assert np.abs(x - y).max() <= TOL["fp32"] * np.abs(x).max()
    lib.close()


def test_fp32_staged_push_skips_dead_and_invalid_particles():
    """Absorbed particles (cell -1) in the middle of a cell-sorted state, and one particle with
    an out-of-range cell, through the staged FP32 push: the status word reports FP_EINVAL, the
    skipped particles keep their state, and the others give the same particles and deposits
    as a push of the state without them."""
    m, orc, lib, sp, e, b = _setup(npart=40_000, speed=0.15, prec=F.FP_FP32)
    d = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    s = d.empty_like()
    lib.sort(d, s)
    n = s.n
    rng = np.random.default_rng(11)
    dead = np.sort(rng.choice(n, 900, replace=False))
    bad = int(dead[450])
    cell = s.cell.clone()
    cell[torch.as_tensor(dead, device="cuda")] = -1
    cell[bad] = orc.n_tets + 3
    keep = np.setdiff1d(np.arange(n), dead)
    kt = torch.as_tensor(keep, device="cuda")
    # the reference: only the live particles (n - 900, a multiple of 4: the same staged kernel)
    r = F.Species(s.cell[kt].contiguous(), s.off[:, kt].contiguous(), s.vel[:, kt].contiguous(), s.q, s.m, s.w)
    assert r.n % 4 == 0
    t = F.Species(cell, s.off.clone(), s.vel.clone(), s.q, s.m, s.w)
    ed = torch.as_tensor(e, device="cuda")
    bd = torch.as_tensor(b, device="cuda")
    out = []
    for sp_ in (t, r):
        dG = torch.empty(orc.n_edges, dtype=torch.float32, device="cuda")
        Q = torch.empty(orc.n_nodes, dtype=torch.float32, device="cuda")
        lib.push_deposit(ed, bd, sp_, 1.0, dG, Q)
        out.append((dG.double().cpu().numpy(), Q.double().cpu().numpy(), lib.status()))
    assert out[0][2] == F.FP_EINVAL and out[1][2] == F.FP_OK
    dt_ = torch.as_tensor(dead, device="cuda")
    assert torch.equal(t.off[:, dt_], s.off[:, dt_]) and torch.equal(t.vel[:, dt_], s.vel[:, dt_])
    assert int(t.cell[bad]) == orc.n_tets + 3
    assert torch.equal(t.cell[kt], r.cell) and torch.equal(t.off[:, kt], r.off) and torch.equal(t.vel[:, kt], r.vel)
    for x, y in ((out[0][0], out[1][0]), (out[0][1], out[1][1])):
        assert np.abs(x - y).max() <= TOL["fp32"] * np.abs(y).max()
    lib.close()
