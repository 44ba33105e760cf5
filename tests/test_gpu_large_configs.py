"""Parity on the larger workload shapes: the two-species 96^3 cube (electrons and ions at mass
ratio 1836, B0 = 0.2 T along x) and the 64^3 cylindrical beam (0.1c drift along z,
Bz = 0.5 T, many face crossings per step), FP32 particle path in the launch configuration
the benchmark times (cell-sorted state, the warp-specialised staged push kernel).

Element by element against the FP64 oracle (Sec. II.A gather/push, Sec. IV.B.1 walk and
deposits): velocities against the oracle push from the same FP32 start state, cells
bit-exact against the oracle walk on the GPU's own FP32 end points, positions, and the
deposits of all species within the FP32 tolerance.  At the 96^3 workload's full 50M + 50M
particles the oracle steps a seeded sample of each species one by one, and the full
deposits are held to what holds at any size: discrete continuity, total charge, D2 b = 0.
"""
import numpy as np
import pytest
import torch

from paper_2103_06737_gb300 import inputs as I
import oracle as O
from helpers import EPS, TOL, assert_deposit_close, fp32_continuity_tol

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_2103_06737_gb300.fem_pic")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2103_06737_gb300 import build
    build.build()


def _fields(cx, B0, amp=1e3, seed=11):
    """Uniform B0 plus a seeded random E of amplitude amp (V/m) times the edge length."""
    rng = np.random.default_rng(seed)
    e = amp * np.linalg.norm(cx.xyz[cx.edges[:, 1]] - cx.xyz[cx.edges[:, 0]], axis=1) * \
        rng.uniform(-1.0, 1.0, cx.n_edges)
    e[cx.boundary_edge] = 0.0
    _, b = cx.project_uniform((0.0, 0.0, 0.0), B0)
    return e, b


def _sorted_species(lib, sp):
    d0 = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    d = d0.empty_like()
    lib.sort(d0, d)
    del d0
    assert d.n % 4 == 0
    return d


def _state(d, idx=None):
    if idx is None:
        return d.cell.cpu().numpy().copy(), d.off.cpu().numpy().copy(), d.vel.cpu().numpy().copy()
    i = torch.as_tensor(idx, device=d.cell.device)
    return (d.cell.index_select(0, i).cpu().numpy(), d.off.index_select(1, i).cpu().numpy(),
            d.vel.index_select(1, i).cpu().numpy())


def _oracle_check(orc, sp, dt, e, b, before, after):
    """Per-particle parity of one species (or a sample of it); returns the oracle walk."""
    cell0, off0, v0 = before
    cell1, off1, v1 = after
    o = orc.origin(cell0)
    Xa = o + off0.T.astype(np.float64)
    Va = v0.T.astype(np.float64)
    live = cell0 >= 0
    ref_push = orc.step(cell0, Xa, Va, e, b, sp.q, sp.m, sp.w, dt)
    assert np.abs(v1.T[live] - ref_push["V"][live]).max() <= TOL["fp32"] * np.abs(ref_push["V"][live]).max()
    end = (off0 + (np.float32(dt) * v1).astype(np.float32)).astype(np.float32)   # as rounded on the GPU
    ref = orc.step(cell0, Xa, Va, e, b, sp.q, sp.m, sp.w, dt, Xend=o + end.T.astype(np.float64), touch=True)
    assert np.array_equal(cell1, ref["cell"])
    alive = cell1 >= 0
    X1 = orc.origin(np.where(alive, cell1, 0)) + off1.T.astype(np.float64)
    assert np.abs(X1[alive] - ref["X"][alive]).max() <= 1e-6
    return ref


def _push_all(lib, ds, ed, bd, dt, R=torch.float32):
    dG = torch.empty(lib.n_edges, dtype=R, device="cuda")
    Q = torch.empty(lib.n_nodes, dtype=R, device="cuda")
    Q0 = torch.empty_like(Q)
    for k, d in enumerate(ds):
        lib.deposit_charge(d, Q0, flags=F.FP_ACCUMULATE if k else 0)
    for k, d in enumerate(ds):   # as the benchmark calls it: the later species reuse the field records
        lib.push_deposit(ed, bd, d, dt, dG, Q, flags=(F.FP_ACCUMULATE | F.FP_SAME_FIELDS) if k else 0)
    st = lib.status()
    res = torch.zeros(6, dtype=torch.float64, device="cuda")
    lib.residuals(dG, Q, Q0, bd, res)
    return st, dG, Q, Q0, res.cpu().numpy()


@pytest.mark.parametrize("idx,scale", [(5, 0.04), (3, 1.0)])
def test_large_shapes_element_by_element(idx, scale):
    """96^3 two species at 2M + 2M particles; the 64^3 beam at its full 20M particles."""
    wl = I.config(idx, scale)
    orc = O.Oracle(wl.mesh.xyz, wl.mesh.tets)
    cx = orc.cx
    e, b = _fields(cx, wl.B0)
    lib = F.FemPic(wl.mesh.xyz, wl.mesh.tets, F.FP_FP32)
    ds = [_sorted_species(lib, sp) for sp in wl.species]
    before = [_state(d) for d in ds]
    st, dG, Q, Q0, r = _push_all(lib, ds, torch.as_tensor(e, device="cuda"), torch.as_tensor(b, device="cuda"),
                                 wl.dt)
    assert st == F.FP_OK, F.fem_pic_last_error(lib.h)
    acc = {k: 0.0 for k in ("dG", "dG_abs", "dG_touch", "Q", "Q_abs", "Q_touch")}
    ncross = 0
    for sp, d, bf in zip(wl.species, ds, before):
        ref = _oracle_check(orc, sp, wl.dt, e, b, bf, _state(d))
        for k in acc:
            acc[k] = acc[k] + ref[k]
        ncross += int(ref["ncross"].sum())
    if idx == 3:
        assert ncross > wl.species[0].n // 50          # the drifting beam crosses faces
    assert_deposit_close(dG.cpu().numpy(), acc["dG"], acc["dG_abs"], TOL["fp32"], "dG", acc["dG_touch"], EPS["fp32"])
    assert_deposit_close(Q.cpu().numpy(), acc["Q"], acc["Q_abs"], TOL["fp32"], "Q", acc["Q_touch"], EPS["fp32"])
    ntot = sum(sp.n for sp in wl.species)
    assert r[0] <= fp32_continuity_tol(ntot, cx.n_nodes, cx.n_edges) * r[1]
    assert r[2] <= 1e-13 * r[3]
    lib.close()


def test_two_species_full_size_sampled():
    """The 96^3 workload at its full 50M electrons + 50M ions in one push call per species:
    a seeded sample of 250,000 particles per species against the oracle one by one, and the
    full deposits against continuity, total charge and D2 b = 0."""
    wl = I.config(5)
    orc = O.Oracle(wl.mesh.xyz, wl.mesh.tets)
    cx = orc.cx
    e, b = _fields(cx, wl.B0)
    lib = F.FemPic(wl.mesh.xyz, wl.mesh.tets, F.FP_FP32)
    ds = []
    for sp in wl.species:
        ds.append(_sorted_species(lib, sp))
    rng = np.random.default_rng(5)
    samples = [np.sort(rng.choice(d.n, 250_000, replace=False)) for d in ds]
    before = [_state(d, s) for d, s in zip(ds, samples)]
    st, dG, Q, Q0, r = _push_all(lib, ds, torch.as_tensor(e, device="cuda"), torch.as_tensor(b, device="cuda"),
                                 wl.dt)
    assert st == F.FP_OK, F.fem_pic_last_error(lib.h)
    for sp, d, s, bf in zip(wl.species, ds, samples, before):
        _oracle_check(orc, sp, wl.dt, e, b, bf, _state(d, s))
    ntot = sum(sp.n for sp in wl.species)
    assert r[0] <= fp32_continuity_tol(ntot, cx.n_nodes, cx.n_edges) * r[1]
    assert r[2] <= 1e-13 * r[3]
    # total charge: every particle alive at the start leaves q w on the nodes (absorbed ones
    # at their wall point), so sum Q = sum Q0 = sum over species of n q w (quasi-neutral: ~0)
    scale = sum(sp.n * abs(sp.q * sp.w) for sp in wl.species)
    tot = sum(sp.n * sp.q * sp.w for sp in wl.species)
    assert abs(float(Q.double().sum()) - tot) <= 1e-6 * scale
    assert abs(float(Q0.double().sum()) - tot) <= 1e-6 * scale
    assert np.isfinite(dG.cpu().numpy()).all()
    lib.close()
