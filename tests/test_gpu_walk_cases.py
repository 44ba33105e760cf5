"""GPU parity of the tet walk on degenerate paths (walk ties, end points on faces, rest,
wall exits; tests/walk_cases.py), through the C ABI, against the oracle walk.

Every case runs as a run of identical particles (so warps hold whole runs and partial
runs) in one push call with zero fields, so the velocity is unchanged and the path is
the case's segment.  FP64 mode: cells and stop points bit-exact (the dyadic cases are
exact on both sides), deposits within 1e-12 under the per-entry reading.  FP32 mode:
cells bit-exact against the oracle walk re-run on the GPU's own FP32 start and end
points, deposits within 1e-5.  The deposits are the Whitney-1 path integrals of
Sec. IV.B.1 along the walked pieces.
"""
import numpy as np
import pytest
import torch

from paper_2103_06737_gb300 import inputs as I
import oracle as O
import walk_cases as W
from helpers import TOL, assert_deposit_close, fp32_continuity_tol

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_2103_06737_gb300.fem_pic")

REP = 40


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2103_06737_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def setup():
    m = I.cube_mesh(W.N_HEX, 1.0, 0.0)
    return m, O.Oracle(m.xyz, m.tets)


def _particles(extra):
    cs = W.cases()
    cell = np.repeat([c[1] for c in cs], REP).astype(np.int32)
    Xa = np.repeat(np.array([c[2] for c in cs]), REP, axis=0)
    V = np.repeat(np.array([c[3] - c[2] for c in cs]), REP, axis=0)
    if extra:   # one more particle at rest: n not a multiple of 4 (grid-stride kernel)
        cell = np.append(cell, cs[-5][1]).astype(np.int32)
        Xa = np.vstack([Xa, cs[-5][2]])
        V = np.vstack([V, np.zeros(3)])
    names = [c[0] for c in cs for _ in range(REP)] + (["rest_extra"] if extra else [])
    return cell, Xa, V, names


@pytest.mark.parametrize("prec,extra,max_cross", [(F.FP_FP64, False, 64), (F.FP_FP64, True, 64),
                                                  (F.FP_FP32, False, 64), (F.FP_FP32, True, 64),
                                                  (F.FP_FP64, False, 2), (F.FP_FP32, False, 2)])
def test_walk_cases_match_oracle(setup, prec, extra, max_cross):
    m, orc = setup
    cx = orc.cx
    cell, Xa, V, names = _particles(extra)
    q, mass, w, dt = -1.0, 1.0, 1.0, 1.0
    lib = F.FemPic(m.xyz, m.tets, prec)
    d = lib.species(cell, Xa, V, q, mass, w)
    R = lib.real
    ez = torch.zeros(lib.n_edges, dtype=torch.float64, device="cuda")
    bz = torch.zeros(lib.n_faces, dtype=torch.float64, device="cuda")
    off0 = d.off.double().cpu().numpy().copy()
    v0 = d.vel.double().cpu().numpy().copy()
    Q0 = torch.empty(lib.n_nodes, dtype=R, device="cuda")
    lib.deposit_charge(d, Q0)
    dG = torch.empty(lib.n_edges, dtype=R, device="cuda")
    Q = torch.empty(lib.n_nodes, dtype=R, device="cuda")
    lib.push_deposit(ez, bz, d, dt, dG, Q, max_cross=max_cross)
    st = lib.status()
    res = torch.zeros(6, dtype=torch.float64, device="cuda")
    lib.residuals(dG, Q, Q0, bz, res)
    cell1 = d.cell.cpu().numpy()
    X1 = lib.positions(d).cpu().numpy()
    # zero fields: the push leaves every velocity as it was (both precisions)
    assert np.array_equal(d.vel.double().cpu().numpy(), v0)
    o = orc.origin(cell)
    Xs = o + off0.T
    if prec == F.FP_FP64:
        Xe = Xs + dt * v0.T
    else:   # the GPU's own FP32 end point: off + dt v rounded as on the device (two roundings)
        end32 = off0.astype(np.float32) + (np.float32(dt) * v0.astype(np.float32)).astype(np.float32)
        Xe = o + end32.astype(np.float32).astype(np.float64).T
    ref = orc.step(cell, Xs, v0.T, np.zeros(cx.n_edges), np.zeros(cx.n_faces), q, mass, w, dt,
                   max_cross=max_cross, Xend=Xe)
    bound = max_cross < 64
    assert st == (F.FP_EWALK if bound else F.FP_OK), F.fem_pic_last_error(lib.h)
    assert (ref["n_bound"] > 0) == bound
    assert np.array_equal(cell1, ref["cell"]), [n for n, a, b in zip(names, cell1, ref["cell"]) if a != b][:5]
    alive = cell1 >= 0
    dyadic = np.array([n != "long" for n in names])
    if prec == F.FP_FP64:
        assert np.array_equal(X1[alive & dyadic], ref["X"][alive & dyadic])
        assert np.abs(X1[alive] - ref["X"][alive]).max() <= 1e-15
    else:
        assert np.abs(X1[alive] - ref["X"][alive]).max() <= 1e-7
    tol = TOL["fp64"] if prec == F.FP_FP64 else TOL["fp32"]
    assert_deposit_close(dG.double().cpu().numpy(), ref["dG"], ref["dG_abs"], tol, "dG")
    assert_deposit_close(Q.double().cpu().numpy(), ref["Q"], ref["Q_abs"], tol, "Q")
    r = res.cpu().numpy()
    ctol = 1e-14 if prec == F.FP_FP64 else fp32_continuity_tol(len(cell), cx.n_nodes, cx.n_edges)
    assert r[0] <= ctol * r[1]
    # the cases reach what they are built for
    by = {n: (a, c) for n, a, c in zip(names, cell1, cell)}
    if not bound:
        assert by["end_on_face"][0] == by["end_on_face"][1]       # strict exit rule: stays
        assert by["rest_on_face"][0] == by["rest_on_face"][1]
        assert by["start_on_face_in"][0] == by["start_on_face_in"][1]
        assert by["start_on_face_out"][0] != by["start_on_face_out"][1]
        assert by["wall_face"][0] == -1 and by["wall_edge"][0] == -1
    lib.close()
