"""Pins of the oracle's tet walk on degenerate paths (Sec. IV.B.1 deposits along the walk).

The paper is silent on the walk; the reading is: an exit needs lambda_k(end) < 0
strictly, the entry face is not an exit candidate, the smallest crossing fraction wins
and ties go to the lowest local face index, a wall absorbs the particle at the wall
point.  Every case of tests/walk_cases.py (paths through mesh edges and vertices, end
points on faces and vertices, starts on faces and edges, rest, wall exits) is held
against what does not depend on that reading:

  * brute-force point location: every sample of the path lies in the tet the walk
    assigns to it, and on a generic path the tets with positive-length pieces are
    exactly the tets brute force finds, in order;
  * the path integral of W1 by the midpoint rule on 2^12 samples with per-sample point
    location equals the walk's deposit (exactly where every crossing fraction is a
    multiple of 2^-12, since the integrand is linear between crossings);
  * continuity D0^T dG = dQ per particle to round-off, and the charge at the end
    point (or at the wall point).
The walk's sequence of cells and crossing points is read from the oracle itself by
bounding the crossings: with max_cross = k the particle stops at its k-th crossing point.
"""
import numpy as np
import pytest

from paper_2103_06737_gb300 import inputs as I
import oracle as O
import walk_cases as W

NS = 1 << 12


@pytest.fixture(scope="module")
def mesh():
    m = I.cube_mesh(W.N_HEX, 1.0, 0.0)
    return O.Oracle(m.xyz, m.tets)


def _zero(orc):
    return np.zeros(orc.n_edges), np.zeros(orc.n_faces)


def _pieces(orc, c0, Xa, Xb, max_cross=64):
    """The walk's pieces: cells[k] and the end points P[k], P[k+1] of piece k."""
    cells, start, stop, end, dG, Q = orc.walk_trace(c0, Xa, Xb, qw=-1.0, max_cross=max_cross)
    P = np.vstack([start, stop[None]])
    return list(cells), P, stop, end, dG, Q


def _containing(orc, P, tol=1e-13):
    """Brute force: for each point, the boolean matrix point x tet of containment."""
    nt = orc.n_tets
    inside = np.zeros((P.shape[0], nt), dtype=bool)
    for t in range(nt):
        lam = orc.bary(np.full(P.shape[0], t, dtype=np.int32), P)
        inside[:, t] = lam.min(axis=1) >= -tol
    return inside


def _grads(cx, t):
    x = cx.xyz[cx.tv[t]]
    J = np.stack([x[1] - x[0], x[2] - x[0], x[3] - x[0]], axis=1)
    Gi = np.linalg.inv(J)
    return np.vstack([-Gi.sum(axis=0), Gi])


@pytest.mark.parametrize("case", W.cases(), ids=[c[0] for c in W.cases()])
def test_walk_case_against_brute_force(mesh, case):
    orc = mesh
    cx = orc.cx
    name, c0, Xa, Xb = case
    lam_a = orc.bary([c0], [Xa])[0]
    assert lam_a.min() >= 0.0, "start point outside its start tet"
    cells, P, stop, end, dG_t, Q_t = _pieces(orc, c0, Xa, Xb)
    e, b = _zero(orc)
    full = orc.step([c0], [Xa], [Xb - Xa], e, b, -1.0, 1.0, 1.0, 1.0)
    # the traced walk is the step's walk
    assert int(full["cell"][0]) == end and np.array_equal(full["X"][0], stop)
    assert np.array_equal(full["dG"], dG_t) and np.array_equal(full["Q"], Q_t)
    assert int(full["ncross"][0]) == len(cells) - 1 + (1 if end < 0 else 0)
    assert cells[0] == c0 and np.array_equal(P[0], Xa)
    if end < 0:
        assert stop[2] == 0.0 or stop[0] == 0.0       # absorbed at the wall point
    else:
        assert np.array_equal(stop, Xb) and cells[-1] == end
    L = np.linalg.norm(stop - Xa)
    # every piece lies in its cell (end points included)
    for j, c in enumerate(cells):
        t = np.linspace(0.0, 1.0, 9)[:, None]
        pts = P[j][None] + t * (P[j + 1] - P[j])[None]
        assert orc.bary(np.full(9, c, dtype=np.int32), pts).min() >= -1e-14, (name, j)
    # the crossing points lie on the path, in order
    s = [float(np.dot(p - Xa, stop - Xa) / L ** 2) if L > 0 else 0.0 for p in P]
    assert s[0] == 0.0 and all(b_ >= a_ for a_, b_ in zip(s, s[1:]))
    if L > 0:
        assert np.abs(s[-1] - 1.0) <= 1e-15
        # brute force over samples of the whole path: each sample lies in the tet of its piece
        ts = (np.arange(NS) + 0.5) / NS
        pts = Xa[None] + ts[:, None] * (stop - Xa)[None]
        inside = _containing(orc, pts)
        assert inside.any(axis=1).all()
        piece = np.searchsorted(np.array(s[1:-1]), ts, side="right")
        assert inside[np.arange(NS), np.array(cells)[piece]].all(), name
        if (inside.sum(axis=1) == 1).all():            # generic path: one tet per sample
            bf = np.argmax(inside, axis=1)
            bf_seq = [bf[0]] + [c for i, c in enumerate(bf[1:], 1) if c != bf[i - 1]]
            walk_seq = [c for j, c in enumerate(cells) if np.linalg.norm(P[j + 1] - P[j]) > 0]
            assert walk_seq == bf_seq, (name, walk_seq, bf_seq)
        # path integral of W1 (times q w = -1) by the midpoint rule with per-sample location
        G = np.zeros(cx.n_edges)
        d = (stop - Xa) / NS
        loc = np.argmax(inside, axis=1)
        for t in np.unique(loc):
            sel = loc == t
            lam = orc.bary(np.full(sel.sum(), t, dtype=np.int32), pts[sel])
            g = _grads(cx, t)
            for k, (a, bb) in enumerate(O.LOCAL_EDGES):
                w = lam[:, a][:, None] * g[bb] - lam[:, bb][:, None] * g[a]
                G[cx.tet_edges[t, k]] += -1.0 * (w @ d).sum()
        # exact for the dyadic cases; "long" crosses faces at generic fractions, where a
        # sample interval that straddles a crossing carries an O(1/NS) error
        tol = 1e-12 if name != "long" else 2.0 * len(cells) / NS
        assert np.abs(full["dG"] - G).max() <= tol * max(np.abs(G).max(), 1e-300), name
    else:
        assert np.abs(full["dG"]).max() == 0.0
    # continuity per particle, and the charge at the stop point
    Q0, _ = orc.charge([c0], [Xa], -1.0, 1.0)
    res = cx.D0().T @ full["dG"] - (full["Q"] - Q0)
    assert np.abs(res).max() <= 1e-14
    lam_e = orc.bary([cells[-1]], [stop])[0]
    assert np.allclose(full["Q"][cx.tv[cells[-1]]], -lam_e, atol=1e-15)


def test_tie_rule_lowest_local_face(mesh):
    """At a crossing through an edge or vertex several faces have the same crossing
    fraction; the walk leaves through the lowest local index among them."""
    orc = mesh
    cx = orc.cx
    n_ties = 0
    for name, c0, Xa, Xb in W.cases():
        cells, P, stop, end, _, _ = _pieces(orc, c0, Xa, Xb)
        nxt_cells = cells[1:] + ([end] if end < 0 else [])
        entry = -1
        for k, nxt in enumerate(nxt_cells):
            c = cells[k]
            la = orc.bary([c], [P[k]])[0]
            lb = orc.bary([c], [Xb])[0]
            cand = [f for f in range(4) if f != entry and lb[f] < 0.0]
            frac = {f: (la[f] / (la[f] - lb[f]) if la[f] - lb[f] > 0 else 0.0) for f in cand}
            smin = min(frac.values())
            tied = [f for f in cand if frac[f] == smin]
            n_ties += len(tied) > 1
            f = min(tied)
            assert cx.neigh[c, f] == nxt, (name, k)
            if nxt < 0:
                break
            shared = set(cx.tv[c])
            entry = [a for a in range(4) if cx.tv[nxt, a] not in shared][0]
    assert n_ties >= 5


def test_walk_bound_stops_at_the_crossing_point(mesh):
    orc = mesh
    name, c0, Xa, Xb = [c for c in W.cases() if c[0] == "long"][0]
    cells, P, stop, end, _, _ = _pieces(orc, c0, Xa, Xb)
    assert len(cells) >= 8
    e, b = _zero(orc)
    for k in (1, 3, 5):
        r = orc.step([c0], [Xa], [Xb - Xa], e, b, -1.0, 1.0, 1.0, 1.0, max_cross=k)
        assert r["n_bound"] == 1 and r["cell"][0] == cells[k]
        assert np.array_equal(r["X"][0], P[k])           # stopped at the k-th crossing point
        Q0, _ = orc.charge([c0], [Xa], -1.0, 1.0)
        assert np.abs(orc.cx.D0().T @ r["dG"] - (r["Q"] - Q0)).max() <= 1e-14
