"""Pins of the oracle's discrete complex (Sec. II.C incidence, Sec. V Euler count)."""
import json
import os

import numpy as np
import pytest

from paper_2103_06737_gb300 import inputs as I
from oracle import Complex

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))


@pytest.mark.parametrize("n", [4, 32])
def test_kuhn_counts_and_euler(n):
    m = I.cube_mesh(n, 1.0, 0.1 if n > 4 else 0.0, seed=1)
    cx = Complex(m.xyz, m.tets)
    g = GOLD["kuhn_cube_counts"][str(n)]
    assert (cx.n_nodes, cx.n_edges, cx.n_faces, cx.n_tets) == \
        (g["n_nodes"], g["n_edges"], g["n_faces"], g["n_tets"])
    assert cx.n_nodes - cx.n_edges + cx.n_faces - cx.n_tets == 1


@pytest.mark.parametrize("n,jit", [(4, 0.0), (6, 0.1)])
def test_exact_sequence(n, jit):
    """[curl][grad] = 0 and [div][curl] = 0 exactly on integers (Sec. IV.B identities)."""
    m = I.cube_mesh(n, 1.0, jit, seed=1)
    cx = Complex(m.xyz, m.tets)
    D0, D1, D2 = cx.D0(), cx.D1(), cx.D2()
    assert (D1 @ D0).count_nonzero() == 0 or abs(D1 @ D0).max() == 0
    assert (D2 @ D1).count_nonzero() == 0 or abs(D2 @ D1).max() == 0
    # each edge has one tail and one head; each tet has 4 faces with +-1
    assert np.all(np.asarray(D0.sum(axis=1)).ravel() == 0)
    assert np.all(abs(D2).sum(axis=1) == 4)
    # rank of D0 is N_n - 1 (connected), of D1 is N_e - N_n + 1 (simply connected)
    if n == 4:
        r0 = np.linalg.matrix_rank(D0.toarray().astype(float))
        r1 = np.linalg.matrix_rank(D1.toarray().astype(float))
        assert r0 == cx.n_nodes - 1
        assert r1 == cx.n_edges - cx.n_nodes + 1


def test_volume_neighbours_boundary():
    n = 5
    m = I.cube_mesh(n, 2.0, 0.1, seed=3)
    cx = Complex(m.xyz, m.tets)
    assert abs(cx.vol.sum() - 8.0) < 1e-13
    # Kuhn tets alternate orientation in sorted-vertex order: both signs occur
    assert set(np.unique(cx.orient)) <= {-1, 1}
    nb = cx.neigh
    t = np.arange(cx.n_tets)
    for k in range(4):
        inner = nb[:, k] >= 0
        # the neighbour lists t back across the same global face
        back = (nb[nb[inner, k]] == t[inner, None]).any(axis=1)
        assert back.all()
        same_face = (cx.tet_faces[nb[inner, k]] == cx.tet_faces[inner, k][:, None]).any(axis=1)
        assert same_face.all()
    # boundary faces of a subdivided cube: 2 triangles per boundary square
    assert cx.boundary_face.sum() == 12 * n * n
    assert cx.boundary_node.sum() == (n + 1) ** 3 - (n - 1) ** 3


def test_two_tet_mesh():
    m = I.two_tet_mesh()
    cx = Complex(m.xyz, m.tets)
    assert (cx.n_nodes, cx.n_edges, cx.n_faces, cx.n_tets) == (5, 9, 7, 2)
    assert cx.neigh[0, 0] == 1 and cx.neigh[1, 3] == 0


def test_table_I_speed_of_light():
    g = GOLD["table_I_beam"]
    assert round(g["v_p"] / I.C_LIGHT, 5) == g["v_p_over_c"]
