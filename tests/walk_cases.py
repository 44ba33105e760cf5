"""Degenerate tet-walk cases on the unjittered 4^3 Kuhn mesh of the unit cube (h = 1/4).

Inputs only: start points, end points and start tets, with dyadic coordinates and
crossing fractions, so every barycentric coordinate and crossing point along these
paths is exact in binary floating point and the walk's ties (a path through a mesh
edge or vertex, an end point on a face) are exact ties on every implementation.  The
start tet is found from the Kuhn lattice: the hex by flooring, the tet by the order of
the local coordinates (tet p of a hex holds u[p0] >= u[p1] >= u[p2], inputs.cube_mesh's
numbering), evaluated at a point a little inside the tet the case names.
"""
import numpy as np

N_HEX = 4
H = 1.0 / N_HEX
_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


def kuhn_cell(P):
    """Tet id of inputs.cube_mesh(4, 1, 0) containing the point P strictly inside a tet."""
    u = np.asarray(P, dtype=np.float64) / H
    hx = np.clip(np.floor(u).astype(int), 0, N_HEX - 1)
    loc = u - hx
    perm = tuple(int(a) for a in np.argsort(-loc, kind="stable"))
    assert len(set(np.round(loc, 12))) == 3, "hint point on a face"
    return 6 * (hx[0] + N_HEX * (hx[1] + N_HEX * hx[2])) + _PERMS.index(perm)


def _c(*a):
    return np.array(a, dtype=np.float64)


def cases():
    """List of (name, start tet, Xa, Xb).  The start tet is the one containing Xa + hint."""
    e = 1.0 / 64.0
    out = []

    def add(name, Xa, Xb, hint=None):
        Xa, Xb = _c(*Xa), _c(*Xb)
        probe = Xa + (hint if hint is not None else (Xb - Xa) * 2.0 ** -10)
        out.append((name, kuhn_cell(probe), Xa, Xb))

    c = 0.375
    # through the interior diagonal of a hex (a mesh edge shared by its six tets), at s = 1/2
    add("hex_diagonal", (c + 2 * e, c, c - 2 * e), (c - 2 * e, c, c + 2 * e))
    # through an axis-parallel mesh edge (x = y = 1/2) shared by four hexes
    add("axis_edge", (0.5 - 3 * e, 0.5 - e, c + 2 * e), (0.5 + 3 * e, 0.5 + e, c - 2 * e))
    # through a face-diagonal mesh edge in the plane z = 1/2
    add("face_diagonal_edge", (c + 2 * e, c - 2 * e, 0.5 - e), (c - 2 * e, c + 2 * e, 0.5 + e))
    # through a mesh vertex (1/2, 1/2, 1/2), generic direction
    add("vertex", (0.5 - 3 * e, 0.5 - 2 * e, 0.5 - e), (0.5 + 3 * e, 0.5 + 2 * e, 0.5 + e))
    # through a mesh vertex along the hex diagonal direction (along mesh edges)
    add("vertex_along_edges", (0.5 - 2 * e, 0.5 - 2 * e, 0.5 - 2 * e), (0.5 + 2 * e, 0.5 + 2 * e, 0.5 + 2 * e),
        hint=_c(e / 8, e / 16, -e / 32))
    # ends exactly on an interior face (the plane x = y inside a hex): stays in its tet
    add("end_on_face", (c + 2 * e, c - e, c - 3 * e), (c + e / 2, c + e / 2, c - 3 * e))
    # ends exactly on a mesh vertex
    add("end_on_vertex", (0.5 - 3 * e, 0.5 - 2 * e, 0.5 - e), (0.5, 0.5, 0.5))
    # starts on an interior face of its tet and leaves through that face
    add("start_on_face_out", (c + e, c + e, c - 2 * e), (c - e, c + 3 * e, c - 2 * e), hint=_c(e / 8, -e / 8, 0))
    # starts on an interior face of its tet and moves into the tet
    add("start_on_face_in", (c + e, c + e, c - 2 * e), (c + 3 * e, c - e, c - 2 * e), hint=_c(e / 8, -e / 8, 0))
    # starts on a mesh edge (the hex diagonal) and leaves its tet through it
    add("start_on_edge_out", (c, c, c), (c - 2 * e, c + e, c + 2 * e), hint=_c(3 * e / 64, 2 * e / 64, e / 64))
    # at rest inside a tet, and at rest on an interior face
    add("rest_inside", (c + 2 * e, c - e, c - 3 * e), (c + 2 * e, c - e, c - 3 * e), hint=_c(0, 0, 0))
    add("rest_on_face", (c + e, c + e, c - 2 * e), (c + e, c + e, c - 2 * e), hint=_c(e / 8, -e / 8, 0))
    # leaves the domain through a wall (z = 0) at an interior point of a boundary face
    add("wall_face", (0.125 + e, 0.125 - e, e), (0.125 + e, 0.125 - e, -e))
    # leaves the domain through a boundary mesh edge (the cube's edge x = z = 0)
    add("wall_edge", (3 * e, 0.375 + e, e), (-3 * e, 0.375 + e, -e))
    # a long path across many tets with generic (non-dyadic) crossing fractions
    add("long", (0.1 + e / 3, 0.2, 0.3), (0.81, 0.67, 0.55))
    return out
