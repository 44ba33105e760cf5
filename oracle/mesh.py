"""Oracle: discrete complex K = {N, E, F, T} of a tet mesh, in plain numpy.  TEST INFRASTRUCTURE.

Sec. II.C: nodes, edges, faces and tets carry Whitney forms W0..W3; the matrices
[grad], [curl], [div] built from M_g, M_c, M_d reduce, for lowest-order Whitney
forms, to signed incidence matrices:
  D0 (N_e x N_n):  edge (i<j):  -1 at i, +1 at j          ((D0 phi)_e = phi_j - phi_i)
  D1 (N_f x N_e):  face (i<j<k): +1 on (i,j), +1 on (j,k), -1 on (i,k)
  D2 (N_t x N_f):  tet (a<b<c<d) with orientation s: s*(-1)^k on the face opposite vertex k
Edges are the sorted pairs, faces the sorted triples, both numbered in
lexicographic order.  Face k of a tet is the face opposite its k-th (sorted) vertex.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

LOCAL_EDGES = ((0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3))
LOCAL_FACES = ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2))


class Complex:
    """Topology + geometry of a tet mesh (Sec. II.C), computed directly from its definition."""

    def __init__(self, xyz: np.ndarray, tets: np.ndarray):
        self.xyz = np.ascontiguousarray(xyz, dtype=np.float64)
        tv = np.sort(np.asarray(tets, dtype=np.int64), axis=1)
        self.tv = tv
        nn = self.xyz.shape[0]
        nt = tv.shape[0]
        self.n_nodes, self.n_tets = nn, nt
        x = self.xyz[tv]
        e1, e2, e3 = x[:, 1] - x[:, 0], x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]
        det = np.einsum("ij,ij->i", e1, np.cross(e2, e3))
        if np.any(det == 0.0):
            raise ValueError("degenerate tet")
        self.orient = np.sign(det).astype(np.int64)
        self.vol = np.abs(det) / 6.0

        # edges: unique sorted pairs
        pairs = np.stack([tv[:, list(a)] for a in LOCAL_EDGES], axis=1)          # [nt,6,2]
        keys = pairs[..., 0] * nn + pairs[..., 1]
        ukeys, inv = np.unique(keys.ravel(), return_inverse=True)
        self.edges = np.stack([ukeys // nn, ukeys % nn], axis=1)
        self.tet_edges = inv.reshape(nt, 6)
        self.n_edges = self.edges.shape[0]
        self._ekeys = ukeys

        # faces: unique sorted triples, face k opposite vertex k
        tri = np.stack([tv[:, list(f)] for f in LOCAL_FACES], axis=1)            # [nt,4,3]
        fkeys = (tri[..., 0] * nn + tri[..., 1]) * nn + tri[..., 2]
        ufk, finv = np.unique(fkeys.ravel(), return_inverse=True)
        self.faces = np.stack([ufk // (nn * nn), (ufk // nn) % nn, ufk % nn], axis=1)
        self.tet_faces = finv.reshape(nt, 4)
        self.n_faces = self.faces.shape[0]

        # neighbours across each face
        owner = np.full((self.n_faces, 2), -1, dtype=np.int64)
        cnt = np.zeros(self.n_faces, dtype=np.int64)
        flat_f = self.tet_faces.ravel()
        flat_t = np.repeat(np.arange(nt), 4)
        order = np.argsort(flat_f, kind="stable")
        fs, ts = flat_f[order], flat_t[order]
        first = np.ones_like(fs, dtype=bool)
        first[1:] = fs[1:] != fs[:-1]
        owner[fs[first], 0] = ts[first]
        owner[fs[~first], 1] = ts[~first]
        np.add.at(cnt, flat_f, 1)
        if cnt.max() > 2:
            raise ValueError("non-manifold mesh")
        self.face_tets = owner
        other = np.where(owner[self.tet_faces, 0] == np.arange(nt)[:, None],
                         owner[self.tet_faces, 1], owner[self.tet_faces, 0])
        self.neigh = other.astype(np.int64)                                     # [nt,4], -1 wall

        bface = cnt == 1
        self.boundary_face = bface
        bnodes = np.zeros(nn, dtype=bool)
        bnodes[self.faces[bface].ravel()] = True
        self.boundary_node = bnodes
        fe = self.face_edges()
        bedge = np.zeros(self.n_edges, dtype=bool)
        bedge[fe[bface].ravel()] = True
        self.boundary_edge = bedge

    def edge_id(self, i, j):
        k = np.asarray(i, dtype=np.int64) * self.n_nodes + np.asarray(j, dtype=np.int64)
        idx = np.searchsorted(self._ekeys, k)
        assert np.all(self._ekeys[idx] == k)
        return idx

    def face_edges(self) -> np.ndarray:
        """[N_f,3] edge ids of (i,j), (j,k), (i,k) for face (i<j<k)."""
        f = self.faces
        return np.stack([self.edge_id(f[:, 0], f[:, 1]), self.edge_id(f[:, 1], f[:, 2]),
                         self.edge_id(f[:, 0], f[:, 2])], axis=1)

    # ---- incidence matrices (Sec. II.C: [grad], [curl], [div] for Whitney forms) ----
    def D0(self) -> sp.csr_matrix:
        ne = self.n_edges
        rows = np.repeat(np.arange(ne), 2)
        cols = self.edges.ravel()
        vals = np.tile([-1, 1], ne)
        return sp.csr_matrix((vals.astype(np.int64), (rows, cols)), shape=(ne, self.n_nodes))

    def D1(self) -> sp.csr_matrix:
        nf = self.n_faces
        rows = np.repeat(np.arange(nf), 3)
        cols = self.face_edges().ravel()
        vals = np.tile([1, 1, -1], nf)
        return sp.csr_matrix((vals.astype(np.int64), (rows, cols)), shape=(nf, self.n_edges))

    def D2(self) -> sp.csr_matrix:
        nt = self.n_tets
        rows = np.repeat(np.arange(nt), 4)
        cols = self.tet_faces.ravel()
        alt = np.array([1, -1, 1, -1])
        vals = (self.orient[:, None] * alt[None, :]).ravel()
        return sp.csr_matrix((vals, (rows, cols)), shape=(nt, self.n_faces))

    # ---- DOFs of uniform fields (circulation along edges, flux through faces) ----
    def project_uniform(self, E0, B0):
        """e_ij = E0 . (x_j - x_i);  b_ijk = B0 . (x_j - x_i) x (x_k - x_i) / 2."""
        E0 = np.asarray(E0, dtype=np.float64)
        B0 = np.asarray(B0, dtype=np.float64)
        x = self.xyz
        e = (x[self.edges[:, 1]] - x[self.edges[:, 0]]) @ E0
        f = self.faces
        area = 0.5 * np.cross(x[f[:, 1]] - x[f[:, 0]], x[f[:, 2]] - x[f[:, 0]])
        b = area @ B0
        return e, b

    def node_volume(self) -> np.ndarray:
        """alpha^0_n = integral of W0_n over the domain = sum over tets containing n of |T|/4."""
        a = np.zeros(self.n_nodes)
        np.add.at(a, self.tv.ravel(), np.repeat(self.vol / 4.0, 4))
        return a

    def c_arrays(self):
        """Contiguous int32 arrays for the C routines."""
        return (np.ascontiguousarray(self.tv, dtype=np.int32),
                np.ascontiguousarray(self.tet_edges, dtype=np.int32),
                np.ascontiguousarray(self.tet_faces, dtype=np.int32),
                np.ascontiguousarray(self.neigh, dtype=np.int32))
