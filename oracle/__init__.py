"""FP64 CPU oracle of the quasi-Helmholtz FEM-PIC hot path.

TEST INFRASTRUCTURE ONLY.  Imported by tests/, by the smoke check and by the
bench's CPU-baseline / reference leg.  The CUDA library never imports, links or
runs anything here, and nothing here imports the library: the two share only
the seeded input generators (paper_2103_06737_gb300/inputs.py).

Parts:
  mesh.Complex       discrete complex, incidence D0/D1/D2, uniform-field DOFs (Sec. II.C)
  particles.c        gather (W1/W2), Boris, tet walk, W1 path-integral deposit, W0 charge
                     (Sec. II.A, II.C, IV.B.1)
  fields.py          Hodge matrices, Newmark wave-equation step, Gauss-law projection,
                     Faraday update, residuals (Sec. II.C, IV.A-B)
  adams.py           fourth-order Adams(-Bashforth) particle mover with start-up, on the
                     same walk and deposits (Sec. IV.B.2)
  cotree.py          tree / co-tree reduced field system (Z-matrices, Eq. reduceMEs and
                     reducedWaveEqn) and the first-order mixed FEM, dense (Sec. IV.B, V, VI.A.1)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

from .mesh import Complex, LOCAL_EDGES, LOCAL_FACES  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile particles.c (plain C, no FMA contraction, OpenMP over particles)."""
    src = os.path.join(_HERE, "particles.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64 = ctypes.c_int64
            d = ctypes.c_double
            i = ctypes.c_int
            _lib.oracle_step.restype = i64
            _lib.oracle_step.argtypes = [i64, i64, P, P, P, P, P, P, P, i64, P, P, P, d, d, d, d, i, i, P,
                                         P, P, P, P, P, i, P, P]
            _lib.oracle_gather.restype = None
            _lib.oracle_gather.argtypes = [P, P, P, P, P, P, i64, P, P, P, P]
            _lib.oracle_bary.restype = None
            _lib.oracle_bary.argtypes = [P, P, i64, P, P, P]
            _lib.oracle_boris.restype = None
            _lib.oracle_boris.argtypes = [i64, P, P, P, d, d, d]
            _lib.oracle_walk_trace.restype = i
            _lib.oracle_walk_trace.argtypes = [i64, i64, P, P, P, P, P, i, P, P, d, i, i, P, P, P, P, P, P, P, P]
            _lib.oracle_charge.restype = None
            _lib.oracle_charge.argtypes = [P, P, i64, i64, P, P, d, P, P]
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class Oracle:
    """Oracle over one mesh: topology from mesh.Complex, particle routines from particles.c."""

    def __init__(self, xyz, tets):
        self.cx = Complex(xyz, tets)
        self.tv32, self.te32, self.tf32, self.nb32 = self.cx.c_arrays()
        self.xyz = self.cx.xyz

    @property
    def n_nodes(self):
        return self.cx.n_nodes

    @property
    def n_edges(self):
        return self.cx.n_edges

    @property
    def n_faces(self):
        return self.cx.n_faces

    @property
    def n_tets(self):
        return self.cx.n_tets

    def origin(self, cell):
        """x of each tet's lowest-id vertex (the offset origin used by the library's state)."""
        return self.xyz[self.cx.tv[np.asarray(cell), 0]]

    def bary(self, cell, X):
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        X = _f64(X, (-1, 3))
        lam = np.empty((cell.shape[0], 4))
        lib().oracle_bary(_p(self.xyz), _p(self.tv32), cell.shape[0], _p(cell), _p(X), _p(lam))
        return lam

    def gather(self, cell, X, e, b):
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        X = _f64(X, (-1, 3))
        e = _f64(e)
        b = _f64(b)
        E = np.empty_like(X)
        B = np.empty_like(X)
        lib().oracle_gather(_p(self.xyz), _p(self.tv32), _p(self.te32), _p(self.tf32), _p(e), _p(b),
                            cell.shape[0], _p(cell), _p(X), _p(E), _p(B))
        return E, B

    def step(self, cell, X, V, e, b, q, m, w, dt, max_cross=64, Xend=None, nthreads=0, touch=False):
        """One particle step (push if Xend is None, else walk to Xend).  Returns a dict; with
        touch=True it also holds dG_touch / Q_touch, the sum of |q w| over the pieces / end
        points that touch each edge / node."""
        cell = np.array(cell, dtype=np.int32, order="C", copy=True)
        X = np.array(X, dtype=np.float64, order="C", copy=True).reshape(-1, 3)
        V = np.array(V, dtype=np.float64, order="C", copy=True).reshape(-1, 3)
        e = _f64(e)
        b = _f64(b)
        n = cell.shape[0]
        dG = np.zeros(self.n_edges)
        dGa = np.zeros(self.n_edges)
        Q = np.zeros(self.n_nodes)
        Qa = np.zeros(self.n_nodes)
        ncross = np.zeros(n, dtype=np.int32)
        Gt = np.zeros(self.n_edges) if touch else None
        Qt = np.zeros(self.n_nodes) if touch else None
        push = 1 if Xend is None else 0
        Xe = _f64(Xend, (-1, 3)) if Xend is not None else np.zeros((1, 3))
        nb = lib().oracle_step(self.n_edges, self.n_nodes, _p(self.xyz), _p(self.tv32), _p(self.te32),
                               _p(self.tf32), _p(self.nb32), _p(e), _p(b), n, _p(cell), _p(X), _p(V),
                               float(q), float(m), float(w), float(dt), int(max_cross), push, _p(Xe),
                               _p(dG), _p(dGa), _p(Q), _p(Qa), _p(ncross), int(nthreads),
                               _p(Gt) if touch else None, _p(Qt) if touch else None)
        out = dict(cell=cell, X=X, V=V, dG=dG, dG_abs=dGa, Q=Q, Q_abs=Qa, ncross=ncross, n_bound=int(nb))
        if touch:
            out["dG_touch"], out["Q_touch"] = Gt, Qt
        return out

    def walk_trace(self, cell, Xa, Xb, qw=1.0, max_cross=64, cap=256):
        """The pieces of one walk: (cells [k], piece start points [k,3], stop point, end cell, dG, Q)."""
        Xa = _f64(Xa, (3,))
        Xb = _f64(Xb, (3,))
        cells = np.zeros(cap, dtype=np.int32)
        start = np.zeros((cap, 3))
        stop = np.zeros(3)
        end = np.zeros(1, dtype=np.int32)
        dG = np.zeros(self.n_edges)
        dGa = np.zeros(self.n_edges)
        Q = np.zeros(self.n_nodes)
        Qa = np.zeros(self.n_nodes)
        k = lib().oracle_walk_trace(self.n_edges, self.n_nodes, _p(self.xyz), _p(self.tv32), _p(self.te32),
                                    _p(self.tf32), _p(self.nb32), int(cell), _p(Xa), _p(Xb), float(qw),
                                    int(max_cross), cap, _p(cells), _p(start), _p(stop), _p(end), _p(dG),
                                    _p(dGa), _p(Q), _p(Qa))
        assert k <= cap
        return cells[:k].copy(), start[:k].copy(), stop, int(end[0]), dG, Q

    def charge(self, cell, X, q, w):
        cell = np.ascontiguousarray(cell, dtype=np.int32)
        X = _f64(X, (-1, 3))
        Q = np.zeros(self.n_nodes)
        Qa = np.zeros(self.n_nodes)
        lib().oracle_charge(_p(self.xyz), _p(self.tv32), self.n_nodes, cell.shape[0], _p(cell), _p(X),
                            float(q * w), _p(Q), _p(Qa))
        return Q, Qa

    @staticmethod
    def boris(V, E, B, q, m, dt):
        V = np.array(V, dtype=np.float64, order="C", copy=True).reshape(-1, 3)
        E = _f64(E, (-1, 3))
        B = _f64(B, (-1, 3))
        lib().oracle_boris(V.shape[0], _p(V), _p(E), _p(B), float(q), float(m), float(dt))
        return V

    def project_uniform(self, E0, B0):
        return self.cx.project_uniform(E0, B0)


def nproc_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:  # pragma: no cover
        return os.cpu_count() or 1


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
