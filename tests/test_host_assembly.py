"""The library's host-side assembly against the oracle, on the CPU (no GPU, no CUDA runtime).

tests/host_harness.cpp compiles the library's own host sources (mesh_build.cpp,
field_build.cpp, mfem_build.cpp) with g++ and exposes what they build.  Checked here:
the discrete complex's numbering and boundary faces; the edge mass [*eps], the curl-curl
matrix [*S] and the node Laplacian L (closed-form element matrices in the library, quadrature
and the paper's products D1^T [*mu^-1] D1, D0^T [*eps] D0 in the oracle) on the free DOFs, with
unit rows on PEC DOFs; the face mass [*mu^-1] and the transposed curl of the comparison
systems; the Lanczos estimate of the top of the Jacobi-scaled spectra.  Both field boundaries.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp

from paper_2103_06737_gb300 import inputs as I
import oracle as O
from oracle import fields as OF

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_2103_06737_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def hh(tmp_path_factory):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    out = str(tmp_path_factory.mktemp("hh") / "libhh.so")
    srcs = [os.path.join(HERE, "host_harness.cpp")] + [os.path.join(CSRC, f) for f in
                                                        ("mesh_build.cpp", "field_build.cpp", "mfem_build.cpp")]
    cmd = [cxx, "-O1", "-std=c++17", "-shared", "-fPIC", "-I" + inc, "-I" + os.path.join(ROOT, "include"),
           *srcs, "-Wl,--no-undefined", "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    lib = ctypes.CDLL(out)
    lib.hh_error.restype = ctypes.c_char_p
    lib.hh_build.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                             ctypes.c_double, ctypes.c_int]
    lib.hh_incidence.restype = ctypes.c_int64
    lib.hh_lambda_max.restype = ctypes.c_double
    lib.hh_lambda_max.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int]
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _build(hh, m, pec):
    xyz = np.ascontiguousarray(m.xyz, np.float64)
    tet = np.ascontiguousarray(m.tets, np.int32)
    st = hh.hh_build(xyz.shape[0], tet.shape[0], _p(xyz), _p(tet), OF.EPS0, OF.MU0, 1 if pec else 0)
    assert st == 0, hh.hh_error().decode()
    s = np.zeros(8, np.int64)
    hh.hh_sizes(_p(s))
    return [int(x) for x in s]


@pytest.fixture(scope="module")
def mesh4():
    m = I.cube_mesh(4, 1.0, 0.1, seed=1)
    return m, O.Complex(m.xyz, m.tets)


def _close(a, b, rel=1e-12):
    a, b = sp.csr_matrix(a), sp.csr_matrix(b)
    scale = abs(b).max()
    return abs(a - b).max() <= rel * scale


@pytest.mark.parametrize("bc", ["pec", "neumann"])
def test_field_operators_match_oracle(hh, mesh4, bc):
    m, cx = mesh4
    nn, ne, nf, nt, enz, nnz_n, fnz, efnz = _build(hh, m, bc == "pec")
    assert (nn, ne, nf, nt) == (cx.n_nodes, cx.n_edges, cx.n_faces, cx.n_tets)
    edges = np.zeros(2 * ne, np.int32)
    faces = np.zeros(3 * nf, np.int32)
    tf = np.zeros(4 * nt, np.int32)
    bface = np.zeros(nf, np.uint8)
    hh.hh_complex(_p(edges), _p(faces), _p(tf), _p(bface))
    assert np.array_equal(edges.reshape(-1, 2), cx.edges)
    assert np.array_equal(faces.reshape(-1, 3), cx.faces)
    assert np.array_equal(tf.reshape(-1, 4), cx.tet_faces)
    assert np.array_equal(bface.astype(bool), cx.boundary_face)

    e_rp, e_col = np.zeros(ne + 1, np.int32), np.zeros(enz, np.int32)
    M, S = np.zeros(enz), np.zeros(enz)
    n_rp, n_col, L = np.zeros(nn + 1, np.int32), np.zeros(nnz_n, np.int32), np.zeros(nnz_n)
    efix, nfix = np.zeros(ne, np.uint8), np.zeros(nn, np.uint8)
    hh.hh_fields(_p(e_rp), _p(e_col), _p(M), _p(S), _p(n_rp), _p(n_col), _p(L), _p(efix), _p(nfix))
    if bc == "pec":
        assert np.array_equal(efix.astype(bool), cx.boundary_edge)
        assert np.array_equal(nfix.astype(bool), cx.boundary_node)
    else:
        assert not efix.any() and not nfix.any()
    fe, fn = np.nonzero(efix == 0)[0], np.nonzero(nfix == 0)[0]
    Mh = sp.csr_matrix((M, e_col, e_rp), shape=(ne, ne))
    Sh = sp.csr_matrix((S, e_col, e_rp), shape=(ne, ne))
    Lh = sp.csr_matrix((L, n_col, n_rp), shape=(nn, nn))
    assert _close(Mh[fe][:, fe], OF.edge_mass(cx)[fe][:, fe])
    assert _close(Sh[fe][:, fe], OF.curl_curl(cx)[fe][:, fe])
    assert _close(Lh[fn][:, fn], OF.node_laplacian(cx)[fn][:, fn])
    # PEC rows: a unit diagonal and nothing else (M, L); no entry in S
    for A, fixed in ((Mh, np.nonzero(efix)[0]), (Lh, np.nonzero(nfix)[0])):
        blk = A[fixed]
        assert abs(blk).sum() == fixed.size
        assert np.array_equal(blk.toarray()[np.arange(fixed.size), fixed], np.ones(fixed.size))
    assert Sh[np.nonzero(efix)[0]].count_nonzero() == 0


def test_face_mass_and_curl_transpose_match_oracle(hh, mesh4):
    m, cx = mesh4
    nn, ne, nf, nt, enz, nnz_n, fnz, efnz = _build(hh, m, True)
    f_rp, f_col, Fm = np.zeros(nf + 1, np.int32), np.zeros(fnz, np.int32), np.zeros(fnz)
    ef_rp, ef_col, ef_sgn = np.zeros(ne + 1, np.int32), np.zeros(efnz, np.int32), np.zeros(efnz, np.int8)
    hh.hh_mfem(_p(f_rp), _p(f_col), _p(Fm), _p(ef_rp), _p(ef_col), _p(ef_sgn))
    Fh = sp.csr_matrix((Fm, f_col, f_rp), shape=(nf, nf))
    assert _close(Fh, OF.face_mass(cx))
    CT = sp.csr_matrix((ef_sgn.astype(np.float64), ef_col, ef_rp), shape=(ne, nf))
    assert abs(CT - cx.D1().T.astype(np.float64)).max() == 0
    # [curl]^T [*mu^-1] [curl] = [*S] (Eq. wave_cont), here from the library's two halves
    assert _close(CT @ Fh @ CT.T, OF.curl_curl(cx))


@pytest.mark.parametrize("bc", ["pec", "neumann"])
def test_lanczos_estimate_of_the_jacobi_spectrum(hh, mesh4, bc):
    """The top of the Jacobi-scaled spectra (the Chebyshev interval's upper end): 40 Lanczos
    steps from the library's fixed start give a lower bound within 1% of the exact largest
    eigenvalue of D^-1 A (numpy, symmetric form D^-1/2 A D^-1/2) for both systems."""
    m, cx = mesh4
    nn, ne, nf, nt, enz, nnz_n, fnz, efnz = _build(hh, m, bc == "pec")
    dt = 0.2 * I.gyro_period(0.1)
    e_rp, e_col = np.zeros(ne + 1, np.int32), np.zeros(enz, np.int32)
    M, S = np.zeros(enz), np.zeros(enz)
    n_rp, n_col, L = np.zeros(nn + 1, np.int32), np.zeros(nnz_n, np.int32), np.zeros(nnz_n)
    efix, nfix = np.zeros(ne, np.uint8), np.zeros(nn, np.uint8)
    hh.hh_fields(_p(e_rp), _p(e_col), _p(M), _p(S), _p(n_rp), _p(n_col), _p(L), _p(efix), _p(nfix))
    for which, A in ((0, sp.csr_matrix((M + 0.25 * dt * dt * S, e_col, e_rp), shape=(ne, ne))),
                     (1, sp.csr_matrix((L, n_col, n_rp), shape=(nn, nn)))):
        d = 1.0 / np.sqrt(A.diagonal())
        lam = np.linalg.eigvalsh((sp.diags(d) @ A @ sp.diags(d)).toarray()).max()
        est = hh.hh_lambda_max(which, dt, 40)
        assert est <= lam * (1 + 1e-9), (which, est, lam)
        assert est >= 0.99 * lam, (which, est, lam)


def test_incidence_neighbours_and_geometry_match_oracle(hh, mesh4):
    """D0, D1, D2 bit-exact, the neighbour table exact, the barycentric gradients and tet
    origins to round-off."""
    m, cx = mesh4
    nn, ne, nf, nt = _build(hh, m, True)[:4]
    for which, ref, rows in ((0, cx.D0(), ne), (1, cx.D1(), nf), (2, cx.D2(), nt)):
        k = int(hh.hh_incidence(which, None, None, None))
        rp, col, val = np.zeros(rows + 1, np.int32), np.zeros(k, np.int32), np.zeros(k, np.int8)
        hh.hh_incidence(which, _p(rp), _p(col), _p(val))
        got = sp.csr_matrix((val.astype(np.int64), col, rp), shape=ref.shape)
        assert (got != ref).nnz == 0, which
    nb = np.zeros(4 * nt, np.int32)
    grad, origin = np.zeros(9 * nt), np.zeros(3 * nt)
    hh.hh_tets(_p(nb), _p(grad), _p(origin))
    assert np.array_equal(nb.reshape(-1, 4), cx.neigh)
    g_ref = OF.grads(cx)[:, 1:, :].reshape(nt, 9)
    assert np.abs(grad.reshape(nt, 9) - g_ref).max() <= 1e-12 * np.abs(g_ref).max()
    assert np.array_equal(origin.reshape(nt, 3), cx.xyz[cx.tv[:, 0]])


def test_build_rejects_bad_meshes(hh):
    """Host-side validation: a node id out of range (FP_EINVAL), a repeated node or a flat tet
    (FP_EGEOM), a face shared by three tets (FP_EGEOM)."""
    xyz = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1], [0.3, 0.3, 0.0], [0.2, 0.2, -1.0]],
                   np.float64)

    def build(tets, pts=xyz):
        t = np.ascontiguousarray(np.array(tets, np.int32))
        x = np.ascontiguousarray(pts)
        return hh.hh_build(x.shape[0], t.shape[0], _p(x), _p(t), OF.EPS0, OF.MU0, 1)

    assert build([[0, 1, 2, 3]]) == 0
    assert build([[0, 1, 2, 9]]) == 1                      # FP_EINVAL
    assert build([[0, 1, 2, 2]]) == 5                      # FP_EGEOM: repeated node
    assert build([[0, 1, 2, 5]]) == 5                      # FP_EGEOM: node 5 lies in the plane z = 0
    assert build([[0, 1, 2, 3], [0, 1, 2, 6]]) == 0
    assert build([[0, 1, 2, 3], [0, 1, 2, 4], [0, 1, 2, 6]]) == 5   # face (0,1,2) in three tets
    assert b"more than two" in hh.hh_error()
