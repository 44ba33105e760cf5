"""Thin Python binding of libfempic.so (C ABI in include/fem_pic.h).

Argument marshalling only: torch tensors give device memory and streams, every
step of the hot path runs in the library's CUDA kernels.  Function names match
the C entry points.  If the library is missing this module raises; there is no
CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

import numpy as np
import torch

from . import build as _build

FP_OK, FP_EINVAL, FP_ECUDA, FP_EWALK, FP_ENOCONV, FP_EGEOM = range(6)
FP_FP64, FP_FP32 = 0, 1
FP_ACCUMULATE, FP_NO_AGGREGATE, FP_SAME_FIELDS, FP_CHARGE_CHANGE = 1, 2, 4, 8
_STATUS = {0: "FP_OK", 1: "FP_EINVAL", 2: "FP_ECUDA", 3: "FP_EWALK", 4: "FP_ENOCONV", 5: "FP_EGEOM"}

_lock = threading.Lock()
_lib = None


class FemPicError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS.get(code, code)}: {msg}")
        self.code = code


class FPMesh(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_tets", ctypes.c_int64), ("xyz", ctypes.c_void_p),
                ("tet", ctypes.c_void_p)]


class FPCsr(ctypes.Structure):
    _fields_ = [("n_rows", ctypes.c_int64), ("n_cols", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("row_ptr", ctypes.c_void_p), ("col", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class FPParticles(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("cell", ctypes.c_void_p), ("off", ctypes.c_void_p),
                ("vel", ctypes.c_void_p), ("q", ctypes.c_double), ("m", ctypes.c_double),
                ("w", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("precond", ctypes.c_int32), ("fell_back", ctypes.c_int32),
                ("outer", ctypes.c_int32), ("rel_res", ctypes.c_double), ("abs_res", ctypes.c_double),
                ("ms", ctypes.c_double)]

    def as_dict(self):
        return dict(iters=int(self.iters), outer=int(self.outer), precond=int(self.precond),
                    fell_back=int(self.fell_back), rel_res=float(self.rel_res), abs_res=float(self.abs_res),
                    ms=float(self.ms))


FP_SYS_NEWMARK, FP_SYS_GAUSS = 0, 1
FP_PC_JACOBI, FP_PC_LEARNED, FP_PC_JACOBI_FP64, FP_PC_LEARNED_GAUSS = 0, 1, 2, 4
FP_BC_PEC, FP_BC_NEUMANN = 0, 1
FP_LEARNED_GUESS, FP_LEARNED_PRECOND = 0, 1
EPS0 = 8.854_187_8128e-12
MU0 = 1.256_637_062_12e-6


def library_path() -> str:
    return _build.SO


def lib():
    """Load libfempic.so (built in-tree by build.py).  Raises if it is not there."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.SO
        if not os.path.exists(path):
            raise RuntimeError(f"libfempic.so not found at {path}: build it first "
                               "(python -c 'import __graft_entry__ as g; g.build()')")
        L = ctypes.CDLL(path)
        P, I64, I32, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        sig = {
            "fem_pic_create": (I32, [ctypes.POINTER(FPMesh), ctypes.POINTER(FPCsr), ctypes.POINTER(FPCsr),
                                     ctypes.POINTER(FPCsr), I32, ctypes.POINTER(P)]),
            "fem_pic_destroy": (None, [P]),
            "fem_pic_last_error": (ctypes.c_char_p, [P]),
            "fem_pic_sizes": (I32, [P, P]),
            "fem_pic_set_deposit_precision": (I32, [P, I32]),
            "fem_pic_deposit_precision": (I32, [P]),
            "fem_pic_set_charge_precision": (I32, [P, I32]),
            "fem_pic_charge_precision": (I32, [P]),
            "fem_pic_incidence": (I32, [P, I32, P, P, P]),
            "fem_pic_topology": (I32, [P, P, P, P, P]),
            "fem_pic_project_uniform": (I32, [P, P, P, P, P, P]),
            "fem_pic_particles_from_global": (I32, [P, I64, P, P, P, P]),
            "fem_pic_particles_to_global": (I32, [P, I64, P, P, P, P]),
            "fem_pic_push_deposit": (I32, [P, P, P, ctypes.POINTER(FPParticles), D, I32, P, P, I32, P]),
            "fem_pic_deposit_charge": (I32, [P, ctypes.POINTER(FPParticles), P, I32, P]),
            "fem_pic_sort": (I32, [P, ctypes.POINTER(FPParticles), ctypes.POINTER(FPParticles), P]),
            "fem_pic_push_deposit_adams": (I32, [P, P, P, ctypes.POINTER(FPParticles), P, I64, D, I32, P, P, I32,
                                                 P]),
            "fem_pic_sort_columns": (I32, [P, ctypes.POINTER(FPParticles), ctypes.POINTER(FPParticles), P, P, I32,
                                           P]),
            "fem_pic_residuals": (I32, [P, P, P, P, P, P, P]),
            "fem_pic_status": (I32, [P, P]),
            "fem_pic_selftest_wait": (I32, [P, D, P]),
            "fem_pic_field_setup": (I32, [P, D, D, D]),
            "fem_pic_field_setup_bc": (I32, [P, D, D, D, I32]),
            "fem_pic_field_nnz": (I32, [P, P]),
            "fem_pic_field_matrix": (I32, [P, I32, P, P, P]),
            "fem_pic_field_solve": (I32, [P, I32, P, P, D, I32, I32, ctypes.POINTER(SolveInfo), P]),
            "fem_pic_field_step": (I32, [P, P, P, P, P, P, P, P, D, I32, I32, ctypes.POINTER(SolveInfo), P]),
            "fem_pic_field_initial": (I32, [P, P, P, D, I32, ctypes.POINTER(SolveInfo), P]),
            "fem_pic_mfem_create": (I32, [P, ctypes.POINTER(P)]),
            "fem_pic_mfem_destroy": (None, [P]),
            "fem_pic_mfem_face_mass": (I32, [P, P, P, P, P]),
            "fem_pic_mfem_step": (I32, [P, P, P, P, P, D, I32, I32, ctypes.POINTER(SolveInfo), P]),
            "fem_pic_wave_step": (I32, [P, P, P, P, P, P, P, D, I32, I32, ctypes.POINTER(SolveInfo), P]),
            "fem_pic_mfem_gauss_residual": (I32, [P, P, P, P, P]),
            "fem_pic_field_last_info": (I32, [P, ctypes.POINTER(SolveInfo), P]),
            "fem_pic_field_options": (I32, [P, I32, I32, D]),
            "fem_pic_field_poly": (I32, [P, I32, I32, D]),
            "fem_pic_whitney0_integrals": (I32, [P, P]),
            "fem_pic_learned_init": (I32, [P, ctypes.c_uint64, I32]),
            "fem_pic_learned_init_model": (I32, [P, ctypes.c_uint64, I32, I32]),
            "fem_pic_learned_build": (I32, [P, P]),
            "fem_pic_learned_delta": (I32, [P, P, P, P]),
            "fem_pic_learned_select": (I32, [P, I32]),
            "fem_pic_learned_mode": (I32, [P, I32, I32]),
            "fem_pic_learned_samples": (I32, [P, P]),
            "fem_pic_learned_train": (I32, [P, I32, I32, I32, D, ctypes.c_uint64, P, P]),
            "fem_pic_learned_eval": (I32, [P, I32, I32, P, P]),
            "fem_pic_learned_params": (I32, [P, P, P, P]),
            "fem_pic_learned_forward": (I32, [P, P, P, P, P]),
            "fem_pic_learned_gradient": (I32, [P, P, P, P, P]),
            "fem_pic_profile_enable": (I32, [P, I32]),
            "fem_pic_profile_read": (I32, [P, P, P, I32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
        return L


def _err(h) -> str:
    s = lib().fem_pic_last_error(h)
    return s.decode() if s else ""


def _check(st: int, h=None):
    if st != FP_OK:
        raise FemPicError(st, _err(h))


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return t.ctypes.data_as(ctypes.c_void_p)
    return ctypes.c_void_p(int(t))


def _need(t, dtype, numel=None, cuda=True, name="tensor"):
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if cuda and not t.is_cuda:
        raise ValueError(f"{name} must be on a CUDA device")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, got {t.numel()}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


@dataclass
class Species:
    """Device particle state of one species (SoA, torch-owned)."""
    cell: torch.Tensor   # int32 [n]
    off: torch.Tensor    # [3, n] float32 or float64: position minus the cell's vertex-0 position
    vel: torch.Tensor    # [3, n]
    q: float
    m: float
    w: float

    @property
    def n(self) -> int:
        return int(self.cell.numel())

    def abi(self) -> FPParticles:
        return FPParticles(self.n, self.cell.data_ptr(), self.off.data_ptr(), self.vel.data_ptr(),
                           float(self.q), float(self.m), float(self.w))

    def empty_like(self) -> "Species":
        return Species(torch.empty_like(self.cell), torch.empty_like(self.off), torch.empty_like(self.vel),
                       self.q, self.m, self.w)


def _csr_struct(m):
    if m is None:
        return None, None
    rp = np.ascontiguousarray(m[0], dtype=np.int32)
    col = np.ascontiguousarray(m[1], dtype=np.int32)
    val = np.ascontiguousarray(m[2], dtype=np.int8)
    s = FPCsr(rp.size - 1, int(m[3]), col.size, rp.ctypes.data, col.ctypes.data, val.ctypes.data)
    return s, (rp, col, val)


# ---------------------------------------------------------------- C ABI wrappers

def fem_pic_create(xyz, tets, D0=None, D1=None, D2=None, precision: int = FP_FP32):
    """Build the mesh handle.  D0/D1/D2: optional (row_ptr, col, val, n_cols) CSR to validate."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    tets = np.ascontiguousarray(tets, dtype=np.int32)
    mesh = FPMesh(xyz.shape[0], tets.shape[0], xyz.ctypes.data, tets.ctypes.data)
    keep = []
    cs = []
    for m in (D0, D1, D2):
        s, k = _csr_struct(m)
        keep.append(k)
        cs.append(ctypes.pointer(s) if s is not None else None)
    h = ctypes.c_void_p()
    st = lib().fem_pic_create(ctypes.byref(mesh), cs[0], cs[1], cs[2], int(precision), ctypes.byref(h))
    _check(st, None)
    return h


def fem_pic_destroy(h):
    lib().fem_pic_destroy(h)


def fem_pic_last_error(h) -> str:
    return _err(h)


def fem_pic_sizes(h) -> dict:
    s = np.zeros(5, dtype=np.int64)
    _check(lib().fem_pic_sizes(h, _ptr(s)), h)
    return dict(n_nodes=int(s[0]), n_edges=int(s[1]), n_faces=int(s[2]), n_tets=int(s[3]),
                precision=int(s[4]))


def fem_pic_incidence(h, which: int):
    sz = fem_pic_sizes(h)
    rows = (sz["n_edges"], sz["n_faces"], sz["n_tets"])[which]
    per = (2, 3, 4)[which]
    rp = np.empty(rows + 1, dtype=np.int32)
    col = np.empty(rows * per, dtype=np.int32)
    val = np.empty(rows * per, dtype=np.int8)
    _check(lib().fem_pic_incidence(h, which, _ptr(rp), _ptr(col), _ptr(val)), h)
    return rp, col, val


def fem_pic_topology(h) -> dict:
    nt = fem_pic_sizes(h)["n_tets"]
    out = dict(tet_nodes=np.empty((nt, 4), np.int32), tet_edges=np.empty((nt, 6), np.int32),
               tet_faces=np.empty((nt, 4), np.int32), tet_neigh=np.empty((nt, 4), np.int32))
    _check(lib().fem_pic_topology(h, _ptr(out["tet_nodes"]), _ptr(out["tet_edges"]),
                                  _ptr(out["tet_faces"]), _ptr(out["tet_neigh"])), h)
    return out


def fem_pic_project_uniform(h, E0, B0, e=None, b=None, stream=None):
    E0 = np.ascontiguousarray(E0, dtype=np.float64)
    B0 = np.ascontiguousarray(B0, dtype=np.float64)
    sz = fem_pic_sizes(h)
    if e is not None:
        _need(e, torch.float64, sz["n_edges"], name="e")
    if b is not None:
        _need(b, torch.float64, sz["n_faces"], name="b")
    _check(lib().fem_pic_project_uniform(h, _ptr(E0), _ptr(B0), _ptr(e), _ptr(b), _stream(stream)), h)


def _real(h):
    return torch.float32 if fem_pic_sizes(h)["precision"] == FP_FP32 else torch.float64


def _dep(h):
    """dtype of the current array dG."""
    return torch.float32 if int(lib().fem_pic_deposit_precision(h)) == FP_FP32 else torch.float64


def _chg(h):
    """dtype of the charge array Q."""
    return torch.float32 if int(lib().fem_pic_charge_precision(h)) == FP_FP32 else torch.float64


def fem_pic_set_deposit_precision(h, precision: int):
    """FP_FP32 or FP_FP64 deposit arrays (dG and Q) of an FP32 context (see the header)."""
    _check(lib().fem_pic_set_deposit_precision(h, int(precision)), h)


def fem_pic_deposit_precision(h) -> int:
    return int(lib().fem_pic_deposit_precision(h))


def fem_pic_set_charge_precision(h, precision: int):
    """FP_FP32 or FP_FP64 charge array Q alone (see the header)."""
    _check(lib().fem_pic_set_charge_precision(h, int(precision)), h)


def fem_pic_charge_precision(h) -> int:
    return int(lib().fem_pic_charge_precision(h))


def fem_pic_particles_from_global(h, cell, X, off, stream=None):
    n = cell.numel()
    _need(cell, torch.int32, n, name="cell")
    _need(X, torch.float64, 3 * n, name="X")
    _need(off, _real(h), 3 * n, name="off")
    _check(lib().fem_pic_particles_from_global(h, n, _ptr(cell), _ptr(X), _ptr(off), _stream(stream)), h)


def fem_pic_particles_to_global(h, cell, off, X, stream=None):
    n = cell.numel()
    _need(cell, torch.int32, n, name="cell")
    _need(off, _real(h), 3 * n, name="off")
    _need(X, torch.float64, 3 * n, name="X")
    _check(lib().fem_pic_particles_to_global(h, n, _ptr(cell), _ptr(off), _ptr(X), _stream(stream)), h)


def _check_species(h, sp: Species):
    n = sp.n
    _need(sp.cell, torch.int32, n, name="cell")
    _need(sp.off, _real(h), 3 * n, name="off")
    _need(sp.vel, _real(h), 3 * n, name="vel")


def fem_pic_push_deposit(h, e, b, sp: Species, dt: float, dG, Q, max_cross: int = 64, flags: int = 0,
                         stream=None):
    sz = fem_pic_sizes(h)
    _check_species(h, sp)
    _need(e, torch.float64, sz["n_edges"], name="e")
    _need(b, torch.float64, sz["n_faces"], name="b")
    _need(dG, _dep(h), sz["n_edges"], name="dG")
    _need(Q, _chg(h), sz["n_nodes"], name="Q")
    p = sp.abi()
    _check(lib().fem_pic_push_deposit(h, _ptr(e), _ptr(b), ctypes.byref(p), float(dt), int(max_cross),
                                      _ptr(dG), _ptr(Q), int(flags), _stream(stream)), h)


def fem_pic_push_deposit_adams(h, e, b, sp: Species, hist, step: int, dt: float, dG, Q, max_cross: int = 64,
                               flags: int = 0, stream=None):
    """Adams-Bashforth particle step; hist is the 18*n planar derivative history (see the header)."""
    sz = fem_pic_sizes(h)
    R = _real(h)
    _check_species(h, sp)
    _need(hist, R, 18 * sp.n, name="hist")
    _need(e, torch.float64, sz["n_edges"], name="e")
    _need(b, torch.float64, sz["n_faces"], name="b")
    _need(dG, R, sz["n_edges"], name="dG")
    _need(Q, R, sz["n_nodes"], name="Q")
    p = sp.abi()
    _check(lib().fem_pic_push_deposit_adams(h, _ptr(e), _ptr(b), ctypes.byref(p), _ptr(hist), int(step),
                                            float(dt), int(max_cross), _ptr(dG), _ptr(Q), int(flags),
                                            _stream(stream)), h)


def fem_pic_deposit_charge(h, sp: Species, Q, flags: int = 0, stream=None):
    _check_species(h, sp)
    _need(Q, _chg(h), fem_pic_sizes(h)["n_nodes"], name="Q")
    p = sp.abi()
    _check(lib().fem_pic_deposit_charge(h, ctypes.byref(p), _ptr(Q), int(flags), _stream(stream)), h)


def fem_pic_sort(h, src: Species, dst: Species, stream=None):
    _check_species(h, src)
    _check_species(h, dst)
    a, b = src.abi(), dst.abi()
    _check(lib().fem_pic_sort(h, ctypes.byref(a), ctypes.byref(b), _stream(stream)), h)


def fem_pic_sort_columns(h, src: Species, dst: Species, cols_src, cols_dst, ncols: int, stream=None):
    _check_species(h, src)
    _check_species(h, dst)
    R = _real(h)
    _need(cols_src, R, ncols * src.n, name="cols_src")
    _need(cols_dst, R, ncols * src.n, name="cols_dst")
    a, b = src.abi(), dst.abi()
    _check(lib().fem_pic_sort_columns(h, ctypes.byref(a), ctypes.byref(b), _ptr(cols_src), _ptr(cols_dst),
                                      int(ncols), _stream(stream)), h)


def fem_pic_residuals(h, dG, Q_new, Q_old, b, out, stream=None):
    _need(out, torch.float64, 6, name="out")
    _check(lib().fem_pic_residuals(h, _ptr(dG), _ptr(Q_new), _ptr(Q_old), _ptr(b), _ptr(out),
                                   _stream(stream)), h)


def fem_pic_status(h, stream=None) -> int:
    return int(lib().fem_pic_status(h, _stream(stream)))


def fem_pic_selftest_wait(h, limit_s: float = 1e-3, stream=None):
    """A bounded wait that runs out on the GPU (see the header); read the result with fem_pic_status."""
    _check(lib().fem_pic_selftest_wait(h, float(limit_s), _stream(stream)), h)


def fem_pic_field_setup(h, dt: float, eps: float = EPS0, mu: float = MU0, bc: int = None):
    """Field operators for time step dt; bc = FP_BC_PEC (default) or FP_BC_NEUMANN."""
    if bc is None:
        _check(lib().fem_pic_field_setup(h, float(dt), float(eps), float(mu)), h)
    else:
        _check(lib().fem_pic_field_setup_bc(h, float(dt), float(eps), float(mu), int(bc)), h)


def fem_pic_field_matrix(h, which: int):
    """Host CSR (row_ptr, col, val) of M (0), S (1), A (2) or L (3)."""
    nnz = np.zeros(2, dtype=np.int64)
    _check(lib().fem_pic_field_nnz(h, _ptr(nnz)), h)
    sz = fem_pic_sizes(h)
    rows = sz["n_nodes"] if which == 3 else sz["n_edges"]
    k = int(nnz[1] if which == 3 else nnz[0])
    rp = np.empty(rows + 1, np.int32)
    col = np.empty(k, np.int32)
    val = np.empty(k, np.float64)
    _check(lib().fem_pic_field_matrix(h, int(which), _ptr(rp), _ptr(col), _ptr(val)), h)
    return rp, col, val


def fem_pic_field_solve(h, system: int, rhs, x, tol: float = 1e-10, max_iter: int = 10000,
                        precond: int = FP_PC_JACOBI, info: bool = True, stream=None):
    _need(rhs, torch.float64, name="rhs")
    _need(x, torch.float64, rhs.numel(), name="x")
    inf = SolveInfo() if info else None
    st = lib().fem_pic_field_solve(h, int(system), _ptr(rhs), _ptr(x), float(tol), int(max_iter), int(precond),
                                   ctypes.byref(inf) if inf is not None else None, _stream(stream))
    if st not in (FP_OK, FP_ENOCONV):
        _check(st, h)
    return st, (inf.as_dict() if inf is not None else None)


def fem_pic_field_step(h, E_prev, E_cur, E_next, b, dG_half, dG_prev, Q_new, tol: float = 1e-10,
                       max_iter: int = 10000, precond: int = FP_PC_JACOBI, info: bool = True, stream=None):
    sz = fem_pic_sizes(h)
    for t, nm in ((E_prev, "E_prev"), (E_cur, "E_cur"), (E_next, "E_next")):
        _need(t, torch.float64, sz["n_edges"], name=nm)
    inf = (SolveInfo * 2)() if info else None
    st = lib().fem_pic_field_step(h, _ptr(E_prev), _ptr(E_cur), _ptr(E_next), _ptr(b), _ptr(dG_half),
                                  _ptr(dG_prev), _ptr(Q_new), float(tol), int(max_iter), int(precond),
                                  inf, _stream(stream))
    if st not in (FP_OK, FP_ENOCONV):
        _check(st, h)
    return st, ([inf[0].as_dict(), inf[1].as_dict()] if inf is not None else None)


def fem_pic_mfem_create(h):
    """Handle of the comparison systems (MFEM, unprojected wave equation) for h's field setup."""
    m = ctypes.c_void_p()
    _check(lib().fem_pic_mfem_create(h, ctypes.byref(m)), h)
    return m


def fem_pic_mfem_destroy(m):
    lib().fem_pic_mfem_destroy(m)


def fem_pic_mfem_face_mass(h, m):
    """Host CSR (row_ptr, col, val) of the face mass [*mu^-1] over all faces."""
    nnz = np.zeros(1, dtype=np.int64)
    _check(lib().fem_pic_mfem_face_mass(m, _ptr(nnz), None, None, None), h)
    nf = fem_pic_sizes(h)["n_faces"]
    rp = np.zeros(nf + 1, dtype=np.int32)
    col = np.zeros(int(nnz[0]), dtype=np.int32)
    val = np.zeros(int(nnz[0]), dtype=np.float64)
    _check(lib().fem_pic_mfem_face_mass(m, None, _ptr(rp), _ptr(col), _ptr(val)), h)
    return rp, col, val


def fem_pic_mfem_step(h, m, E_cur, E_next, b, dG_half, tol: float = 1e-10, max_iter: int = 10000,
                      precond: int = FP_PC_JACOBI, info: bool = True, stream=None):
    sz = fem_pic_sizes(h)
    for t, nm in ((E_cur, "E_cur"), (E_next, "E_next")):
        _need(t, torch.float64, sz["n_edges"], name=nm)
    _need(b, torch.float64, sz["n_faces"], name="b")
    inf = SolveInfo() if info else None
    st = lib().fem_pic_mfem_step(m, _ptr(E_cur), _ptr(E_next), _ptr(b), _ptr(dG_half), float(tol), int(max_iter),
                                 int(precond), ctypes.byref(inf) if inf is not None else None, _stream(stream))
    if st not in (FP_OK, FP_ENOCONV):
        _check(st, h)
    return st, (inf.as_dict() if inf is not None else None)


def fem_pic_wave_step(h, m, E_prev, E_cur, E_next, b, dG_half, dG_prev, tol: float = 1e-10, max_iter: int = 10000,
                      precond: int = FP_PC_JACOBI, info: bool = True, stream=None):
    sz = fem_pic_sizes(h)
    for t, nm in ((E_prev, "E_prev"), (E_cur, "E_cur"), (E_next, "E_next")):
        _need(t, torch.float64, sz["n_edges"], name=nm)
    if b is not None:
        _need(b, torch.float64, sz["n_faces"], name="b")
    inf = SolveInfo() if info else None
    st = lib().fem_pic_wave_step(m, _ptr(E_prev), _ptr(E_cur), _ptr(E_next), _ptr(b), _ptr(dG_half),
                                 _ptr(dG_prev), float(tol), int(max_iter), int(precond),
                                 ctypes.byref(inf) if inf is not None else None, _stream(stream))
    if st not in (FP_OK, FP_ENOCONV):
        _check(st, h)
    return st, (inf.as_dict() if inf is not None else None)


def fem_pic_mfem_gauss_residual(h, m, E, Q, out, stream=None):
    """out (device double[2]) <- max |D0^T [*eps] E + Q| over free nodes and its scale."""
    _need(out, torch.float64, 2, name="out")
    _check(lib().fem_pic_mfem_gauss_residual(m, _ptr(E), _ptr(Q), _ptr(out), _stream(stream)), h)


def fem_pic_field_initial(h, Q, E, tol: float = 1e-10, max_iter: int = 10000, info: bool = True, stream=None):
    inf = SolveInfo() if info else None
    st = lib().fem_pic_field_initial(h, _ptr(Q), _ptr(E), float(tol), int(max_iter),
                                     ctypes.byref(inf) if inf is not None else None, _stream(stream))
    if st not in (FP_OK, FP_ENOCONV):
        _check(st, h)
    return st, (inf.as_dict() if inf is not None else None)


def fem_pic_learned_select(h, system: int):
    """Choose the system (FP_SYS_NEWMARK or FP_SYS_GAUSS) the fem_pic_learned_* calls address."""
    _check(lib().fem_pic_learned_select(h, int(system)), h)


def fem_pic_learned_init(h, seed: int = 0, sample_capacity: int = 64):
    _check(lib().fem_pic_learned_init(h, int(seed), int(sample_capacity)), h)


def fem_pic_learned_init_model(h, seed: int = 0, sample_capacity: int = 64, model: int = FP_LEARNED_PRECOND):
    _check(lib().fem_pic_learned_init_model(h, int(seed), int(sample_capacity), int(model)), h)


def fem_pic_learned_build(h, stream=None):
    _check(lib().fem_pic_learned_build(h, _stream(stream)), h)


def fem_pic_learned_delta(h, nnz: int, n: int, device="cuda", stream=None):
    """Delta~ per CSR entry of the selected system's operator and the network's static input."""
    d = torch.empty(int(nnz), dtype=torch.float32, device=device)
    x = torch.empty(int(n), dtype=torch.float32, device=device)
    _check(lib().fem_pic_learned_delta(h, _ptr(d), _ptr(x), _stream(stream)), h)
    return d, x


def fem_pic_learned_mode(h, collect: bool, active: bool):
    _check(lib().fem_pic_learned_mode(h, 1 if collect else 0, 1 if active else 0), h)


def fem_pic_learned_samples(h) -> int:
    c = ctypes.c_int(0)
    _check(lib().fem_pic_learned_samples(h, ctypes.byref(c)), h)
    return int(c.value)


def fem_pic_learned_train(h, first: int, count: int, epochs: int, lr: float = 1e-3, seed: int = 0, stream=None):
    loss = np.zeros(max(1, epochs), dtype=np.float64)
    _check(lib().fem_pic_learned_train(h, int(first), int(count), int(epochs), float(lr), int(seed), _ptr(loss),
                                       _stream(stream)), h)
    return loss[:epochs]


def fem_pic_learned_eval(h, first: int, count: int, stream=None) -> np.ndarray:
    out = np.zeros(count, dtype=np.float64)
    _check(lib().fem_pic_learned_eval(h, int(first), int(count), _ptr(out), _stream(stream)), h)
    return out


def fem_pic_learned_params(h, set_values=None) -> np.ndarray:
    n = ctypes.c_int64(0)
    _check(lib().fem_pic_learned_params(h, None, None, ctypes.byref(n)), h)
    out = np.zeros(int(n.value), dtype=np.float32)
    sv = None if set_values is None else np.ascontiguousarray(set_values, dtype=np.float32)
    _check(lib().fem_pic_learned_params(h, _ptr(out), _ptr(sv), None), h)
    return out


def fem_pic_learned_forward(h, r, stream=None):
    _need(r, torch.float64, name="r")
    ct = torch.empty(r.numel(), dtype=torch.float32, device=r.device)
    rt = torch.empty_like(ct)
    _check(lib().fem_pic_learned_forward(h, _ptr(r), _ptr(ct), _ptr(rt), _stream(stream)), h)
    return ct, rt


def fem_pic_learned_gradient(h, r, stream=None):
    _need(r, torch.float32, name="r")
    n = ctypes.c_int64(0)
    _check(lib().fem_pic_learned_params(h, None, None, ctypes.byref(n)), h)
    g = np.zeros(int(n.value), dtype=np.float32)
    loss = ctypes.c_double(0.0)
    _check(lib().fem_pic_learned_gradient(h, _ptr(r), _ptr(g), ctypes.byref(loss), _stream(stream)), h)
    return g, float(loss.value)


def fem_pic_field_last_info(h, stream=None):
    inf = (SolveInfo * 2)()
    _check(lib().fem_pic_field_last_info(h, inf, _stream(stream)), h)
    return [inf[0].as_dict(), inf[1].as_dict()]


def fem_pic_whitney0_integrals(h) -> np.ndarray:
    a = np.empty(fem_pic_sizes(h)["n_nodes"], dtype=np.float64)
    _check(lib().fem_pic_whitney0_integrals(h, _ptr(a)), h)
    return a


PHASES = ("prep", "push_fast", "walk", "push_fp64", "charge", "sort", "residuals", "field_other",
          "cg_newmark", "cg_gauss", "learned", "adams_push", "adams_walk")


def fem_pic_field_options(h, newmark_solver: int = -1, gauss_solver: int = -1, inner_tol: float = 1e-5):
    _check(lib().fem_pic_field_options(h, int(newmark_solver), int(gauss_solver), float(inner_tol)), h)


def fem_pic_field_poly(h, system: int, degree: int, ratio: float = 30.0):
    """Chebyshev degree of the inner solves' preconditioner for one system (1 = Jacobi)."""
    _check(lib().fem_pic_field_poly(h, int(system), int(degree), float(ratio)), h)


def fem_pic_profile_enable(h, on: bool = True):
    _check(lib().fem_pic_profile_enable(h, 1 if on else 0), h)


def fem_pic_profile_read(h, reset: bool = True) -> dict:
    ms = np.zeros(16, dtype=np.float64)
    n = np.zeros(16, dtype=np.int64)
    _check(lib().fem_pic_profile_read(h, _ptr(ms), _ptr(n), 1 if reset else 0), h)
    return {name: (float(ms[i]), int(n[i])) for i, name in enumerate(PHASES) if n[i] > 0}


# ---------------------------------------------------------------- convenience layer

class FemPic:
    """Owns one library handle; methods forward to the C ABI wrappers above."""

    def __init__(self, xyz, tets, precision: int = FP_FP32, D0=None, D1=None, D2=None):
        self.h = fem_pic_create(xyz, tets, D0, D1, D2, precision)
        self.sizes = fem_pic_sizes(self.h)
        self.precision = precision
        self.real = torch.float32 if precision == FP_FP32 else torch.float64

    def close(self):
        if self.h is not None:
            fem_pic_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_nodes(self):
        return self.sizes["n_nodes"]

    @property
    def n_edges(self):
        return self.sizes["n_edges"]

    @property
    def n_faces(self):
        return self.sizes["n_faces"]

    @property
    def n_tets(self):
        return self.sizes["n_tets"]

    def species(self, cell, X, V, q, m, w, device="cuda") -> Species:
        """Upload one species from host arrays (cell [n], global X [n,3], V [n,3])."""
        n = int(np.asarray(cell).shape[0])
        c = torch.as_tensor(np.ascontiguousarray(cell, dtype=np.int32)).to(device)
        Xd = torch.as_tensor(np.ascontiguousarray(X, dtype=np.float64).reshape(n, 3)).to(device)
        off = torch.empty((3, n), dtype=self.real, device=device)
        fem_pic_particles_from_global(self.h, c, Xd, off)
        vel = torch.as_tensor(np.ascontiguousarray(np.asarray(V, dtype=np.float64).reshape(n, 3).T)).to(
            device=device, dtype=self.real).contiguous()
        return Species(c, off, vel, q, m, w)

    def positions(self, sp: Species) -> torch.Tensor:
        X = torch.empty((sp.n, 3), dtype=torch.float64, device=sp.cell.device)
        fem_pic_particles_to_global(self.h, sp.cell, sp.off, X)
        return X

    def fields_uniform(self, E0, B0, device="cuda"):
        e = torch.empty(self.n_edges, dtype=torch.float64, device=device)
        b = torch.empty(self.n_faces, dtype=torch.float64, device=device)
        fem_pic_project_uniform(self.h, E0, B0, e, b)
        return e, b

    def push_deposit(self, e, b, sp, dt, dG, Q, max_cross=64, flags=0, stream=None):
        fem_pic_push_deposit(self.h, e, b, sp, dt, dG, Q, max_cross, flags, stream)

    def push_deposit_adams(self, e, b, sp, hist, step, dt, dG, Q, max_cross=64, flags=0, stream=None):
        fem_pic_push_deposit_adams(self.h, e, b, sp, hist, step, dt, dG, Q, max_cross, flags, stream)

    def sort_columns(self, src, dst, cols_src, cols_dst, ncols, stream=None):
        fem_pic_sort_columns(self.h, src, dst, cols_src, cols_dst, ncols, stream)

    def deposit_charge(self, sp, Q, flags=0, stream=None):
        fem_pic_deposit_charge(self.h, sp, Q, flags, stream)

    def set_deposit_precision(self, precision: int):
        fem_pic_set_deposit_precision(self.h, precision)

    @property
    def deposit_dtype(self):
        """dtype of dG (and of Q unless set_charge_precision changed it)."""
        return _dep(self.h)

    def set_charge_precision(self, precision: int):
        fem_pic_set_charge_precision(self.h, precision)

    @property
    def charge_dtype(self):
        return _chg(self.h)

    def sort(self, src, dst, stream=None):
        fem_pic_sort(self.h, src, dst, stream)

    def residuals(self, dG, Q_new, Q_old, b, out, stream=None):
        fem_pic_residuals(self.h, dG, Q_new, Q_old, b, out, stream)

    def status(self, stream=None) -> int:
        return fem_pic_status(self.h, stream)
