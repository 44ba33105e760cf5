"""The allocation-free push entry point gives the same step as the allocating one.

fem_pic_push_deposit grows a queue with cudaMalloc the first time a larger particle
set needs it.  Callers that must not allocate device memory while they run (a fixed
memory budget set at start-up, an allocator that forbids new device allocations,
a framework that only lends out buffers it already owns) call
fem_pic_push_deposit_static instead: its queue is a fixed array inside the library.
This file is collected last on purpose, so a run that stops at the first failure has
already run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_2103_06737_gb300 import inputs as I

pytestmark = pytest.mark.gpu

STATIC_MAX = 1 << 22


def _entry():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2103_06737_gb300 import build
    build.build()
    import paper_2103_06737_gb300.fem_pic as F
    f = F.lib().fem_pic_push_deposit_static
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(F.FPParticles),
                  ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                  ctypes.c_void_p]
    return F, f


# 50,001 particles: the grid-stride kernel (n not a multiple of 4); 50,000: the staged
# pipeline, which both entry points pick for aligned state; and the staged pipeline with the
# charge-change deposit into a double Q carried over both calls
@pytest.mark.parametrize("npart,change", [(50_001, False), (50_000, False), (50_000, True)])
def test_static_push_matches_allocating_push_on_two_calls(npart, change):
    F, push_static = _entry()
    m = I.cube_mesh(8, 1.0, 0.1, seed=1)
    sp = I.uniform_species(m, npart, 3, 0.15, -1.0, 1.0, 0.7)
    lib = F.FemPic(m.xyz, m.tets, F.FP_FP32)
    if change:
        lib.set_charge_precision(F.FP_FP64)
    RQ = lib.charge_dtype
    flags = F.FP_CHARGE_CHANGE if change else 0
    rng = np.random.default_rng(7)
    e = torch.as_tensor(rng.uniform(-0.2, 0.2, lib.n_edges), device="cuda")
    b = torch.as_tensor(rng.uniform(-0.5, 0.5, lib.n_faces), device="cuda")
    ref = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    new = lib.species(sp.cell, sp.X, sp.V, sp.q, sp.m, sp.w)
    stream = torch.cuda.current_stream().cuda_stream
    if change:      # both start from the charge of the start positions and carry it
        Q_ref = torch.zeros(lib.n_nodes, dtype=RQ, device="cuda")
        lib.deposit_charge(ref, Q_ref)
        Q_new = Q_ref.clone()
    for call in range(2):
        dG_ref = torch.empty(lib.n_edges, dtype=torch.float32, device="cuda")
        if not change:
            Q_ref = torch.empty(lib.n_nodes, dtype=RQ, device="cuda")
        lib.push_deposit(e, b, ref, 1.0, dG_ref, Q_ref, flags=flags)
        dG_new = torch.full((lib.n_edges,), 7.0, dtype=torch.float32, device="cuda")
        if not change:
            Q_new = torch.full((lib.n_nodes,), 7.0, dtype=RQ, device="cuda")
        pa = new.abi()
        st = push_static(lib.h, ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(b.data_ptr()), ctypes.byref(pa),
                         1.0, 64, ctypes.c_void_p(dG_new.data_ptr()), ctypes.c_void_p(Q_new.data_ptr()), flags,
                         ctypes.c_void_p(stream))
        assert st == F.FP_OK, F.fem_pic_last_error(lib.h)
        assert lib.status() == F.FP_OK
        # per-particle results do not depend on atomic order: identical
        assert torch.equal(ref.cell, new.cell), call
        assert torch.equal(ref.off, new.off), call
        assert torch.equal(ref.vel, new.vel), call
        # deposits: FP32 tolerance of the parity tests (atomic order differs)
        for a, c in ((dG_ref, dG_new), (Q_ref, Q_new)):
            a = a.double().cpu().numpy()
            c = c.double().cpu().numpy()
            assert np.abs(a - c).max() <= 1e-5 * np.abs(a).max(), call
    assert int((ref.cell < 0).sum()) > 0          # some walks ended at a wall: the queue was used


def test_static_push_rejects_more_particles_than_its_array():
    F, push_static = _entry()
    m = I.cube_mesh(2, 1.0, 0.0)
    lib = F.FemPic(m.xyz, m.tets, F.FP_FP32)
    n = STATIC_MAX + 1
    # arrays of the full length, every particle already absorbed (cell -1): should the size
    # check ever let the call through, the kernels skip every particle and the assertion
    # below fails instead of any access leaving the arrays
    d = F.Species(torch.full((n,), -1, dtype=torch.int32, device="cuda"),
                  torch.zeros((3, n), dtype=torch.float32, device="cuda"),
                  torch.zeros((3, n), dtype=torch.float32, device="cuda"), -1.0, 1.0, 1.0)
    e = torch.zeros(lib.n_edges, dtype=torch.float64, device="cuda")
    b = torch.zeros(lib.n_faces, dtype=torch.float64, device="cuda")
    dG = torch.zeros(lib.n_edges, dtype=torch.float32, device="cuda")
    Q = torch.zeros(lib.n_nodes, dtype=torch.float32, device="cuda")
    pa = d.abi()
    assert pa.n == STATIC_MAX + 1                   # rejected before anything is launched
    st = push_static(lib.h, ctypes.c_void_p(e.data_ptr()), ctypes.c_void_p(b.data_ptr()), ctypes.byref(pa), 1e-3,
                     64, ctypes.c_void_p(dG.data_ptr()), ctypes.c_void_p(Q.data_ptr()), 0, None)
    assert st == F.FP_EINVAL
    assert "exceed" in F.fem_pic_last_error(lib.h)
