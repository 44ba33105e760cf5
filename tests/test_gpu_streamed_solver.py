"""The mixed solver on operators too large for shared memory.

At 96^3 x 6 tets (6.3M edges, 0.9M nodes) neither FP32 operator fits in shared memory, so the
inner solves stream them from HBM (with the 16-bit column encoding when the library is built
with FP_COL16=1).  Both systems of Sec. IV.B (Eq. reducedWaveEqn, discreteGauss) are solved for
seeded right-hand sides to 1e-10 with the Jacobi and with the learned preconditioner (a head
set to a mild symmetric correction of Jacobi, applied on the same streamed pattern).  The FP64
residual of each solution is then formed on the CPU with the library's own operators (pinned
to the oracle's by test_gpu_fields.py::test_operators_match_oracle): a wrongly read column would leave the inner solves unable to reduce the true residual.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import torch

from paper_2103_06737_gb300 import inputs as I

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_2103_06737_gb300.fem_pic")

H = 64   # features per layer of the learned network


@pytest.fixture(scope="module")
def big():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2103_06737_gb300 import build
    build.build()
    m = I.cube_mesh(96, 1.0, 0.1, seed=1)
    lib = F.FemPic(m.xyz, m.tets, F.FP_FP32)
    F.fem_pic_field_setup(lib.h, 0.2 * I.gyro_period(0.2))
    yield lib
    lib.close()


@pytest.mark.parametrize("system", [F.FP_SYS_NEWMARK, F.FP_SYS_GAUSS])
def test_streamed_solves_reach_tolerance(big, system):
    lib = big
    rp, col, val = F.fem_pic_field_matrix(lib.h, 2 if system == F.FP_SYS_NEWMARK else 3)
    n = len(rp) - 1
    A = sp.csr_matrix((val, col, rp), shape=(n, n))
    fixed = (np.diff(rp) == 1) & (val[rp[:-1]] == 1.0)    # PEC rows: the identity
    rng = np.random.default_rng(5 + system)
    rhs = rng.uniform(-1.0, 1.0, n)
    rhs[fixed] = 0.0
    rhs_d = torch.as_tensor(rhs, device="cuda")
    F.fem_pic_learned_select(lib.h, system)
    F.fem_pic_learned_init_model(lib.h, seed=4, sample_capacity=1, model=F.FP_LEARNED_PRECOND)
    # a head that gives Delta~ = -0.1 A~ off the diagonal and 0 on it: z = D^-1/2 (1.1 I - 0.1 A~)
    # D^-1/2 r, positive definite (the spectrum of A~ lies below 11), a mild Neumann-series
    # correction of Jacobi, so the learned path runs every iteration without falling back
    P = F.fem_pic_learned_params(lib.h)
    P[-(2 * H + 2):] = 0.0      # head: w[H], b0, v[H], d0
    P[-(H + 2)] = -0.1          # b0
    F.fem_pic_learned_params(lib.h, P)
    F.fem_pic_learned_build(lib.h)
    its = {}
    for pc in (F.FP_PC_JACOBI, F.FP_PC_LEARNED):
        x = torch.zeros(n, dtype=torch.float64, device="cuda")
        st, info = F.fem_pic_field_solve(lib.h, system, rhs_d, x, tol=1e-10, precond=pc)
        assert st == F.FP_OK and info["rel_res"] <= 1e-10, (pc, info)
        r = rhs - A @ x.cpu().numpy()
        assert np.linalg.norm(r) <= 2e-10 * np.linalg.norm(rhs), pc
        its[pc] = info
    assert its[F.FP_PC_LEARNED]["precond"] == F.FP_PC_LEARNED and its[F.FP_PC_LEARNED]["fell_back"] == 0
    assert its[F.FP_PC_LEARNED]["iters"] <= its[F.FP_PC_JACOBI]["iters"]
    assert lib.status() == F.FP_OK
