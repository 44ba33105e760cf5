"""The learned preconditioner (network model FP_LEARNED_PRECOND): the correction Delta~ and
the loss gradient against a plain PyTorch CPU reference of the same network (BF16 rounding
emulated at the same points), training on residuals the method produces, learned
preconditioned solves and field steps reaching the same 1e-10 tolerance and the same
fields as plain Jacobi-CG with fewer iterations, and the fallback to Jacobi when the learned
operator is not positive.  The systems are the Newmark edge system and the Gauss-law node
Laplacian of Sec. IV.B (Eq. reducedWaveEqn, discreteGauss); the paper gives no solver, so
plain Jacobi-CG at the same tolerance is the reference.
"""
import numpy as np
import pytest
import torch

from paper_2103_06737_gb300 import inputs as I

pytestmark = pytest.mark.gpu

F = pytest.importorskip("paper_2103_06737_gb300.fem_pic")

H, K, NL = 64, 128, 3


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2103_06737_gb300 import build
    build.build()


def _bf(x):
    return x.to(torch.bfloat16).to(torch.float32)


def _unpack(P):
    P = torch.as_tensor(P, dtype=torch.float32)
    we, be = P[0:64], P[64:128]
    W, b = [], []
    o = 128
    for _ in range(NL):
        W.append(P[o:o + K * H].reshape(K, H))
        b.append(P[o + K * H:o + K * H + H])
        o += K * H + H
    w, b0 = P[o:o + H], P[o + H]
    v, d0 = P[o + H + 1:o + 2 * H + 1], P[o + 2 * H + 1]
    return we, be, W, b, w, b0, v, d0


def _setup(n_hex=5, system=F.FP_SYS_NEWMARK):
    m = I.cube_mesh(n_hex, 1.0, 0.1, seed=1)
    dt = 0.2 * I.gyro_period(0.1)
    lib = F.FemPic(m.xyz, m.tets, F.FP_FP64)
    F.fem_pic_field_setup(lib.h, dt)
    F.fem_pic_learned_select(lib.h, system)
    rp, col, val = F.fem_pic_field_matrix(lib.h, 2 if system == F.FP_SYS_NEWMARK else 3)
    n = len(rp) - 1
    rows = np.repeat(np.arange(n), np.diff(rp))
    d = val[rp[:-1] + np.array([np.nonzero(col[rp[i]:rp[i + 1]] == i)[0][0] for i in range(n)])]
    dis = 1.0 / np.sqrt(d)
    at = (val * dis[rows] * dis[col]).astype(np.float32)
    fixed = np.array([(rp[i + 1] - rp[i] == 1) and val[rp[i]] == 1.0 for i in range(n)])
    return m, lib, dt, dict(rp=rp, col=col, rows=rows, at=torch.as_tensor(at), dis=dis, fixed=fixed, n=n)


def _dense(S, vals):
    A = torch.zeros((S["n"], S["n"]), dtype=torch.float32)
    A[torch.as_tensor(S["rows"]), torch.as_tensor(S["col"])] = vals
    return A


def reference(params, S, r=None):
    """Delta~ per CSR entry, and for a residual r the loss ||A~ (r~ + Delta~ r~) - r~||^2 / n_free."""
    we, be, W, b, w, b0, v, d0 = params
    fixed = torch.as_tensor(S["fixed"])
    free = ~fixed
    Atil = _dense(S, S["at"])
    xin = torch.where(fixed, torch.zeros(S["n"]), Atil.sum(1))
    xin = xin / torch.sqrt((xin[free] ** 2).sum() / free.sum())
    h = _bf(torch.relu(xin[:, None] * we[None, :] + be[None, :]))
    for l in range(NL):
        m = _bf(Atil @ h)
        h = _bf(torch.relu(torch.cat([h, m], 1) @ _bf(W[l]) + b[l]))
    rows = torch.as_tensor(S["rows"])
    cols = torch.as_tensor(S["col"]).long()
    diag = rows == cols
    pair = (h[rows] * h[cols] * w[None, :]).sum(1)
    dsq = ((h ** 2) * v[None, :]).sum(1)
    delta = torch.where(diag, d0 + dsq[rows], S["at"] * (b0 + pair))
    delta = torch.where(fixed[rows], torch.zeros_like(delta), delta)
    if r is None:
        return delta, xin, None
    x = torch.where(fixed, torch.zeros(S["n"]), torch.as_tensor(r, dtype=torch.float32) *
                    torch.as_tensor(S["dis"], dtype=torch.float32))
    rt = x / torch.sqrt((x[free] ** 2).sum() / free.sum())
    u = rt + _dense(S, delta) @ rt
    e = torch.where(fixed, torch.zeros(S["n"]), Atil @ u - rt)
    return delta, xin, (e ** 2).sum() / free.sum()


@pytest.mark.parametrize("system", [F.FP_SYS_NEWMARK, F.FP_SYS_GAUSS])
def test_delta_and_gradient_match_reference(system):
    m, lib, dt, S = _setup(n_hex=5 if system == F.FP_SYS_NEWMARK else 8, system=system)
    F.fem_pic_learned_init_model(lib.h, seed=3, sample_capacity=2, model=F.FP_LEARNED_PRECOND)
    P = F.fem_pic_learned_params(lib.h)
    # move the head away from its near-zero start so every term is exercised
    P = P.copy()
    rng = np.random.default_rng(1)
    o = 128 + NL * (K * H + H)
    P[o:o + H] = rng.normal(0, 0.05, H)
    P[o + H] = 0.3
    P[o + H + 1:o + 2 * H + 1] = rng.normal(0, 0.05, H)
    P[o + 2 * H + 1] = -0.2
    F.fem_pic_learned_params(lib.h, P)
    nnz = len(S["col"])
    d_gpu, x_gpu = F.fem_pic_learned_delta(lib.h, nnz, S["n"])
    leaves = list(_unpack(P))
    flat = [leaves[0], leaves[1]] + leaves[2] + leaves[3] + leaves[4:]
    for t in flat:
        t.requires_grad_(True)
    r = rng.normal(0, 1e-12, S["n"])
    r[S["fixed"]] = 0.0
    delta, xin, loss = reference((leaves[0], leaves[1], leaves[2], leaves[3], *leaves[4:]), S, r)
    assert torch.allclose(x_gpu.cpu(), xin.detach(), rtol=1e-5, atol=1e-6)
    err = (d_gpu.cpu() - delta.detach()).abs().max() / delta.detach().abs().max()
    assert err < 2e-2, float(err)
    loss.backward()
    we, be, W, b, w, b0, v, d0 = leaves
    g_ref = torch.cat([we.grad, be.grad] + sum([[W[l].grad.reshape(-1), b[l].grad] for l in range(NL)], []) +
                      [w.grad, b0.grad.reshape(1), v.grad, d0.grad.reshape(1)]).numpy()
    g_gpu, loss_gpu = F.fem_pic_learned_gradient(lib.h, torch.as_tensor(r, dtype=torch.float32, device="cuda"))
    assert g_gpu.shape == g_ref.shape
    assert abs(loss_gpu - loss.item()) <= 2e-2 * loss.item()
    rel = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    assert rel < 5e-2, rel
    cos = (g_gpu @ g_ref) / (np.linalg.norm(g_gpu) * np.linalg.norm(g_ref))
    assert cos > 0.998, cos
    assert np.array_equal(F.fem_pic_learned_params(lib.h), P)   # the gradient call changes nothing
    lib.close()


def _run_steps(lib, nsteps, precond, seed=5):
    """Field steps driven by a seeded random current that respects continuity."""
    n_e, n_n = lib.n_edges, lib.n_nodes
    rng = np.random.default_rng(seed)
    rp, col, val = F.fem_pic_incidence(lib.h, 0)
    D0 = np.zeros((n_e, n_n))
    D0[np.repeat(np.arange(n_e), 2), col] = val
    Q = torch.zeros(n_n, dtype=torch.float64, device="cuda")
    E = [torch.zeros(n_e, dtype=torch.float64, device="cuda") for _ in range(3)]
    b = torch.zeros(lib.n_faces, dtype=torch.float64, device="cuda")
    dGp = torch.zeros(n_e, dtype=torch.float64, device="cuda")
    infos = []
    base = rng.normal(0, 1e-13, n_e)
    for k in range(nsteps):
        dG = base * np.cos(0.3 * k) + rng.normal(0, 2e-14, n_e)
        Q += torch.as_tensor(D0.T @ dG, device="cuda")
        dGt = torch.as_tensor(dG, device="cuda")
        st, info = F.fem_pic_field_step(lib.h, E[0], E[1], E[2], b, dGt, dGp, Q, tol=1e-10, precond=precond)
        assert st == F.FP_OK, info
        infos.append(info)
        E = [E[1], E[2], E[0]]
        dGp = dGt
    return E[1], infos


@pytest.mark.parametrize("system", [F.FP_SYS_NEWMARK, F.FP_SYS_GAUSS])
def test_training_and_learned_solves_beat_jacobi_iterations(system):
    m, lib, dt, S = _setup(n_hex=8, system=system)
    bit = F.FP_PC_LEARNED if system == F.FP_SYS_NEWMARK else F.FP_PC_LEARNED_GAUSS
    F.fem_pic_learned_init_model(lib.h, seed=1, sample_capacity=40, model=F.FP_LEARNED_PRECOND)
    F.fem_pic_learned_mode(lib.h, collect=True, active=False)
    E_plain, info_plain = _run_steps(lib, 40, F.FP_PC_JACOBI)
    assert F.fem_pic_learned_samples(lib.h) == 40
    before = F.fem_pic_learned_eval(lib.h, 32, 8)
    loss = F.fem_pic_learned_train(lib.h, 0, 32, epochs=30, lr=2e-3, seed=0)
    after = F.fem_pic_learned_eval(lib.h, 32, 8)
    assert loss[-1] < loss[0]
    assert after.mean() < 0.9 * before.mean()
    F.fem_pic_learned_mode(lib.h, collect=False, active=False)
    F.fem_pic_learned_build(lib.h)
    E_learn, info_learn = _run_steps(lib, 40, bit)
    k = 0 if system == F.FP_SYS_NEWMARK else 1
    assert all(i[k]["precond"] == F.FP_PC_LEARNED and i[k]["fell_back"] == 0 for i in info_learn)
    assert all(i[0]["rel_res"] <= 1e-10 and i[1]["rel_res"] <= 1e-10 for i in info_learn)
    err = (E_learn - E_plain).abs().max() / E_plain.abs().max()
    assert float(err) < 1e-7
    it_plain = np.mean([i[k]["iters"] for i in info_plain])
    it_learn = np.mean([i[k]["iters"] for i in info_learn])
    assert it_learn < 0.8 * it_plain, (it_learn, it_plain)
    # a direct solve of one system with the learned preconditioner: same solution
    n = S["n"]
    rhs = torch.as_tensor(np.where(S["fixed"], 0.0, np.random.default_rng(4).normal(0, 1, n)), device="cuda")
    x0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    x1 = torch.zeros_like(x0)
    st0, i0 = F.fem_pic_field_solve(lib.h, system, rhs, x0, tol=1e-10, precond=F.FP_PC_JACOBI)
    st1, i1 = F.fem_pic_field_solve(lib.h, system, rhs, x1, tol=1e-10, precond=F.FP_PC_LEARNED)
    assert st0 == F.FP_OK and st1 == F.FP_OK and i1["precond"] == F.FP_PC_LEARNED and i1["fell_back"] == 0
    assert float((x1 - x0).abs().max() / x0.abs().max()) < 1e-8
    assert i1["iters"] < i0["iters"]
    lib.close()


def test_indefinite_learned_operator_falls_back_to_jacobi():
    m, lib, dt, S = _setup(n_hex=6)
    F.fem_pic_learned_init_model(lib.h, seed=2, sample_capacity=2, model=F.FP_LEARNED_PRECOND)
    P = F.fem_pic_learned_params(lib.h).copy()
    o = 128 + NL * (K * H + H)
    P[o + 2 * H + 1] = -3.0          # Delta~_ii = -3: z = -2 D^-1 r, r.z < 0
    F.fem_pic_learned_params(lib.h, P)
    F.fem_pic_learned_build(lib.h)
    n = S["n"]
    rhs = torch.as_tensor(np.where(S["fixed"], 0.0, np.random.default_rng(6).normal(0, 1, n)), device="cuda")
    x0 = torch.zeros(n, dtype=torch.float64, device="cuda")
    x1 = torch.zeros_like(x0)
    F.fem_pic_field_solve(lib.h, F.FP_SYS_NEWMARK, rhs, x0, tol=1e-10, precond=F.FP_PC_JACOBI)
    st, info = F.fem_pic_field_solve(lib.h, F.FP_SYS_NEWMARK, rhs, x1, tol=1e-10, precond=F.FP_PC_LEARNED)
    assert st == F.FP_OK and info["fell_back"] == 1 and info["rel_res"] <= 1e-10
    assert float((x1 - x0).abs().max() / x0.abs().max()) < 1e-8
    # a network without a build is refused
    F.fem_pic_learned_init_model(lib.h, seed=2, sample_capacity=2, model=F.FP_LEARNED_PRECOND)
    with pytest.raises(F.FemPicError):
        F.fem_pic_field_solve(lib.h, F.FP_SYS_NEWMARK, rhs, x1, tol=1e-10, precond=F.FP_PC_LEARNED)
    lib.close()
