"""The learned corrections (Newmark edge system and Gauss-law node system): forward pass and
gradients against a plain PyTorch CPU reference of the same network (BF16 rounding emulated
at the same points), training on residuals the method produces, and the fallback-guarded
field step matching plain CG.
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


def _unpack(P):
    P = torch.as_tensor(P, dtype=torch.float32)
    we, be = P[0:64], P[64:128]
    W, b = [], []
    o = 128
    for _ in range(NL):
        W.append(P[o:o + K * H].reshape(K, H))
        b.append(P[o + K * H:o + K * H + H])
        o += K * H + H
    wh, bh = P[o:o + H], P[o + H]
    return we, be, W, b, wh, bh


def _bf(x):
    return x.to(torch.bfloat16).to(torch.float32)


def forward_loss(params, Atil, dis, fixed, r):
    we, be, W, b, wh, bh = params
    free = ~fixed
    x = torch.where(fixed, torch.zeros_like(r), r * dis)
    s = torch.sqrt((x[free] ** 2).sum() / free.sum())
    rt = x / s
    h = _bf(torch.relu(rt[:, None] * we[None, :] + be[None, :]))
    for l in range(NL):
        m = _bf(Atil @ h)
        h = _bf(torch.relu(torch.cat([h, m], 1) @ _bf(W[l]) + b[l]))
    ct = torch.where(fixed, torch.zeros_like(rt), rt + h @ wh + bh)
    e = torch.where(fixed, torch.zeros_like(rt), Atil @ ct - rt)
    loss = (e ** 2).sum() / free.sum()
    return ct, rt, loss


def _setup(n_hex=5, steps=10, seed=1, system=F.FP_SYS_NEWMARK):
    m = I.cube_mesh(n_hex, 1.0, 0.1, seed=1)
    dt = 0.2 * I.gyro_period(0.1)
    lib = F.FemPic(m.xyz, m.tets, F.FP_FP64)
    F.fem_pic_field_setup(lib.h, dt)
    F.fem_pic_learned_select(lib.h, system)
    rp, col, val = F.fem_pic_field_matrix(lib.h, 2 if system == F.FP_SYS_NEWMARK else 3)
    n = lib.n_edges if system == F.FP_SYS_NEWMARK else lib.n_nodes
    A = np.zeros((n, n))
    for i in range(n):
        A[i, col[rp[i]:rp[i + 1]]] = val[rp[i]:rp[i + 1]]
    d = np.diag(A)
    dis = 1.0 / np.sqrt(d)
    Atil = (A * dis[:, None] * dis[None, :]).astype(np.float32)
    fixed = np.array([(rp[i + 1] - rp[i] == 1) and A[i, i] == 1.0 for i in range(n)])
    return m, lib, torch.as_tensor(Atil), torch.as_tensor(dis.astype(np.float32)), torch.as_tensor(fixed), dt


@pytest.mark.parametrize("system", [F.FP_SYS_NEWMARK, F.FP_SYS_GAUSS])
def test_forward_and_gradient_match_reference(system):
    m, lib, Atil, dis, fixed, dt = _setup(n_hex=5 if system == F.FP_SYS_NEWMARK else 8, system=system)
    F.fem_pic_learned_init(lib.h, seed=3, sample_capacity=4)
    P = F.fem_pic_learned_params(lib.h)
    rng = np.random.default_rng(0)
    r = rng.normal(0, 1e-12, Atil.shape[0])
    r[fixed.numpy()] = 0.0
    ct_g, rt_g = F.fem_pic_learned_forward(lib.h, torch.as_tensor(r, device="cuda"))
    we, be, W, b, wh, bh = _unpack(P)
    leaves = [we, be] + W + b + [wh, bh]
    for t in leaves:
        t.requires_grad_(True)
    ct, rt, loss = forward_loss((we, be, W, b, wh, bh), Atil, dis, fixed, torch.as_tensor(r, dtype=torch.float32))
    assert torch.allclose(rt_g.cpu(), rt.detach(), rtol=1e-5, atol=1e-6)
    err = (ct_g.cpu() - ct.detach()).abs().max() / ct.detach().abs().max()
    assert err < 2e-2, float(err)
    # gradients
    loss.backward()
    g_ref = torch.cat([we.grad, be.grad] + sum([[W[l].grad.reshape(-1), b[l].grad] for l in range(NL)], []) +
                      [wh.grad, bh.grad.reshape(1)]).numpy()
    g_gpu, loss_gpu = F.fem_pic_learned_gradient(lib.h, torch.as_tensor(r, dtype=torch.float32, device="cuda"))
    assert abs(loss_gpu - loss.item()) <= 2e-2 * loss.item()
    rel = np.linalg.norm(g_gpu - g_ref) / np.linalg.norm(g_ref)
    assert rel < 5e-2, rel
    cos = (g_gpu @ g_ref) / (np.linalg.norm(g_gpu) * np.linalg.norm(g_ref))
    assert cos > 0.998, cos
    # the gradient call leaves the weights unchanged
    assert np.array_equal(F.fem_pic_learned_params(lib.h), P)
    lib.close()


def _run_steps(lib, m, dt, nsteps, precond=F.FP_PC_JACOBI_FP64, seed=5):
    """Field steps driven by a seeded random current pattern (a cheap stand-in for the
    particle push) that still respects continuity: dG only, Q accumulated from it."""
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


def test_training_lowers_the_loss_and_learned_steps_match_plain():
    m, lib, Atil, dis, fixed, dt = _setup(n_hex=6)
    F.fem_pic_learned_init(lib.h, seed=1, sample_capacity=32)
    F.fem_pic_learned_mode(lib.h, collect=True, active=False)
    E_plain, info_plain = _run_steps(lib, m, dt, 24)
    assert F.fem_pic_learned_samples(lib.h) == 24
    before = F.fem_pic_learned_eval(lib.h, 20, 4)
    loss = F.fem_pic_learned_train(lib.h, 0, 20, epochs=40, lr=2e-3, seed=0)
    after = F.fem_pic_learned_eval(lib.h, 20, 4)
    assert loss[-1] < loss[0]
    assert after.mean() < before.mean()
    # learned field steps reach the same tolerance and the same field
    F.fem_pic_learned_mode(lib.h, collect=False, active=False)
    E_learn, info_learn = _run_steps(lib, m, dt, 24, precond=F.FP_PC_LEARNED)
    assert all(i[0]["precond"] == F.FP_PC_LEARNED for i in info_learn)
    assert all(i[0]["rel_res"] <= 1e-10 for i in info_learn)
    err = (E_learn - E_plain).abs().max() / E_plain.abs().max()
    assert float(err) < 1e-7
    lib.close()


def test_gauss_training_and_learned_projection_match_plain():
    """The node-graph network on the Gauss-law projection: samples are the projection's
    right-hand sides (zero start), training lowers the held-out loss, and field steps with
    FP_PC_LEARNED_GAUSS reach the same tolerance and the same field as plain CG."""
    m, lib, Atil, dis, fixed, dt = _setup(n_hex=6, system=F.FP_SYS_GAUSS)
    F.fem_pic_learned_init(lib.h, seed=2, sample_capacity=32)
    F.fem_pic_learned_mode(lib.h, collect=True, active=False)
    E_plain, info_plain = _run_steps(lib, m, dt, 24, precond=F.FP_PC_JACOBI)
    assert F.fem_pic_learned_samples(lib.h) == 24
    before = F.fem_pic_learned_eval(lib.h, 20, 4)
    loss = F.fem_pic_learned_train(lib.h, 0, 20, epochs=40, lr=2e-3, seed=0)
    after = F.fem_pic_learned_eval(lib.h, 20, 4)
    assert loss[-1] < loss[0]
    assert after.mean() < before.mean()
    F.fem_pic_learned_mode(lib.h, collect=False, active=False)
    E_learn, info_learn = _run_steps(lib, m, dt, 24, precond=F.FP_PC_LEARNED_GAUSS)
    assert all(i[1]["precond"] == F.FP_PC_LEARNED for i in info_learn)
    assert all(i[0]["precond"] != F.FP_PC_LEARNED for i in info_learn)
    assert all(i[0]["rel_res"] <= 1e-10 and i[1]["rel_res"] <= 1e-10 for i in info_learn)
    err = (E_learn - E_plain).abs().max() / E_plain.abs().max()
    assert float(err) < 1e-7
    # both corrections at once need both networks; the Newmark one was never initialised
    with pytest.raises(F.FemPicError):
        _run_steps(lib, m, dt, 1, precond=F.FP_PC_LEARNED | F.FP_PC_LEARNED_GAUSS)
    lib.close()
