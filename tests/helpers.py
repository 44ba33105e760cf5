"""Shared helpers for the tests (tolerances follow the stated reading).

Deposit tolerance (per entry, relative to the sum of absolute contributions):
  |G_gpu - G_ref|_e <= tol * sum_p |g_{p,e}| + 64 eps max|G_ref|
  and   max|G_gpu - G_ref| <= tol * max|G_ref|
with tol = 1e-12 in FP64 mode and 1e-5 in FP32 mode, eps = 2^-52.  A plain relative
bound per entry is ill-posed where thermal contributions cancel.  The 64 eps term is
the oracle's own FP64 rounding floor: its 2-point Gauss-Legendre nodes are not dyadic,
so an entry whose exact value is zero (a piece on which the edge's two barycentric
coordinates stay proportional, e.g. one of them zero throughout) comes out as rounding
noise of order eps there.
"""
import numpy as np

TOL = {"fp64": 1e-12, "fp32": 1e-5}
EPS = {"fp64": 2.0 ** -53, "fp32": 2.0 ** -24}


def fp32_continuity_tol(n_particles, n_nodes, n_edges):
    """Relative bound on the FP32 continuity residual |D0^T dG - dQ| against the node scale.

    The deposits are FP32 sums of k terms each (k ~ 4 N_p / N_n per node charge, 6 N_p / N_e
    per edge current); their rounding grows like sqrt(k) * 2^-24 for independent roundings.
    The bound takes 8 times that, and never less than 1e-6.
    """
    k = max(4.0 * n_particles / n_nodes, 6.0 * n_particles / n_edges, 1.0)
    return max(1e-6, 8.0 * 2.0 ** -24 * k ** 0.5)


def assert_deposit_close(got, ref, ref_abs, tol, what="dG", touch=None, eps=None):
    """Per-entry and max-norm deposit bound.  With touch (the oracle's sum of |q w| over the
    pieces / end points touching each entry) and eps (the unit roundoff of the precision the
    deposits were computed in) the per-entry floor is 4 eps touch instead of 64 eps_64 max|ref|:
    barycentric coordinates in [0, 1] carry an absolute rounding of order eps, so an entry
    formed from near-zero contributions (a particle near the opposite face, a start point that
    rounding put a hair outside its tet and that the walk first moves onto the face) is held
    to that absolute scale per touching particle, not to its own tiny value."""
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref)
    scale = np.maximum(ref_abs, np.finfo(np.float64).tiny)
    if touch is not None:
        floor = 4.0 * eps * np.asarray(touch)
    else:
        floor = 64.0 * np.finfo(np.float64).eps * np.abs(ref).max()
    bad = err > tol * scale + floor + 1e-300
    assert not bad.any(), (f"{what}: {bad.sum()} entries beyond {tol} * sum|contrib| "
                           f"(worst ratio {np.max(err / scale):.3e})")
    assert err.max() <= tol * max(np.abs(ref).max(), np.finfo(np.float64).tiny) + 1e-300, \
        f"{what}: max error {err.max():.3e} vs {tol} * max|ref| {np.abs(ref).max():.3e}"


def csr_tuple(m, n_cols):
    m = m.tocsr()
    m.sort_indices()
    return (m.indptr.astype(np.int32), m.indices.astype(np.int32), m.data.astype(np.int8), n_cols)


def continuity_run(m, cx, fo, dt, n_steps, seed, q_sign=-1.0):
    """Deposits from the oracle's own particle steps on the library reading's fields.

    The reduced system rests on continuity at every free node.  A particle absorbed by the
    wall leaves the particle set after its step, so the next step's node charge no longer
    holds its wall charge; under the natural boundary those wall nodes are free.  The run
    therefore keeps absorbed charge on the wall: Q^{n+1} = Q^n + D0^T dG^{n+1/2}, which
    equals the particles' own W0 charge wherever no particle was absorbed."""
    from paper_2103_06737_gb300 import inputs as I
    import oracle as O

    orc = O.Oracle(m.xyz, m.tets)
    sp_ = I.uniform_species(m, 800, seed, 0.02 * I.C_LIGHT, q_sign * I.Q_E, I.M_E, 1e6)
    _, b0 = cx.project_uniform((0, 0, 0), (0, 0, 0.1))
    Q0, _ = orc.charge(sp_.cell, sp_.X, sp_.q, sp_.w)
    E0 = fo.initial_field(Q0)
    E_prev, E, b = E0.copy(), E0.copy(), b0.copy()
    dG_prev = np.zeros(cx.n_edges)
    cell, X, V = sp_.cell, sp_.X, sp_.V
    D0T = cx.D0().T.astype(np.float64)
    Q = Q0.copy()
    out = []
    for _ in range(n_steps):
        r = orc.step(cell, X, V, E, b, sp_.q, sp_.m, sp_.w, dt)
        cell, X, V = r["cell"], r["X"], r["V"]
        Q = Q + D0T @ r["dG"]
        assert np.abs(Q - r["Q"])[~cx.boundary_node].max() <= 1e-13 * np.abs(Q).max()
        E1, b1 = fo.step(E, E_prev, b, r["dG"], dG_prev, Q)
        out.append(dict(dG=r["dG"], dG_prev=dG_prev, Q=Q.copy(), E=E1, b=b1))
        E_prev, E, b, dG_prev = E, E1, b1, r["dG"]
    return Q0, E0, b0, out
