"""Fourth-order Adams particle mover of the oracle (FP64, plain numpy).

TEST INFRASTRUCTURE ONLY: used by tests/ and the bench's CPU legs, never by the library.

Sec. IV.B.2 states that the particles' trajectories and velocities are advanced by a
fourth-order Adams method, with the scheme itself given in another paper.  Reading used
here (and by the library): the explicit Adams-Bashforth method on the first-order system

    dx/dt = v,    dv/dt = a(x, v) = (q/m) (E(x) + v x B(x)),

with x and v at the same time level (no staggering), the fields frozen at time level n for
the whole step, and the k-step formula

    y^{n+1} = y^n + dt * sum_{j=0}^{k-1} beta_{k,j} f^{n-j},    f = (v, a),

where k = min(s + 1, 4) on a particle's s-th step (s earlier derivative values known), so
the first three steps start the method at orders 1, 2, 3.  The position moves along the
straight segment x^n -> x^{n+1}; the walk and the Whitney-1 / Whitney-0 deposits on that
segment are the Boris path's (Sec. IV.B.1), so the discrete continuity equation still holds.

The coefficients are not typed in: beta_{k,j} = (1/dt) * integral over [t_n, t_{n+1}] of the
Lagrange basis polynomial that is 1 at t_{n-j} and 0 at the other k-1 nodes, integrated
exactly in rational arithmetic (the definition of the Adams-Bashforth family).
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def _poly_mul(p, q):
    out = [Fraction(0)] * (len(p) + len(q) - 1)
    for i, a in enumerate(p):
        for j, b in enumerate(q):
            out[i + j] += a * b
    return out


def ab_coefficients_exact(k: int):
    """beta_{k,0..k-1} as Fractions, time in units of dt with t_n = 0, t_{n-j} = -j."""
    if not 1 <= k <= 8:
        raise ValueError("order 1..8")
    beta = []
    for j in range(k):
        # Lagrange basis for node -j over nodes {0, -1, ..., -(k-1)}: prod_{i != j} (t + i)/(i - j)
        poly = [Fraction(1)]
        for i in range(k):
            if i == j:
                continue
            poly = _poly_mul(poly, [Fraction(i, i - j), Fraction(1, i - j)])   # (i + t)/(i - j)
        # integral over t in [0, 1] of sum c_p t^p
        beta.append(sum(c / (p + 1) for p, c in enumerate(poly)))
    return beta


def ab_coefficients(k: int) -> np.ndarray:
    return np.array([float(c) for c in ab_coefficients_exact(k)])


def order_for(step: int) -> int:
    """Order of the step taken by a particle with `step` earlier steps (start-up at 1, 2, 3)."""
    if step < 0:
        raise ValueError("step >= 0")
    return min(step + 1, 4)


def lorentz(V, E, B, q, m):
    """a = (q/m)(E + v x B), FP64 (Sec. II.A, non-relativistic)."""
    V = np.asarray(V, dtype=np.float64).reshape(-1, 3)
    return (q / m) * (np.asarray(E, dtype=np.float64).reshape(-1, 3) + np.cross(V, np.asarray(B, np.float64).reshape(-1, 3)))


def ab_update(X, V, A, hist_v, hist_a, step, dt):
    """One Adams-Bashforth update of (x, v) from f^n = (V, A) and the history.

    hist_v, hist_a: [3, n, 3] with slot (step - j) % 3 holding f^{n-j}, j = 1..min(step, 3).
    Returns (X1, V1).  Pure arithmetic: no field evaluation, no mesh.
    """
    k = order_for(step)
    beta = ab_coefficients(k)
    dx = beta[0] * np.asarray(V, np.float64)
    dv = beta[0] * np.asarray(A, np.float64)
    for j in range(1, k):
        s = (step - j) % 3
        dx = dx + beta[j] * hist_v[s]
        dv = dv + beta[j] * hist_a[s]
    return np.asarray(X, np.float64) + dt * dx, np.asarray(V, np.float64) + dt * dv


def adams_step(orc, cell, X, V, hist_v, hist_a, step, e, b, q, m, w, dt, max_cross=64, Xend=None,
               nthreads=0):
    """One Adams particle step on the mesh: gather E, B at x^n (Whitney-1/2, Sec. II.C), the
    Lorentz acceleration, the Adams-Bashforth update, then the walk and deposits along the
    straight segment to x^{n+1} (or to Xend when given: the walk on another program's end
    points).  The history is updated in a copy (slot step % 3 takes f^n).

    Returns a dict: cell, X (end points; the wall point for absorbed particles), V (v^{n+1}),
    Xab (the Adams end points), dG, dG_abs, Q, Q_abs, hist_v, hist_a, n_bound.
    """
    cell = np.asarray(cell, dtype=np.int32)
    X = np.asarray(X, np.float64).reshape(-1, 3)
    V = np.asarray(V, np.float64).reshape(-1, 3)
    alive = cell >= 0
    E, B = orc.gather(np.where(alive, cell, 0), X, e, b)
    A = lorentz(V, E, B, q, m)
    X1, V1 = ab_update(X, V, A, hist_v, hist_a, step, dt)
    X1[~alive] = X[~alive]
    V1[~alive] = V[~alive]
    hv = np.array(hist_v, dtype=np.float64, copy=True)
    ha = np.array(hist_a, dtype=np.float64, copy=True)
    s = step % 3
    hv[s][alive] = V[alive]
    ha[s][alive] = A[alive]
    r = orc.step(cell, X, V, e, b, q, m, w, dt, max_cross=max_cross, Xend=X1 if Xend is None else Xend,
                 nthreads=nthreads)
    return dict(cell=r["cell"], X=r["X"], V=V1, Xab=X1, A=A, dG=r["dG"], dG_abs=r["dG_abs"], Q=r["Q"],
                Q_abs=r["Q_abs"], hist_v=hv, hist_a=ha, n_bound=r["n_bound"])
