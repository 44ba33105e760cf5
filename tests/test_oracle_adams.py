"""Pins of the oracle's fourth-order Adams particle mover (Sec. IV.B.2 names the method; the
reading is the explicit Adams-Bashforth family with start-up at orders 1, 2, 3).

Pinned by:
  * the coefficient tables and error constants of the Adams-Bashforth methods (standard
    tables, tests/golden/closed_forms.json), against the oracle's exact integration of the
    Lagrange basis;
  * exactness: order k integrates a derivative that is a polynomial of degree k-1 in t
    exactly, and misses degree k by the tabulated error constant;
  * the gyro orbit in a uniform B: the global error after one period falls as dt^4;
  * on the mesh: a uniform E (B = 0) started from the exact history lands on the exact
    parabola to round-off; the history ring takes f^n; continuity D0^T dG = dQ and total
    charge hold along the Adams segments, including absorbed particles.
"""
import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_2103_06737_gb300 import inputs as I
import oracle as O
from oracle import adams as AD

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))["adams_bashforth"]


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_coefficients_match_tables(k):
    got = AD.ab_coefficients_exact(k)
    want = [Fraction(a, b) for a, b in GOLD["beta"][str(k)]]
    assert got == want


def _history_from(f, step, n=1):
    """hist[s] = f(-j) for the slot s = (step - j) % 3, j = 1..3 (time in units of dt, t_n = 0)."""
    h = np.zeros((3, n, 3))
    for j in range(1, min(step, 3) + 1):
        h[(step - j) % 3] = f(-j)
    return h


@pytest.mark.parametrize("k", [1, 2, 3, 4])
def test_exact_for_polynomials_and_error_constant(k):
    rng = np.random.default_rng(k)
    step = k - 1                               # order k
    assert AD.order_for(step) == k
    # f(t) = sum_p c_p t^p with deg k-1 (vector valued, 3 components); dt = 1
    c = rng.normal(size=(k, 3))
    f = lambda t: sum(c[p] * t ** p for p in range(k))[None, :]
    exact = sum(c[p] / (p + 1) for p in range(k))
    hv = _history_from(f, step)
    # f as both the velocity (position update) and the acceleration (velocity update)
    X1, V1 = AD.ab_update(np.zeros((1, 3)), f(0.0), f(0.0), hv, hv, step, 1.0)
    assert np.abs(X1[0] - exact).max() <= 1e-14 * (1 + np.abs(exact).max())
    assert np.abs(V1[0] - f(0.0)[0] - exact).max() <= 1e-14 * (1 + np.abs(exact).max())
    # degree k: error = C_{k+1} * y^{(k+1)} with y' = t^k, y^{(k+1)} = k!
    g = lambda t: np.full((1, 3), float(t) ** k)
    hg = _history_from(g, step)
    Xg, _ = AD.ab_update(np.zeros((1, 3)), g(0.0), g(0.0), hg, hg, step, 1.0)
    err = 1.0 / (k + 1) - Xg[0, 0]
    a, b = GOLD["error_constant"][str(k)]
    assert abs(err - a / b * math.factorial(k)) <= 1e-13 * math.factorial(k)


def _gyro_error(n_per_period):
    """Global error of the Adams mover after one gyro period in a uniform B (E = 0), started
    from the exact orbit's history."""
    q, m, B0 = -I.Q_E, I.M_E, 0.1
    wc = abs(q) * B0 / m
    T = 2 * math.pi / wc
    dt = T / n_per_period
    vp = 1e6
    rL = vp / wc
    # electrons gyrate counter-clockwise about +z: v = vp (-sin(wc t), cos(wc t)) with centre
    # offset so that x(0) = (rL, 0)
    def exact(t):
        x = np.array([[rL * math.cos(wc * t), rL * math.sin(wc * t), 0.0]])
        v = np.array([[-vp * math.sin(wc * t), vp * math.cos(wc * t), 0.0]])
        return x, v
    Bv = np.array([[0.0, 0.0, B0]])
    hv = np.zeros((3, 1, 3))
    ha = np.zeros((3, 1, 3))
    for j in range(1, 4):
        _, vj = exact(-j * dt)
        hv[(3 - j) % 3] = vj
        ha[(3 - j) % 3] = AD.lorentz(vj, np.zeros((1, 3)), Bv, q, m)
    X, V = exact(0.0)
    step = 3
    for _ in range(n_per_period):
        A = AD.lorentz(V, np.zeros((1, 3)), Bv, q, m)
        X1, V1 = AD.ab_update(X, V, A, hv, ha, step, dt)
        hv[step % 3], ha[step % 3] = V, A
        X, V, step = X1, V1, step + 1
    x_ex, _ = exact(T)
    return np.linalg.norm(X - x_ex) / rL


def test_gyro_orbit_fourth_order():
    e1, e2, e3 = _gyro_error(200), _gyro_error(400), _gyro_error(800)
    assert e1 < 1e-4
    for a, b in ((e1, e2), (e2, e3)):
        assert 13.0 < a / b < 19.0          # 2^4 = 16


def test_uniform_field_parabola_on_mesh():
    """B = 0, uniform E: v is linear and x quadratic in t, which order >= 2 integrates exactly."""
    m = I.cube_mesh(4, 1.0, 0.1, seed=1)
    orc = O.Oracle(m.xyz, m.tets)
    cx = orc.cx
    Ev = np.array([3.0e3, -1.0e3, 2.0e3])
    e, b = orc.project_uniform(Ev, [0.0, 0.0, 0.0])
    q, mass = -I.Q_E, I.M_E
    acc = q / mass * Ev
    sp = I.uniform_species(m, 300, 5, 2e5, q, mass)
    dt = 2e-8
    n = sp.n
    for step in (0, 1, 2, 3, 7):
        # exact history at t_{n-j} = -j dt of the parabola through (X, V) at t_n = 0
        hv = np.zeros((3, n, 3))
        ha = np.zeros((3, n, 3))
        for j in range(1, min(step, 3) + 1):
            hv[(step - j) % 3] = sp.V - j * dt * acc
            ha[(step - j) % 3] = acc
        r = AD.adams_step(orc, sp.cell, sp.X, sp.V, hv, ha, step, e, b, q, mass, 1.0, dt)
        want_v = sp.V + dt * acc
        assert np.abs(r["V"] - want_v).max() <= 1e-12 * np.abs(want_v).max()
        want_x = sp.X + dt * sp.V + 0.5 * dt * dt * acc
        err = np.abs(r["Xab"] - want_x).max()
        if step == 0:       # forward Euler misses the dt^2/2 term
            assert abs(err - 0.5 * dt * dt * np.abs(acc).max()) <= 1e-3 * 0.5 * dt * dt * np.abs(acc).max()
        else:
            assert err <= 1e-14
        # the ring takes f^n in slot step % 3 and keeps the others
        s = step % 3
        assert np.array_equal(r["hist_v"][s], sp.V)
        assert np.abs(r["hist_a"][s] - acc).max() <= 1e-12 * np.abs(acc).max()
        for o in range(3):
            if o != s:
                assert np.array_equal(r["hist_v"][o], hv[o])


def test_continuity_along_adams_segments():
    m = I.cube_mesh(4, 1.0, 0.1, seed=2)
    orc = O.Oracle(m.xyz, m.tets)
    cx = orc.cx
    rng = np.random.default_rng(4)
    e = rng.uniform(-1, 1, cx.n_edges)
    b = rng.uniform(-1, 1, cx.n_faces)
    n = 2000
    sp = I.uniform_species(m, n, 6, 0.0, -1.0, 1.0)
    V = rng.normal(size=(n, 3)) * 0.4
    hv = rng.normal(size=(3, n, 3)) * 0.4
    ha = rng.normal(size=(3, n, 3))
    q, mass, w, dt = -1.0, 1.0, 2.0, 0.5
    Q0, Q0a = orc.charge(sp.cell, sp.X, q, w)
    r = AD.adams_step(orc, sp.cell, sp.X, V, hv, ha, 3, e, b, q, mass, w, dt)
    assert (r["cell"] < 0).sum() > 10
    D0 = cx.D0()
    res = D0.T @ r["dG"] - (r["Q"] - Q0)
    scale = abs(D0.T) @ r["dG_abs"] + r["Q_abs"] + Q0a
    assert np.abs(res).max() <= 1e-14 * scale.max()
    assert abs(r["Q"].sum() - n * q * w) <= 1e-12 * n * w
    # live particles end at the Adams end point
    live = r["cell"] >= 0
    assert np.abs(r["X"][live] - r["Xab"][live]).max() <= 1e-14
