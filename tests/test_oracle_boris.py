"""Pins of the oracle's non-relativistic Boris push against closed forms of the discrete map.

The paper moves particles by the Lorentz force and Newton's law in the
non-relativistic regime (Sec. I, II.A); the mover here is Boris.  Closed forms:
  * E = 0: |v| is conserved and v turns by theta = 2 atan(w_c dt/2) per step;
    the leapfrog orbit is a regular polygon of circumradius (v_perp/w_c) sqrt(1+(w_c dt/2)^2);
    theta/dt -> w_c with error O(dt^2);
  * E perpendicular to B with v = E x B / B^2: a fixed point of the map for any dt.
"""
import json
import math
import os

import numpy as np

from paper_2103_06737_gb300 import inputs as I
import oracle as O

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
q, m = -I.Q_E, I.M_E


def _run(v0, E, B, dt, n):
    V = np.array([v0], dtype=np.float64)
    out = [V[0].copy()]
    for _ in range(n):
        V = O.Oracle.boris(V, [E], [B], q, m, dt)
        out.append(V[0].copy())
    return np.array(out)


def test_rotation_angle_and_speed():
    B0 = 0.1
    wc = abs(q) * B0 / m
    g = GOLD["boris_discrete_gyration"]
    dt = g["omega_dt"] / wc
    vs = _run([1e6, 2e5, 3e5], [0, 0, 0], [0, 0, B0], dt, 400)
    speed = np.linalg.norm(vs, axis=1)
    assert np.abs(speed / speed[0] - 1).max() < 1e-13
    assert np.abs(vs[:, 2] - 3e5).max() == 0.0 or np.abs(vs[:, 2] - 3e5).max() < 1e-9
    ang = np.arctan2(vs[1:, 1], vs[1:, 0]) - np.arctan2(vs[:-1, 1], vs[:-1, 0])
    ang = np.abs((ang + np.pi) % (2 * np.pi) - np.pi)
    assert np.abs(ang - g["theta"]).max() < 1e-12
    # electrons (q<0) gyrate counter-clockwise about +z
    cz = np.cross(vs[0], vs[1])[2]
    assert cz > 0


def test_orbit_circumradius():
    B0 = 0.1
    wc = abs(q) * B0 / m
    g = GOLD["boris_discrete_gyration"]
    dt = g["omega_dt"] / wc
    vperp = 1e6
    vs = _run([vperp, 0, 0], [0, 0, 0], [0, 0, B0], dt, 50)
    x = np.concatenate([[0.0, 0.0, 0.0]], axis=0)[None]
    xs = np.cumsum(np.vstack([np.zeros(3), dt * vs[1:]]), axis=0)
    a, b, c = xs[0, :2], xs[1, :2], xs[2, :2]
    d = 2 * (a[0] * (b[1] - c[1]) + b[0] * (c[1] - a[1]) + c[0] * (a[1] - b[1]))
    ux = ((a @ a) * (b[1] - c[1]) + (b @ b) * (c[1] - a[1]) + (c @ c) * (a[1] - b[1])) / d
    uy = ((a @ a) * (c[0] - b[0]) + (b @ b) * (a[0] - c[0]) + (c @ c) * (b[0] - a[0])) / d
    R = np.hypot(xs[:, 0] - ux, xs[:, 1] - uy)
    rL = vperp / wc
    assert np.abs(R / rL - g["R_over_rL"]).max() < 1e-9
    del x


def test_gyrofrequency_converges_second_order():
    B0 = 0.1
    wc = abs(q) * B0 / m
    errs = []
    for frac in (0.1, 0.05, 0.025):
        dt = frac * math.pi / wc
        vs = _run([1e6, 0, 0], [0, 0, 0], [0, 0, B0], dt, 3)
        th = abs(math.atan2(vs[1, 1], vs[1, 0]))
        errs.append(abs(th / dt - wc) / wc)
    assert errs[0] / errs[1] > 3.8 and errs[1] / errs[2] > 3.9


def test_exb_drift_fixed_point():
    B = np.array([0.0, 0.0, 0.2])
    E = np.array([3e4, -1e4, 0.0])
    vE = np.cross(E, B) / (B @ B)
    wc = abs(q) * 0.2 / m
    for dt in (0.1 / wc, 1.2566 / wc, 5.0 / wc):
        vs = _run(vE, E, B, dt, 100)
        assert np.abs(vs - vE).max() < 1e-9 * np.linalg.norm(vE)


def test_exb_mean_drift_with_gyration():
    B = np.array([0.0, 0.0, 0.2])
    E = np.array([2e4, 0.0, 0.0])
    vE = np.cross(E, B) / (B @ B)
    wc = abs(q) * 0.2 / m
    dt = 0.4 * math.pi / wc             # 5 steps per (discrete) revolution-ish
    vs = _run(vE + np.array([3e5, 0, 0]), E, B, dt, 20000)
    mean = vs[1:].mean(axis=0)
    assert np.abs(mean - vE).max() < 2e-3 * 3e5
