"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module only *draws* inputs: a jittered cube mesh (node coordinates and tet
connectivity), particle clouds (start tet, global position, velocity) and random
field-DOF vectors.  It contains none of the method's arithmetic: no incidence
matrices, no Whitney functions, no push, walk or deposit.  Both the CUDA library
and the oracle derive everything else from these arrays on their own.

Workloads follow the paper's setting (a PEC cavity filled with electrons and,
optionally, ions; Sec. VI) at the sizes of the five synthetic configurations:

* cube n^3 split into 6 Kuhn tets per hex (conforming, shares the main diagonal),
  interior nodes optionally jittered by U(-jit*h, jit*h) per coordinate;
* particles uniform in space (tet chosen with probability proportional to its
  volume, then a point uniform inside it) or a cylindrical beam (rejection of the
  uniform cloud outside a radius), velocities Maxwellian with per-axis standard
  deviation v_th plus a drift.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# CODATA 2018 constants (SI).
C_LIGHT = 299_792_458.0
Q_E = 1.602_176_634e-19
M_E = 9.109_383_7015e-31
EPS0 = 8.854_187_8128e-12
MU0 = 1.256_637_062_12e-6
MASS_RATIO_ION = 1836.0

# the 6 permutations of the axes; tet k of a hex follows the monotone lattice path
# 000 -> e[p0] -> e[p0]+e[p1] -> 111 (Kuhn / Freudenthal subdivision)
_KUHN_PERMS = ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0))


@dataclass
class Mesh:
    """Unstructured tetrahedral mesh as plain arrays (node coordinates, connectivity)."""
    xyz: np.ndarray        # float64 [n_nodes, 3]
    tets: np.ndarray       # int32   [n_tets, 4] (any vertex order)
    n: int                 # hexes per axis
    length: float          # cube side (m)

    @property
    def n_nodes(self) -> int:
        return int(self.xyz.shape[0])

    @property
    def n_tets(self) -> int:
        return int(self.tets.shape[0])


def cube_mesh(n: int, length: float = 1.0, jitter: float = 0.0, seed: int = 1) -> Mesh:
    """Cube [0,L]^3 with n^3 hexes, each cut into 6 tets; interior nodes jittered.

    Node id = i + (n+1)*(j + (n+1)*k); tet id = 6*(i + n*(j + n*k)) + perm.
    """
    if n < 1:
        raise ValueError("n must be >= 1")
    h = length / n
    ax = np.arange(n + 1, dtype=np.float64) * h
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")  # [i,j,k]
    # node id = i + (n+1)*(j + (n+1)*k): flatten with k slowest
    xyz = np.stack([X.transpose(2, 1, 0).ravel(), Y.transpose(2, 1, 0).ravel(),
                    Z.transpose(2, 1, 0).ravel()], axis=1).copy()
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        d = rng.uniform(-jitter * h, jitter * h, size=xyz.shape)
        ii = np.arange(n + 1)
        I, J, K = np.meshgrid(ii, ii, ii, indexing="ij")
        inner = ((I > 0) & (I < n) & (J > 0) & (J < n) & (K > 0) & (K < n))
        inner = inner.transpose(2, 1, 0).ravel()
        xyz[inner] += d[inner]
    m = n + 1
    ci = np.arange(n)
    I, J, K = np.meshgrid(ci, ci, ci, indexing="ij")
    I = I.transpose(2, 1, 0).ravel()
    J = J.transpose(2, 1, 0).ravel()
    K = K.transpose(2, 1, 0).ravel()

    def nid(di, dj, dk):
        return (I + di) + m * ((J + dj) + m * (K + dk))

    tets = np.empty((n * n * n, 6, 4), dtype=np.int64)
    for p, perm in enumerate(_KUHN_PERMS):
        step = [0, 0, 0]
        verts = [nid(0, 0, 0)]
        for a in perm:
            step[a] += 1
            verts.append(nid(*step))
        tets[:, p, :] = np.stack(verts, axis=1)
    return Mesh(xyz=xyz, tets=tets.reshape(-1, 4).astype(np.int32), n=n, length=length)


@dataclass
class Particles:
    """One species: start tet, global position, velocity, and its constants."""
    cell: np.ndarray       # int32 [np]
    X: np.ndarray          # float64 [np, 3]
    V: np.ndarray          # float64 [np, 3]
    q: float
    m: float
    w: float               # macro weight (physical particles per macro-particle)

    @property
    def n(self) -> int:
        return int(self.cell.shape[0])


def _tet_volumes(mesh: Mesh) -> np.ndarray:
    # only to draw positions uniformly in space (sampling weights)
    x = mesh.xyz[mesh.tets]
    d = np.einsum("ij,ij->i", x[:, 1] - x[:, 0], np.cross(x[:, 2] - x[:, 0], x[:, 3] - x[:, 0]))
    return np.abs(d) / 6.0


def _uniform_points(mesh: Mesh, n: int, rng: np.random.Generator, tet_subset=None):
    vol = _tet_volumes(mesh)
    ids = np.arange(mesh.n_tets) if tet_subset is None else np.asarray(tet_subset)
    p = vol[ids] / vol[ids].sum()
    cell = ids[rng.choice(ids.shape[0], size=n, p=p)].astype(np.int32)
    # uniform point in a simplex: spacings of 3 sorted uniforms
    u = np.sort(rng.random((n, 3)), axis=1)
    lam = np.diff(np.concatenate([np.zeros((n, 1)), u, np.ones((n, 1))], axis=1), axis=1)
    x = mesh.xyz[mesh.tets[cell]]                       # [n,4,3]
    X = np.einsum("nk,nkd->nd", lam, x)
    return cell, X


def maxwellian(n: int, v_th: float, rng: np.random.Generator, drift=(0.0, 0.0, 0.0)) -> np.ndarray:
    """Velocities with per-axis normal spread v_th (the reading of 'Maxwellian v_th')."""
    return rng.normal(0.0, v_th, size=(n, 3)) + np.asarray(drift, dtype=np.float64)[None, :]


def uniform_species(mesh: Mesh, n: int, seed: int, v_th: float, q: float, m: float,
                    w: float = 1.0, drift=(0.0, 0.0, 0.0)) -> Particles:
    rng = np.random.default_rng(seed)
    cell, X = _uniform_points(mesh, n, rng)
    V = maxwellian(n, v_th, rng, drift)
    return Particles(cell=cell, X=X, V=V, q=q, m=m, w=w)


def beam_species(mesh: Mesh, n: int, seed: int, radius: float, v_th: float, drift,
                 q: float, m: float, w: float = 1.0) -> Particles:
    """Uniform cylinder of the given radius about the axis x = y = L/2, all z."""
    rng = np.random.default_rng(seed)
    c = 0.5 * mesh.length
    x = mesh.xyz[mesh.tets]
    # keep tets whose bounding box meets the cylinder's bounding square (cheap superset)
    lo = x.min(axis=1)
    hi = x.max(axis=1)
    near = (hi[:, 0] >= c - radius) & (lo[:, 0] <= c + radius) & \
           (hi[:, 1] >= c - radius) & (lo[:, 1] <= c + radius)
    subset = np.nonzero(near)[0]
    cells, Xs = [], []
    have = 0
    while have < n:
        want = int((n - have) * 1.4) + 1024
        cell, X = _uniform_points(mesh, want, rng, subset)
        keep = (X[:, 0] - c) ** 2 + (X[:, 1] - c) ** 2 < radius * radius
        cells.append(cell[keep])
        Xs.append(X[keep])
        have += int(keep.sum())
    cell = np.concatenate(cells)[:n]
    X = np.concatenate(Xs)[:n]
    V = maxwellian(n, v_th, rng, drift)
    return Particles(cell=cell.astype(np.int32), X=X, V=V, q=q, m=m, w=w)


def random_dofs(n: int, seed: int, scale: float = 1.0) -> np.ndarray:
    """Uniform U(-scale, scale) vector (random field DOFs for parity tests)."""
    return np.random.default_rng(seed).uniform(-scale, scale, size=n)


def gyro_period(B0: float, q: float = Q_E, m: float = M_E) -> float:
    return 2.0 * math.pi * m / (abs(q) * B0)


@dataclass
class Workload:
    name: str
    mesh: Mesh
    species: list = field(default_factory=list)
    dt: float = 0.0
    B0: tuple = (0.0, 0.0, 0.0)
    E_amp: float = 0.0     # amplitude of the seeded random edge field (V/m), 0 = none
    steps: int = 1
    n0: float = 1e14       # plasma density used for the macro weight
    background_ions: bool = False   # uniform immobile neutralising ion background


def _weight(n0: float, volume: float, n_macro: int) -> float:
    return n0 * volume / max(1, n_macro)


def config(idx: int, scale: float = 1.0, mesh_n: int = 0) -> Workload:
    """The five synthetic workloads (1-based index).  `scale` < 1 shrinks particle counts.

    1: 4^3x6 tets, no jitter, 1,000 e-, v_th=0.01c, seed 0, Bz=0.1 T, dt=0.2*T_ce, 100 steps
    2: 32^3x6, +-10% jitter (seed 1), 2M e-, v_th=0.01c, Bz=0.1 T, 200 steps
    3: 64^3x6, jitter, 20M e- beam r=0.2L drifting 0.1c along z, v_th=0.005c, Bz=0.5 T,
       random edge field amplitude 1e3 V/m, 100 steps
    5: 96^3x6, jitter, 50M e- + 50M ions, v_th_e=0.02c, Bx=0.2 T, 50 steps

    mesh_n > 0 replaces the workload's mesh resolution n by mesh_n with the same particles per
    tet (counts times (mesh_n / n)^3) and the same displacement per step in cells (dt times
    n / mesh_n): a smaller case of the same character, named after its sizes.
    """
    L = 1.0
    base_n = {1: 4, 2: 32, 3: 64, 5: 96}.get(idx)
    if base_n is None:
        raise ValueError(f"unknown workload {idx}")
    n = mesh_n if mesh_n > 0 else base_n
    f = (n / base_n) ** 3 if mesh_n > 0 else 1.0
    tdt = base_n / n

    def count(c):
        return max(1, int(c * scale * f))

    def named(default, parts):
        return default if mesh_n <= 0 else f"cube{n}" + parts
    if idx == 1:
        mesh = cube_mesh(n, L, 0.0)
        npart = count(1000)
        B0 = 0.1
        sp = [uniform_species(mesh, npart, 0, 0.01 * C_LIGHT, -Q_E, M_E, _weight(1e14, L ** 3, npart))]
        return Workload(named("cube4_e1k", f"_e{npart}"), mesh, sp, 0.2 * gyro_period(B0) * tdt, (0.0, 0.0, B0),
                        0.0, 100, background_ions=True)
    if idx == 2:
        mesh = cube_mesh(n, L, 0.1, seed=1)
        npart = count(2_000_000)
        B0 = 0.1
        sp = [uniform_species(mesh, npart, 2, 0.01 * C_LIGHT, -Q_E, M_E, _weight(1e14, L ** 3, npart))]
        return Workload(named("cube32_jit_e2M", f"_jit_e{npart}"), mesh, sp, 0.2 * gyro_period(B0) * tdt,
                        (0.0, 0.0, B0), 0.0, 200, background_ions=True)
    if idx == 3:
        mesh = cube_mesh(n, L, 0.1, seed=1)
        npart = count(20_000_000)
        B0 = 0.5
        r = 0.2 * L
        sp = [beam_species(mesh, npart, 3, r, 0.005 * C_LIGHT, (0.0, 0.0, 0.1 * C_LIGHT), -Q_E, M_E,
                           _weight(1e14, math.pi * r * r * L, npart))]
        return Workload(named("cube64_jit_beam20M", f"_jit_beam{npart}"), mesh, sp, 0.2 * gyro_period(B0) * tdt,
                        (0.0, 0.0, B0), 1e3, 100)
    mesh = cube_mesh(n, L, 0.1, seed=1)
    npart = count(50_000_000)
    B0 = 0.2
    vte = 0.02 * C_LIGHT
    w = _weight(1e14, L ** 3, npart)
    sp = [uniform_species(mesh, npart, 5, vte, -Q_E, M_E, w),
          uniform_species(mesh, npart, 55, vte / math.sqrt(MASS_RATIO_ION), Q_E, MASS_RATIO_ION * M_E, w)]
    return Workload(named("cube96_jit_e50M_i50M", f"_jit_e{npart}_i{npart}"), mesh, sp,
                    0.2 * gyro_period(B0) * tdt, (B0, 0.0, 0.0), 0.0, 50)


def two_tet_mesh() -> Mesh:
    """Two tets sharing the face (1,2,3): 5 nodes, 9 edges, 7 faces."""
    xyz = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0],
                    [0.9, 0.8, 0.7]], dtype=np.float64)
    tets = np.array([[0, 1, 2, 3], [1, 2, 3, 4]], dtype=np.int32)
    return Mesh(xyz=xyz, tets=tets, n=1, length=1.0)
