"""The seeded workload generator: the stated workloads keep their names, sizes and time steps,
and a resolution override keeps particles per tet and displacement per step in cells."""
import numpy as np

from paper_2103_06737_gb300 import inputs as I


def test_workload_two_as_stated():
    wl = I.config(2, 0.05)
    assert wl.name == "cube32_jit_e2M" and wl.mesh.n == 32
    assert [s.n for s in wl.species] == [100_000]
    assert wl.dt == 0.2 * I.gyro_period(0.1)


def test_resolution_override_keeps_density_and_cell_displacement():
    a = I.config(2, 0.05)
    b = I.config(2, 0.05, mesh_n=16)
    assert b.mesh.n == 16 and b.name == "cube16_jit_e12500"
    ta, tb = len(a.mesh.tets), len(b.mesh.tets)
    assert tb * 8 == ta
    assert a.species[0].n / ta == b.species[0].n / tb          # particles per tet
    assert np.isclose(b.dt / (1.0 / 16), a.dt / (1.0 / 32))     # dt over the cell size
    assert np.all((b.species[0].cell >= 0) & (b.species[0].cell < tb))
