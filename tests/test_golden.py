"""Golden fixtures: the paper's printed geometry and an oracle regression file."""
import os

import numpy as np

from oracle import Oracle
from workloads import heat as H

GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _read(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        if not line.strip() or line.startswith("#"):
            continue
        key, *vals = line.split()
        out.setdefault(key, []).append([float(v) for v in vals])
    return out


def test_cell_geometry_matches_paper_figure():
    g = _read("paper_geometry.txt")
    np.testing.assert_array_equal(H.R_FACES_CELL, g["cell_r_faces"][0])
    np.testing.assert_array_equal(H.Z_FACES_CELL, g["cell_z_faces"][0])
    p = H.config1()
    o = Oracle(p)
    reg = o.grid()["region"]
    # terminal cap covers the whole top segment, void is r in (2, 4.2) x z in (8, 10)
    assert np.all(reg[-1] == H.TERMINAL)
    assert np.all(reg[0, :31] == H.COOLER) and np.all(reg[0, 31:46] == H.INSULATOR)


def test_paper_grid_shape():
    g = _read("paper_geometry.txt")
    p = H.config_paper_grid()
    np.testing.assert_array_equal(p.r_faces, g["paper_r_faces"][0])
    np.testing.assert_array_equal(p.r_cells, g["paper_r_cells"][0])
    np.testing.assert_array_equal(p.z_faces, g["paper_z_faces"][0])
    assert (p.Nr, p.Nz) == tuple(int(v) for v in g["paper_grid"][0])
    o = Oracle(p)
    reg = o.grid()["region"]
    core = reg[:, 0] >= 0
    other = reg[:, 900] >= 0
    assert core.sum() == g["paper_core_z_cells"][0][0]
    assert other.sum() == g["paper_other_z_cells"][0][0]
    assert p.T_init == g["paper_T0"][0][0]


def test_oracle_regression_config1():
    g = _read("oracle_config1.txt")
    p = H.config1()
    o = Oracle(p)
    tau = H.DT_FACTOR * o.tau_exp()
    assert abs(tau - g["tau"][0][0]) <= 1e-14 * tau
    o.step(tau, H.STEPS["config1"])
    T = o.field()
    E1, F1, _ = o.energy()
    assert abs(E1 - g["E1"][0][0]) <= 1e-12 * abs(E1)
    for k, v in g["T"]:
        assert abs(T.flat[int(k)] - v) <= 1e-12 * abs(v)
