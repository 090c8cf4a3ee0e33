"""The headless VTU writer (paper_2001_08849_gb300/vtu.py): structure of the
file and exact round trip of every array (CPU only)."""
import xml.etree.ElementTree as ET

import numpy as np
import pytest

from inputs.kuhn_beam import kuhn_beam
from paper_2001_08849_gb300 import vtu


def test_round_trip(tmp_path):
    m = kuhn_beam(2, 1, 1, (2.0, 1.0, 1.0), 0.1, seed=3)
    rng = np.random.default_rng(1)
    pd = {"displacement": rng.standard_normal((m.n_nodes, 3)), "von_mises": rng.random(m.n_nodes)}
    cd = {"region": np.arange(m.n_tets, dtype=np.int32), "stress": rng.standard_normal((m.n_tets, 6))}
    path = tmp_path / "beam.vtu"
    vtu.write_vtu(str(path), m.xyz, m.tets, point_data=pd, cell_data=cd)
    root = ET.parse(path).getroot()
    assert root.get("type") == "UnstructuredGrid" and root.get("header_type") == "UInt64"
    got = vtu.read_vtu_arrays(str(path))
    assert got["NumberOfPoints"] == m.n_nodes and got["NumberOfCells"] == m.n_tets
    assert np.array_equal(got["Points"], m.xyz)
    assert np.array_equal(got["connectivity"], m.tets.reshape(-1))
    assert np.array_equal(got["offsets"], 4 * np.arange(1, m.n_tets + 1))
    assert np.all(got["types"] == vtu.VTK_TETRA)
    for k, v in {**pd, **cd}.items():
        assert np.array_equal(got[k], v), k


def test_rejects_bad_shapes(tmp_path):
    m = kuhn_beam(1, 1, 1, (1.0, 1.0, 1.0), 0.0, seed=1)
    with pytest.raises(ValueError):
        vtu.write_vtu(str(tmp_path / "a.vtu"), m.xyz, m.tets, point_data={"u": np.zeros(m.n_nodes + 1)})
    with pytest.raises(ValueError):
        vtu.write_vtu(str(tmp_path / "b.vtu"), m.xyz, m.tets + m.n_nodes)
