"""Headless VTU output of results (the paper's post-processing, Sec. 3.4:
the mesh with its displacements, strains and stresses written as a "vtu"
file for ParaView).

write_vtu writes a VTK XML UnstructuredGrid: points, 4-node tets
(VTK_TETRA), point data and cell data arrays, each stored inline as base64
"binary" data preceded by its byte count (UInt64, little endian).
write_solution adds the recovered nodal strain, stress and von Mises stress
of a displacement field (sfem_recover) to the displacements.
"""
from __future__ import annotations

import base64

import numpy as np

VTK_TETRA = 10
_TYPES = {
    np.dtype(np.float64): "Float64",
    np.dtype(np.float32): "Float32",
    np.dtype(np.int64): "Int64",
    np.dtype(np.int32): "Int32",
    np.dtype(np.uint8): "UInt8",
}


def _encode(a: np.ndarray) -> str:
    raw = np.ascontiguousarray(a).astype(a.dtype.newbyteorder("<"), copy=False).tobytes()
    return base64.b64encode(np.uint64(len(raw)).astype("<u8").tobytes() + raw).decode("ascii")


def _array_xml(name: str, a: np.ndarray, indent: str) -> str:
    a = np.asarray(a)
    if a.dtype not in _TYPES:
        a = a.astype(np.float64)
    ncomp = 1 if a.ndim == 1 else a.shape[1]
    return (f'{indent}<DataArray type="{_TYPES[a.dtype]}" Name="{name}" NumberOfComponents="{ncomp}" '
            f'format="binary">{_encode(a)}</DataArray>\n')


def write_vtu(path: str, xyz, tets, point_data: dict | None = None, cell_data: dict | None = None) -> None:
    """Write the tet mesh (xyz: n x 3, tets: m x 4, 0-based) with point data
    (name -> array of n rows) and cell data (name -> array of m rows)."""
    xyz = np.asarray(xyz, dtype=np.float64)
    tets = np.asarray(tets, dtype=np.int64)
    n, m = xyz.shape[0], tets.shape[0]
    if xyz.ndim != 2 or xyz.shape[1] != 3 or tets.ndim != 2 or tets.shape[1] != 4:
        raise ValueError("xyz must be n x 3 and tets m x 4")
    if m and (tets.min() < 0 or tets.max() >= n):
        raise ValueError("tet node index out of range")
    for kind, data, rows in (("point", point_data, n), ("cell", cell_data, m)):
        for k, v in (data or {}).items():
            if np.asarray(v).shape[0] != rows:
                raise ValueError(f"{kind} data '{k}' must have {rows} rows")
    out = ['<?xml version="1.0"?>\n',
           '<VTKFile type="UnstructuredGrid" version="1.0" byte_order="LittleEndian" header_type="UInt64">\n',
           '  <UnstructuredGrid>\n',
           f'    <Piece NumberOfPoints="{n}" NumberOfCells="{m}">\n']
    if point_data:
        out.append("      <PointData>\n")
        out += [_array_xml(k, v, "        ") for k, v in point_data.items()]
        out.append("      </PointData>\n")
    if cell_data:
        out.append("      <CellData>\n")
        out += [_array_xml(k, v, "        ") for k, v in cell_data.items()]
        out.append("      </CellData>\n")
    out.append("      <Points>\n")
    out.append(_array_xml("Points", xyz, "        "))
    out.append("      </Points>\n      <Cells>\n")
    out.append(_array_xml("connectivity", tets.reshape(-1), "        "))
    out.append(_array_xml("offsets", 4 * np.arange(1, m + 1, dtype=np.int64), "        "))
    out.append(_array_xml("types", np.full(m, VTK_TETRA, dtype=np.uint8), "        "))
    out.append("      </Cells>\n    </Piece>\n  </UnstructuredGrid>\n</VTKFile>\n")
    with open(path, "w") as fh:
        fh.writelines(out)


def read_vtu_arrays(path: str) -> dict:
    """Decode every DataArray of a file written by write_vtu (name -> numpy
    array, rows x components); also 'NumberOfPoints' and 'NumberOfCells'."""
    import xml.etree.ElementTree as ET
    inv = {v: k for k, v in _TYPES.items()}
    root = ET.parse(path).getroot()
    piece = root.find("UnstructuredGrid/Piece")
    out = {"NumberOfPoints": int(piece.get("NumberOfPoints")), "NumberOfCells": int(piece.get("NumberOfCells"))}
    for da in root.iter("DataArray"):
        raw = base64.b64decode(da.text)
        nbytes = int(np.frombuffer(raw[:8], "<u8")[0])
        a = np.frombuffer(raw[8:8 + nbytes], dtype=inv[da.get("type")].newbyteorder("<"))
        k = int(da.get("NumberOfComponents", "1"))
        out[da.get("Name")] = a.reshape(-1, k) if k > 1 else a
    return out


def write_solution(path: str, h, xyz, tets, u) -> dict:
    """Recover strains and stresses of the displacement u (CUDA float64
    tensor, 3 n values) on context h and write the mesh with the point data
    displacement, strain, stress and von_mises.  Returns the host arrays."""
    from . import sfem as S
    rec = S.sfem_recover(h, u, faces=False, nodes=True)
    pd = {"displacement": u.detach().cpu().numpy().reshape(-1, 3),
          "strain": rec["node_strain"].cpu().numpy(),
          "stress": rec["node_stress"].cpu().numpy(),
          "von_mises": rec["node_vm"].cpu().numpy()}
    write_vtu(path, xyz, tets, point_data=pd)
    return pd
