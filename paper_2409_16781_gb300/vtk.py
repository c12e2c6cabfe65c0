"""Legacy-VTK output of the macroscopic fields (the paper's use cases write
VTK files for viewing in ParaView, Sec. 3.3): plain file I/O on the host.

``write_vtk(path, rho, u, flags=None)`` writes a binary legacy VTK file
(version 3.0, big-endian as the format requires) with one STRUCTURED_POINTS
dataset of nx x ny x nz points (x fastest, the library's cell order), the
point data SCALARS rho (float64), VECTORS u (float64) and, when given,
SCALARS flags (unsigned_char).  ``read_vtk`` reads such a file back (it
understands exactly what write_vtk writes).
"""
from __future__ import annotations

import numpy as np


def write_vtk(path: str, rho: np.ndarray, u: np.ndarray, flags=None, spacing=(1.0, 1.0, 1.0),
              origin=(0.0, 0.0, 0.0), title: str = "lbgb fields") -> None:
    rho = np.asarray(rho, dtype=np.float64)
    if rho.ndim != 3:
        raise ValueError("rho must be (nz, ny, nx)")
    nz, ny, nx = rho.shape
    u = np.asarray(u, dtype=np.float64)
    if u.shape != (3, nz, ny, nx):
        raise ValueError(f"u must be (3, {nz}, {ny}, {nx}), got {u.shape}")
    title = title.replace("\n", " ")[:255]
    n = nx * ny * nz
    with open(path, "wb") as fh:
        head = (f"# vtk DataFile Version 3.0\n{title}\nBINARY\nDATASET STRUCTURED_POINTS\n"
                f"DIMENSIONS {nx} {ny} {nz}\nORIGIN {origin[0]:.17g} {origin[1]:.17g} {origin[2]:.17g}\n"
                f"SPACING {spacing[0]:.17g} {spacing[1]:.17g} {spacing[2]:.17g}\nPOINT_DATA {n}\n")
        fh.write(head.encode("ascii"))
        fh.write(b"SCALARS rho double 1\nLOOKUP_TABLE default\n")
        fh.write(rho.reshape(-1).astype(">f8").tobytes())
        fh.write(b"\nVECTORS u double\n")
        # one (ux, uy, uz) triple per point, points in x-fastest order
        fh.write(np.ascontiguousarray(u.reshape(3, n).T).astype(">f8").tobytes())
        if flags is not None:
            fl = np.asarray(flags, dtype=np.uint8).reshape(-1)
            if fl.size != n:
                raise ValueError(f"flags has {fl.size} entries, the lattice {n}")
            fh.write(b"\nSCALARS flags unsigned_char 1\nLOOKUP_TABLE default\n")
            fh.write(fl.tobytes())
        fh.write(b"\n")


def read_vtk(path: str) -> dict:
    """Fields of a file written by write_vtk: dims (nx, ny, nz), origin,
    spacing, rho (nz, ny, nx), u (3, nz, ny, nx) and, if present, flags."""
    data = open(path, "rb").read()
    pos = 0

    def line():
        nonlocal pos
        end = data.index(b"\n", pos)
        s = data[pos:end].decode("ascii")
        pos = end + 1
        return s

    if not line().startswith("# vtk DataFile Version"):
        raise ValueError("not a legacy VTK file")
    line()  # title
    if line().strip() != "BINARY" or line().strip() != "DATASET STRUCTURED_POINTS":
        raise ValueError("not a binary STRUCTURED_POINTS file")
    out = {}
    while True:
        key, *vals = line().split()
        if key == "DIMENSIONS":
            out["dims"] = tuple(int(v) for v in vals)
        elif key == "ORIGIN":
            out["origin"] = tuple(float(v) for v in vals)
        elif key == "SPACING":
            out["spacing"] = tuple(float(v) for v in vals)
        elif key == "POINT_DATA":
            n = int(vals[0])
            break
    nx, ny, nz = out["dims"]
    while pos < len(data):
        words = line().split()
        if not words:
            continue
        if words[0] == "SCALARS":
            name, typ = words[1], words[2]
            line()  # LOOKUP_TABLE
            dt = {"double": ">f8", "unsigned_char": "u1"}[typ]
            size = np.dtype(dt).itemsize * n
            arr = np.frombuffer(data, dtype=dt, count=n, offset=pos).astype(
                np.float64 if typ == "double" else np.uint8)
            pos += size
            out[name] = arr.reshape(nz, ny, nx)
        elif words[0] == "VECTORS":
            arr = np.frombuffer(data, dtype=">f8", count=3 * n, offset=pos).astype(np.float64)
            pos += 24 * n
            out[words[1]] = np.ascontiguousarray(arr.reshape(n, 3).T).reshape(3, nz, ny, nx)
    return out
