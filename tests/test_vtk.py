"""Legacy-VTK output of the fields (host file I/O): round trip, the header
a VTK reader expects, big-endian binary payloads."""
import numpy as np
import pytest

from paper_2409_16781_gb300.vtk import read_vtk, write_vtk


def test_round_trip_exact(tmp_path):
    rng = np.random.default_rng(7)
    nz, ny, nx = 3, 4, 5
    rho = 1 + 0.01 * rng.standard_normal((nz, ny, nx))
    u = 0.05 * rng.standard_normal((3, nz, ny, nx))
    flags = rng.integers(0, 4, (nz, ny, nx)).astype(np.uint8)
    p = tmp_path / "f.vtk"
    write_vtk(str(p), rho, u, flags, spacing=(0.5, 0.5, 2.0), origin=(1.0, 0.0, -1.0))
    r = read_vtk(str(p))
    assert r["dims"] == (nx, ny, nz) and r["spacing"] == (0.5, 0.5, 2.0) and r["origin"] == (1.0, 0.0, -1.0)
    assert np.array_equal(r["rho"], rho) and np.array_equal(r["u"], u) and np.array_equal(r["flags"], flags)


def test_header_and_byte_order(tmp_path):
    rho = np.arange(6, dtype=np.float64).reshape(1, 2, 3)
    u = np.zeros((3, 1, 2, 3))
    u[0, 0, 1, 2] = 0.25     # the last point (x = 2, y = 1)
    p = tmp_path / "g.vtk"
    write_vtk(str(p), rho, u)
    data = p.read_bytes()
    head = data[:data.index(b"LOOKUP_TABLE")].decode("ascii").splitlines()
    assert head[0] == "# vtk DataFile Version 3.0"
    assert head[2:6] == ["BINARY", "DATASET STRUCTURED_POINTS", "DIMENSIONS 3 2 1", "ORIGIN 0 0 0"]
    assert "POINT_DATA 6" in head and "SCALARS rho double 1" in head
    # rho payload: points in x-fastest order, big-endian doubles
    start = data.index(b"LOOKUP_TABLE default\n") + len(b"LOOKUP_TABLE default\n")
    assert np.array_equal(np.frombuffer(data[start:start + 48], ">f8"), np.arange(6.0))
    # u payload: (ux, uy, uz) per point; the last triple is (0.25, 0, 0)
    vstart = data.index(b"VECTORS u double\n") + len(b"VECTORS u double\n")
    trip = np.frombuffer(data[vstart:vstart + 144], ">f8").reshape(6, 3)
    assert trip[5].tolist() == [0.25, 0.0, 0.0] and not trip[:5].any()
    assert b"flags" not in data


def test_bad_shapes_rejected(tmp_path):
    with pytest.raises(ValueError):
        write_vtk(str(tmp_path / "a.vtk"), np.ones((2, 2)), np.zeros((3, 2, 2)))
    with pytest.raises(ValueError):
        write_vtk(str(tmp_path / "b.vtk"), np.ones((2, 2, 2)), np.zeros((3, 2, 2, 3)))
    with pytest.raises(ValueError):
        write_vtk(str(tmp_path / "c.vtk"), np.ones((2, 2, 2)), np.zeros((3, 2, 2, 2)), flags=np.zeros(7))
