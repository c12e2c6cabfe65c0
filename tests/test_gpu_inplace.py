"""In-place lattices (lb_options.inplace = 1: one population array, the AA
access pattern) against the FP64 oracle and against the two-array scheme.

The in-place steps alternate two layouts of one array; after any number of
steps -- even or odd -- the exported populations, moments and totals are
those of the two-array update.  Tolerances as in the parity tests: f64
populations 1e-12 relative; the other forms velocity, max |du| / max |u|:
1e-5 (f32), 2e-3 (f16s), 3e-2 (bf16s), 1e-6 (f32d).  Against the two-array
one-cell-per-thread kernel (variant 1) the result is bitwise identical: both
run the same collision on the same pulled values.
"""
import numpy as np
import pytest

import oracle as O
from parity import fluid_mask, lib_to_oracle_perm, pop_rel_err, to_lib_order, vel_err
from paper_2409_16781_gb300 import Lattice, LbDiverged, bytes_required
from paper_2409_16781_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STORAGES = ["f64", "f32", "f16s", "bf16s", "f32d", "e3m12s"]
VEL_TOL = {"f32": 1e-5, "f16s": 2e-3, "bf16s": 3e-2, "f32d": 1e-6, "e3m12s": 5e-4}


@pytest.fixture(scope="module")
def perm():
    return lib_to_oracle_perm()


def _check(ora, gpu, storage, perm, flags):
    mask = fluid_mask(flags, gpu.shape)
    rho_o, u_o = ora.moments()
    rho_g, u_g = gpu.moments()
    if storage == "f64":
        assert pop_rel_err(gpu.populations(), to_lib_order(ora.A, perm), mask) <= 1e-12
        assert vel_err(u_g, u_o, mask) <= 1e-11
    else:
        assert vel_err(u_g, u_o, mask) <= VEL_TOL[storage]
    assert np.all(rho_g[~mask] == 0) and np.all(u_g[:, ~mask] == 0)


CASES = [
    # nx, ny, nz, tau, flags-spec, u_lid, force
    (1, 1, 1, 0.7, None, (0, 0, 0), (1e-4, -2e-4, 3e-4)),
    (3, 5, 7, 0.65, ("random", 9), (0.05, 0.02, 0.0), (1e-4, 0, -1e-4)),
    (17, 9, 4, 0.8, ("random", 4), (0.08, 0.0, 0.01), (0, 0, 0)),
    (33, 5, 3, 0.55, None, (0, 0, 0), (2e-5, 1e-5, 0)),
    (70, 3, 2, 0.9, ("cavity", 0), (0.1, 0, 0), (0, 0, 0)),
    (66, 5, 4, 0.7, ("random", 22), (0.02, 0.0, 0.0), (5e-5, 0, 1e-4)),
    # nx a multiple of 64 up to 1024: 16-bit rows from the swapped layout in
    # one block each -- all-fluid rows (aligned stores only), rows with walls
    # (the general stores), a mix, and the largest block (16 warps)
    (128, 4, 3, 0.6, None, (0, 0, 0), (1e-5, 2e-5, 0)),
    (64, 6, 5, 0.7, ("random", 5), (0.04, 0.0, 0.01), (3e-5, 0, -2e-5)),
    (64, 7, 6, 0.75, ("sparse", 8), (0.03, 0.0, 0.0), (0, 0, 0)),
    (1024, 2, 3, 0.65, None, (0, 0, 0), (0, 1e-5, 0)),
    (192, 3, 4, 0.65, ("sparse", 3), (0.02, 0.01, 0.0), (0, 0, 0)),
]


def _flags(spec, nx, ny, nz):
    if spec is None:
        return None
    kind, seed = spec
    if kind == "random":
        return W.random_flags(nx, ny, nz, seed=seed, p_wall=0.2, p_lid=0.1)
    if kind == "sparse":  # about half the 64-cell rows without a wall
        return W.random_flags(nx, ny, nz, seed=seed, p_wall=0.01, p_lid=0.005)
    return W.cavity_flags(nx, ny, nz)


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("steps", [1, 2, 7, 12])
@pytest.mark.parametrize("storage", STORAGES)
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}x{c[2]}")
def test_inplace_matches_oracle_and_two_arrays(case, storage, steps, kernel, perm):
    """Kernel 2 (two cells per thread, packed FP32) applies to FP32 and
    16-bit storage with even nx; elsewhere it runs the one-cell kernel."""
    nx, ny, nz, tau, spec, ulid, g = case
    flags = _flags(spec, nx, ny, nz)
    rho0, u0 = W.random_fields(nx, ny, nz, seed=nx * 100 + ny * 10 + nz, du=0.06, drho=0.02)
    ora = O.Lattice(nx, ny, nz, tau, u_lid=ulid, flags=flags, force=g)
    ora.init_fields(rho0, u0)
    aa = Lattice(nx, ny, nz, tau, u_lid=ulid, flags=flags, storage=storage, force=g, inplace=True, kernel=kernel)
    ab = Lattice(nx, ny, nz, tau, u_lid=ulid, flags=flags, storage=storage, force=g, kernel=1)
    for lat in (aa, ab):
        lat.init_fields(rho0, u0)
        lat.step(steps)
    ora.step(steps)
    _check(ora, aa, storage, perm, flags)
    mask = fluid_mask(flags, aa.shape)
    assert np.array_equal(aa.populations()[:, mask], ab.populations()[:, mask])
    ma, pa = aa.totals()
    mb, pb = ab.totals()
    assert ma == mb and np.array_equal(pa, pb)
    aa.close()
    ab.close()


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("trt", [0.0, 3 / 16])
@pytest.mark.parametrize("steps", [500, 501])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
def test_inplace_cavity_32(storage, steps, trt, kernel, perm):
    """32^3 lid-driven cavity (tau 0.6, lid (0.1,0,0)), an even and an odd
    number of steps, BGK and TRT, one and two cells per thread."""
    n = 32
    flags = W.cavity_flags(n, n, n)
    om = O.trt_omega_minus(0.6, trt) if trt else None
    ora = O.Lattice(n, n, n, 0.6, u_lid=(0.1, 0, 0), flags=flags, omega_minus=om)
    aa = Lattice(n, n, n, 0.6, u_lid=(0.1, 0, 0), flags=flags, storage=storage, inplace=True, trt_magic=trt,
                 kernel=kernel)
    ora.step(steps)
    aa.step(steps)
    _check(ora, aa, storage, perm, flags)
    m_o, p_o = ora.totals()
    m_g, p_g = aa.totals()
    if storage == "f64":
        assert abs(m_g - m_o) <= 1e-12 * m_o and np.abs(p_g - p_o).max() <= 1e-12 * m_o


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
def test_inplace_taylor_green_and_porous(storage, perm):
    n = 48
    rho0, u0 = W.taylor_green_fields(n, n, n, u0=0.05)
    ora = O.Lattice(n, n, n, 0.55)
    ora.init_fields(rho0, u0)
    aa = Lattice(n, n, n, 0.55, storage=storage, inplace=True)
    aa.init_fields(rho0, u0)
    ora.step(61)
    aa.step(61)
    _check(ora, aa, storage, perm, None)
    nx, ny, nz = 40, 36, 32
    flags = W.porous_flags(nx, ny, nz, n_spheres=10, r_min=3, r_max=6, seed=2409)
    ora = O.Lattice(nx, ny, nz, 0.8, flags=flags, force=(1e-5, 0, 0))
    aa = Lattice(nx, ny, nz, 0.8, flags=flags, storage=storage, force=(1e-5, 0, 0), inplace=True)
    ora.step(101)
    aa.step(101)
    _check(ora, aa, storage, perm, flags)


@pytest.mark.parametrize("storage", STORAGES)
def test_inplace_populations_in_both_layouts(storage, perm):
    """Export/import and sampled reads after an even and an odd number of
    steps; import resets the layout; an arbitrary state steps like the
    oracle."""
    nx, ny, nz = 13, 8, 6
    flags = W.random_flags(nx, ny, nz, seed=12, p_wall=0.15, p_lid=0.1)
    mask = fluid_mask(flags, (nz, ny, nx))
    _, w = O.velocity_set()
    f = W.random_populations(nx, ny, nz, seed=5, w=w, amp=0.02)  # oracle order
    ora = O.Lattice(nx, ny, nz, 0.75, u_lid=(0.03, -0.02, 0.01), flags=flags, force=(1e-4, 0, 2e-4))
    ora.set_populations(f)
    aa = Lattice(nx, ny, nz, 0.75, u_lid=(0.03, -0.02, 0.01), flags=flags, storage=storage,
                 force=(1e-4, 0, 2e-4), inplace=True)
    aa.set_populations(to_lib_order(f, perm))
    cells = np.array([0, 7, 66, 300, nx * ny * nz - 1])
    for k in range(4):
        g = aa.populations()
        at = aa.populations_at(cells)
        assert np.array_equal(at, g.reshape(19, -1)[:, cells].T)
        if storage == "f64":
            assert pop_rel_err(g, to_lib_order(ora.A, perm), mask) <= 1e-13
        # re-importing the exported state changes nothing, in either layout
        aa.set_populations(g)
        assert np.array_equal(aa.populations()[:, mask], g[:, mask])
        ora.step(1)
        aa.step(1)
    _check(ora, aa, storage, perm, flags)


def test_inplace_init_fields_midway_and_rest_state(perm):
    nx, ny, nz = 20, 9, 7
    flags = W.random_flags(nx, ny, nz, seed=3, p_wall=0.1, p_lid=0.0)
    aa = Lattice(nx, ny, nz, 0.6, flags=flags, storage="f32", inplace=True)
    f0 = aa.populations()
    aa.step(25)  # rest state, no lid motion, no force: stays exactly at rest
    assert np.array_equal(aa.populations(), f0)
    rho0, u0 = W.random_fields(nx, ny, nz, seed=9, du=0.04, drho=0.01)
    aa.step(1)  # odd layout, then re-initialise
    aa.init_fields(rho0, u0)
    ora = O.Lattice(nx, ny, nz, 0.6, flags=flags)
    ora.init_fields(rho0, u0)
    aa.step(9)
    ora.step(9)
    _check(ora, aa, "f32", perm, flags)


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_inplace_autotune_keeps_state(storage, perm, tmp_path, monkeypatch):
    monkeypatch.setenv("LBGB_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    nx, ny, nz = 64, 12, 10
    flags = W.random_flags(nx, ny, nz, seed=31, p_wall=0.05, p_lid=0.02)
    aa = Lattice(nx, ny, nz, 0.6, u_lid=(0.05, 0, 0), flags=flags, storage=storage, inplace=True)
    aa.step(3)  # odd layout
    f0 = aa.populations()
    v, b, ms = aa.autotune(reps=3)
    assert v in (1, 2) and b in (32, 64, 128, 256, 512) and ms > 0
    assert np.array_equal(aa.populations(), f0)
    ora = O.Lattice(nx, ny, nz, 0.6, u_lid=(0.05, 0, 0), flags=flags)
    ora.step(3)
    ora.step(20)
    aa.step(20)
    _check(ora, aa, storage, perm, flags)


def test_inplace_memory_and_divergence():
    n = 16
    # exactly one population array less (19 planes of 16^3 FP32 values)
    assert bytes_required(n, n, n, "f32") - bytes_required(n, n, n, "f32", inplace=True) == 19 * n ** 3 * 4
    aa = Lattice(n, n, n, 0.7, storage="f32", inplace=True)
    aa.step(1)
    f = aa.populations()
    f[3, 2, 2, 2] = np.nan
    aa.set_populations(f)
    aa.step(1)
    with pytest.raises(LbDiverged):
        aa.totals()


@pytest.mark.parametrize("kernel", [1, 2])
@pytest.mark.parametrize("steps", [300, 301])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16s"])
def test_inplace_flow_past_cylinder(storage, steps, kernel, perm):
    """Far-field inflow / outflow planes in place: a pull from a far-field
    cell reads no memory, so the in-place ownership argument still holds."""
    nx, ny, nz, D = 64, 32, 3, 8
    flags = W.cylinder_flags(nx, ny, nz, diameter=D, cx=2 * D, cy=ny / 2 + 0.5)
    ora = O.Lattice(nx, ny, nz, 0.6, u_lid=(0.05, 0.0, 0.0), flags=flags)
    aa = Lattice(nx, ny, nz, 0.6, u_lid=(0.05, 0.0, 0.0), flags=flags, storage=storage, inplace=True,
                 kernel=kernel)
    ora.step(steps)
    aa.step(steps)
    _check(ora, aa, storage, perm, flags)
