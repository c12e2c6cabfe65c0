"""Stochastic rounding of 16-bit stored deviations (lb_options.rounding = 1).

* The random bits are a function of (cell, direction, steps taken) only, so
  every step variant, the in-place kernels and a batch slot give bitwise the
  same state, and a checkpoint restart is bit-exact.
* Round-to-nearest loses a body-force increment that is below half a unit in
  the last place of the stored values; stochastic rounding keeps it on
  average.  In a forced periodic box the FP64 momentum must grow by mass * g
  per step (exact for the update in exact arithmetic): within 1 % with
  stochastic rounding, while nearest rounding falls far short.
* Against the FP64 oracle on the 64^3 cavity over 1000 steps the FP16 form
  stays within the FP16S tolerance 2e-3 of max |u|, the E3M12 form within
  5e-4.
"""
import numpy as np
import pytest

import oracle as O
from parity import fluid_mask, vel_err
from paper_2409_16781_gb300 import Lattice, LbError
from paper_2409_16781_gb300 import workloads as W
from paper_2409_16781_gb300.batch import Batch

pytestmark = pytest.mark.gpu

DIMS = (38, 11, 9)
TAU = 0.58


def _case():
    nx, ny, nz = DIMS
    flags = W.random_flags(nx, ny, nz, seed=5, p_wall=0.08, p_lid=0.04)
    flags[:, :, 0] = W.FARFIELD
    rho, u = W.random_fields(nx, ny, nz, seed=6)
    return flags, rho, u


def _run(storage, variant=0, steps=13, inplace=False, force=(3e-5, 0.0, 1e-5)):
    flags, rho, u = _case()
    lat = Lattice(*DIMS, TAU, u_lid=(0.07, 0.0, 0.0), flags=flags, storage=storage, force=force,
                  kernel=variant, inplace=inplace, rounding="stochastic")
    lat.init_fields(rho, u)
    lat.step(steps)
    return lat


@pytest.mark.parametrize("storage", ["f16s", "bf16s", "e3m12s"])
def test_every_variant_rounds_alike(storage):
    ref = _run(storage, 1).populations()
    for v in (0, 2, 3, 4, 6, 8, 13, 14, 15, 16, 17, 18, 19):
        assert np.array_equal(_run(storage, v).populations(), ref), f"variant {v}"
    for v in (1, 2):
        for steps in (12, 13):
            a = _run(storage, v, steps=steps, inplace=True).populations()
            b = _run(storage, 1, steps=steps).populations()
            fl = _case()[0] == 0
            assert np.array_equal(a[:, fl], b[:, fl]), f"in place variant {v}, {steps} steps"


@pytest.mark.parametrize("storage", ["f16s", "bf16s", "e3m12s"])
def test_stochastic_differs_from_nearest_and_is_reproducible(storage):
    a = _run(storage, 15).populations()
    b = _run(storage, 15).populations()
    assert np.array_equal(a, b)
    flags, rho, u = _case()
    rn = Lattice(*DIMS, TAU, u_lid=(0.07, 0.0, 0.0), flags=flags, storage=storage, force=(3e-5, 0.0, 1e-5))
    rn.init_fields(rho, u)
    rn.step(13)
    assert not np.array_equal(a, rn.populations())


def test_checkpoint_restart_is_bit_exact():
    full = _run("f16s", 15, steps=20).populations()
    part = _run("f16s", 15, steps=8)
    snap = part.checkpoint()
    flags, _, _ = _case()
    fresh = Lattice(*DIMS, TAU, u_lid=(0.07, 0.0, 0.0), flags=flags, storage="f16s", force=(3e-5, 0.0, 1e-5),
                    rounding="stochastic")
    fresh.restore(snap)
    fresh.step(12)
    assert np.array_equal(fresh.populations(), full)


def test_batch_slot_equals_lattice_alone():
    flags, rho, u = _case()
    alone = _run("f16s", 0, steps=11).populations()
    with Batch(capacity_bytes=64 << 20, max_slots=8) as b:
        other = b.add(20, 6, 7, 0.7, storage="f16s", steps=11, rounding="stochastic")
        s = b.add(*DIMS, TAU, u_lid=(0.07, 0.0, 0.0), flags=flags, storage="f16s", force=(3e-5, 0.0, 1e-5),
                  steps=11, rounding="stochastic")
        b.init_fields(s, rho, u)
        b.step(11)
        b.sync()
        got = b.populations(s)
        assert other >= 0
    assert np.array_equal(got, alone)


@pytest.mark.parametrize("storage", ["f16s", "bf16s", "e3m12s"])
def test_weak_force_is_kept_on_average(storage):
    """Periodic box, all fluid, at rest, g = 2e-7 along x: the FP64 momentum
    grows by exactly mass * g per step in exact arithmetic."""
    n, steps, g = 32, 1500, 2e-7
    res = {}
    for rounding in ("nearest", "stochastic"):
        lat = Lattice(n, n, n, 0.8, storage=storage, force=(g, 0.0, 0.0), rounding=rounding)
        m0, p0 = lat.totals()
        lat.step(steps)
        m, p = lat.totals()
        res[rounding] = (p[0] - p0[0]) / (m0 * g * steps)
    assert abs(res["stochastic"] - 1.0) < 0.01, res
    assert abs(res["nearest"] - 1.0) > 0.05, res


def test_cavity_64_against_oracle():
    n, steps = 64, 1000
    fl = W.cavity_flags(n, n, n)
    ora = O.Lattice(n, n, n, 0.6, u_lid=(0.1, 0, 0), flags=fl)
    ora.step(steps)
    _, u_o = ora.moments()
    for storage, tol in (("f16s", 2e-3), ("e3m12s", 5e-4)):
        lat = Lattice(n, n, n, 0.6, u_lid=(0.1, 0, 0), flags=fl, storage=storage, rounding="stochastic")
        lat.step(steps)
        _, u_g = lat.moments()
        assert vel_err(u_g, u_o, fluid_mask(fl, u_o.shape[1:])) <= tol, storage


def test_rounding_needs_16_bit_storage():
    with pytest.raises(LbError):
        Lattice(8, 4, 4, 0.7, storage="f32", rounding="stochastic")
    with pytest.raises(LbError):
        Lattice(8, 4, 4, 0.7, storage="f16s", rounding=2)
