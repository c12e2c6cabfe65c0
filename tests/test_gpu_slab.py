"""Z-slab lattices (lb_options.halo_z, lb_halo_pack / lb_halo_unpack) on one GPU.

Two to four slabs of one lattice live in one process on one GPU and trade
their halo planes directly (a ring of device buffers, no process group):
after every step each slab packs, then each unpacks its neighbours'
messages.  Nothing waits on anything else on the device; this is the
exchange that SlabExchange runs between GPUs, with the messages handed over
in place of sent.  The slabs' own planes must equal the whole lattice run by
the same kernel bitwise, for every storage form and several step variants,
the summed FP64 totals its totals, and (FP64) the oracle to 1e-12.
"""
import numpy as np
import pytest

import oracle as O
from parity import lib_to_oracle_perm, pop_rel_err, to_lib_order
from paper_2409_16781_gb300 import Lattice
from paper_2409_16781_gb300 import workloads as W
from paper_2409_16781_gb300.slab import SlabLattice, slab_range

pytestmark = pytest.mark.gpu

NX, NY, NZ, TAU = 36, 9, 14, 0.62
U_LID = (0.06, -0.02, 0.0)
FORCE = (2e-5, 1e-5, -3e-5)


class _Nothing:
    def __call__(self, local):
        pass

    def sum(self, values):
        return np.asarray(values, dtype=np.float64)


def _ring(slabs):
    for s in slabs:
        lo, hi, _, _ = s.halo_buffers()
        s.halo_pack(lo, hi)
    W_ = len(slabs)
    for r, s in enumerate(slabs):
        below, above = slabs[(r - 1) % W_], slabs[(r + 1) % W_]
        s.halo_unpack(below.halo_buffers()[1], above.halo_buffers()[0])


def _inputs():
    flags = W.random_flags(NX, NY, NZ, seed=21, p_wall=0.1, p_lid=0.05)
    flags[:, :, 0] = W.FARFIELD
    rho, u = W.random_fields(NX, NY, NZ, seed=22)
    return flags, rho, u


def _run(storage, variant, world, steps):
    import torch
    flags, rho, u = _inputs()
    whole = Lattice(NX, NY, NZ, TAU, u_lid=U_LID, flags=flags, storage=storage, force=FORCE, kernel=variant)
    whole.init_fields(rho, u)
    slabs = [SlabLattice(NX, NY, NZ, TAU, u_lid=U_LID, flags=flags, storage=storage, force=FORCE, rank=r,
                         world=world, exchange=_Nothing(), kernel=variant) for r in range(world)]
    for s in slabs:
        s.lattice.init_fields(*_ghosted_fields(s, rho, u))
    _ring(slabs)
    for _ in range(steps):
        whole.step(1)
        for s in slabs:
            s.lattice.step(1)
        _ring(slabs)
    torch.cuda.synchronize()
    return whole, slabs


def _ghosted_fields(s, rho, u):
    from paper_2409_16781_gb300.slab import ghosted
    return ghosted(rho, s.z0, s.z1), ghosted(u, s.z0, s.z1, axis=1)


@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s", "f32d", "e3m12s"])
@pytest.mark.parametrize("world", [2, 3])
def test_slabs_equal_whole_lattice(storage, world):
    whole, slabs = _run(storage, 0, world, 7)
    f = whole.populations()
    mass, mom = whole.totals()
    m_sum, p_sum = 0.0, np.zeros(3)
    for s in slabs:
        assert np.array_equal(s.own_populations(), f[:, s.z0:s.z1])
        m, p = s.lattice.totals()
        m_sum += m
        p_sum += p
        rho, u = s.own_moments()
        wr, wu = whole.moments()
        assert np.array_equal(rho, wr[s.z0:s.z1]) and np.array_equal(u, wu[:, s.z0:s.z1])
    # FP32 arithmetic: each thread sums several cells in FP32 before the FP64
    # fold, and the slabs group their cells differently from the whole lattice
    tol = 1e-12 if storage in ("f64", "f32d") else 1e-9
    assert abs(m_sum - mass) <= tol * mass
    assert np.abs(p_sum - mom).max() <= tol * mass


@pytest.mark.parametrize("storage,variant", [("f32", 1), ("f32", 4), ("f32", 13), ("f32", 16),
                                             ("f16s", 15), ("f16s", 17), ("f16s", 8), ("bf16s", 6)])
def test_slab_variants(storage, variant):
    whole, slabs = _run(storage, variant, 4, 5)
    f = whole.populations()
    for s in slabs:
        assert np.array_equal(s.own_populations(), f[:, s.z0:s.z1])


def test_f64_slabs_match_the_oracle():
    flags, rho, u = _inputs()
    _, slabs = _run("f64", 0, 3, 9)
    ora = O.Lattice(NX, NY, NZ, TAU, u_lid=U_LID, flags=flags, force=FORCE)
    ora.init_fields(rho, u)
    ora.step(9)
    perm = lib_to_oracle_perm()
    ref = to_lib_order(ora.A, perm)
    fluid = flags == 0
    for s in slabs:
        assert pop_rel_err(s.own_populations(), ref[:, s.z0:s.z1], fluid[s.z0:s.z1]) <= 1e-12


def test_halo_arguments():
    import torch
    from paper_2409_16781_gb300 import LbError
    lat = Lattice(8, 4, 6, 0.7)
    assert lat.halo_bytes() == 0
    buf = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(LbError):
        lat.halo_pack(buf, buf)
    with pytest.raises(LbError):
        Lattice(8, 4, 2, 0.7, halo_z=True)
    with pytest.raises(LbError):
        Lattice(8, 4, 6, 0.7, halo_z=True, inplace=True)
    s = Lattice(8, 4, 6, 0.7, storage="f16s", halo_z=True)
    assert s.halo_bytes() == 5 * 8 * 4 * 2
    assert slab_range(14, 3, 1) == (5, 10)
