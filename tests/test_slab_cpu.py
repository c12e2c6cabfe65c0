"""Z-slab decomposition (paper_2409_16781_gb300.slab) on the CPU.

The slab scheme -- plane ranges, ghosted inputs, the per-step exchange of
the c_z = +-1 populations with the z-neighbours over torch.distributed, and
the all-reduce of the totals -- runs here with slabs of the FP64 oracle as
the local lattices, in gloo ranks (world sizes 2 and 3) and in one process
(world size 1, the slab its own neighbour).  The slabs' populations after
the steps must equal the whole-lattice oracle's bitwise, and the summed
totals its totals to FP64 rounding.
"""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))

NX, NY, NZ, TAU, STEPS = 10, 9, 13, 0.62, 6
U_LID = (0.06, -0.02, 0.0)
FORCE = (2e-5, 1e-5, -3e-5)


def _inputs():
    from paper_2409_16781_gb300 import workloads as W
    flags = W.random_flags(NX, NY, NZ, seed=11, p_wall=0.12, p_lid=0.06)
    flags[:, :, 0] = W.FARFIELD
    rho, u = W.random_fields(NX, NY, NZ, seed=12)
    return flags, rho, u


def _whole():
    import oracle as O
    flags, rho, u = _inputs()
    ora = O.Lattice(NX, NY, NZ, TAU, u_lid=U_LID, flags=flags, force=FORCE)
    ora.init_fields(rho, u)
    ora.step(STEPS)
    return ora.A.copy(), ora.totals()


def _run_slab(rank, world, group=None):
    from paper_2409_16781_gb300.slab import SlabExchange
    from slab_oracle import OracleSlab
    flags, rho, u = _inputs()
    slab = OracleSlab(NX, NY, NZ, TAU, U_LID, flags, FORCE, rank, world)
    ex = SlabExchange(rank, world, group)
    slab.init_fields(rho, u)
    ex(slab)
    for _ in range(STEPS):
        slab.step()
        ex(slab)
    m, p = slab.own_totals()
    tot = ex.sum([m, p[0], p[1], p[2]])
    return slab.z0, slab.z1, slab.own_populations(), tot


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path[:0] = [ROOT, HERE]
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        q.put((rank,) + _run_slab(rank, world))
    finally:
        dist.destroy_process_group()


def _check(results):
    A, (mass, mom) = _whole()
    got = np.empty_like(A)
    covered = np.zeros(NZ, dtype=int)
    for _, z0, z1, pops, tot in results:
        got[:, z0:z1] = pops
        covered[z0:z1] += 1
        assert abs(tot[0] - mass) <= 1e-12 * mass
        assert np.abs(tot[1:] - mom).max() <= 1e-12 * mass
    assert (covered == 1).all()
    assert np.array_equal(got, A)


def test_slab_range_and_ghosts():
    from paper_2409_16781_gb300.slab import ghosted, slab_range
    for nz in (3, 7, 13, 256):
        for world in range(1, min(nz, 9) + 1):
            spans = [slab_range(nz, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == nz
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            lens = [b - a for a, b in spans]
            assert max(lens) - min(lens) <= 1 and min(lens) >= 1
    with pytest.raises(ValueError):
        slab_range(2, 3, 0)
    a = np.arange(5 * 2 * 3).reshape(5, 2, 3)
    g = ghosted(a, 0, 2)
    assert np.array_equal(g[0], a[4]) and np.array_equal(g[1:3], a[0:2]) and np.array_equal(g[3], a[2])
    v = np.arange(3 * 5 * 2 * 3).reshape(3, 5, 2, 3)
    gv = ghosted(v, 3, 5, axis=1)
    assert np.array_equal(gv[:, 0], v[:, 2]) and np.array_equal(gv[:, -1], v[:, 0])


def test_one_slab_is_its_own_neighbour():
    sys.path.insert(0, HERE)
    _check([(0,) + _run_slab(0, 1)])


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_over_gloo_ranks_equal_the_whole_lattice(world):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    results = [q.get(timeout=180) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    _check(results)


def test_bench_slab_inputs_are_the_ghosted_global_fields():
    """bench.py builds each z-slab's Taylor-Green fields without the whole
    lattice's arrays: they must equal the ghosted slices of the global ones."""
    sys.path.insert(0, ROOT)
    import bench
    from paper_2409_16781_gb300 import workloads as W
    from paper_2409_16781_gb300.slab import ghosted, slab_range
    n, world = 12, 3
    nz = n * world
    rho, u = W.taylor_green_fields(n, n, nz, u0=0.05)
    for r in range(world):
        z0, z1 = slab_range(nz, world, r)
        rl, ul = bench.tgv_slab_inputs(n, nz, z0, z1)
        assert np.allclose(rl, ghosted(rho, z0, z1), rtol=0, atol=0)
        assert np.allclose(ul, ghosted(u, z0, z1, axis=1), rtol=0, atol=1e-15)
