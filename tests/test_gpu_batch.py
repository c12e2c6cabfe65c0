"""Batches of lattices (lb_batch_*): every lattice gives the same result alone
and in the mix, per-slot step budgets, the captured-graph path, HBM-budget
admission, and the serving loop end to end.

Tolerances as in the parity tests: f64 populations 1e-12 relative; the
others compare velocity fields, max |du| / max |u| <= 1e-5 (f32), 2e-3
(f16s), 3e-2 (bf16s).  A lattice alone runs through lb_step (one thread per
cell, variant 1); in the batch it runs the batched kernel with other
lattices of other sizes and storage types.
"""
import numpy as np
import pytest

import oracle as O
from parity import fluid_mask, lib_to_oracle_perm, pop_rel_err, to_lib_order, vel_err
from paper_2409_16781_gb300 import Lattice, LbError
from paper_2409_16781_gb300 import _lib as L
from paper_2409_16781_gb300 import workloads as W
from paper_2409_16781_gb300.batch import Batch, slot_bytes
from paper_2409_16781_gb300.serve import BatchBackend, SequentialBackend, serve

pytestmark = pytest.mark.gpu

VEL_TOL = {"f32": 1e-5, "f16s": 2e-3, "bf16s": 3e-2, "f32d": 1e-6, "e3m12s": 5e-4}
# relative mass agreement: the storage rounding of each deviation bounds how
# closely two kernels' conserved sums agree (16-bit: about one ulp per cell)
MASS_TOL = {"f64": 1e-12, "f32": 1e-8, "f16s": 1e-5, "bf16s": 1e-4, "f32d": 1e-8, "e3m12s": 1e-5}

MIX = [
    # nx, ny, nz, tau, storage, kind, steps
    (17, 12, 9, 0.7, "f32", "cavity", 40),
    (32, 20, 16, 0.56, "f16s", "channel", 33),
    (9, 7, 13, 0.9, "f64", "cavity", 25),
    (40, 10, 12, 0.6, "bf16s", "channel", 30),
    (22, 14, 10, 0.62, "e3m12s", "cavity", 27),
    (24, 24, 24, 0.52, "f32", "channel", 57),
    (5, 31, 6, 0.8, "f16s", "cavity", 11),
    (64, 3, 2, 0.65, "f32", "random", 21),
    (15, 11, 7, 0.75, "f32d", "cavity", 19),
    (30, 12, 3, 0.6, "f32", "cylinder", 45),
    (28, 12, 4, 0.6, "f16s", "cylinder", 38),
]


def _geom(nx, ny, nz, kind):
    if kind == "cavity":
        return W.cavity_flags(nx, ny, nz), (0.06, 0.0, 0.0), (0.0, 0.0, 0.0)
    if kind == "cylinder":
        return (W.cylinder_flags(nx, ny, nz, diameter=ny / 3, cx=nx / 3, cy=ny / 2 + 0.5), (0.05, 0.0, 0.0),
                (0.0, 0.0, 0.0))
    if kind == "channel":
        return W.channel_flags(nx, ny, nz, walls=("y", "z")), (0.0, 0.0, 0.0), (2e-5, 0.0, 0.0)
    return W.random_flags(nx, ny, nz, seed=nx, p_wall=0.1, p_lid=0.05), (0.03, 0.01, 0.0), (1e-5, 0, 1e-5)


def _compare(f_batch, f_alone, u_batch, u_alone, storage, flags, shape):
    mask = fluid_mask(flags, shape)
    if storage == "f64":
        assert pop_rel_err(f_batch, f_alone, mask) <= 1e-12
    else:
        assert vel_err(u_batch, u_alone, mask) <= VEL_TOL[storage]


def test_same_alone_and_in_the_mix():
    b = Batch(capacity_bytes=64 << 20, max_slots=16)
    slots = []
    for nx, ny, nz, tau, storage, kind, steps in MIX:
        flags, ulid, g = _geom(nx, ny, nz, kind)
        s = b.add(nx, ny, nz, tau, steps, u_lid=ulid, flags=flags, storage=storage, force=g)
        slots.append(s)
    b.step(60)          # more than any budget: each slot stops at its own count
    done = set(b.poll())
    assert done == set(slots)
    bitwise = 0
    for s, (nx, ny, nz, tau, storage, kind, steps) in zip(slots, MIX):
        q = b.query(s)
        assert q["done"] == steps and q["remaining"] == 0
        flags, ulid, g = _geom(nx, ny, nz, kind)
        alone = Lattice(nx, ny, nz, tau, u_lid=ulid, flags=flags, storage=storage, force=g, kernel=1)
        alone.step(steps)
        fb, fa = b.populations(s), alone.populations()
        _, ub = b.moments(s)
        _, ua = alone.moments()
        _compare(fb, fa, ub, ua, storage, flags, alone.shape)
        mask = fluid_mask(flags, alone.shape)
        bitwise += int(np.array_equal(fb[:, mask], fa[:, mask]))
        mb, _ = b.totals(s)
        ma, _ = alone.totals()
        assert abs(mb - ma) <= MASS_TOL[storage] * ma
        alone.close()
    print(f"bitwise-identical slots: {bitwise}/{len(MIX)}")
    b.close()


def test_batch_matches_oracle_f64():
    perm = lib_to_oracle_perm()
    b = Batch(capacity_bytes=16 << 20, max_slots=4)
    cases = [(11, 9, 7, 0.65, "cavity", 30), (16, 6, 10, 0.8, "random", 19)]
    slots = []
    for nx, ny, nz, tau, kind, steps in cases:
        flags, ulid, g = _geom(nx, ny, nz, kind)
        slots.append(b.add(nx, ny, nz, tau, steps, u_lid=ulid, flags=flags, storage="f64", force=g))
    b.step(31)
    for s, (nx, ny, nz, tau, kind, steps) in zip(slots, cases):
        flags, ulid, g = _geom(nx, ny, nz, kind)
        ora = O.Lattice(nx, ny, nz, tau, u_lid=ulid, flags=flags, force=g)
        ora.step(steps)
        err = pop_rel_err(b.populations(s), to_lib_order(ora.A, perm), fluid_mask(flags, (nz, ny, nx)))
        assert err <= 1e-12
    b.close()


def test_batch_trt_matches_oracle():
    """Slots with the two-relaxation-time collision (per-slot magic
    parameter) next to a BGK slot, against the oracle's TRT / BGK steps."""
    perm = lib_to_oracle_perm()
    b = Batch(capacity_bytes=16 << 20, max_slots=4)
    cases = [(11, 9, 7, 0.52, "cavity", 30, 3 / 16), (16, 6, 10, 0.8, "random", 19, 1 / 4),
             (12, 8, 6, 0.7, "channel", 25, 0.0)]
    slots = []
    for nx, ny, nz, tau, kind, steps, magic in cases:
        flags, ulid, g = _geom(nx, ny, nz, kind)
        slots.append(b.add(nx, ny, nz, tau, steps, u_lid=ulid, flags=flags, storage="f64", force=g,
                           trt_magic=magic))
    b.step(31)
    for s, (nx, ny, nz, tau, kind, steps, magic) in zip(slots, cases):
        flags, ulid, g = _geom(nx, ny, nz, kind)
        om = O.trt_omega_minus(tau, magic) if magic else None
        ora = O.Lattice(nx, ny, nz, tau, u_lid=ulid, flags=flags, force=g, omega_minus=om)
        ora.step(steps)
        err = pop_rel_err(b.populations(s), to_lib_order(ora.A, perm), fluid_mask(flags, (nz, ny, nx)))
        assert err <= 1e-12
    b.close()


def test_graph_path_and_init_fields():
    """Step counts above the graph size (8) replay captured graphs; the
    result equals the single-lattice run."""
    nx, ny, nz = 20, 14, 12
    rho0, u0 = W.random_fields(nx, ny, nz, seed=4, du=0.04, drho=0.01)
    b = Batch(capacity_bytes=16 << 20, max_slots=4)
    s = b.add(nx, ny, nz, 0.6, 1000, storage="f32")
    b.init_fields(s, rho0, u0)
    b.step(8 * 5 + 3)
    assert b.query(s)["done"] == 43
    alone = Lattice(nx, ny, nz, 0.6, storage="f32", kernel=1)
    alone.init_fields(rho0, u0)
    alone.step(43)
    _, ub = b.moments(s)
    _, ua = alone.moments()
    assert vel_err(ub, ua, np.ones((nz, ny, nx), bool)) <= 1e-5
    b.close()


def test_admission_limits():
    nbytes = slot_bytes(16, 16, 16, "f32")
    small_bytes = slot_bytes(4, 4, 4, "f32")
    assert small_bytes < nbytes
    b = Batch(capacity_bytes=2 * nbytes + small_bytes, max_slots=3)
    s0 = b.add(16, 16, 16, 0.7, 10)
    s1 = b.add(16, 16, 16, 0.7, 10)
    with pytest.raises(LbError) as e:
        b.add(16, 16, 16, 0.7, 10)
    assert e.value.status == L.LB_ENOMEM
    assert b.try_add(16, 16, 16, 0.7, 10) is None
    small = b.add(4, 4, 4, 0.7, 10)          # still fits
    with pytest.raises(LbError) as e:
        b.add(2, 2, 2, 0.7, 10)
    assert e.value.status == L.LB_EBUSY       # 3 slots in use
    b.remove(s0)
    s2 = b.add(16, 16, 16, 0.7, 10)           # memory and slot came back
    assert s2 == s0
    b.step(10)
    assert set(b.poll()) == {s1, s2, small}
    for s in (s1, s2, small):
        b.remove(s)
    free_bytes, free_slots = b.free()
    assert free_slots == 3 and free_bytes == 2 * nbytes + small_bytes  # fully coalesced
    b.close()


def _same_fields_as_alone(results, reqs):
    """Each served request's rho and u against the same request run alone
    by the one-at-a-time baseline (same storage), element by element over
    its fluid cells."""
    got = {r.rid: r.fields for r in results}
    for req in reqs:
        st1 = serve([req], SequentialBackend(storage=req.storage, keep_fields=True))
        rho_a, u_a = st1.results[0].fields
        rho_b, u_b = got[req.rid]
        mask = req.flags() == 0
        tol = VEL_TOL[req.storage]
        assert vel_err(u_b, u_a, mask) <= tol, (req.rid, req.storage)
        assert np.abs(rho_b[mask] - rho_a[mask]).max() <= tol * np.abs(rho_a[mask]).max(), req.rid
        assert np.abs(u_a[:, mask]).max() > 0


@pytest.mark.parametrize("policy", ["fifo", "srpt"])
def test_serve_end_to_end_same_as_sequential(policy):
    """A small request stream through the batched server and through the
    one-at-a-time baseline (same storage per request) gives the same rho and
    u fields element by element, and every request completes."""
    reqs = W.request_stream(n=10, rate_hz=200.0, seed=5, min_cells=6 ** 3, max_cells=20 ** 3,
                            steps_range=(20, 120))
    be = BatchBackend(capacity_bytes=128 << 20, max_slots=8, keep_fields=True)
    st = serve(reqs, be, chunk_ms=2.0, policy=policy, target_cells=5000)
    be.close()
    assert len(st.results) == len(reqs) and not st.rejected
    _same_fields_as_alone(st.results, reqs)
    s = st.summary()
    assert s["requests"] == len(reqs) and s["p99_s"] >= s["p50_s"]


class _CountingBackend(BatchBackend):
    """Records every positive quota the scheduler grants: per request, the
    list of (chunk number, quota)."""

    def __init__(self, *a, **kw):
        super().__init__(*a, **kw)
        self.grants = {}
        self.slot_rid = {}
        self.chunk = 0
        self.clock = None

    def admit(self, req):
        h = super().admit(req)
        if h is not None:
            self.slot_rid[h] = req.rid
            self.grants[req.rid] = []
        return h

    def set_quotas(self, quotas):
        for h, q in quotas.items():
            if q > 0:
                self.grants[self.slot_rid[h]].append((self.chunk, int(q)))
        super().set_quotas(quotas)

    def step(self, n):
        super().step(n)
        self.chunk += 1
        if self.clock is not None:
            self.clock.t += 1e-3


class _ChunkClock:
    """Scheduler time that advances 1 ms per issued chunk (and by the sleeps
    of an idle scheduler), so that which request arrives during which chunk
    -- and so the whole schedule -- does not depend on the host's speed."""

    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


@pytest.mark.parametrize("rounding", ["nearest", "stochastic"])
def test_serve_chunked_quotas_and_pauses_same_as_alone(rounding):
    """Through serve() with the srpt policy: every request is granted its
    steps in at least 3 chunks (max_chunk caps a chunk), some requests are
    paused (left without a quota) between grants while shorter ones that
    arrived later run, and each result equals the request run alone element
    by element."""
    reqs = W.request_stream(n=12, rate_hz=400.0, seed=7, min_cells=6 ** 3, max_cells=18 ** 3,
                            steps_range=(60, 160))
    clock = _ChunkClock()
    be = _CountingBackend(capacity_bytes=128 << 20, max_slots=12, keep_fields=True, rounding=rounding)
    be.clock = clock
    st = serve(reqs, be, chunk_ms=1.0, policy="srpt", target_cells=3000, max_chunk=16, min_chunk=4,
               clock=clock, sleep=clock.sleep)
    be.close()
    assert len(st.results) == len(reqs) and not st.rejected
    paused_between = 0
    for req in reqs:
        g = be.grants[req.rid]
        chunks = [c for c, _ in g]
        assert sum(q for _, q in g) == req.steps
        assert len(g) >= 3, (req.rid, g)
        if chunks[-1] - chunks[0] + 1 > len(chunks):  # chunks ran without it in between
            paused_between += 1
    assert paused_between > 0
    if rounding == "nearest":
        _same_fields_as_alone(st.results, reqs)
    else:
        got = {r.rid: r.fields for r in st.results}
        for req in reqs:  # the same request alone, with the same rounding
            st1 = serve([req], SequentialBackend(storage=req.storage, keep_fields=True, rounding=rounding))
            rho_a, u_a = st1.results[0].fields
            rho_b, u_b = got[req.rid]
            mask = req.flags() == 0
            assert np.array_equal(u_b[:, mask], u_a[:, mask]) and np.array_equal(rho_b[mask], rho_a[mask])


def test_step_quotas():
    """lb_batch_set_steps_many grants per-slot quotas: a slot with quota 0 is
    not stepped; quotas are consumed by the steps that follow."""
    b = Batch(capacity_bytes=16 << 20, max_slots=4)
    s0 = b.add(12, 10, 8, 0.7, 0, flags=W.cavity_flags(12, 10, 8), u_lid=(0.05, 0, 0))
    s1 = b.add(12, 10, 8, 0.7, 0, flags=W.cavity_flags(12, 10, 8), u_lid=(0.05, 0, 0))
    b.set_steps_many([s0, s1], [7, 0])
    b.step(10)
    b.set_steps_many([s1], [3])
    b.step(10)
    assert b.query(s0)["done"] == 7 and b.query(s1)["done"] == 3
    a7 = Lattice(12, 10, 8, 0.7, flags=W.cavity_flags(12, 10, 8), u_lid=(0.05, 0, 0), kernel=1)
    a7.step(7)
    _, u0 = b.moments(s0)
    _, ua = a7.moments()
    assert vel_err(u0, ua, W.cavity_flags(12, 10, 8) == 0) <= 1e-5
    b.close()


def test_inplace_slots_in_the_mix():
    """In-place slots (one population array each) next to two-array slots of
    every storage: each gives the same result as the lattice alone (bitwise
    for the fluid cells: same pull, same collision), after odd and even
    step counts; fetch reads them back through the staging area."""
    b = Batch(capacity_bytes=64 << 20, max_slots=16)
    slots = []
    for k, (nx, ny, nz, tau, storage, kind, steps) in enumerate(MIX):
        flags, ulid, g = _geom(nx, ny, nz, kind)
        slots.append(b.add(nx, ny, nz, tau, steps, u_lid=ulid, flags=flags, storage=storage, force=g,
                           inplace=(k % 2 == 0)))
    b.step(60)
    assert set(b.poll()) == set(slots)
    for k, (s, (nx, ny, nz, tau, storage, kind, steps)) in enumerate(zip(slots, MIX)):
        flags, ulid, g = _geom(nx, ny, nz, kind)
        alone = Lattice(nx, ny, nz, tau, u_lid=ulid, flags=flags, storage=storage, force=g, kernel=1)
        alone.step(steps)
        mask = fluid_mask(flags, alone.shape)
        fb, fa = b.populations(s), alone.populations()
        assert np.array_equal(fb[:, mask], fa[:, mask]), (k, storage)
        rb, ub = b.moments(s)
        ra, ua = alone.moments()
        assert np.array_equal(ub, ua) and np.array_equal(rb, ra)
        mb, pb = b.totals(s)
        ma, pa = alone.totals()
        assert mb == ma and np.array_equal(pb, pa)
        # asynchronous read-back (the in-place slots through the staging area)
        rho = np.empty((nz, ny, nx))
        u = np.empty((3, nz, ny, nx))
        b.fetch(s, rho, u)
        while not b.fetch_done(s):
            pass
        assert np.array_equal(rho, ra) and np.array_equal(u, ua)
        alone.close()
    b.close()


def test_inplace_admission_and_init_fields():
    """A pool that holds two two-array FP32 slots holds three in-place ones;
    re-initialising an in-place slot after an odd number of steps resets its
    layout; adding the first in-place slot after graph replays re-captures
    the step graph."""
    two = slot_bytes(16, 16, 16, "f32")
    one = slot_bytes(16, 16, 16, "f32", inplace=True)
    assert two - one == 19 * 16 ** 3 * 4
    b = Batch(capacity_bytes=2 * two, max_slots=4)
    s0 = b.add(16, 16, 16, 0.7, 100)
    b.step(16)  # graph path with the two-array kernel only
    b.remove(s0)
    ss = [b.add(16, 16, 16, 0.7, 100, inplace=True) for _ in range(3)]
    assert b.try_add(16, 16, 16, 0.7, 10, inplace=True) is None
    rho0, u0 = W.random_fields(16, 16, 16, seed=2, du=0.04, drho=0.01)
    b.step(17)                     # odd: streamed layout
    b.init_fields(ss[1], rho0, u0)  # back to the swapped layout
    b.step(24)                     # graph re-captured with the in-place kernel
    alone = Lattice(16, 16, 16, 0.7, storage="f32", kernel=1)
    alone.step(41)
    ref = Lattice(16, 16, 16, 0.7, storage="f32", kernel=1)
    ref.init_fields(rho0, u0)
    ref.step(24)
    for s in ss:
        f = b.populations(s)
        want = ref.populations() if s == ss[1] else alone.populations()
        assert np.array_equal(f, want)
    b.close()


def test_serve_inplace_same_as_sequential():
    """The batched server with in-place slots gives the same velocity fields
    as the one-at-a-time baseline."""
    reqs = W.request_stream(n=8, rate_hz=200.0, seed=9, min_cells=6 ** 3, max_cells=20 ** 3,
                            steps_range=(20, 120))
    be = BatchBackend(capacity_bytes=64 << 20, max_slots=8, keep_fields=True, inplace=True)
    st = serve(reqs, be, chunk_ms=2.0, policy="srpt", target_cells=5000)
    be.close()
    assert len(st.results) == len(reqs) and not st.rejected
    _same_fields_as_alone(st.results, reqs)
