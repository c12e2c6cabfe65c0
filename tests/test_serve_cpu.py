"""The serving scheduler's admission / stepping / retirement logic on the CPU,
against a fake backend with a byte budget and a virtual clock."""
from dataclasses import dataclass

import pytest

from paper_2409_16781_gb300.serve import Scheduler
from paper_2409_16781_gb300 import workloads as W


class VirtualClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(dt, 1e-6)


class FakeBackend:
    """Pool of `capacity` bytes, `slots` slots; a step of n costs n * 1e-4 s
    of virtual time; each request needs cells * 100 bytes."""

    def __init__(self, capacity, slots, clock):
        self.capacity, self.slots, self.clock = capacity, slots, clock
        self.used = 0
        self.active = {}
        self.next = 0
        self.log = []

    def admit(self, req):
        need = req.cells * 100
        if len(self.active) >= self.slots or self.used + need > self.capacity:
            return None
        self.next += 1
        self.active[self.next] = [req, req.steps, need]
        self.used += need
        self.log.append(("admit", req.rid, self.clock.t))
        return self.next

    def set_quotas(self, quotas):
        self.quota = getattr(self, "quota", {})
        self.quota.update(quotas)

    def step(self, n):
        assert n >= 1
        q = getattr(self, "quota", None)
        for h, a in self.active.items():
            take = n if q is None or h not in q else min(n, q[h])
            if q is not None and h in q:
                q[h] -= take
            a[1] = max(0, a[1] - take)
        self.clock.t += n * 1e-4

    def finished(self):
        q = getattr(self, "quota", None)
        return [h for h, a in self.active.items() if a[1] == 0 or (q is not None and q.get(h, 1) == 0)]

    def start_retire(self, h):
        req, _, need = self.active.pop(h)
        self.used -= need
        self.log.append(("retire", req.rid, self.clock.t))
        self.done = getattr(self, "done", []) + [(h, float(req.rid))]

    def collect(self):
        out, self.done = getattr(self, "done", []), []
        return out


@dataclass
class Req:
    rid: int
    arrival_s: float
    cells: int
    steps: int
    storage: str = "f32"


def test_fifo_admission_within_budget_and_all_finish():
    clk = VirtualClock()
    be = FakeBackend(capacity=1000 * 100 * 3, slots=8, clock=clk)
    reqs = [Req(i, 0.001 * i, 1000, 50 + 10 * i) for i in range(10)]
    st = Scheduler(be, clock=clk, sleep=clk.sleep, max_chunk=16).run(reqs)
    assert len(st.results) == 10 and not st.rejected
    admits = [rid for kind, rid, _ in be.log if kind == "admit"]
    assert admits == sorted(admits)                     # arrival order
    # never more than 3 resident at once (byte budget)
    live = 0
    for kind, _, _ in be.log:
        live += 1 if kind == "admit" else -1
        assert 0 <= live <= 3
    for r in st.results:
        assert r.finished >= r.admitted >= r.arrival - 1e-12
        assert r.fields == float(r.rid)
    s = st.summary()
    assert s["requests"] == 10 and s["p99_s"] >= s["p50_s"] > 0


def test_slot_limit_and_oversized_request_is_rejected():
    clk = VirtualClock()
    be = FakeBackend(capacity=10 ** 9, slots=2, clock=clk)
    reqs = [Req(0, 0.0, 10, 30), Req(1, 0.0, 10, 30), Req(2, 0.0, 10, 30), Req(3, 0.5, 10 ** 9, 5)]
    st = Scheduler(be, clock=clk, sleep=clk.sleep, max_chunk=8).run(reqs)
    assert sorted(r.rid for r in st.results) == [0, 1, 2]
    assert [r.rid for r in st.rejected] == [3]
    # request 2 waited for a slot: admitted only after one of 0/1 retired
    t_retire_first = min(t for kind, rid, t in be.log if kind == "retire")
    t_admit_2 = [t for kind, rid, t in be.log if kind == "admit" and rid == 2][0]
    assert t_admit_2 >= t_retire_first


def test_chunks_follow_the_work_estimate_and_keep_work_queued():
    """Chunk length ~ chunk_ms of estimated work; all issued steps cover the
    longest request; a request that ends inside a chunk is still retired."""
    clk = VirtualClock()
    be = FakeBackend(capacity=10 ** 12, slots=8, clock=clk)
    steps_seen = []
    orig = be.step
    be.step = lambda n: (steps_seen.append(n), orig(n))
    reqs = [Req(0, 0.0, 10, 5), Req(1, 0.0, 10 ** 6, 400)]
    sch = Scheduler(be, clock=clk, sleep=clk.sleep, chunk_ms=8.0, est_gbs=1000.0, max_chunk=1000)
    st = sch.run(reqs)
    # 1e6 cells * 153 B at 1000 GB/s = 0.153 ms per step -> 52 steps per 8 ms chunk
    assert steps_seen[0] == 52
    assert sum(steps_seen) >= 400
    assert {r.rid for r in st.results} == {0, 1}


def test_idle_until_next_arrival():
    clk = VirtualClock()
    be = FakeBackend(capacity=10 ** 9, slots=4, clock=clk)
    st = Scheduler(be, clock=clk, sleep=clk.sleep, max_chunk=8).run([Req(0, 2.0, 10, 8)])
    assert st.results[0].admitted >= 2.0


def test_request_stream_shape():
    reqs = W.request_stream(n=300, rate_hz=5.0, seed=1)
    assert len(reqs) == 300
    for r in reqs:
        dims = (r.nx, r.ny, r.nz)
        assert max(dims) / min(dims) <= 4.0 + 1e-9
        assert 4 ** 3 <= r.cells <= 260 ** 3
        assert 0.52 <= r.tau <= 1.0 and 200 <= r.steps <= 5000
        assert r.kind in ("cavity", "channel") and r.storage in ("f32", "f16s")
    arr = [r.arrival_s for r in reqs]
    assert arr == sorted(arr)
    gaps = [b - a for a, b in zip(arr, arr[1:])]
    assert 0.1 < sum(gaps) / len(gaps) < 0.4   # mean inter-arrival ~ 1/rate


def test_srpt_runs_least_remaining_work_first():
    """Under "srpt" with a small target, a short request admitted behind a
    long one is stepped first and finishes first; both complete."""
    clk = VirtualClock()
    be = FakeBackend(capacity=10 ** 12, slots=8, clock=clk)
    reqs = [Req(0, 0.0, 10 ** 6, 2000), Req(1, 0.0, 10 ** 4, 50)]
    st = Scheduler(be, clock=clk, sleep=clk.sleep, policy="srpt", target_cells=1, max_chunk=64).run(reqs)
    fin = {r.rid: r.finished for r in st.results}
    assert set(fin) == {0, 1} and fin[1] < fin[0]
    # fifo for comparison: both progress together; the short one still ends first
    clk2 = VirtualClock()
    be2 = FakeBackend(capacity=10 ** 12, slots=8, clock=clk2)
    st2 = Scheduler(be2, clock=clk2, sleep=clk2.sleep, policy="fifo", max_chunk=64).run(reqs)
    assert {r.rid for r in st2.results} == {0, 1}


def _overload(max_wait_s):
    """One large request at t = 0 (50 chunks of 64 steps), then a small
    request (4 chunks) every 20 ms for 2 s; one request runs per chunk
    (target_cells = 1) and a chunk costs 6.4 ms, so the small requests alone
    keep the backend busy."""
    clk = VirtualClock()
    be = FakeBackend(capacity=10 ** 12, slots=256, clock=clk)
    reqs = [Req(0, 0.0, 10 ** 6, 64 * 50)]
    reqs += [Req(i, 0.02 * i, 10 ** 3, 64 * 4) for i in range(1, 101)]
    st = Scheduler(be, clock=clk, sleep=clk.sleep, policy="srpt", target_cells=1, max_chunk=64, min_chunk=64,
                   max_wait_s=max_wait_s).run(reqs)
    assert len(st.results) == 101 and not st.rejected
    return {r.rid: r.finished for r in st.results}


def test_srpt_max_wait_bounds_starvation():
    """Pure shortest-remaining-work-first leaves the large request paused
    until the stream of small ones ends; with max_wait_s it is granted once
    it has waited that long, oldest first, and finishes well before."""
    starve = _overload(None)
    bounded = _overload(0.5)
    last_small = max(t for rid, t in starve.items() if rid != 0)
    assert starve[0] >= 0.9 * last_small
    assert 0.5 < bounded[0] < 0.5 + 50 * 0.0064 + 0.05
    # the small requests still all finish
    assert all(bounded[i] > 0 for i in range(1, 101))


def test_per_request_jsonl_records(tmp_path):
    """Every finished and every rejected request gets one JSON line; the
    latency is finished - arrival and the p50 of the lines matches the
    summary's."""
    import json

    import numpy as np
    clk = VirtualClock()
    be = FakeBackend(capacity=20000, slots=4, clock=clk)   # the last request never fits
    reqs = [Req(i, 0.01 * i, 10 + 5 * i, 8 + i) for i in range(12)] + [Req(99, 0.2, 10 ** 6, 4)]
    st = Scheduler(be, clock=clk, sleep=clk.sleep, max_chunk=8).run(reqs)
    path = tmp_path / "serve.jsonl"
    n = st.write_jsonl(str(path))
    lines = [json.loads(l) for l in path.read_text().splitlines()]
    assert n == len(lines) == 13
    done = [l for l in lines if not l.get("rejected")]
    assert len(done) == 12 and [l["rid"] for l in done] == list(range(12))
    assert [l["rid"] for l in lines if l.get("rejected")] == [99]
    for l in done:
        assert abs(l["latency_s"] - (l["finished_s"] - l["arrival_s"])) < 1e-5
        assert l["arrival_s"] <= l["admitted_s"] <= l["finished_s"]
    assert abs(np.percentile([l["latency_s"] for l in done], 50) - st.summary()["p50_s"]) < 1e-3


def test_storage_policy_promotes_slowly_driven_16_bit_requests():
    """A 16-bit request whose predicted deviations (U/6 for flow speed U) lie
    below 2^-13 is served in FP32: FP16 keeps its 11 significant bits only
    above 2^-14."""
    from paper_2409_16781_gb300.serve import MIN_DEV_16, predicted_deviation, served_storage
    assert MIN_DEV_16 == 2.0 ** -13
    cav = W.Request(0, 0.0, 32, 32, 32, 0.6, 1000, "cavity", "f16s", u_lid=(0.05, 0.0, 0.0))
    assert predicted_deviation(cav) == pytest.approx(0.05 / 6)
    assert served_storage(cav) == "f16s"
    # a narrow, viscous duct: its laminar centre speed g H^2 / (8 nu) bounds U
    duct = W.Request(1, 0.0, 65, 54, 18, 0.978, 3115, "channel", "f16s", u_lid=(0.0, 0.0, 0.0),
                     force=(1e-6, 0.0, 0.0))
    nu, h = (0.978 - 0.5) / 3, 16
    assert predicted_deviation(duct) == pytest.approx(1e-6 * h * h / (8 * nu) / 6)
    assert served_storage(duct) == "f32"
    assert served_storage(duct, promote=False) == "f16s"
    # a wide duct: the free acceleration g t bounds U
    wide = W.Request(2, 0.0, 105, 207, 77, 0.953, 4312, "channel", "f16s", u_lid=(0.0, 0.0, 0.0),
                     force=(1e-6, 0.0, 0.0))
    assert predicted_deviation(wide) == pytest.approx(1e-6 * 4312 / 6)
    assert served_storage(wide) == "f16s"
    fp32 = W.Request(3, 0.0, 8, 8, 8, 0.9, 200, "channel", "f32", force=(1e-6, 0.0, 0.0))
    assert served_storage(fp32) == "f32"


def test_scheduler_records_the_served_storage():
    clock = VirtualClock()
    be = FakeBackend(capacity=10 ** 9, slots=8, clock=clock)
    be.storage_of = lambda req: "f32" if req.rid % 2 else req.storage
    reqs = [W.Request(k, 0.0, 8, 8, 8, 0.7, 50, "cavity", "f16s") for k in range(4)]
    st = Scheduler(be, clock=clock, sleep=clock.sleep).run(reqs)
    assert sorted((r.rid, r.storage) for r in st.results) == [(0, "f16s"), (1, "f32"), (2, "f16s"), (3, "f32")]
