"""Continuous-batching server for lattice simulations.

Requests (size, tau, storage, steps, geometry) arrive over time.  The
scheduler admits waiting requests in arrival order as slots and pool memory
free up (HBM-budget admission), advances everything admitted together in
shared batched launches, retires finished simulations (their rho and u are
copied back to the host) and records time-to-result = completion - arrival
on the host's monotonic clock.

Backends:
  BatchBackend      -- liblbgb batches (lb_batch_*): the serving form;
  SequentialBackend -- one plain lattice at a time, one launch per step (the
                       baseline the batched form is compared with);
the scheduler itself only needs admit / step / finished / retire, so its
admission logic is tested on the CPU against a fake backend.
"""
from __future__ import annotations

import time
from collections import deque
from dataclasses import dataclass, field

import numpy as np


BYTES_PER_UPDATE = {"f64": 305, "f32": 153, "f16s": 77, "bf16s": 77, "f32d": 153, "e3m12s": 77}


@dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    cells: int
    steps: int
    storage: str
    fields: tuple = None       # (rho, u) on the host when kept

    @property
    def latency(self) -> float:
        return self.finished - self.arrival

    @property
    def checksum(self) -> float:
        """RMS speed of the returned velocity field (needs kept fields)."""
        return _checksum(self.fields[1])


@dataclass
class ServeStats:
    results: list = field(default_factory=list)
    rejected: list = field(default_factory=list)
    makespan: float = 0.0
    launches: int = 0

    def records(self):
        """One dict per finished request (times in seconds from the start of
        the run on the host's monotonic clock)."""
        for r in sorted(self.results, key=lambda r: r.rid):
            yield {"rid": r.rid, "arrival_s": round(r.arrival, 6), "admitted_s": round(r.admitted, 6),
                   "finished_s": round(r.finished, 6), "latency_s": round(r.latency, 6), "cells": r.cells,
                   "steps": r.steps, "storage": r.storage}
        for q in self.rejected:
            yield {"rid": q.rid, "arrival_s": round(q.arrival_s, 6), "rejected": True,
                   "cells": q.cells, "steps": q.steps, "storage": getattr(q, "storage", "f32")}

    def write_jsonl(self, path: str) -> int:
        """Write records() as JSON lines; returns the number written."""
        import json
        n = 0
        with open(path, "w") as fh:
            for rec in self.records():
                fh.write(json.dumps(rec) + "\n")
                n += 1
        return n

    def summary(self) -> dict:
        lat = np.array([r.latency for r in self.results]) if self.results else np.zeros(1)
        lups = float(sum(r.cells * r.steps for r in self.results))
        return {
            "requests": len(self.results),
            "rejected": len(self.rejected),
            "makespan_s": round(self.makespan, 4),
            "mlups": round(lups / self.makespan / 1e6, 1) if self.makespan > 0 else 0.0,
            "p50_s": round(float(np.percentile(lat, 50)), 4),
            "p99_s": round(float(np.percentile(lat, 99)), 4),
            "mean_s": round(float(lat.mean()), 4),
            "chunks": self.launches,
        }


class Scheduler:
    """Admission in arrival order, chunked stepping, two-phase retirement.

    Steps are issued in chunks sized to about ``chunk_ms`` of estimated GPU
    work (admitted cells x bytes per update at ``est_gbs``), and up to
    ``depth`` chunks stay queued: the scheduler waits only for the oldest
    chunk's counters (backend.finished()), starts the read-back of the
    requests that completed (backend.start_retire), admits waiting requests
    and issues the next chunk while the queued ones run; finished read-backs
    are collected with backend.collect().

    Policies for sharing the device between admitted requests:
      "fifo" -- every admitted request takes every step of every chunk;
      "srpt" -- each chunk grants step quotas to the requests with the least
                remaining work (cells x steps x bytes per update), in that
                order, until ``target_cells`` cells are running; the others
                stay resident but paused (backend.set_quotas).
    ``max_wait_s`` (srpt only) bounds starvation: requests that arrived more
    than ``max_wait_s`` seconds ago are granted first, oldest first, ahead of
    the least-remaining-work order.  Pure shortest-remaining-work-first
    leaves the largest requests paused for as long as arrivals exceed the
    capacity, so its p99 time-to-result grows past that of plain FIFO; with
    the bound, requests past it are served in arrival order.
    ``max_active_cells`` optionally bounds the cells admitted at once.
    Backends with ``whole_requests`` true (one request at a time) get each
    request's remaining steps as one chunk."""

    def __init__(self, backend, chunk_ms: float = 8.0, depth: int = 3, clock=time.monotonic, sleep=time.sleep,
                 max_active_cells=None, est_gbs: float = 5500.0, max_chunk: int = 256, min_chunk: int = 4,
                 policy: str = "fifo", target_cells: int = 8_000_000, max_wait_s=None):
        self.backend = backend
        self.chunk_ms = float(chunk_ms)
        self.depth = max(1, int(depth))
        self.clock = clock
        self.sleep = sleep
        self.max_active_cells = max_active_cells
        self.est_gbs = float(est_gbs)
        self.max_chunk = int(max_chunk)
        self.min_chunk = int(min_chunk)
        if policy not in ("fifo", "srpt"):
            raise ValueError(policy)
        self.policy = policy
        self.target_cells = int(target_cells)
        self.max_wait_s = None if max_wait_s is None else float(max_wait_s)

    def _storage(self, req):
        fn = getattr(self.backend, "storage_of", None)
        return fn(req) if fn is not None else getattr(req, "storage", "f32")

    def _bpu(self, req):
        return BYTES_PER_UPDATE.get(self._storage(req), 153)

    def _chunk(self, running):
        if getattr(self.backend, "whole_requests", False):
            return max(a[2] for a in running)
        bytes_per_step = sum(a[0].cells * self._bpu(a[0]) for a in running)
        step_s = max(4e-6, bytes_per_step / (self.est_gbs * 1e9))
        n = int(self.chunk_ms * 1e-3 / step_s)
        return max(self.min_chunk, min(self.max_chunk, n))

    def _select(self, live, now=0.0):
        """The requests that step in the next chunk."""
        if self.policy == "fifo" or getattr(self.backend, "whole_requests", False):
            return live
        late = self.max_wait_s

        def key(a):
            if late is not None and now - a[0].arrival_s > late:
                return (0, a[0].arrival_s)
            return (1, a[2] * a[0].cells * self._bpu(a[0]))
        order = sorted(live, key=key)
        out, cells = [], 0
        for a in order:
            if out and cells >= self.target_cells:
                break
            out.append(a)
            cells += a[0].cells
        return out

    def run(self, requests) -> ServeStats:
        reqs = sorted(requests, key=lambda r: r.arrival_s)
        stats = ServeStats()
        t0 = self.clock()
        i = 0
        waiting = deque()
        # handle -> [request, admitted time, steps not yet granted, chunk of the last grant]
        active = {}
        retiring = {}   # handle -> (request, admitted time)
        issued = 0      # chunks issued
        polled = 0      # chunks whose counters have been read
        srpt = self.policy == "srpt" and not getattr(self.backend, "whole_requests", False)
        while i < len(reqs) or waiting or active or retiring:
            now = self.clock() - t0
            while i < len(reqs) and reqs[i].arrival_s <= now:
                waiting.append(reqs[i])
                i += 1
            cells = sum(a[0].cells for a in active.values())
            while waiting:
                head = waiting[0]
                if (self.max_active_cells is not None and active
                        and cells + head.cells > self.max_active_cells):
                    break
                h = self.backend.admit(head)
                if h is None:
                    break
                waiting.popleft()
                # under srpt a request starts paused (quota 0) until selected
                active[h] = [head, self.clock() - t0, head.steps, -1]
                if srpt:
                    self.backend.set_quotas({h: 0})
                cells += head.cells
            live = [a for a in active.values() if a[2] > 0]
            if live and issued - polled < self.depth:
                run_now = self._select(live, self.clock() - t0)
                n = self._chunk(run_now)
                if srpt:
                    quotas = {}
                    for h, a in active.items():
                        if a in run_now:
                            quotas[h] = min(n, a[2])
                    self.backend.set_quotas(quotas)
                    for h, a in active.items():
                        if h in quotas:
                            a[2] -= quotas[h]
                            a[3] = issued
                else:
                    for a in run_now:
                        a[2] = max(0, a[2] - n)
                        a[3] = issued
                self.backend.step(n)
                issued += 1
                stats.launches += 1
                if issued - polled < self.depth and any(a[2] > 0 for a in active.values()):
                    continue       # keep more work queued before waiting
            progressed = False
            if issued > polled or (active and not live):
                chunk_done = polled if issued > polled else issued - 1
                if issued > polled:
                    polled += 1
                for h in self.backend.finished():
                    a = active.get(h)
                    # complete: every step granted, and the chunk of the last grant has run
                    if a is not None and a[2] == 0 and a[3] <= chunk_done:
                        del active[h]
                        self.backend.start_retire(h)
                        retiring[h] = (a[0], a[1])
                        progressed = True
            for h, payload in self.backend.collect():
                req, t_adm = retiring.pop(h)
                stats.results.append(Result(req.rid, req.arrival_s, t_adm, self.clock() - t0, req.cells,
                                            req.steps, self._storage(req), payload))
                progressed = True
            if issued > polled or progressed:
                continue
            if retiring:
                self.sleep(2e-4)   # read-backs in flight
                continue
            if not active:
                if waiting:
                    # nothing running and the head does not fit an empty backend
                    stats.rejected.append(waiting.popleft())
                    continue
                if i < len(reqs):
                    self.sleep(max(0.0, reqs[i].arrival_s - (self.clock() - t0)))
        if stats.results:
            stats.makespan = max(r.finished for r in stats.results) - min(r.arrival for r in stats.results)
        return stats


# Storage policy for 16-bit requests.  FP16 keeps 11 significant bits only
# for |d| >= 2^-14; below that its steps are a fixed 2^-24, so a request
# whose deviations stay small (a slowly driven flow) loses relative
# precision in FP16 whatever the rounding.  Its deviation scale is
# predicted from the request: the axis populations carry w 3 c.u = U/6 for
# a flow speed U, with U the lid speed for a cavity, and for a duct driven
# by a body force g from rest the smaller of the free acceleration g t and
# the laminar centre speed g H^2 / (8 nu) (H the narrower wall-to-wall width,
# nu = (tau - 1/2) / 3).  A 16-bit request predicted below MIN_DEV_16 is
# served in FP32 instead.
MIN_DEV_16 = 2.0 ** -13


def predicted_deviation(req) -> float:
    """The deviation scale U/6 a request's flow reaches (see above)."""
    ulid = float(np.linalg.norm(getattr(req, "u_lid", (0.0, 0.0, 0.0))))
    g = float(np.linalg.norm(getattr(req, "force", (0.0, 0.0, 0.0))))
    u = ulid
    if g > 0.0:
        h = max(1, min(req.ny, req.nz) - 2)
        nu = (req.tau - 0.5) / 3.0
        u = max(u, min(g * req.steps, g * h * h / (8.0 * nu)))
    return u / 6.0


def served_storage(req, promote: bool = True) -> str:
    """The storage a request is served in: its own, except that a 16-bit
    request whose predicted deviations are below MIN_DEV_16 gets FP32."""
    st = getattr(req, "storage", "f32")
    if promote and st in ("f16s", "bf16s", "e3m12s") and predicted_deviation(req) < MIN_DEV_16:
        return "f32"
    return st


def _rounding_for(storage: str, rounding: str) -> str:
    """Stochastic rounding applies to 16-bit storage only."""
    return rounding if storage in ("f16s", "bf16s", "e3m12s") else "nearest"


def _checksum(u):
    return float(np.sqrt(np.mean(np.sum(u * u, axis=0))))


def _host_fields(shape, pinned=True):
    """rho (nz,ny,nx) and u (3,nz,ny,nx) float64 host arrays, in page-locked
    memory when torch is available (its caching host allocator)."""
    if pinned:
        try:
            import torch
            rho = torch.empty(shape, dtype=torch.float64, pin_memory=True)
            u = torch.empty((3,) + tuple(shape), dtype=torch.float64, pin_memory=True)
            return rho.numpy(), u.numpy(), (rho, u)
        except (ImportError, RuntimeError):
            pass
    return np.empty(shape), np.empty((3,) + tuple(shape)), None


class BatchBackend:
    """The serving form: every admitted request is a slot of one lb_batch;
    results come back asynchronously (lb_batch_fetch) into pinned buffers."""

    def __init__(self, capacity_bytes: int, max_slots: int = 1024, device=None, keep_fields: bool = False,
                 inplace: bool = False, rounding: str = "nearest", promote: bool = False):
        from .batch import Batch
        self.batch = Batch(capacity_bytes, max_slots=max_slots, device=device)
        self.keep = keep_fields
        self.inplace = inplace  # one population array per slot: about twice the requests per budget
        self.rounding = rounding  # of 16-bit requests (lb_options.rounding)
        self.promote = promote    # 16-bit requests with small predicted deviations served in FP32
        self.pending = {}

    def storage_of(self, req) -> str:
        return served_storage(req, self.promote)

    def admit(self, req):
        st = self.storage_of(req)
        return self.batch.try_add(req.nx, req.ny, req.nz, req.tau, req.steps, u_lid=req.u_lid,
                                  flags=req.flags(), storage=st, force=req.force,
                                  inplace=self.inplace, rounding=_rounding_for(st, self.rounding))

    def step(self, n):
        self.batch.step(n)

    def set_quotas(self, quotas):
        if quotas:
            self.batch.set_steps_many(list(quotas.keys()), list(quotas.values()))

    def finished(self):
        return self.batch.poll()

    def start_retire(self, slot):
        nx, ny, nz, _ = self.batch.meta[slot]
        rho, u, owner = _host_fields((nz, ny, nx))
        self.batch.fetch(slot, rho, u)
        self.pending[slot] = (rho, u, owner)

    def collect(self):
        out = []
        for slot in list(self.pending):
            if self.batch.fetch_done(slot):
                rho, u, _ = self.pending.pop(slot)
                self.batch.remove(slot)
                out.append((slot, (rho.copy(), u.copy()) if self.keep else None))
        return out

    def close(self):
        self.batch.close()


class SequentialBackend:
    """Baseline: one plain lattice at a time, one launch per time step, in
    the given storage (FP32 for the comparison); results read back
    synchronously into the same kind of pinned buffers."""

    whole_requests = True

    def __init__(self, storage: str = "f32", device=None, keep_fields: bool = False, rounding: str = "nearest"):
        self.storage = storage
        self.rounding = rounding
        self.device = device
        self.keep = keep_fields
        self.lat = None
        self.left = 0
        self.key = 0
        self.done = []

    def admit(self, req):
        if self.lat is not None:
            return None
        from .lattice import Lattice
        self.lat = Lattice(req.nx, req.ny, req.nz, req.tau, u_lid=req.u_lid, flags=req.flags(),
                           storage=self.storage, force=req.force, device=self.device,
                           rounding=_rounding_for(self.storage, self.rounding))
        self.left = req.steps
        self.key += 1
        return self.key

    def step(self, n):
        k = min(n, self.left)
        self.lat.step(k)
        self.left -= k

    def finished(self):
        return [self.key] if (self.lat is not None and self.left == 0) else []

    def start_retire(self, key):
        import ctypes
        rho, u, _ = _host_fields(self.lat.shape)
        st = self.lat.lib.lb_moments(self.lat.handle, ctypes.c_void_p(rho.ctypes.data),
                                     ctypes.c_void_p(u.ctypes.data))
        if st != 0:
            raise RuntimeError(f"lb_moments failed: {st}")
        self.lat.close()
        self.lat = None
        self.done.append((key, (rho.copy(), u.copy()) if self.keep else None))

    def collect(self):
        out, self.done = self.done, []
        return out

    def close(self):
        if self.lat is not None:
            self.lat.close()


def serve(requests, backend, **kw) -> ServeStats:
    return Scheduler(backend, **kw).run(requests)
