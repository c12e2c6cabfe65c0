#!/usr/bin/env python
"""Benchmark of the fused D3Q19 BGK lattice update on GB300.

Default workload: 3D periodic Taylor-Green vortex, 256^3 lattice, FP32
populations (stored as f - w), tau = 0.55, u0 = 0.05, k = 2*pi/256 -- the
configuration the MLUPS metric is quoted on.  One bench step = one
lb_step(1) (one fused stream-collide launch over all 16.8 M cells) plus, every
``--check-every`` steps and once at the end, the FP64 mass/momentum
reduction used as the divergence check.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun, one rank per GPU.  By default the lattice is
decomposed into z-slabs (--decomp slab): rank r owns 256 z-planes of one
256 x 256 x (256 N) Taylor-Green lattice (weak scaling) and trades the five
c_z = +-1 populations of its boundary planes with its z-neighbours after
every step (NCCL send/recv); --decomp replicas runs an independent lattice
per rank instead.  value = all ranks' cell updates / max-over-ranks time.

Besides the headline line's TGV measurement, the default run measures the
other configurations (``configs``): the 512^3 porous channel in FP32 and
shifted FP16, the 768^3 cavity precision study (5000 steps, three tau), and
the 2000-request serving stream at 0.5x and 2x the sequential FP32
capacity; --no-configs skips them.

The reference arm (--impl reference) times the FP64 CPU oracle on the host
cores, each step a bounded sample (a z-slab of the same lattice).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

T_START = time.time()  # process start: the configs sections stop starting after --configs-deadline-s

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "D3Q19 MLUPS & fraction of HBM roofline; batched-serve p50/p99 vs plain FP32 launches"
STORAGE_BYTES = {"f64": 8, "f32": 4, "f16s": 2, "bf16s": 2, "f32d": 4, "e3m12s": 2}
FALLBACK_HBM_GBS = 6800.0
# the files that make up the step kernel (hashed to tie ncu figures to it)
# the CUDA sources of the step kernels: shared headers, then the two-array
# kernels' and the in-place kernels' own files
STEP_SOURCES = ("lb_common.cuh", "lb_fpconv.cuh", "lb_internal.h", "lb_kernels.cuh", "lb_pairs.cuh", "lb_mbarrier.cuh",
                "lb_step.cu", "lb_inplace.cu")
STEP_SOURCES_OF = {"two_arrays": tuple(n for n in STEP_SOURCES if n != "lb_inplace.cu"),
                   "inplace": tuple(n for n in STEP_SOURCES if n not in ("lb_step.cu", "lb_mbarrier.cuh"))}


def bytes_per_update(storage: str) -> int:
    """Algorithmic bytes per lattice update: 19 reads + 19 writes + 1 flag byte."""
    return 2 * 19 * STORAGE_BYTES[storage] + 1


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--storage", choices=list(STORAGE_BYTES), default="f32")
    ap.add_argument("--n", type=int, default=256, help="lattice edge (default 256)")
    ap.add_argument("--kernel", type=int, default=0, help="step kernel variant (0 = library choice)")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--inplace", action="store_true",
                    help="one population array updated in place (AA pattern) instead of two")
    ap.add_argument("--trt-magic", type=float, default=0.0,
                    help="two-relaxation-time collision with this magic parameter (0 = BGK)")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the short runs of the other storage / layout forms in the default line")
    ap.add_argument("--check-every", type=int, default=100)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the library default variant instead of the autotuner's choice")
    ap.add_argument("--workload", choices=["tgv", "serve", "porous", "precision", "vks"], default="tgv",
                    help="tgv: the 256^3 Taylor-Green line (default); serve: a full serving run; "
                         "porous: the 512^3 porous channel; precision: the 768^3 cavity precision study; "
                         "vks: flow past a cylinder (von Karman street), 1024x256x64")
    ap.add_argument("--vks-steps", type=int, default=40000,
                    help="steps of the von Karman street run that measures the shedding frequency")
    ap.add_argument("--taus", default="0.52,0.56,0.6", help="relaxation times of the precision study")
    ap.add_argument("--serve-requests", type=int, default=None,
                    help="requests of the serving run: default 80 in the default line's serving section "
                         "(0 = skip it), 2000 for --workload serve")
    ap.add_argument("--serve-budget-gb", type=float, default=64.0, help="HBM budget of the batch pool")
    ap.add_argument("--serve-rates", default="0.5,2",
                    help="arrival rates of --workload serve, as multiples of the sequential FP32 capacity")
    ap.add_argument("--serve-max-wait", type=float, default=60.0,
                    help="seconds after which a waiting request is served oldest-first (0 = no bound)")
    ap.add_argument("--serve-log", default=None,
                    help="path prefix for per-request JSON-lines records of the serving runs")
    ap.add_argument("--serve-tight-gb", type=float, default=0.75,
                    help="HBM budget of the memory-bound serving comparison (two arrays vs in place; 0 = skip)")
    ap.add_argument("--serve-rounding", choices=["nearest", "stochastic"], default="stochastic",
                    help="rounding of the 16-bit requests' stored values in the batched server")
    ap.add_argument("--rounding", choices=["nearest", "stochastic"], default="nearest",
                    help="rounding of the headline lattice's 16-bit stored values")
    ap.add_argument("--decomp", choices=["slab", "replicas"], default="slab",
                    help="N > 1: z-slabs of one lattice with a halo exchange (default), or replicas")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the porous 512^3, cavity 768^3 precision and 2000-request serving sections")
    ap.add_argument("--precision-steps", type=int, default=5000, help="steps of the 768^3 precision study")
    ap.add_argument("--configs-deadline-s", type=float, default=2400.0,
                    help="a configs section that would start later than this many seconds after the "
                         "process started is skipped (reported as skipped), so the line is always printed")
    return ap.parse_args(argv)


# ---------------------------------------------------------------- distributed
class Dist:
    """Rank bookkeeping; a process group only when WORLD_SIZE > 1."""

    def __init__(self, backend=None):
        self.rank = int(os.environ.get("RANK", "0"))
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.local_rank = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = False
        self.backend = None
        if self.world > 1:
            import torch.distributed as dist
            if backend is None:
                import torch
                backend = "nccl" if torch.cuda.is_available() else "gloo"
            self.backend = backend
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend)
            self.pg = True

    def device_tensor(self, v):
        import torch
        dev = f"cuda:{self.local_rank}" if getattr(self, "backend", "gloo") == "nccl" else "cpu"
        return torch.tensor([float(v)], dtype=torch.float64, device=dev)

    def barrier(self):
        if self.pg:
            import torch.distributed as dist
            dist.barrier()

    def max(self, v: float) -> float:
        if not self.pg:
            return float(v)
        import torch.distributed as dist
        t = self.device_tensor(v)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    def sum(self, v: float) -> float:
        if not self.pg:
            return float(v)
        import torch.distributed as dist
        t = self.device_tensor(v)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg:
            import torch.distributed as dist
            dist.destroy_process_group()


def aggregate_replicas(dist: Dist, cells_per_rank: float, steps: int, seconds_local: float):
    """Whole-job throughput of independent replicas: all ranks' updates over
    the slowest rank's time.  Returns (MLUPS, max seconds)."""
    t = dist.max(seconds_local)
    total = dist.sum(cells_per_rank * steps)
    return total / t / 1e6, t


# ---------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, enabled=True):
        self.gpu = gpu_index
        self.enabled = enabled
        self.proc = None
        self.lines = []          # (host monotonic time of arrival, line)
        self.window = None       # (start, end) of the timed region, host monotonic
        self.continued = False   # the window is the same load continued after a short region

    def mark(self, start: bool):
        """Note the host time at which the timed region starts / ends (the
        sampler runs from before the warm-up so that it is already sampling
        when a short region starts)."""
        t = time.monotonic()
        if start:
            self.window = (t, None)
        elif self.window is not None:
            self.window = (self.window[0], t)

    def start(self):
        if not self.enabled:
            return
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except (OSError, ValueError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.monotonic(), line.strip()))

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        return self.summary()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = self.lines
        where = "whole run"
        if self.window is not None and self.window[1] is not None:
            # samples taken during the region (one sampling period of slack at
            # the end); a region shorter than the period gets the first
            # sample after it started
            t0, t1 = self.window
            lines = [(t, ln) for t, ln in self.lines if t0 <= t <= t1 + 0.05]
            where = ("the same steps continued untimed for 0.5 s right after the timed region (shorter "
                     "than the 100 ms sampling period)" if self.continued else "timed region")
            if not lines:
                after = [(t, ln) for t, ln in self.lines if t >= t0]
                lines = after[:1]
                where = "first sample after the window started"
        for _, ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "sampled": where}


# ---------------------------------------------------------------- helpers
def strip_comments(src: str) -> str:
    """C/C++ source without its comments and with runs of blank space
    collapsed (string and character literals kept verbatim): the code the
    compiler sees, so that editing a comment does not change the hash."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def kernel_source_hash(kind: str = "two_arrays") -> str:
    """Hash of the CUDA code (comments excluded) of the two-array or the
    in-place step kernels (`kind`); a committed ncu figure is only reported
    while it matches the kernels being timed."""
    h = hashlib.sha256()
    cs = os.path.join(ROOT, "paper_2409_16781_gb300", "csrc")
    for name in STEP_SOURCES_OF[kind]:
        with open(os.path.join(cs, name), encoding="utf-8") as fh:
            h.update(name.encode() + b"\0" + strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


NOMINAL_HBM_GBS = 8000.0   # GB300 HBM3e, nominal (the 8 TB/s the >= 80 % target is stated against)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback"


def ncu_figure(profile_key: str, variant=None, field: str = "dram_bytes_per_launch"):
    """A committed ncu figure (profiles/traffic.json: per workload key, the
    source hash and one record per kernel variant), if it was taken on the
    current kernel sources and for the kernel variant being timed."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        rec = d.get(profile_key)
        kind = "inplace" if profile_key.endswith("_inplace") else "two_arrays"
        if rec and rec.get("source_hash") == kernel_source_hash(kind):
            per = rec.get("variants", {})
            hit = per.get(str(variant)) if variant is not None else None
            if hit:
                return hit.get(field)
    except (OSError, ValueError):
        pass
    return None


def ncu_traffic(profile_key: str, variant=None):
    """Per-launch DRAM bytes (read + write) from the committed ncu figures."""
    return ncu_figure(profile_key, variant, "dram_bytes_per_launch")


# FP64-pipe peak of a GB300 (the FP64 and Mixed2 forms are bound by it):
# 2 FP64 thread instructions per SM per clock -- the nominal 1.25 TFLOP/s
# FP64 (an FMA counting 2) over 152 SMs at 2.07 GHz, and what the ncu pipe
# counters of the FP64 step kernel imply (one warp instruction per 16 clocks
# per SM at 100 % pipe activity).
FP64_PIPE_INST_PER_SM_CLK = 2
GB300_SMS = 152
GB300_MAX_SM_GHZ = 2.07


def fp64_alu_roofline(storage, variant, glups):
    """The ALU roofline of an FP64-arithmetic form: FP64-pipe thread
    instructions per update (ncu, profiles/traffic.json) x updates per second
    against the pipe's peak; None without a figure for this variant."""
    per = ncu_figure(f"step_{storage}_tgv256", variant, "fp64_pipe_inst_per_update")
    if not per:
        return None
    peak = GB300_SMS * FP64_PIPE_INST_PER_SM_CLK * GB300_MAX_SM_GHZ   # G inst / s
    achieved = glups * per
    return {"bound": "alu", "unit": "G FP64-pipe inst/s", "inst_per_update": per,
            "achieved": round(achieved, 1), "peak": round(peak, 1), "frac": round(achieved / peak, 4),
            "peak_kind": "derived: 152 SMs x 2 FP64 inst/clk x 2.07 GHz"}


def tgv_inputs(n):
    from paper_2409_16781_gb300 import workloads as W
    return W.taylor_green_fields(n, n, n, u0=0.05)


def tgv_slab_inputs(n, nz, z0, z1, u0=0.05):
    """Taylor-Green fields of an n x n x nz lattice (wavenumber 2 pi / edge
    on each axis) on planes z0-1 .. z1 (periodic): a z-slab with its ghost
    planes, without building the whole lattice's fields."""
    import numpy as np
    kx = ky = 2 * math.pi / n
    kz = 2 * math.pi / nz
    x = np.arange(n)[None, None, :]
    y = np.arange(n)[None, :, None]
    z = np.array([(z0 - 1) % nz] + list(range(z0, z1)) + [z1 % nz])[:, None, None]
    u = np.zeros((3, len(z), n, n))
    u[0] = u0 * np.sin(kx * x) * np.cos(ky * y) * np.cos(kz * z)
    u[1] = -u0 * np.cos(kx * x) * np.sin(ky * y) * np.cos(kz * z)
    return np.ones((len(z), n, n)), u


# ---------------------------------------------------------------- our arm
def run_ours(args, dist: Dist):
    import numpy as np
    import torch

    from paper_2409_16781_gb300 import Lattice

    dev = torch.device("cuda", dist.local_rank)
    torch.cuda.set_device(dev)
    n = args.n
    N = n ** 3           # cells this rank updates per step
    tau = 0.55
    stream = torch.cuda.current_stream(dev)
    slab = None
    if dist.world > 1 and args.decomp == "slab":
        # z-slabs of one n x n x (n * world) lattice, n own planes per rank
        from paper_2409_16781_gb300.slab import SlabExchange, SlabLattice
        if args.inplace:
            raise SystemExit("--decomp slab needs two population arrays (no --inplace)")
        nzg = n * dist.world
        slab = SlabLattice(n, n, nzg, tau, storage=args.storage, rank=dist.rank, world=dist.world,
                           exchange=SlabExchange(dist.rank, dist.world,
                                                 device=dev if dist.backend == "nccl" else None),
                           device=dev, stream=stream,
                           kernel=args.kernel, block=args.block)
        lat = slab.lattice
        rho0, u0 = tgv_slab_inputs(n, nzg, slab.z0, slab.z1)
        lat.init_fields(rho0, u0)
        slab.halo()
    else:
        rho0, u0 = tgv_inputs(n)
        lat = Lattice(n, n, n, tau, storage=args.storage, device=dev, stream=stream,
                      kernel=args.kernel, block=args.block, inplace=args.inplace, trt_magic=args.trt_magic,
                      rounding=args.rounding)
        lat.init_fields(rho0, u0)
    tuned = None
    if args.kernel == 0 and not args.no_autotune:
        tuned = lat.autotune(reps=20, cache=False)

    def step():
        lat.step(1)
        if slab is not None:
            slab.halo()

    def totals():
        return slab.totals() if slab is not None else lat.totals()

    launches_per_check = 2  # reduction kernel + finalize kernel
    clocks = ClockSampler(dist.local_rank, enabled=not args.no_clocks and dist.local_rank == 0)
    clocks.start()  # already sampling when the timed region starts
    for _ in range(args.warmup):
        step()
    totals()
    torch.cuda.synchronize(dev)

    K = args.steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    n_checks = 0
    dist.barrier()
    torch.cuda.synchronize(dev)
    clocks.mark(True)
    t_start.record(stream)
    for k in range(K):
        ev[k][0].record(stream)
        lat.step(1)
        ev[k][1].record(stream)
        if slab is not None:
            slab.halo()
        if args.check_every > 0 and (k + 1) % args.check_every == 0 and k + 1 < K:
            totals()
            n_checks += 1
    mass, mom = totals()
    n_checks += 1
    t_end.record(stream)
    torch.cuda.synchronize(dev)
    clocks.mark(False)
    seconds = t_start.elapsed_time(t_end) / 1e3
    if clocks.enabled and seconds < 0.5:
        # a region shorter than a few 100 ms sampling periods: keep the same
        # load (untimed step launches, no halo exchange, so that no other rank
        # takes part; the state is re-initialised by the e2e run below) for
        # about half a second and sample that
        extra = int(math.ceil(0.5 / max(seconds / K, 1e-6)))
        clocks.mark(True)
        for _ in range(extra):
            lat.step(1)
        torch.cuda.synchronize(dev)
        clocks.mark(False)
        clocks.continued = True
    dist.barrier()
    clock_summary = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    kernel_ms = statistics.mean(step_ms)
    value, t_max = aggregate_replicas(dist, N, K, seconds)

    # end-to-end through the C ABI with host buffers: upload the initial
    # fields from pinned memory, K steps, download rho and u.
    e2e = None
    if not args.no_e2e:
        rho_h = torch.from_numpy(np.ascontiguousarray(rho0)).pin_memory()
        u_h = torch.from_numpy(np.ascontiguousarray(u0)).pin_memory()
        rho_out = torch.empty_like(rho_h).pin_memory()
        u_out = torch.empty_like(u_h).pin_memory()
        lat.sync()
        dist.barrier()
        t0 = time.perf_counter()
        lat.lib.lb_init_fields(lat.handle, rho_h.data_ptr(), u_h.data_ptr())
        if slab is None:
            lat.step(K)
        else:
            slab.halo()
            for _ in range(K):
                step()
        st = lat.lib.lb_moments(lat.handle, rho_out.data_ptr(), u_out.data_ptr())
        t1 = time.perf_counter()
        assert st == 0
        dist.barrier()
        e2e_val, _ = aggregate_replicas(dist, N, K, t1 - t0)
        moved = dist.sum(32 * rho_h.numel())  # rho + u, 8 + 24 bytes per cell, all ranks
        e2e = {"value": round(e2e_val, 1), "unit": "MLUPS",
               "h2d_bytes_per_step": int(moved / K), "d2h_bytes_per_step": int(moved / K),
               "what": "lb_init_fields(host rho,u) + lb_step(K) + lb_moments(host rho,u), pinned host buffers"
                       + ("; z-slab halo exchange after every step" if slab is not None else "")}

    peak, peak_kind = measured_peaks()
    bpu = bytes_per_update(args.storage)
    achieved = bpu * N / (kernel_ms / 1e3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
            "frac": round(achieved / peak, 4), "peak_kind": peak_kind,
            "traffic": ncu_traffic(f"step_{args.storage}_tgv{n}" + ("_inplace" if args.inplace else ""),
                                   tuned[0] if tuned else args.kernel),
            "algorithmic_bytes_per_launch": bpu * N, "kernel": "lb step kernel",
            "kernel_ms_mean": round(kernel_ms, 5), "kernel_ms_median": round(statistics.median(step_ms), 5),
            # the same figure against the nominal HBM3e bandwidth, for context
            "frac_of_nominal": round(achieved / NOMINAL_HBM_GBS, 4), "nominal_peak": NOMINAL_HBM_GBS}

    line = {
        "metric": METRIC, "value": round(value, 1), "unit": "MLUPS", "n_gpus": dist.world,
        "steps": K, "warmup": args.warmup, "ms_per_step": round(t_max * 1e3 / K, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"f64": "f64", "f32": "f32", "f16s": "f16", "bf16s": "bf16", "f32d": "f32+f64",
                  "e3m12s": "e3m12"}[args.storage],
        "data": "synthetic",
        "config": {**reference_config(args),
                   "workload": (f"taylor-green vortex {n}^3, D3Q19 BGK, {args.storage} populations "
                                f"(f - w), tau={tau}, u0=0.05, k=2pi/{n}") if slab is None else
                               (f"taylor-green vortex {n}x{n}x{n * dist.world} in {dist.world} z-slabs of "
                                f"{n}^3, D3Q19 BGK, {args.storage} populations (f - w), tau={tau}, u0=0.05"),
                   "lattice": [n, n, n * (dist.world if slab is not None else 1)],
                   "parallelism": ("single" if dist.world == 1 else
                                   "replicas" if slab is None else
                                   f"z-slabs over {dist.world} GPUs, halo exchange by NCCL send/recv")},
        "kernel": ({"variant": tuned[0], "block": tuned[1], "chosen_by": "lb_autotune"}
                   if tuned else {"variant": args.kernel, "block": args.block, "chosen_by": "command line"}),
        "roofline": roof,
        "e2e": e2e,
        # step launches, 2 per FP64 check; z-slabs: + halo pack and unpack per step
        "gpu_launches": K + launches_per_check * n_checks + (2 * K if slab is not None else 0),
        "clocks": clock_summary,
        "mass_drift_rel": abs(mass - N * dist.world) / (N * dist.world) if slab is not None else abs(mass - N) / N,
    }
    lat.close()
    return line


# ---------------------------------------------------------------- other forms
def forms_section(n, steps=200, device=None):
    """Short timed runs of the same Taylor-Green lattice in the other storage
    forms, the in-place layout and the TRT collision (autotuned kernel, CUDA
    events on the lattice's stream, 5 warm-up steps): GLUPS and the fraction
    of the measured HBM bandwidth at the algorithmic bytes per update."""
    import torch

    from paper_2409_16781_gb300 import Lattice
    peak, peak_kind = measured_peaks()
    rho0, u0 = tgv_inputs(n)
    out = []
    for storage, inplace, trt, rounding in (("f16s", False, 0.0, "nearest"), ("f16s", False, 0.0, "stochastic"),
                                            ("bf16s", False, 0.0, "nearest"), ("f64", False, 0.0, "nearest"),
                                            ("f32d", False, 0.0, "nearest"), ("f32", False, 3 / 16, "nearest"),
                                            ("f32", True, 0.0, "nearest"), ("f16s", True, 0.0, "nearest"),
                                            ("e3m12s", False, 0.0, "stochastic")):
        stream = torch.cuda.current_stream(device)
        lat = Lattice(n, n, n, 0.55, storage=storage, stream=stream, device=device, inplace=inplace,
                      trt_magic=trt, rounding=rounding)
        lat.init_fields(rho0, u0)
        v, b, _ = lat.autotune(reps=10, cache=False)
        k = steps if STORAGE_BYTES[storage] <= 4 and storage != "f32d" else steps // 4
        lat.step(5)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(device)
        e0.record(stream)
        lat.step(k)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1) / k
        glups = n ** 3 / ms / 1e6
        gbs = glups * bytes_per_update(storage)
        out.append({"storage": storage, "populations": "in place" if inplace else "two arrays",
                    "collision": "TRT 3/16" if trt else "BGK", "rounding": rounding,
                    "variant": v, "block": b, "steps": k,
                    "glups": round(glups, 2), "gbs": round(gbs, 1),
                    "frac": round(gbs / peak, 4), "peak_kind": peak_kind,
                    "bytes_per_update": bytes_per_update(storage)})
        if storage in ("f64", "f32d"):
            out[-1]["alu"] = fp64_alu_roofline(storage, v, glups)
        lat.close()
        del lat
    return out


# ---------------------------------------------------------------- serving
def run_serving(n_requests, rate_multipliers=(2.0,), budget_gb=64.0, seed=16781, calib=16,
                device=None, tight_budget_gb=0.75, max_wait_s=60.0, log_prefix=None, rounding="stochastic",
                accuracy_every=1):
    """Continuous-batching serving of a seeded Poisson stream of cavity /
    channel requests (sizes log-uniform 16^3..192^3, aspect <= 4, tau in
    [0.52, 1], steps in [200, 5000], FP32 / shifted-FP16 50/50, the FP16
    requests' stored values rounded as `rounding`), against the same stream
    served one plain FP32 lattice at a time.  Arrival rates are set as
    multiples of the measured sequential FP32 capacity.  The velocity error
    of the FP16 requests (every `accuracy_every`-th of them) against FP32 is
    in f16s_accuracy."""
    import torch

    from paper_2409_16781_gb300 import workloads as W
    from paper_2409_16781_gb300.serve import BatchBackend, SequentialBackend, serve

    torch.cuda.synchronize()
    # sequential FP32 capacity: service time of the first `calib` requests
    # presented at once (arrivals zeroed)
    base = W.request_stream(n=n_requests, rate_hz=1.0, seed=seed)
    cal = [W.Request(**{**r.__dict__, "arrival_s": 0.0}) for r in base[:calib]]
    st = serve(cal, SequentialBackend("f32", device=device))
    capacity = len(cal) / max(st.makespan, 1e-9)      # requests per second
    out = {"requests": n_requests, "capacity_req_per_s": round(capacity, 3),
           "hbm_budget_gb": budget_gb,
           "storage_mix": f"f32/f16s 50/50, f16s rounded {rounding}; f16s requests whose predicted "
                          "deviations are below 2^-13 served in f32 (batched); f32 (sequential)",
           "policy": "batched: shortest remaining work first"
                     + (f", requests waiting over {max_wait_s:g} s first (oldest first)" if max_wait_s else "")
                     + ", 4M-cell occupancy target, 8 ms chunks, 3 queued; sequential: FIFO, one lattice "
                       "at a time, one launch per step",
           "runs": []}
    out["f16s_accuracy"] = f16s_accuracy(base, every=accuracy_every, device=device, rounding=rounding)
    for mult in rate_multipliers:
        reqs = W.request_stream(n=n_requests, rate_hz=mult * capacity, seed=seed)
        be = BatchBackend(int(budget_gb * (1 << 30)), max_slots=1024, device=device, rounding=rounding,
                          promote=True)
        sb = serve(reqs, be, policy="srpt", target_cells=4_000_000, max_wait_s=max_wait_s)
        be.close()
        torch.cuda.synchronize()
        ss = serve(reqs, SequentialBackend("f32", device=device))
        torch.cuda.synchronize()
        if log_prefix:   # one JSON line per request (serve.ServeStats.records)
            sb.write_jsonl(f"{log_prefix}_{mult:g}x_batched.jsonl")
            ss.write_jsonl(f"{log_prefix}_{mult:g}x_sequential.jsonl")
        out["runs"].append({"rate_multiplier": mult, "rate_hz": round(mult * capacity, 3),
                            "batched": sb.summary(), "sequential_fp32": ss.summary()})
    if tight_budget_gb:
        # the same stream against a small HBM budget, where admission is bound
        # by memory: slots with two population arrays vs in-place slots (one
        # array, about half the bytes per request)
        mult = rate_multipliers[-1]
        reqs = W.request_stream(n=n_requests, rate_hz=mult * capacity, seed=seed)
        tight = {"budget_gb": tight_budget_gb, "rate_multiplier": mult}
        for name, inplace in (("two_arrays", False), ("in_place", True)):
            be = BatchBackend(int(tight_budget_gb * (1 << 30)), max_slots=1024, device=device, inplace=inplace,
                              rounding=rounding, promote=True)
            st = serve(reqs, be, policy="srpt", target_cells=4_000_000, max_wait_s=max_wait_s)
            be.close()
            torch.cuda.synchronize()
            tight[name] = st.summary()
        out["memory_bound"] = tight
    return out


def f16s_accuracy(requests, every=1, device=None, rounding="stochastic"):
    """Velocity error of the FP16-storage requests as the batched server
    serves them: every `every`-th FP16 request (in request order) that the
    storage policy keeps in FP16 runs alone in FP16S, rounded as the server
    rounds it (a slot gives bitwise the lattice-alone result), and in FP32;
    max |u16 - u32| / max |u32| over fluid cells.  Requests the policy
    serves in FP32 are counted as promoted."""
    from paper_2409_16781_gb300 import Lattice
    from paper_2409_16781_gb300.serve import served_storage
    sixteen = [r for r in requests if r.storage == "f16s"]
    promoted = sum(served_storage(r) != "f16s" for r in sixteen)
    pick = [r for r in sixteen if served_storage(r) == "f16s"][::max(1, int(every))]
    errs = []
    for r in pick:
        u = {}
        for storage, rnd in (("f32", "nearest"), ("f16s", rounding)):
            lat = Lattice(r.nx, r.ny, r.nz, r.tau, u_lid=r.u_lid, flags=r.flags(), storage=storage,
                          force=r.force, device=device, rounding=rnd)
            lat.step(r.steps)
            u[storage] = lat.moments()[1]
            lat.close()
        mask = r.flags() == 0
        ref = u["f32"][:, mask]
        errs.append(float(abs(u["f16s"][:, mask] - ref).max() / max(abs(ref).max(), 1e-30)))
    worst = sorted(zip(errs, pick), key=lambda t: -t[0])[:5]
    return {"checked": len(errs), "of_f16s_requests": len(sixteen), "promoted_to_f32": promoted,
            "rounding": rounding, "max_err": max(errs) if errs else None,
            "median_err": sorted(errs)[len(errs) // 2] if errs else None,
            "within_2e-3": sum(e <= 2e-3 for e in errs),
            "worst": [{"rid": r.rid, "dims": [r.nx, r.ny, r.nz], "tau": round(r.tau, 3), "steps": r.steps,
                       "kind": r.kind, "err": e} for e, r in worst]}


# ---------------------------------------------------------------- oracle
def oracle_slab_run(n, planes, steps):
    """Run the FP64 oracle for `steps` steps on an n x n x planes slab of the
    Taylor-Green lattice; returns (seconds, cells)."""
    import oracle as O
    from paper_2409_16781_gb300 import workloads as W
    rho, u = W.taylor_green_fields(n, n, n, u0=0.05)
    L = O.Lattice(n, n, planes, 0.55)
    L.init_fields(rho[:planes], u[:, :planes])
    t0 = time.perf_counter()
    L.step(steps)
    return time.perf_counter() - t0, n * n * planes


def oracle_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v else (os.cpu_count() or 1)


def cpu_baseline(n, budget_s=12.0, single_budget_s=4.0):
    """Oracle MLUPS on a bounded sample: an n x n x 16 slab, as many steps as
    fit in about budget_s seconds (at least 2), on all host cores; and the
    same on one thread (a child process with OMP_NUM_THREADS=1, a smaller
    sample of about single_budget_s seconds)."""
    planes = 16
    t1, cells = oracle_slab_run(n, planes, 1)
    steps = max(2, min(200, int(budget_s / max(t1, 1e-3))))
    t, cells = oracle_slab_run(n, planes, steps)
    out = {"value": round(cells * steps / t / 1e6, 2), "unit": "MLUPS", "cores": oracle_threads(),
           "kind": "oracle",
           "sample": f"{steps} steps of a {n}x{n}x{planes} slab of the {n}^3 Taylor-Green lattice "
                     f"(FP64 C oracle, OpenMP over z)"}
    code = ("import sys, json; sys.path.insert(0, %r); import bench; "
            "t1, c = bench.oracle_slab_run(%d, 4, 1); k = max(2, min(100, int(%f / max(t1, 1e-3)))); "
            "t, c = bench.oracle_slab_run(%d, 4, k); print(json.dumps([c * k / t / 1e6, k]))"
            % (ROOT, n, single_budget_s, n))
    try:
        r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=120,
                           env={**os.environ, "OMP_NUM_THREADS": "1"})
        v, k = json.loads(r.stdout.strip().splitlines()[-1])
        out["single_thread"] = {"value": round(v, 2), "unit": "MLUPS", "cores": 1,
                                "sample": f"{k} steps of a {n}x{n}x4 slab, OMP_NUM_THREADS=1"}
    except (subprocess.SubprocessError, ValueError, IndexError, OSError):
        out["single_thread"] = None
    return out


def reference_config(args):
    """The `config` of our arm's line for the same arguments (N = 1), so that
    the two arms' lines name the same workload."""
    n, tau = args.n, 0.55
    return {"workload": f"taylor-green vortex {n}^3, D3Q19 BGK, {args.storage} populations "
                        f"(f - w), tau={tau}, u0=0.05, k=2pi/{n}",
            "lattice": [n, n, n], "storage": args.storage, "tau": tau,
            "populations": "one array, in place (AA pattern)" if args.inplace else "two arrays (A -> B)",
            "collision": f"TRT, magic {args.trt_magic}" if args.trt_magic else "BGK",
            "check_every": args.check_every,
            "l2": f"no flush: working set {2 * 19 * STORAGE_BYTES[args.storage] * n ** 3 / 1e9:.2f} GB "
                  "> 129 MB L2",
            "parallelism": "single"}


def run_reference(args, dist: Dist):
    n = args.n
    # calibrate: one step on an 8-plane slab, then size the per-step sample
    t_cal, cells_cal = oracle_slab_run(n, 8, 1)
    rate = cells_cal / max(t_cal, 1e-6)           # cells per second
    budget = 60.0                                  # seconds for the timed steps
    planes = int(max(1, min(n, budget * rate / max(1, args.steps) / (n * n))))
    import oracle as O
    from paper_2409_16781_gb300 import workloads as W
    rho, u = W.taylor_green_fields(n, n, n, u0=0.05)
    L = O.Lattice(n, n, planes, 0.55)
    L.init_fields(rho[:planes], u[:, :planes])
    for _ in range(args.warmup):
        L.step(1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        L.step(1)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    cells = n * n * planes
    value = cells * args.steps / total / 1e6
    sample = (f"each step: one oracle update of a {n}x{n}x{planes} slab ({cells} cells) of the "
              f"{n}^3 Taylor-Green lattice, FP64 C oracle, OpenMP over z")
    return {
        "metric": METRIC, "value": round(value, 3), "unit": "MLUPS", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total * 1e3 / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": reference_config(args),
        "cpu_baseline": {"value": round(value, 3), "unit": "MLUPS", "cores": oracle_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": "MLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }


def main(argv=None):
    args = parse_args(argv)
    if args.impl == "reference":
        rank = int(os.environ.get("RANK", "0"))
        if rank != 0:
            return 0
        print(json.dumps(run_reference(args, _single())))
        return 0
    dist = Dist()
    try:
        if args.workload in ("serve", "porous", "precision", "vks"):
            fn = {"serve": serve_line, "porous": porous_line, "precision": precision_line,
                  "vks": vks_line}[args.workload]
            if dist.rank == 0:
                print(json.dumps(fn(args)), flush=True)
            return 0
        line = run_ours(args, dist)

        def soft(fn):  # a failed extra section is reported in the line, which is still printed
            try:
                return fn()
            except Exception as e:
                return {"error": f"{type(e).__name__}: {e}"}
        if dist.rank == 0 and dist.world == 1 and not args.no_forms:
            line["other_forms"] = soft(lambda: forms_section(args.n))
        n_serve = 80 if args.serve_requests is None else args.serve_requests
        if dist.rank == 0 and dist.world == 1 and n_serve > 0:
            line["serving"] = soft(lambda: run_serving(n_serve, (2.0,), args.serve_budget_gb,
                                                       tight_budget_gb=args.serve_tight_gb,
                                                       max_wait_s=args.serve_max_wait or None,
                                                       rounding=args.serve_rounding))
        elif dist.rank == 0:
            line["serving"] = None
        if dist.rank == 0 and dist.world == 1 and not args.no_configs:
            line["configs"] = configs_section(args)
        if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = soft(lambda: cpu_baseline(args.n))
        elif dist.rank == 0:
            line["cpu_baseline"] = None
        if dist.rank == 0:
            print(json.dumps(line), flush=True)
    finally:
        dist.close()
    return 0


def configs_section(args):
    """The other configurations of the workload list, measured in the
    default run: porous channel 512^3 (FP32, and FP16 rounded
    stochastically), the 768^3 cavity precision study, and the
    2000-request serving stream at 0.5x and 2x the sequential FP32
    capacity (p50 / p99 for both servers; the FP16 requests' error checked
    on every tenth of them)."""
    import torch
    out = {}
    t0 = time.time()
    sections = (
        ("porous_512", porous_section),
        ("cavity_768_precision",
         lambda: precision_section(args.precision_steps, tuple(float(t) for t in args.taus.split(",")))),
        ("serving_2000",
         lambda: run_serving(2000, (0.5, 2.0), args.serve_budget_gb, tight_budget_gb=0,
                             max_wait_s=args.serve_max_wait or None, rounding=args.serve_rounding,
                             accuracy_every=10)),
    )
    for name, fn in sections:
        t1 = time.time()
        if t1 - T_START > args.configs_deadline_s:
            out[name] = {"skipped": f"started {t1 - T_START:.0f} s after the process, past the "
                                    f"{args.configs_deadline_s:.0f} s deadline"}
            continue
        try:
            out[name] = fn()
        except Exception as e:  # a failed section is reported, the line still printed
            out[name] = {"error": f"{type(e).__name__}: {e}"}
        out[name + "_wall_s"] = round(time.time() - t1, 1)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
    out["wall_s"] = round(time.time() - t0, 1)
    return out


def porous_section(forms=(("f32", "nearest"), ("f16s", "stochastic")), steps=200, warmup=5):
    """Porous channel 512^3, tau 0.8, g = 1e-6 x, walls on the y/z faces,
    400 spheres (radius U[8,24], SplitMix64 seed 2409), in each storage
    form: GLUPS over all cells and over fluid cells (CUDA events on the
    lattice's stream around `steps` steps, autotuned kernel), the fraction of
    the measured HBM bandwidth at the algorithmic bytes per update, and the
    FP64 mass drift and momentum."""
    import torch

    from paper_2409_16781_gb300 import Lattice
    from paper_2409_16781_gb300 import workloads as W
    n = 512
    flags = W.porous_flags(n, n, n, n_spheres=400, r_min=8, r_max=24, seed=2409)
    fluid = int((flags == 0).sum())
    N = n ** 3
    peak, kind = measured_peaks()
    stream = torch.cuda.current_stream()
    out = {"lattice": [n, n, n], "solid_fraction": round(1 - fluid / N, 4), "steps": steps, "peak_kind": kind,
           "forms": []}
    for storage, rounding in forms:
        lat = Lattice(n, n, n, 0.8, flags=flags, storage=storage, force=(1e-6, 0.0, 0.0), stream=stream,
                      rounding=rounding)
        v, b, _ = lat.autotune(reps=10, cache=False)
        lat.step(warmup)
        m0, _ = lat.totals()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        e1.synchronize()
        sec = e0.elapsed_time(e1) / 1e3
        m1, p1 = lat.totals()
        lat.close()
        glups = N * steps / sec / 1e9
        gbs = glups * bytes_per_update(storage)
        out["forms"].append({"storage": storage, "rounding": rounding, "variant": v, "block": b,
                             "glups": round(glups, 2), "fluid_glups": round(glups * fluid / N, 2),
                             "gbs": round(gbs, 1), "frac": round(gbs / peak, 4),
                             "mass_drift_rel": abs(m1 - m0) / m0, "momentum_x": p1[0]})
    return out


def porous_line(args):
    """The porous channel (porous_section) in --storage as its own line."""
    rounding = "stochastic" if STORAGE_BYTES[args.storage] == 2 else "nearest"
    sec = porous_section(((args.storage, rounding),), steps=args.steps, warmup=args.warmup)
    f = sec["forms"][0]
    peak, kind = measured_peaks()
    return {"metric": METRIC, "value": round(f["glups"] * 1e3, 1), "unit": "MLUPS", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(512 ** 3 / f["glups"] / 1e6, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.storage,
            "data": "synthetic",
            "config": {"workload": "porous channel 512^3, D3Q19 BGK, tau 0.8, g 1e-6 x, 400 spheres r U[8,24]",
                       "solid_fraction": sec["solid_fraction"], "rounding": rounding,
                       "kernel": {"variant": f["variant"], "block": f["block"], "chosen_by": "lb_autotune"}},
            "fluid_mlups": round(f["fluid_glups"] * 1e3, 1),
            "roofline": {"bound": "hbm", "achieved": f["gbs"], "peak": peak, "unit": "GB/s", "frac": f["frac"],
                         "peak_kind": kind},
            "mass_drift_rel": f["mass_drift_rel"], "momentum_x": f["momentum_x"]}


def vks_line(args):
    """Flow past a cylinder, the paper's von Karman street use case in 3D:
    1024 x 256 x 64 cells, a cylinder along z of diameter D = 32 at x = 8D,
    far-field (free stream) planes at x = 0 and x = nx-1, periodic y and z,
    free stream U = 0.05 along x, Re = U D / nu = 100.  Throughput: CUDA
    events around 2000 steps (autotuned kernel); then a longer run started
    from the free stream with a small asymmetric kick measures the shedding
    frequency from u_y one diameter pair behind the cylinder (Strouhal
    number St = f D / U; about 0.16-0.19 expected at Re 100 for an
    unconfined to 1/8-blocked cylinder -- a check of the physics, not a
    parity pin)."""
    import numpy as np
    import torch

    from paper_2409_16781_gb300 import Lattice, velocity_set
    from paper_2409_16781_gb300 import workloads as W
    nx, ny, nz, D, U, Re = 1024, 256, 64, 32, 0.05, 100.0
    tau = 0.5 + 3.0 * U * D / Re
    cx, cy = 8 * D, ny / 2 + 0.5
    flags = W.cylinder_flags(nx, ny, nz, diameter=D, cx=cx, cy=cy)
    N = nx * ny * nz
    fluid = int((flags == 0).sum())
    stream = torch.cuda.current_stream()
    lat = Lattice(nx, ny, nz, tau, u_lid=(U, 0.0, 0.0), flags=flags, storage=args.storage, stream=stream,
                  trt_magic=args.trt_magic, inplace=args.inplace)
    u0 = np.zeros((3, nz, ny, nx))
    u0[0] = U
    u0[0][flags != 0] = 0.0
    # an asymmetric kick behind the cylinder so that shedding starts early
    kick = np.zeros((nz, ny, nx), bool)
    kick[:, int(cy):int(cy) + D, int(cx) + D // 2:int(cx) + 3 * D] = True
    u0[1][kick & (flags == 0)] = 0.2 * U
    lat.init_fields(None, u0)
    v, b, _ = lat.autotune(reps=10, cache=False)
    lat.step(20)
    K = 2000
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    lat.step(K)
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1) / K
    mlups = N / ms / 1e3
    # shedding frequency
    lat.init_fields(None, u0)
    c, _ = velocity_set()
    probe = np.array([int(cx + 2 * D) + nx * (int(cy) + ny * (nz // 2))])
    every, uy = 25, []
    for _ in range(args.vks_steps // every):
        lat.step(every)
        f = lat.populations_at(probe)[0]
        uy.append(float(f @ c[:, 1]) / float(f.sum()))
    uy = np.array(uy)
    # the period from the zero crossings (linear interpolation) of u_y over
    # the second half of the run, once the street is established
    tail = uy[len(uy) // 2:] - uy[len(uy) // 2:].mean()
    t = (np.arange(len(tail)) + len(uy) - len(tail)) * every
    up = np.nonzero((tail[:-1] < 0) & (tail[1:] >= 0))[0]
    tc = t[up] + every * (-tail[up]) / (tail[up + 1] - tail[up])
    st = float(D / (U * np.diff(tc).mean())) if len(tc) >= 2 else None
    m, _ = lat.totals()
    lat.close()
    peak, peak_kind = measured_peaks()
    gbs = mlups * 1e6 * bytes_per_update(args.storage) / 1e9
    return {
        "metric": METRIC, "value": round(mlups, 1), "unit": "MLUPS", "n_gpus": 1, "steps": K, "warmup": 20,
        "ms_per_step": round(ms, 5), "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.storage, "data": "synthetic",
        "config": {"workload": f"von Karman street (flow past a cylinder) {nx}x{ny}x{nz}, D={D}, "
                               f"U={U}, Re={Re:g}, tau={tau:.4f}, {args.storage} populations, far-field "
                               "inflow/outflow planes, periodic y and z",
                   "kernel": {"variant": v, "block": b}, "inplace": bool(args.inplace),
                   "collision": f"TRT {args.trt_magic}" if args.trt_magic else "BGK"},
        "fluid_mlups": round(mlups * fluid / N, 1),
        "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(gbs / peak, 4), "peak_kind": peak_kind, "traffic": None},
        "shedding": {"strouhal": None if st is None else round(st, 4), "periods_seen": int(max(len(tc) - 1, 0)),
                     "probe": "u_y at (x0 + 2D, y0, nz/2)",
                     "samples": len(uy), "every_steps": every, "steps": args.vks_steps,
                     "uy_amplitude_over_U": round(float(np.abs(tail).max()) / U, 4)},
        "mass_per_fluid_cell": m / fluid,
        "gpu_launches": K,
    }


# every tau: the two forms gated at 2e-3; the last tau also the contrasts
# (FP16 rounded to nearest, BF16)
PRECISION_FORMS = (("f16s", "stochastic"), ("e3m12s", "stochastic"))
PRECISION_CONTRASTS = (("f16s", "nearest"), ("bf16s", "stochastic"))


def precision_section(steps=5000, taus=(0.52, 0.56, 0.6), n=768, small=64):
    """Lid-driven cavity n^3 (lid (0.1, 0, 0)) with the populations stored as
    f - w in FP16 (rounded to nearest even, and stochastically), E3M12 and
    BF16 (stochastically), FP32 math, against the FP32 run of the same case:
    max |u - u_f32| / max |u_f32| over the lattice after `steps` steps, mass
    drift from the FP64 reduction, GLUPS and the fraction of the measured
    HBM bandwidth; plus the small^3 copy of the case (tau 0.6) against the
    FP64 oracle."""
    import numpy as np
    import torch

    import oracle as O
    from paper_2409_16781_gb300 import Lattice, LbDiverged
    from paper_2409_16781_gb300 import workloads as W
    K = int(steps)
    flags = W.cavity_flags(n, n, n)
    peak, peak_kind = measured_peaks()
    out = {"lattice": [n, n, n], "steps": K, "lid": [0.1, 0.0, 0.0], "peak_kind": peak_kind, "runs": []}
    stream = torch.cuda.current_stream()

    def run(storage, rounding, tau):
        lat = Lattice(n, n, n, tau, u_lid=(0.1, 0, 0), flags=flags, storage=storage, stream=stream,
                      rounding=rounding)
        v, b, _ = lat.autotune(reps=3, cache=False)
        m0, _ = lat.totals()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        done, diverged, sec = 0, None, 0.0
        while done < K:
            k = min(1000, K - done)
            e0.record(stream)
            lat.step(k)
            e1.record(stream)
            e1.synchronize()
            sec += e0.elapsed_time(e1) / 1e3
            done += k
            try:
                m1, _ = lat.totals()
            except LbDiverged:
                diverged = done
                break
        u = None if diverged else lat.moments_device()[1]
        lat.close()
        glups = done * n ** 3 / sec / 1e9
        rec = {"glups": round(glups, 2), "frac": round(glups * bytes_per_update(storage) / peak, 4),
               "variant": v, "block": b, "mass_drift": None if diverged else abs(m1 - m0) / m0,
               "diverged_at": diverged}
        return u, rec

    for tau in taus:
        u32, rec32 = run("f32", "nearest", tau)
        rec = {"tau": tau, "f32": rec32}
        umax = None if u32 is None else u32.abs().max().item()
        for storage, rounding in PRECISION_FORMS + (PRECISION_CONTRASTS if tau == taus[-1] else ()):
            u, r = run(storage, rounding, tau)
            r["u_err_vs_f32"] = None if (u is None or u32 is None) else (u - u32).abs().max().item() / umax
            rec[f"{storage}_{rounding}"] = r
            del u
            torch.cuda.empty_cache()
        del u32
        torch.cuda.empty_cache()
        out["runs"].append(rec)
    # the small copy against the FP64 oracle
    m = small
    fl = W.cavity_flags(m, m, m)
    ks = min(K, 5000)
    ora = O.Lattice(m, m, m, 0.6, u_lid=(0.1, 0, 0), flags=fl)
    ora.step(ks)
    _, u_o = ora.moments()
    mask = fl == 0
    vs = {"lattice": [m, m, m], "tau": 0.6, "steps": ks}
    for storage, rounding in (("f32", "nearest"),) + PRECISION_FORMS + PRECISION_CONTRASTS:
        lat = Lattice(m, m, m, 0.6, u_lid=(0.1, 0, 0), flags=fl, storage=storage, rounding=rounding)
        lat.step(ks)
        _, u_g = lat.moments()
        lat.close()
        vs[f"{storage}_{rounding}"] = float(np.abs(u_g[:, mask] - u_o[:, mask]).max() / np.abs(u_o[:, mask]).max())
    out["vs_oracle"] = vs
    return out


def precision_line(args):
    """The 768^3 cavity precision study (precision_section) as its own line."""
    taus = tuple(float(t) for t in args.taus.split(","))
    out = precision_section(args.precision_steps if args.precision_steps else args.steps, taus)
    last = out["runs"][-1]["f16s_stochastic"]
    return {"metric": METRIC, "value": round(last["glups"] * 1e3, 1), "unit": "MLUPS", "n_gpus": 1,
            "steps": out["steps"], "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f16", "data": "synthetic",
            "config": {"workload": "cavity 768^3 precision study: f - w stored in FP16 / BF16, FP32 math, "
                                   "vs the FP32 GPU run and the FP64 oracle at 64^3"},
            "precision": out}


def serve_line(args):
    """A full serving run: the request stream at 0.5x and 2x the sequential
    FP32 capacity; value = batched aggregate MLUPS at 2x."""
    n = args.serve_requests if args.serve_requests else 2000
    rates = tuple(float(r) for r in args.serve_rates.split(","))
    sv = run_serving(n, rates, args.serve_budget_gb, tight_budget_gb=args.serve_tight_gb,
                     max_wait_s=args.serve_max_wait or None, log_prefix=args.serve_log,
                     rounding=args.serve_rounding, accuracy_every=10 if n > 200 else 1)
    hi = sv["runs"][-1]
    return {"metric": METRIC, "value": hi["batched"]["mlups"], "unit": "MLUPS", "n_gpus": 1,
            "steps": None, "warmup": 0, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f16", "data": "synthetic",
            "config": {"workload": f"serving: {n} seeded Poisson cavity/channel requests, 16^3-192^3, "
                                   f"tau U[0.52,1], steps U[200,5000]",
                       "parallelism": "single"},
            "serving": sv}


def _single():
    d = Dist.__new__(Dist)
    d.rank, d.world, d.local_rank, d.pg = 0, int(os.environ.get("WORLD_SIZE", "1")), 0, False
    return d


if __name__ == "__main__":
    sys.exit(main())
