"""Python binding of a batch of lattices (argument marshalling over lb_batch_*).

PyTorch provides the device memory (one uint8 tensor handed to
lb_batch_create_in) and a dedicated CUDA stream; all work runs in liblbgb.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib as L
from .lattice import make_options

Q = L.Q


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def slot_bytes(nx, ny, nz, storage="f32", inplace=False) -> int:
    return int(L.lib().lb_batch_slot_bytes(int(nx), int(ny), int(nz), L.STORAGE[storage], 1 if inplace else 0))


def _bcheck(status: int, what: str):
    if status == L.LB_OK:
        return
    lib = L.lib()
    msg = lib.lb_batch_last_error().decode() or lib.lb_status_string(status).decode()
    cls = L.LbDiverged if status == L.LB_EDIVERGED else L.LbError
    raise cls(status, f"{what}: {msg}")


class Batch:
    """Many lattices with their own sizes, tau, storage and step budgets,
    resident in one device pool of ``capacity_bytes`` and advanced together."""

    def __init__(self, capacity_bytes: int, max_slots: int = 1024, device=None, stream=None,
                 library_memory: bool = False):
        import torch
        self.lib = L.lib()
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        # a non-default stream: the batch captures CUDA graphs on it
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        self.max_slots = int(max_slots)
        h = ctypes.c_void_p()
        fixed = int(self.lib.lb_batch_fixed_bytes(self.max_slots))
        if fixed == 0:
            raise L.LbError(L.LB_EINVAL, f"bad max_slots {max_slots}")
        with torch.cuda.device(self.device):
            if library_memory:
                self._buf = None
                st = self.lib.lb_batch_create(ctypes.byref(h), int(capacity_bytes), self.max_slots,
                                              ctypes.c_void_p(self.stream.cuda_stream))
            else:
                nbytes = fixed + int(capacity_bytes)
                self._buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
                torch.cuda.current_stream(self.device).synchronize()
                st = self.lib.lb_batch_create_in(ctypes.byref(h), ctypes.c_void_p(self._buf.data_ptr()),
                                                 nbytes, self.max_slots,
                                                 ctypes.c_void_p(self.stream.cuda_stream))
        _bcheck(st, "lb_batch_create")
        self._h = h
        self.meta = {}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            st = self.lib.lb_batch_destroy(self._h)
            self._h = None
            _bcheck(st, "lb_batch_destroy")
        self._buf = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------------
    def add(self, nx, ny, nz, tau, steps, u_lid=(0.0, 0.0, 0.0), flags=None, storage="f32",
            force=(0.0, 0.0, 0.0), trt_magic=0.0, inplace=False, rounding="nearest") -> int:
        """Admit a lattice; returns its slot.  Raises LbError with status
        LB_ENOMEM (pool full) or LB_EBUSY (no free slot) when it does not fit.
        trt_magic > 0 selects the two-relaxation-time collision; inplace keeps
        one population array (half the population memory)."""
        opts = make_options(storage, force, trt_magic=trt_magic, inplace=inplace, rounding=rounding)
        ulid = (ctypes.c_double * 3)(*[float(v) for v in u_lid])
        fl = None
        if flags is not None:
            fl = np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
            if fl.size != nx * ny * nz:
                raise ValueError("flags have the wrong size")
        slot = ctypes.c_int(-1)
        st = self.lib.lb_batch_add(self._h, int(nx), int(ny), int(nz), float(tau), ulid,
                                   None if fl is None else _dptr(fl), ctypes.byref(opts),
                                   int(steps), ctypes.byref(slot))
        _bcheck(st, "lb_batch_add")
        self.meta[slot.value] = (int(nx), int(ny), int(nz), storage)
        return slot.value

    def try_add(self, *args, **kw):
        """As add, but returns None instead of raising when the pool or the
        slot table is full."""
        try:
            return self.add(*args, **kw)
        except L.LbError as e:
            if e.status in (L.LB_ENOMEM, L.LB_EBUSY):
                return None
            raise

    def init_fields(self, slot, rho=None, u=None):
        r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        _bcheck(self.lib.lb_batch_init_fields(self._h, int(slot), None if r is None else _dptr(r),
                                              None if uu is None else _dptr(uu)), "lb_batch_init_fields")

    def set_steps(self, slot, steps):
        _bcheck(self.lib.lb_batch_set_steps(self._h, int(slot), int(steps)), "lb_batch_set_steps")

    def set_steps_many(self, slots, steps):
        ids = np.ascontiguousarray(slots, dtype=np.int32)
        cnt = np.ascontiguousarray(steps, dtype=np.int64)
        _bcheck(self.lib.lb_batch_set_steps_many(self._h, int(ids.size), _dptr(ids), _dptr(cnt)),
                "lb_batch_set_steps_many")

    def step(self, n: int = 1):
        _bcheck(self.lib.lb_batch_step(self._h, int(n)), "lb_batch_step")

    def poll(self):
        """Slots that have taken all their steps."""
        buf = (ctypes.c_int * self.max_slots)()
        nd = ctypes.c_int()
        _bcheck(self.lib.lb_batch_poll(self._h, buf, self.max_slots, ctypes.byref(nd)), "lb_batch_poll")
        return list(buf[:min(nd.value, self.max_slots)])

    def query(self, slot):
        rem = ctypes.c_int64()
        done = ctypes.c_int64()
        dims = (ctypes.c_int * 3)()
        st = ctypes.c_int()
        _bcheck(self.lib.lb_batch_query(self._h, int(slot), ctypes.byref(rem), ctypes.byref(done), dims,
                                        ctypes.byref(st)), "lb_batch_query")
        return {"remaining": rem.value, "done": done.value, "dims": tuple(dims), "storage": st.value}

    def moments(self, slot):
        nx, ny, nz, _ = self.meta[slot]
        rho = np.empty((nz, ny, nx))
        u = np.empty((3, nz, ny, nx))
        _bcheck(self.lib.lb_batch_moments(self._h, int(slot), _dptr(rho), _dptr(u)), "lb_batch_moments")
        return rho, u

    def totals(self, slot):
        m = ctypes.c_double()
        p = (ctypes.c_double * 3)()
        _bcheck(self.lib.lb_batch_totals(self._h, int(slot), ctypes.byref(m), p), "lb_batch_totals")
        return m.value, np.array(p[:])

    def populations(self, slot):
        nx, ny, nz, _ = self.meta[slot]
        f = np.empty((Q, nz, ny, nx))
        _bcheck(self.lib.lb_batch_get_populations(self._h, int(slot), _dptr(f)), "lb_batch_get_populations")
        return f

    def fetch(self, slot, rho, u):
        """Start the asynchronous read-back of a finished slot into host
        arrays rho (nz,ny,nx) and u (3,nz,ny,nx), float64, C-contiguous
        (pinned memory makes it truly asynchronous); keep them alive until
        fetch_done(slot) is True."""
        _bcheck(self.lib.lb_batch_fetch(self._h, int(slot), ctypes.c_void_p(rho.ctypes.data),
                                        ctypes.c_void_p(u.ctypes.data)), "lb_batch_fetch")

    def fetch_done(self, slot) -> bool:
        st = self.lib.lb_batch_fetch_done(self._h, int(slot))
        if st < 0:
            _bcheck(st, "lb_batch_fetch_done")
        return st == 1

    def remove(self, slot):
        _bcheck(self.lib.lb_batch_remove(self._h, int(slot)), "lb_batch_remove")
        self.meta.pop(slot, None)

    def free(self):
        fb = ctypes.c_size_t()
        fs = ctypes.c_int()
        _bcheck(self.lib.lb_batch_free_bytes(self._h, ctypes.byref(fb), ctypes.byref(fs)), "lb_batch_free_bytes")
        return fb.value, fs.value

    def sync(self):
        _bcheck(self.lib.lb_batch_sync(self._h), "lb_batch_sync")
