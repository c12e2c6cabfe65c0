"""Python binding of one D3Q19 lattice (argument marshalling over the C ABI).

PyTorch provides the device memory (one uint8 tensor handed to
``lb_create_in``) and the CUDA stream; every step of the computation runs in
the kernels of liblbgb.so.
"""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

from . import _lib as L

Q = L.Q


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def velocity_set():
    """(c[19,3], w[19]) in the library's order (include/lbgb.h)."""
    c = np.zeros(57, dtype=np.int32)
    w = np.zeros(19, dtype=np.float64)
    L.lib().lb_velocity_set(_dptr(c), _dptr(w))
    return c.reshape(19, 3).astype(np.int64), w


ROUNDING = {"nearest": 0, "stochastic": 1}


def make_options(storage="f32", force=(0.0, 0.0, 0.0), stream=None, kernel=0, block=0, trt_magic=0.0,
                 inplace=False, halo_z=False, rounding="nearest"):
    o = L.LbOptions()
    L.lib().lb_default_options(ctypes.byref(o))
    o.storage = L.STORAGE[storage] if isinstance(storage, str) else int(storage)
    o.kernel = int(kernel)
    o.block = int(block)
    o.trt_magic = float(trt_magic)
    o.inplace = 1 if inplace else 0
    o.halo_z = 1 if halo_z else 0
    o.rounding = ROUNDING[rounding] if isinstance(rounding, str) else int(rounding)
    for a in range(3):
        o.force[a] = float(force[a])
    o.stream = stream
    return o


def bytes_required(nx, ny, nz, storage="f32", inplace=False) -> int:
    o = make_options(storage, inplace=inplace)
    return int(L.lib().lb_bytes_required(int(nx), int(ny), int(nz), ctypes.byref(o)))


def autotune_key(device_name, storage, dims, force, flags, trt_magic=0.0, inplace=False,
                 rounding="nearest") -> str:
    """The autotune cache key: GPU, storage, dims, forcing, geometry (a digest
    of the flags, or "nowalls" when every cell is fluid), collision,
    population layout and rounding -- everything the fastest step kernel
    depends on."""
    import hashlib
    fl = None if flags is None else np.ascontiguousarray(flags, dtype=np.uint8)
    geo = ("walls:" + hashlib.blake2b(fl.tobytes(), digest_size=8).hexdigest()
           if fl is not None and fl.any() else "nowalls")
    nx, ny, nz = dims
    return "|".join([str(device_name), str(storage), f"{nx}x{ny}x{nz}", "force" if force else "noforce", geo]
                    + (["trt"] if trt_magic else []) + (["inplace"] if inplace else [])
                    + (["sr"] if rounding in ("stochastic", 1) else []))


class Lattice:
    """A lattice advanced by liblbgb on one GPU.

    Arrays follow the library's layout: scalar fields (nz, ny, nx), vector
    fields (3, nz, ny, nx), populations (19, nz, ny, nx) in the library's
    velocity order; flags uint8 (nz, ny, nx) with 0 fluid, 1 wall, 2 lid, 3 far field.
    trt_magic: 0 = BGK collision; > 0 = two-relaxation-time collision with
    that magic parameter (lb_options.trt_magic).
    inplace: one population array updated in place (lb_options.inplace).
    halo_z: a z-slab of a decomposed lattice, planes 0 and nz-1 being ghost
    planes (lb_options.halo_z; see halo_pack / halo_unpack and slab.py).
    rounding: "nearest" (default) or "stochastic" for 16-bit storage
    (lb_options.rounding).
    """

    def __init__(self, nx, ny, nz, tau, u_lid=(0.0, 0.0, 0.0), flags=None, storage="f32",
                 force=(0.0, 0.0, 0.0), device=None, stream=None, kernel=0, block=0,
                 library_memory=False, trt_magic=0.0, inplace=False, halo_z=False, rounding="nearest"):
        import torch

        self.lib = L.lib()
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.N = self.nx * self.ny * self.nz
        self.shape = (self.nz, self.ny, self.nx)
        self.tau = float(tau)
        self.storage = storage
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None \
            else torch.device(device)
        if stream is None:
            stream = torch.cuda.current_stream(self.device)
        self.stream = stream
        opts = make_options(storage, force, ctypes.c_void_p(stream.cuda_stream), kernel, block, trt_magic,
                            inplace, halo_z, rounding)
        self.halo_z = bool(halo_z)
        self.rounding = rounding
        self.trt_magic = float(trt_magic)
        self.inplace = bool(inplace)
        ulid = (ctypes.c_double * 3)(*[float(v) for v in u_lid])
        fl = None
        if flags is not None:
            fl = np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
            if fl.size != self.N:
                raise ValueError(f"flags has {fl.size} entries, lattice has {self.N}")
        self._flags = fl
        self._force = any(float(v) != 0.0 for v in force)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            if library_memory:
                self._buf = None
                st = self.lib.lb_create(ctypes.byref(h), self.nx, self.ny, self.nz, self.tau, ulid,
                                        None if fl is None else _dptr(fl), ctypes.byref(opts))
            else:
                nbytes = self.lib.lb_bytes_required(self.nx, self.ny, self.nz, ctypes.byref(opts))
                if nbytes == 0:
                    raise L.LbError(L.LB_EINVAL, f"bad lattice size {nx}x{ny}x{nz}")
                self._buf = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
                st = self.lib.lb_create_in(ctypes.byref(h), self.nx, self.ny, self.nz, self.tau, ulid,
                                           None if fl is None else _dptr(fl), ctypes.byref(opts),
                                           ctypes.c_void_p(self._buf.data_ptr()), nbytes)
        L.check(st, "lb_create")
        self._h = h

    # ------------------------------------------------------------------
    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            st = self.lib.lb_destroy(self._h)
            self._h = None
            L.check(st, "lb_destroy")
        self._buf = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ------------------------------------------------------------------
    def init_fields(self, rho=None, u=None):
        r = None if rho is None else np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        uu = None if u is None else np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        if r is not None and r.size != self.N:
            raise ValueError("rho has the wrong size")
        if uu is not None and uu.size != 3 * self.N:
            raise ValueError("u has the wrong size")
        L.check(self.lib.lb_init_fields(self._h, None if r is None else _dptr(r),
                                        None if uu is None else _dptr(uu)), "lb_init_fields")

    def step(self, n: int = 1):
        L.check(self.lib.lb_step(self._h, int(n)), "lb_step")

    def sync(self):
        L.check(self.lib.lb_sync(self._h), "lb_sync")

    def moments(self):
        rho = np.empty(self.shape)
        u = np.empty((3,) + self.shape)
        L.check(self.lib.lb_moments(self._h, _dptr(rho), _dptr(u)), "lb_moments")
        return rho, u

    def write_vtk(self, path: str, title: str = "lbgb fields"):
        """rho, u (lb_moments) and the flags as a legacy VTK file (vtk.write_vtk)."""
        from .vtk import write_vtk
        rho, u = self.moments()
        flags = None if self._flags is None else self._flags.reshape(self.shape)
        write_vtk(path, rho, u, flags, title=title)

    def moments_device(self, rho=None, u=None):
        """(rho, u) as float64 CUDA tensors, issued on the lattice's stream."""
        import torch
        if rho is None:
            rho = torch.empty(self.shape, dtype=torch.float64, device=self.device)
        if u is None:
            u = torch.empty((3,) + self.shape, dtype=torch.float64, device=self.device)
        L.check(self.lib.lb_moments_device(self._h, ctypes.c_void_p(rho.data_ptr()),
                                           ctypes.c_void_p(u.data_ptr())), "lb_moments_device")
        return rho, u

    def totals(self, check=True):
        m = ctypes.c_double()
        p = (ctypes.c_double * 3)()
        st = self.lib.lb_totals(self._h, ctypes.byref(m), p)
        if check:
            L.check(st, "lb_totals")
        return m.value, np.array(p[:])

    def populations(self):
        f = np.empty((Q,) + self.shape)
        L.check(self.lib.lb_get_populations(self._h, _dptr(f)), "lb_get_populations")
        return f

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64).reshape(-1)
        if f.size != Q * self.N:
            raise ValueError("populations have the wrong size")
        L.check(self.lib.lb_set_populations(self._h, _dptr(f)), "lb_set_populations")

    def checkpoint(self) -> bytes:
        """Bit-exact snapshot of the state (lb_checkpoint_save)."""
        n = int(self.lib.lb_checkpoint_bytes(self._h))
        buf = np.empty(n, dtype=np.uint8)
        L.check(self.lib.lb_checkpoint_save(self._h, _dptr(buf), n), "lb_checkpoint_save")
        return buf.tobytes()

    def restore(self, snapshot: bytes):
        """Restore a snapshot taken by checkpoint() of a lattice of the same
        dims, storage and population scheme (lb_checkpoint_load)."""
        buf = np.frombuffer(snapshot, dtype=np.uint8)
        L.check(self.lib.lb_checkpoint_load(self._h, _dptr(np.ascontiguousarray(buf)), int(buf.size)),
                "lb_checkpoint_load")

    def populations_at(self, cells):
        cells = np.ascontiguousarray(cells, dtype=np.int64).reshape(-1)
        out = np.empty((cells.size, Q))
        L.check(self.lib.lb_get_populations_at(self._h, _dptr(cells), int(cells.size), _dptr(out)),
                "lb_get_populations_at")
        return out

    def halo_bytes(self) -> int:
        """Bytes of one halo message (lb_halo_bytes; 0 without ghost planes)."""
        return int(self.lib.lb_halo_bytes(self._h))

    def halo_pack(self, send_lo, send_hi):
        """lb_halo_pack into two device tensors of halo_bytes() bytes each."""
        L.check(self.lib.lb_halo_pack(self._h, ctypes.c_void_p(send_lo.data_ptr()),
                                      ctypes.c_void_p(send_hi.data_ptr())), "lb_halo_pack")

    def halo_unpack(self, recv_lo, recv_hi):
        """lb_halo_unpack from two device tensors of halo_bytes() bytes each."""
        L.check(self.lib.lb_halo_unpack(self._h, ctypes.c_void_p(recv_lo.data_ptr()),
                                        ctypes.c_void_p(recv_hi.data_ptr())), "lb_halo_unpack")

    def set_kernel(self, variant: int, block: int = 0):
        L.check(self.lib.lb_set_kernel(self._h, int(variant), int(block)), "lb_set_kernel")

    def autotune(self, reps: int = 20, cache: bool = True):
        """Pick the fastest step-kernel variant and block size for this
        lattice (lb_autotune), remembering the choice in a JSON file keyed by
        GPU, storage, dims, forcing and geometry (a digest of the flags: the
        best kernel depends on how many cells are next to a wall)
        (LBGB_AUTOTUNE_CACHE, default ~/.cache/lbgb/autotune.json).
        Returns (variant, block, ms/step)."""
        import torch
        key = autotune_key(torch.cuda.get_device_name(self.device), self.storage, (self.nx, self.ny, self.nz),
                           self._force, self._flags, self.trt_magic, self.inplace, self.rounding)
        path = os.environ.get("LBGB_AUTOTUNE_CACHE",
                              os.path.join(os.path.expanduser("~"), ".cache", "lbgb", "autotune.json"))
        table = {}
        if cache and os.path.exists(path):
            try:
                with open(path) as fh:
                    table = json.load(fh)
            except (OSError, ValueError):
                table = {}
            if key in table:
                v, b, ms = table[key]
                self.set_kernel(v, b)
                return v, b, ms
        v = ctypes.c_int()
        b = ctypes.c_int()
        ms = ctypes.c_float()
        L.check(self.lib.lb_autotune(self._h, int(reps), ctypes.byref(v), ctypes.byref(b),
                                     ctypes.byref(ms)), "lb_autotune")
        if cache:
            table[key] = [v.value, b.value, ms.value]
            try:
                os.makedirs(os.path.dirname(path), exist_ok=True)
                tmp = f"{path}.{os.getpid()}"
                with open(tmp, "w") as fh:
                    json.dump(table, fh, indent=1, sort_keys=True)
                os.replace(tmp, path)
            except OSError:
                pass
        return v.value, b.value, ms.value

    def query(self):
        dims = (ctypes.c_int * 3)()
        st = ctypes.c_int()
        steps = ctypes.c_int64()
        L.check(self.lib.lb_query(self._h, dims, ctypes.byref(st), ctypes.byref(steps)), "lb_query")
        return tuple(dims), st.value, steps.value
