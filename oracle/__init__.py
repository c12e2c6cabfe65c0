"""FP64 CPU oracle for the D3Q19 BGK lattice update -- TEST INFRASTRUCTURE.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never imports, links or executes it, and it imports
nothing from the product package.

The arithmetic lives in ``lb_oracle.c`` (plain C, FP64, one loop per step of
arXiv 2409.16781 Eq. 1-3 and the fused pull scheme of Sec. 3.1); this module
compiles it with gcc and marshals numpy arrays.  Populations use the oracle's
own velocity order, reported by :func:`velocity_set`; callers that compare
with another implementation match directions by velocity vector.

Parity pins: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_pins.py`` (lattice isotropy, equilibrium and source moment
closed forms, rest fixed point, pure-streaming transport, conservation laws,
shear-wave and Taylor-Green decay rates, Couette and Poiseuille steady
profiles, Galilean advection, mirror symmetry, and a brute-force push stepper;
for the TRT collision: reduction to BGK, conservation, Lambda-independent
viscosity, and the exact Poiseuille parabola at Lambda = 3/16 for any tau).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lb_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblb_oracle.so")
_lock = threading.Lock()
_lib = None

Q = 19
FLUID, WALL, LID, FARFIELD = 0, 1, 2, 3


def compile_source(src: str, out: str) -> str:
    """gcc -O2 -fopenmp a C source of the oracle into a shared library."""
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11",
           "-o", tmp, src, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def build(force: bool = False) -> str:
    """Compile ``lb_oracle.c`` into ``liblb_oracle.so`` (gcc, -O2, OpenMP)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    return compile_source(_SRC, _LIB_PATH)


def load_library(path: str):
    """Load an oracle shared library and declare its C signatures."""
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    I = ctypes.c_int
    D = ctypes.c_double
    lib.lbo_velocity_set.argtypes = [P, P]
    lib.lbo_velocity_set.restype = I
    lib.lbo_equilibrium.argtypes = [D, P, P]
    lib.lbo_source.argtypes = [D, D, P, P, P]
    lib.lbo_init.argtypes = [I, I, I, P, P, P]
    lib.lbo_step.argtypes = [I, I, I, D, P, P, P, P, P]
    lib.lbo_run.argtypes = [I, I, I, D, P, P, P, P, P, I]
    lib.lbo_run.restype = I
    lib.lbo_moments.argtypes = [I, I, I, P, P, P, P, P, P]
    lib.lbo_totals.argtypes = [I, I, I, P, P, P, P, P]
    lib.lbo_step_trt.argtypes = [I, I, I, D, D, P, P, P, P, P]
    lib.lbo_run_trt.argtypes = [I, I, I, D, D, P, P, P, P, P, I]
    lib.lbo_run_trt.restype = I
    return lib


def trt_omega_minus(tau: float, magic: float = 3.0 / 16.0) -> float:
    """omega- from the TRT parameter Lambda = (1/omega+ - 1/2)(1/omega- - 1/2)."""
    return 1.0 / (magic / (tau - 0.5) + 0.5)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = load_library(build())
        return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def _flags(flags, n):
    if flags is None:
        return None
    f = np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
    if f.size != n:
        raise ValueError(f"flags has {f.size} entries, lattice has {n}")
    return f


def _lib_or_default(lib):
    return _load() if lib is None else lib


def velocity_set(lib=None):
    """(c[19,3] int, w[19] float64) in the oracle's order."""
    lib = _lib_or_default(lib)
    c = np.zeros((Q, 3), dtype=np.int32)
    w = np.zeros(Q, dtype=np.float64)
    lib.lbo_velocity_set(_ptr(c), _ptr(w))
    return c.astype(np.int64), w


def equilibrium(rho: float, u, lib=None) -> np.ndarray:
    """f^eq(rho, u) (Eq. 2-3) in the oracle's order."""
    lib = _lib_or_default(lib)
    u = _f64(u, (3,))
    out = np.zeros(Q)
    lib.lbo_equilibrium(float(rho), _ptr(u), _ptr(out))
    return out


def source(tau: float, rho: float, u, g, lib=None) -> np.ndarray:
    """Guo source S_i (the S_i of Eq. 1) in the oracle's order."""
    lib = _lib_or_default(lib)
    u = _f64(u, (3,))
    g = _f64(g, (3,))
    out = np.zeros(Q)
    lib.lbo_source(float(tau), float(rho), _ptr(u), _ptr(g), _ptr(out))
    return out


class Lattice:
    """A D3Q19 lattice on the CPU: post-collision array ``A`` of shape
    (19, nz, ny, nx) in the oracle's velocity order, plus a scratch ``B``."""

    def __init__(self, nx, ny, nz, tau, u_lid=(0.0, 0.0, 0.0), flags=None,
                 force=(0.0, 0.0, 0.0), lib=None, omega_minus=None):
        """omega_minus: None = BGK; otherwise the TRT odd-part rate."""
        self.lib = _lib_or_default(lib)
        self.omega_minus = None if omega_minus is None else float(omega_minus)
        self.nx, self.ny, self.nz = int(nx), int(ny), int(nz)
        self.N = self.nx * self.ny * self.nz
        self.tau = float(tau)
        self.u_lid = _f64(u_lid, (3,))
        self.g = _f64(force, (3,))
        self.flags = _flags(flags, self.N)
        self.A = np.zeros((Q, self.nz, self.ny, self.nx))
        self.B = np.zeros_like(self.A)
        self.init_fields()

    def init_fields(self, rho=None, u=None):
        """A <- f^eq(rho, u); rho is (nz,ny,nx) or None (=1), u is
        (3,nz,ny,nx) or None (=0).  B gets the same values."""
        r = None if rho is None else _f64(rho, (self.N,))
        uu = None if u is None else _f64(u, (3 * self.N,))
        self.lib.lbo_init(self.nx, self.ny, self.nz, _ptr(r), _ptr(uu), _ptr(self.A))
        self.B[...] = self.A

    def set_populations(self, f):
        """A <- f (19, nz, ny, nx) in the oracle's order; B gets a copy."""
        self.A[...] = _f64(f, self.A.shape)
        self.B[...] = self.A

    def step(self, n: int = 1):
        """n fused pull steps (the C loop alternates A and B)."""
        n = int(n)
        if n <= 0:
            return
        if self.omega_minus is None:
            which = self.lib.lbo_run(self.nx, self.ny, self.nz, self.tau, _ptr(self.u_lid),
                                     _ptr(self.g), _ptr(self.flags), _ptr(self.A),
                                     _ptr(self.B), n)
        else:
            which = self.lib.lbo_run_trt(self.nx, self.ny, self.nz, self.tau, self.omega_minus,
                                         _ptr(self.u_lid), _ptr(self.g), _ptr(self.flags),
                                         _ptr(self.A), _ptr(self.B), n)
        if which == 1:
            self.A, self.B = self.B, self.A

    def moments(self):
        """(rho (nz,ny,nx), u (3,nz,ny,nx)); solid cells are 0."""
        rho = np.zeros((self.nz, self.ny, self.nx))
        u = np.zeros((3, self.nz, self.ny, self.nx))
        self.lib.lbo_moments(self.nx, self.ny, self.nz, _ptr(self.u_lid), _ptr(self.g),
                             _ptr(self.flags), _ptr(self.A), _ptr(rho), _ptr(u))
        return rho, u

    def totals(self):
        """(mass, momentum[3]) over fluid cells."""
        out = np.zeros(4)
        self.lib.lbo_totals(self.nx, self.ny, self.nz, _ptr(self.u_lid), _ptr(self.g),
                            _ptr(self.flags), _ptr(self.A), _ptr(out))
        return float(out[0]), out[1:].copy()


def step_array(nx, ny, nz, tau, u_lid, force, flags, A, lib=None, omega_minus=None):
    """One step on a caller-supplied array A (19*N float64, oracle order);
    returns the new post-collision array (solid cells copied from A)."""
    lib = _lib_or_default(lib)
    A = _f64(A, (Q * nx * ny * nz,))
    B = A.copy()
    fl = _flags(flags, nx * ny * nz)
    if omega_minus is None:
        lib.lbo_step(int(nx), int(ny), int(nz), float(tau), _ptr(_f64(u_lid, (3,))),
                     _ptr(_f64(force, (3,))), _ptr(fl), _ptr(A), _ptr(B))
    else:
        lib.lbo_step_trt(int(nx), int(ny), int(nz), float(tau), float(omega_minus),
                         _ptr(_f64(u_lid, (3,))), _ptr(_f64(force, (3,))), _ptr(fl), _ptr(A), _ptr(B))
    return B
