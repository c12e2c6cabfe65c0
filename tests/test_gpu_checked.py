"""Bounds-checked build (liblbgb_checked.so, -DLBGB_CHECKED): the same
sources with every population load and store of the step kernels checked
against its launch's arrays -- loads inside the array the step reads, stores
inside the array it writes.  An access outside would be counted and skipped
(never performed), so this finds a wrong index without faulting the GPU.
Every step variant, storage form and population layout runs on ragged
lattices with walls, lids, far-field cells and a body force; the test asserts
that the checks ran, that none failed, and that the checked build computes
exactly what the product build computes."""
import ctypes

import numpy as np
import pytest

from paper_2409_16781_gb300 import _lib as L
from paper_2409_16781_gb300 import build as B
from paper_2409_16781_gb300 import workloads as W
from paper_2409_16781_gb300.lattice import make_options

pytestmark = pytest.mark.gpu

SHAPES = ((34, 7, 6), (35, 6, 5), (48, 5, 4), (1, 1, 1), (2, 3, 1), (66, 3, 2), (64, 4, 3), (128, 3, 2))
STEPS = 3


@pytest.fixture(scope="module")
def libs():
    B.build()
    checked = L.load(B.build_checked())
    for name in ("lbgb_checked_violations_step", "lbgb_checked_violations_inplace"):
        fn = getattr(checked, name)
        fn.restype = ctypes.c_ulonglong
        fn.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_ulonglong)]
    return L.lib(), checked


def _violations(checked):
    total_v, total_c = 0, 0
    for name in ("lbgb_checked_violations_step", "lbgb_checked_violations_inplace"):
        c = ctypes.c_ulonglong()
        v = getattr(checked, name)(1, ctypes.byref(c))
        assert v != 2 ** 64 - 1, f"{name}: CUDA error"
        total_v += v
        total_c += c.value
    return total_v, total_c


def _flags(nx, ny, nz, seed):
    f = W.random_flags(nx, ny, nz, seed=seed, p_wall=0.15, p_lid=0.08)
    rng = np.random.default_rng(seed + 1)
    f.reshape(-1)[rng.random(f.size) < 0.05] = W.FARFIELD
    return f


def _run(lib, nx, ny, nz, storage, inplace, force, flags, rho, u, schedule):
    o = make_options(storage, force, None, 0, 0, 0.0, inplace)
    h = ctypes.c_void_p()
    ulid = (ctypes.c_double * 3)(0.05, 0.0, -0.02)
    L.check(lib.lb_create(ctypes.byref(h), nx, ny, nz, 0.7, ulid, flags.ctypes.data_as(ctypes.c_void_p),
                          ctypes.byref(o)), "lb_create")
    try:
        L.check(lib.lb_init_fields(h, rho.ctypes.data_as(ctypes.c_void_p), u.ctypes.data_as(ctypes.c_void_p)),
                "lb_init_fields")
        for v, block in schedule:
            L.check(lib.lb_set_kernel(h, v, block), "lb_set_kernel")
            L.check(lib.lb_step(h, STEPS), "lb_step")
        f = np.empty(19 * nx * ny * nz)
        L.check(lib.lb_get_populations(h, f.ctypes.data_as(ctypes.c_void_p)), "lb_get_populations")
        return f
    finally:
        lib.lb_destroy(h)


@pytest.mark.parametrize("inplace", [False, True], ids=["two_arrays", "in_place"])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s", "f32d", "e3m12s"])
def test_every_access_inside_its_array(libs, storage, inplace):
    plain, checked = libs
    variants = range(20) if not inplace else (0, 1, 2)
    schedule = [(v, b) for v in variants for b in (0, 32, 96)]
    _violations(checked)  # reset
    min_checks = 0
    for nx, ny, nz in SHAPES:
        flags = _flags(nx, ny, nz, seed=nx * 11 + nz)
        fluid = int((flags == 0).sum())
        rho, u = (np.ascontiguousarray(a, dtype=np.float64)
                  for a in W.random_fields(nx, ny, nz, seed=5, du=0.04, drho=0.01))
        for force in ((0.0, 0.0, 0.0), (1e-5, -2e-6, 3e-6)):
            a = _run(plain, nx, ny, nz, storage, inplace, force, flags, rho, u, schedule)
            b = _run(checked, nx, ny, nz, storage, inplace, force, flags, rho, u, schedule)
            assert np.array_equal(a.view(np.uint64), b.view(np.uint64)), \
                f"checked build differs: {storage} {nx}x{ny}x{nz} force={force}"
            # each launch stores every fluid cell's 19 values (and loads them,
            # through shared memory in the TMA variants), at most four values
            # per checked access
            min_checks += len(schedule) * STEPS * (fluid * 19 // 4)
    bad, checks = _violations(checked)
    assert bad == 0, f"{bad} population accesses outside their arrays ({storage}, in place={inplace})"
    assert checks >= min_checks > 0
