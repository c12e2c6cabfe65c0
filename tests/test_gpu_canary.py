"""Out-of-bounds write detection without a sanitizer: the library works in a
caller-owned device buffer (lb_create_in, lb_batch_create_in), so each test
places that buffer inside a larger torch allocation whose guard bands before
and after are filled with a pattern, runs every step variant (two arrays
and in place, every storage form, ragged row lengths, walls, lids, far-field
cells and a body force) and checks that the guard bands still hold the
pattern.  A kernel that stores past either end of its arrays changes a
guard byte."""
import ctypes

import numpy as np
import pytest

from paper_2409_16781_gb300 import _lib as L
from paper_2409_16781_gb300 import workloads as W
from paper_2409_16781_gb300.lattice import make_options

pytestmark = pytest.mark.gpu

GUARD = 1 << 16      # bytes before and after; a multiple of the 256-byte alignment
PATTERN = 0xA5
SHAPES = ((34, 7, 6), (35, 6, 5), (48, 5, 4), (1, 1, 1), (66, 3, 2), (64, 4, 3), (128, 3, 2))


def _flags(nx, ny, nz, seed):
    f = W.random_flags(nx, ny, nz, seed=seed, p_wall=0.15, p_lid=0.08)
    rng = np.random.default_rng(seed)
    f.reshape(-1)[rng.random(f.size) < 0.05] = W.FARFIELD
    return f


def _guarded(torch, nbytes):
    buf = torch.full((GUARD + nbytes + GUARD,), PATTERN, dtype=torch.uint8, device="cuda")
    torch.cuda.synchronize()
    return buf


def _guards_intact(torch, buf, nbytes):
    torch.cuda.synchronize()
    head = buf[:GUARD]
    tail = buf[GUARD + nbytes:]
    bad_head = int((head != PATTERN).sum())
    bad_tail = int((tail != PATTERN).sum())
    return bad_head, bad_tail


@pytest.mark.parametrize("inplace", [False, True], ids=["two_arrays", "in_place"])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16s", "bf16s", "f32d", "e3m12s"])
def test_step_variants_stay_inside_their_buffer(storage, inplace):
    import torch
    lib = L.lib()
    variants = range(0, 18) if not inplace else (0, 1, 2)
    for nx, ny, nz in SHAPES:
        flags = _flags(nx, ny, nz, seed=nx * 7 + ny)
        rho, u = (np.ascontiguousarray(a, dtype=np.float64)
                  for a in W.random_fields(nx, ny, nz, seed=3, du=0.04, drho=0.01))
        for force in ((0.0, 0.0, 0.0), (1e-5, -2e-6, 3e-6)):
            o = make_options(storage, force, None, 0, 0, 0.0, inplace)
            nbytes = int(lib.lb_bytes_required(nx, ny, nz, ctypes.byref(o)))
            assert nbytes > 0
            buf = _guarded(torch, nbytes)
            h = ctypes.c_void_p()
            ulid = (ctypes.c_double * 3)(0.05, 0.0, -0.02)
            L.check(lib.lb_create_in(ctypes.byref(h), nx, ny, nz, 0.7, ulid, flags.ctypes.data_as(ctypes.c_void_p),
                                     ctypes.byref(o), ctypes.c_void_p(buf.data_ptr() + GUARD), nbytes),
                    "lb_create_in")
            try:
                L.check(lib.lb_init_fields(h, rho.ctypes.data_as(ctypes.c_void_p),
                                           u.ctypes.data_as(ctypes.c_void_p)), "lb_init_fields")
                for v in variants:
                    for block in (0, 32, 96):
                        L.check(lib.lb_set_kernel(h, v, block), "lb_set_kernel")
                        L.check(lib.lb_step(h, 3), "lb_step")
                L.check(lib.lb_sync(h), "lb_sync")
                head, tail = _guards_intact(torch, buf, nbytes)
                assert head == 0 and tail == 0, \
                    f"{storage} {'in place' if inplace else 'two arrays'} {nx}x{ny}x{nz}: " \
                    f"{head} guard bytes changed before the buffer, {tail} after"
            finally:
                lib.lb_destroy(h)


def test_batch_pool_stays_inside_its_buffer():
    """A batch of mixed slots (every storage form, two arrays and in place,
    ragged shapes) stepping in shared launches writes only inside its pool."""
    import torch
    lib = L.lib()
    max_slots = 40
    fixed = int(lib.lb_batch_fixed_bytes(max_slots))
    cap = 64 << 20
    nbytes = fixed + cap
    buf = _guarded(torch, nbytes)
    stream = torch.cuda.Stream()
    h = ctypes.c_void_p()
    L.check(lib.lb_batch_create_in(ctypes.byref(h), ctypes.c_void_p(buf.data_ptr() + GUARD), nbytes, max_slots,
                                   ctypes.c_void_p(stream.cuda_stream)), "lb_batch_create_in")
    try:
        k = 0
        for storage in ("f64", "f32", "f16s", "bf16s", "f32d", "e3m12s"):
            for inplace in (False, True):
                for nx, ny, nz in SHAPES[:3]:
                    flags = _flags(nx, ny, nz, seed=k)
                    o = make_options(storage, (1e-5, 0.0, 0.0) if k % 2 else (0.0, 0.0, 0.0), None, 0, 0,
                                     0.0, inplace)
                    slot = ctypes.c_int()
                    ulid = (ctypes.c_double * 3)(0.05, 0.0, 0.0)
                    st = lib.lb_batch_add(h, nx, ny, nz, 0.7, ulid, flags.ctypes.data_as(ctypes.c_void_p),
                                          ctypes.byref(o), 25 + k, ctypes.byref(slot))
                    assert st == L.LB_OK, lib.lb_batch_last_error().decode()
                    k += 1
        for _ in range(4):
            assert lib.lb_batch_step(h, 8) == L.LB_OK
        assert lib.lb_batch_sync(h) == L.LB_OK
        head, tail = _guards_intact(torch, buf, nbytes)
        assert head == 0 and tail == 0, f"{head} guard bytes changed before the pool, {tail} after"
    finally:
        lib.lb_batch_destroy(h)
