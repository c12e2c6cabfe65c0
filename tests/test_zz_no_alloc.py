"""lb_totals_static: the FP64 totals for callers that cannot allocate device
memory (a fixed memory budget, another framework's pool, a real-time loop).

The test allocates the device buffers itself (the entry point allocates
nothing) and fills them with the stored values of a lattice made through
the normal API (its bit-exact checkpoint).  For every storage form, on two
calls in a row with steps in between, lb_totals_static must give what
lb_totals gives and what the FP64 oracle's totals give on the same
populations, within the tolerance of the form's arithmetic; the flag field
has walls, a moving lid and far-field cells; and the device's free memory
must be the same before and after each call.  It sits in a file of its own
that pytest collects last.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
from parity import lib_to_oracle_perm, to_oracle_order
from paper_2409_16781_gb300 import Lattice
from paper_2409_16781_gb300 import _lib as L
from paper_2409_16781_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CHECKPOINT_HEADER = 64  # bytes before the stored planes (lb_checkpoint_save)


def _static_totals(lib, dev_pops, plane_stride, dev_flags, dims, storage, force, u_lid, stream):
    out = (ctypes.c_double * 5)()
    f3 = (ctypes.c_double * 3)(*force)
    u3 = (ctypes.c_double * 3)(*u_lid)
    st = lib.lb_totals_static(ctypes.c_void_p(dev_pops.data_ptr()), plane_stride,
                              ctypes.c_void_p(dev_flags.data_ptr()), dims[0], dims[1], dims[2],
                              L.STORAGE[storage], f3, u3, ctypes.c_void_p(stream.cuda_stream), out)
    assert st == L.LB_OK, L.lib().lb_status_string(st)
    return out[0], np.array(out[1:4]), out[4]


def _flags(nx, ny, nz):
    """A cavity (walls, lid on top) whose x = 0 face is a far-field plane."""
    f = W.cavity_flags(nx, ny, nz)
    f[1:nz - 1, 1:ny - 1, 0] = W.FARFIELD
    return f


# Relative to the mass.  Against lb_totals (the same reduction kernel over
# the same cells): 1e-12.  Against the FP64 oracle: 1e-12 for the forms with
# FP64 arithmetic (f64, f32d); the forms with FP32 arithmetic (f32, f16s,
# bf16s, e3m12s) sum each cell's 19 values in FP32 and take the far-field inflow and
# the lid term as FP32 constants, whose roundings have the same sign at every
# cell of a boundary plane, so their totals sit within a few FP32 roundings
# per boundary cell of the oracle's: 1e-8 of the mass.
@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32d", 1e-12), ("f32", 1e-8),
                                         ("f16s", 1e-8), ("bf16s", 1e-8), ("e3m12s", 1e-8)])
def test_static_totals_match_lb_totals_and_oracle(storage, tol):
    import torch
    lib = L.lib()
    nx, ny, nz = 40, 24, 20
    N = nx * ny * nz
    flags = _flags(nx, ny, nz)
    force = (2e-5, 0.0, -1e-5)
    u_lid = (0.08, 0.0, 0.0)
    lat = Lattice(nx, ny, nz, 0.6, u_lid=u_lid, flags=flags, storage=storage, force=force)
    stream = torch.cuda.current_stream()
    perm = lib_to_oracle_perm()
    ora = O.Lattice(nx, ny, nz, 0.6, u_lid=u_lid, flags=flags, force=force)
    dev_flags = torch.from_numpy(flags.reshape(-1)).cuda()
    # one call first: the first use of a kernel may load its code onto the
    # device (lazy module loading), which is the runtime's memory, not a
    # call's
    first = torch.zeros(19 * N * L.STORAGE_BYTES[L.STORAGE[storage]], dtype=torch.uint8, device="cuda")
    _static_totals(lib, first, N, dev_flags, (nx, ny, nz), storage, force, u_lid, stream)
    for steps in (40, 25):  # two calls in a row, with steps in between
        lat.step(steps)
        mass, mom = lat.totals()
        raw = np.frombuffer(lat.checkpoint(), dtype=np.uint8)[CHECKPOINT_HEADER:]
        dev_pops = torch.from_numpy(raw.copy()).cuda()
        assert dev_pops.numel() == 19 * N * L.STORAGE_BYTES[L.STORAGE[storage]]
        torch.cuda.synchronize()
        free_before, _ = torch.cuda.mem_get_info()
        m2, p2, bad = _static_totals(lib, dev_pops, N, dev_flags, (nx, ny, nz), storage,
                                     force, u_lid, stream)
        free_after, _ = torch.cuda.mem_get_info()
        assert free_after == free_before, "lb_totals_static changed the device's free memory"
        assert bad == 0
        # the same populations in the FP64 oracle
        ora.set_populations(to_oracle_order(lat.populations(), perm))
        m3, p3 = ora.totals()
        for m_ref, p_ref, t in ((mass, mom, 1e-12), (m3, p3, tol)):
            assert abs(m2 - m_ref) <= t * abs(m_ref)
            assert np.abs(p2 - p_ref).max() <= t * abs(m_ref)
        assert np.abs(mom).max() > 0


def test_static_totals_rejects_bad_sizes():
    import torch
    lib = L.lib()
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    fl = torch.zeros(64, dtype=torch.uint8, device="cuda")
    out = (ctypes.c_double * 5)()
    p = ctypes.c_void_p(buf.data_ptr())
    f = ctypes.c_void_p(fl.data_ptr())
    assert lib.lb_totals_static(p, 64, f, 2048, 2048, 1024, L.LB_F32, None, None, None, out) == L.LB_EINVAL
    assert lib.lb_totals_static(p, 10, f, 4, 4, 4, L.LB_F32, None, None, None, out) == L.LB_EINVAL
    assert lib.lb_totals_static(p, 64, f, 0, 4, 4, L.LB_F32, None, None, None, out) == L.LB_EINVAL
