"""lb_totals_static: the FP64 totals for callers that cannot allocate device
memory (a fixed memory budget, another framework's pool, a real-time loop).

The test allocates the device buffers itself (the entry point allocates
nothing), fills them with the state of a lattice made through the normal
API, and checks that lb_totals_static gives what lb_totals gives -- within
the FP64 tolerance of the parity tests (1e-12 relative) -- on two calls in a
row with steps in between.  It sits in a file of its own that pytest
collects last.
"""
import ctypes

import numpy as np
import pytest

from paper_2409_16781_gb300 import Lattice, velocity_set
from paper_2409_16781_gb300 import _lib as L
from paper_2409_16781_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _static_totals(lib, dev_pops, plane_stride, dev_flags, dims, storage, force, u_lid, stream):
    out = (ctypes.c_double * 5)()
    f3 = (ctypes.c_double * 3)(*force)
    u3 = (ctypes.c_double * 3)(*u_lid)
    st = lib.lb_totals_static(ctypes.c_void_p(dev_pops.data_ptr()), plane_stride,
                              ctypes.c_void_p(dev_flags.data_ptr()), dims[0], dims[1], dims[2],
                              L.STORAGE[storage], f3, u3, ctypes.c_void_p(stream.cuda_stream), out)
    assert st == L.LB_OK, L.lib().lb_status_string(st)
    return out[0], np.array(out[1:4]), out[4]


# f64: the parity tests' FP64 tolerance.  f32: per-cell sums are FP32 and the
# two kernels group cells differently before folding into FP64, so the sums
# may differ by a few FP32 roundings of |rho - 1| ~ 1e-3 per group.
@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-10)])
def test_static_totals_match_lb_totals(storage, tol):
    import torch
    lib = L.lib()
    nx, ny, nz = 40, 24, 20
    N = nx * ny * nz
    flags = W.cavity_flags(nx, ny, nz)
    force = (2e-5, 0.0, -1e-5)
    u_lid = (0.08, 0.0, 0.0)
    lat = Lattice(nx, ny, nz, 0.6, u_lid=u_lid, flags=flags, storage=storage, force=force)
    stream = torch.cuda.current_stream()
    _, w = velocity_set()
    dtype = {"f64": torch.float64, "f32": torch.float32}[storage]
    dev_flags = torch.from_numpy(flags.reshape(-1)).cuda()
    for steps in (40, 25):  # two calls in a row, with steps in between
        lat.step(steps)
        mass, mom = lat.totals()
        f = lat.populations().reshape(19, N)
        d = f - w[:, None]               # exact: the stored deviations
        dev_pops = torch.from_numpy(d).to(dtype).cuda().contiguous()
        torch.cuda.synchronize()
        m2, p2, bad = _static_totals(lib, dev_pops, N, dev_flags, (nx, ny, nz), storage,
                                     force, u_lid, stream)
        assert bad == 0
        assert abs(m2 - mass) <= tol * abs(mass)
        assert np.abs(p2 - mom).max() <= tol * abs(mass)
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
