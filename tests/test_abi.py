"""The C-ABI library loads and exports every symbol that include/lbgb.h
declares, and its host-side validation answers without a GPU (CPU only)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2409_16781_gb300 import _lib as L
from paper_2409_16781_gb300 import build as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbgb.h")


@pytest.fixture(scope="module")
def lib():
    B.build()
    return L.lib()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(lb_[a-z_]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lb_create", "lb_step", "lb_moments", "lb_destroy", "lb_totals",
                     "lb_init_fields", "lb_get_populations", "lb_set_populations"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", L.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (lb_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"
    assert set(L.SIGNATURES) == set(declared_functions())


def test_velocity_set_is_d3q19(lib):
    from paper_2409_16781_gb300 import velocity_set
    c, w = velocity_set()
    gold = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "d3q19_velocity_set.txt")):
        if line.strip() and not line.startswith("#"):
            a, b, cc, ww = line.split()
            num, den = ww.split("/")
            gold[(int(a), int(b), int(cc))] = int(num) / int(den)
    assert {tuple(v) for v in c.tolist()} == set(gold)
    for i in range(19):
        assert w[i] == gold[tuple(c[i].tolist())]
    # opposites at (2k-1, 2k) as the header states
    for k in range(1, 10):
        assert np.array_equal(c[2 * k - 1], -c[2 * k])


def test_bytes_required(lib):
    from paper_2409_16781_gb300 import bytes_required
    n = bytes_required(256, 256, 256, "f32")
    assert n >= 2 * 19 * 256 ** 3 * 4 + 256 ** 3
    assert bytes_required(256, 256, 256, "f16s") < n < bytes_required(256, 256, 256, "f64")
    assert bytes_required(0, 4, 4) == 0
    assert bytes_required(2048, 2048, 1024) == 0  # >= 2^31 cells


@pytest.mark.parametrize("args,what", [
    ((0, 4, 4, 0.6), "zero dim"),
    ((4, 4, 4, 0.5), "tau = 1/2"),
    ((4, 4, 4, float("nan")), "tau nan"),
    ((4, 4, -1, 0.7), "negative dim"),
])
def test_create_rejects_bad_arguments(lib, args, what):
    h = ctypes.c_void_p()
    st = lib.lb_create(ctypes.byref(h), *args, None, None, None)
    assert st == L.LB_EINVAL, what
    assert h.value is None
    assert lib.lb_last_error().decode()


def test_create_rejects_bad_flags(lib):
    h = ctypes.c_void_p()
    flags = np.zeros(64, dtype=np.uint8)
    flags[17] = 4  # 0..3 are fluid, wall, lid, far field
    st = lib.lb_create(ctypes.byref(h), 4, 4, 4, 0.7, None,
                       flags.ctypes.data_as(ctypes.c_void_p), None)
    assert st == L.LB_EINVAL
    assert "17" in lib.lb_last_error().decode()


def test_null_handle_calls(lib):
    assert lib.lb_step(None, 1) == L.LB_EINVAL
    assert lib.lb_moments(None, None, None) == L.LB_EINVAL
    assert lib.lb_destroy(None) == L.LB_OK
    assert lib.lb_status_string(L.LB_EDIVERGED) == b"simulation diverged"


def test_options_layout_and_trt_validation(lib):
    """lb_options keeps its 80-byte layout; a negative or non-finite TRT
    magic parameter is rejected before any device work."""
    assert ctypes.sizeof(L.LbOptions) == 80
    assert L.LbOptions.trt_magic.offset == 48
    assert L.LbOptions.inplace.offset == 56
    for bad in (-0.1, float("nan"), float("inf")):
        o = L.LbOptions()
        lib.lb_default_options(ctypes.byref(o))
        assert o.trt_magic == 0.0
        o.trt_magic = bad
        h = ctypes.c_void_p()
        st = lib.lb_create(ctypes.byref(h), 4, 4, 4, 0.7, None, None, ctypes.byref(o))
        assert st == L.LB_EINVAL
        assert "trt_magic" in lib.lb_last_error().decode()


def test_inplace_option(lib):
    """One population array halves the population memory; inplace must be
    0 or 1."""
    from paper_2409_16781_gb300 import bytes_required
    two = bytes_required(128, 128, 128, "f32")
    one = bytes_required(128, 128, 128, "f32", inplace=True)
    pops = 19 * 128 ** 3 * 4
    assert two - one == pops
    o = L.LbOptions()
    lib.lb_default_options(ctypes.byref(o))
    assert o.inplace == 0
    o.inplace = 2
    assert lib.lb_bytes_required(8, 8, 8, ctypes.byref(o)) == 0
    h = ctypes.c_void_p()
    assert lib.lb_create(ctypes.byref(h), 8, 8, 8, 0.7, None, None, ctypes.byref(o)) == L.LB_EINVAL
    assert "inplace" in lib.lb_last_error().decode()


def test_selftest_wait_rejects_bad_deadlines(lib):
    """lb_selftest_wait validates its deadline before any device work."""
    for bad in (0.0, -1.0, 6.0, float("nan")):
        assert lib.lb_selftest_wait(bad, None) == L.LB_EINVAL


C_PROGRAM = r"""
#include <stdio.h>
#include "lbgb.h"
int main(void) {
    lb_options o;
    lb_default_options(&o);
    o.storage = LB_F32;
    size_t two = lb_bytes_required(64, 32, 16, &o);
    o.inplace = 1;
    size_t one = lb_bytes_required(64, 32, 16, &o);
    int c[57];
    double w[19];
    lb_velocity_set(c, w);
    printf("%zu %zu %d %d %d %.17g %s\n", two, one, c[3], c[4], c[5], w[0], lb_status_string(LB_EINVAL));
    return 0;
}
"""


def test_header_is_plain_c_and_links(lib, tmp_path):
    """include/lbgb.h compiles as strict C99 with warnings as errors, and a C
    program links liblbgb.so and calls its host-only entry points."""
    import shutil
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "t.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "t"
    libdir = os.path.dirname(L.LIB_PATH)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", libdir, "-llbgb", f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    two, one = int(out[0]), int(out[1])
    assert two - one == 19 * 64 * 32 * 16 * 4       # one population array fewer in place
    assert out[2:5] == ["1", "0", "0"]               # c_1 = (+1, 0, 0)
    assert float(out[5]) == 1 / 3
    assert " ".join(out[6:]) == "invalid argument"


def test_batch_sizes(lib):
    """Slot sizes: 19 planes of round_up(N, 128) values per population
    array plus N code bytes, each rounded to 256 bytes; in place one array
    fewer; bad arguments give 0.  The fixed area grows with max_slots and
    holds at least the 16 MiB staging area."""
    def rup(v, a):
        return (v + a - 1) // a * a
    sizes = {L.LB_F64: 8, L.LB_F32: 4, L.LB_F16S: 2, L.LB_BF16S: 2, L.LB_F32D: 4}
    for (nx, ny, nz) in ((16, 16, 16), (33, 5, 7), (1, 1, 1), (192, 96, 64)):
        n = nx * ny * nz
        ps = rup(n, 128)
        for st, sb in sizes.items():
            pops = rup(19 * ps * sb, 256)
            assert lib.lb_batch_slot_bytes(nx, ny, nz, st, 0) == 2 * pops + rup(n, 256)
            assert lib.lb_batch_slot_bytes(nx, ny, nz, st, 1) == pops + rup(n, 256)
    for bad in ((0, 4, 4, L.LB_F32, 0), (4, 4, 4, 9, 0), (4, 4, 4, L.LB_F32, 2), (2048, 2048, 512, L.LB_F32, 0)):
        assert lib.lb_batch_slot_bytes(*bad) == 0
    f1, f1k = lib.lb_batch_fixed_bytes(1), lib.lb_batch_fixed_bytes(1024)
    assert f1 >= 16 << 20 and f1k > f1
    assert lib.lb_batch_fixed_bytes(0) == 0 and lib.lb_batch_fixed_bytes(65537) == 0
