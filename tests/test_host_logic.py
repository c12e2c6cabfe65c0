"""Host-side logic that needs no GPU: the autotune cache key, the FP64-pipe
roofline the bench reports for the FP64 forms, the committed ncu figures'
source-hash guard, and the serving command-line defaults."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2409_16781_gb300.lattice import autotune_key  # noqa: E402


def test_autotune_key_separates_geometries():
    """The best kernel depends on how many cells are next to a wall, so two
    lattices of the same size and storage but different flags get different
    keys; all-fluid flags and no flags share one."""
    dims = (16, 8, 4)
    none = autotune_key("GB300", "f32", dims, False, None)
    fluid = autotune_key("GB300", "f32", dims, False, np.zeros(16 * 8 * 4, np.uint8))
    assert none == fluid and none.endswith("nowalls")
    a = np.zeros(16 * 8 * 4, np.uint8)
    a[5] = 1
    b = a.copy()
    b[6] = 1
    ka = autotune_key("GB300", "f32", dims, False, a)
    kb = autotune_key("GB300", "f32", dims, False, b)
    assert ka != kb and ka != none
    assert ka == autotune_key("GB300", "f32", dims, False, a.reshape(4, 8, 16))
    # storage, forcing, collision and layout each change the key
    keys = {autotune_key("GB300", s, dims, f, a, t, i)
            for s in ("f32", "f16s") for f in (False, True) for t in (0.0, 0.1875) for i in (False, True)}
    assert len(keys) == 16


def test_fp64_alu_roofline_from_committed_figures():
    """The FP64 forms' ALU roofline: FP64-pipe instructions per update (from
    the committed ncu figures, valid for the current sources) x updates per
    second against 152 SMs x 2 per clock x 2.07 GHz."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        t = json.load(fh)
    if t["step_f64_tgv256"]["source_hash"] != bench.kernel_source_hash():
        # figures taken on other sources are never reported
        assert bench.fp64_alu_roofline("f64", 4, 3.5) is None
        return
    per = t["step_f64_tgv256"]["variants"]["4"]["fp64_pipe_inst_per_update"]
    r = bench.fp64_alu_roofline("f64", 4, 3.5)
    assert r["bound"] == "alu" and r["inst_per_update"] == per
    assert abs(r["peak"] - 152 * 2 * 2.07) < 0.1
    assert abs(r["frac"] - 3.5 * per / (152 * 2 * 2.07)) < 1e-3
    assert bench.fp64_alu_roofline("f64", 13, 3.5) is None      # no figure for that variant
    assert bench.fp64_alu_roofline("f32", 1, 40.0) is None      # not an FP64 form


def test_ncu_figures_need_the_current_sources(monkeypatch):
    """A figure recorded under another source hash is not reported."""
    with open(os.path.join(ROOT, "profiles", "traffic.json")) as fh:
        t = json.load(fh)
    current = t["step_f32_tgv256"]["source_hash"] == bench.kernel_source_hash()
    assert (bench.ncu_traffic("step_f32_tgv256", 1) is not None) == current
    monkeypatch.setattr(bench, "kernel_source_hash", lambda kind="two_arrays": "0" * 16)
    assert bench.ncu_traffic("step_f32_tgv256", 1) is None
    assert bench.fp64_alu_roofline("f64", 4, 3.5) is None


def test_source_hash_per_kernel_family():
    """The two-array figures depend on the two-array kernels' sources only,
    the in-place figures on the in-place kernels' only; both on the shared
    headers."""
    two, inp = bench.STEP_SOURCES_OF["two_arrays"], bench.STEP_SOURCES_OF["inplace"]
    assert "lb_step.cu" in two and "lb_inplace.cu" not in two
    assert "lb_inplace.cu" in inp and "lb_step.cu" not in inp
    for shared in ("lb_common.cuh", "lb_kernels.cuh", "lb_pairs.cuh", "lb_fpconv.cuh", "lb_internal.h"):
        assert shared in two and shared in inp
    assert bench.kernel_source_hash("two_arrays") != bench.kernel_source_hash("inplace")


def test_step_sources_exist_and_cover_the_step_code():
    """Every file named in the hash exists, and every step-kernel source of
    the library is named."""
    csrc = os.path.join(ROOT, "paper_2409_16781_gb300", "csrc")
    for name in bench.STEP_SOURCES:
        assert os.path.exists(os.path.join(csrc, name)), name
    for name in os.listdir(csrc):
        if name.endswith(".cuh"):
            assert name in bench.STEP_SOURCES, name


def test_serving_defaults():
    a = bench.parse_args([])
    assert a.serve_requests is None and a.serve_max_wait == 60.0 and a.serve_tight_gb == 0.75
    a = bench.parse_args(["--workload", "serve", "--serve-rates", "2", "--serve-max-wait", "0"])
    assert a.serve_rates == "2" and not a.serve_max_wait


def test_source_hash_ignores_comments_only():
    """The hash behind the committed ncu figures covers code, not comments:
    editing a comment keeps it, changing a token changes it, and comment
    markers inside string or character literals are code."""
    s = bench.strip_comments
    code = 'int a = 1; // the cell\'s "own" value\n/* block\n comment */ int b = 2;'
    assert s(code) == "int a = 1; int b = 2;"
    assert s(code.replace("the cell's", "a cell's")) == s(code)
    assert s(code.replace("b = 2", "b = 3")) != s(code)
    assert s('const char* p = "// not a comment"; char q = \'/\';') == \
        'const char* p = "// not a comment"; char q = \'/\';'
    assert s('x = "a\\"b // c"; y;') == 'x = "a\\"b // c"; y;'


def test_configs_sections_skip_past_the_deadline(monkeypatch):
    """A configs section that would start after --configs-deadline-s is
    reported as skipped (no GPU work), so the line is still printed."""
    args = bench.parse_args(["--configs-deadline-s", "-1"])
    out = bench.configs_section(args)
    for name in ("porous_512", "cavity_768_precision", "serving_2000"):
        assert "skipped" in out[name], out[name]
    assert "wall_s" in out
