"""Planted mistakes in copies of the oracle must each fail at least one pin.

Each mutant is the oracle's C source with one plausible slip (a dropped or
mis-scaled term, a flipped sign, a transposed index, a wrong opposite
direction); it is compiled to a temporary library on the CPU and the full pin
set is run against it.  A mutant that passes every pin would mean the pins
cannot tell that slip from the paper's method.
"""
import os

import numpy as np
import pytest

import oracle as O
import oracle_pins as P

SRC = os.path.join(os.path.dirname(os.path.abspath(O.__file__)), "lb_oracle.c")

MUTANTS = {
    "quadratic_coeff": ("4.5 * cu * cu", "3.0 * cu * cu"),
    "linear_sign": ("(1.0 + 3.0 * cu", "(1.0 - 3.0 * cu"),
    "uu_sign": ("- 1.5 * uu", "+ 1.5 * uu"),
    "weights_swapped": ("1.0 / 18.0 : 1.0 / 36.0", "1.0 / 36.0 : 1.0 / 18.0"),
    "lid_sign": ("f[i] += 6.0 * lbo_w[i]", "f[i] -= 6.0 * lbo_w[i]"),
    "lid_scale": ("6.0 * lbo_w[i] * 1.0 * cu", "3.0 * lbo_w[i] * 1.0 * cu"),
    "pull_sign_x": ("lbo_wrap(x - lbo_c[i][0], nx)", "lbo_wrap(x + lbo_c[i][0], nx)"),
    "pull_axis_swap": ("lbo_wrap(y - lbo_c[i][1], ny)", "lbo_wrap(y - lbo_c[i][2], ny)"),
    "bounce_same_dir": ("A[(size_t)lbo_opp[i] * N + cell]", "A[(size_t)i * N + cell]"),
    "guo_prefactor": ("double pref = 1.0 - 0.5 / tau;", "double pref = 1.0;"),
    "guo_u_sign": ("(3.0 * (lbo_c[i][a] - u[a])", "(3.0 * (lbo_c[i][a] + u[a])"),
    "guo_cc_coeff": ("9.0 * cu * lbo_c[i][a]", "3.0 * cu * lbo_c[i][a]"),
    "no_half_force": ("u[a] = j[a] / r + 0.5 * g[a];", "u[a] = j[a] / r;"),
    "omega_is_tau": ("double omega = 1.0 / tau;", "double omega = 2.0 - 1.0 / tau;"),
    "trt_odd_rate_is_even": ("- wm * (fm - em)", "- wp * (fm - em)"),
    "trt_even_rate_is_odd": ("- wp * (fp - ep)", "- wm * (fp - ep)"),
    "trt_guo_odd_scale": ("(1.0 - 0.5 * wm) * gm", "(1.0 - 0.5 * wp) * gm"),
    "trt_guo_even_scale": ("(1.0 - 0.5 * wp) * gp", "(1.0 - 0.5 * wm) * gp"),
    "trt_odd_part_sign": ("fm = 0.5 * (f[i] - f[o])", "fm = 0.5 * (f[o] - f[i])"),
    "farfield_as_wall": ("flags[src] == LBO_FARFIELD", "flags[src] == 99"),
    "farfield_density": ("lbo_equilibrium(1.0, ulid, f_free)", "lbo_equilibrium(1.02, ulid, f_free)"),
    "farfield_at_rest": ("lbo_equilibrium(1.0, ulid, f_free)", "lbo_equilibrium(1.0, (double[3]){0, 0, 0}, f_free)"),
    "layout_transposed": ("(size_t)x + (size_t)nx * ((size_t)y + (size_t)ny * (size_t)z)",
                          "(size_t)y + (size_t)ny * ((size_t)x + (size_t)nx * (size_t)z)"),
}


@pytest.fixture(scope="module")
def source_text():
    with open(SRC) as fh:
        return fh.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, source_text, tmp_path):
    old, new = MUTANTS[name]
    assert source_text.count(old) >= 1, f"mutation site for {name} not found"
    src = tmp_path / f"mut_{name}.c"
    src.write_text(source_text.replace(old, new))
    so = O.compile_source(str(src), str(tmp_path / f"libmut_{name}.so"))
    lib = O.load_library(so)
    caught = []
    for pin in P.ALL_PINS:
        try:
            # a mutant may blow up (overflow, log of a NaN); the pin must still fail
            with np.errstate(all="ignore"):
                pin(lib)
        except AssertionError:
            caught.append(pin.__name__)
        except (FloatingPointError, ValueError, ZeroDivisionError, OverflowError):
            caught.append(pin.__name__ + " (error)")
    assert caught, f"mutant {name} passed every pin"
