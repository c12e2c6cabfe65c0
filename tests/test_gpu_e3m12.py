"""The E3M12 storage form (LB_E3M12S): the library's conversions against the
format written out from its definition (tests/e3m12_ref.py), bit for bit.

* decoding: all 65536 codes are loaded verbatim (checkpoint) and exported as
  FP64 f = w + d; d must be the definition's value of each code;
* encoding (rounding to nearest, ties to even, saturating): deviations
  imported through lb_set_populations must be stored as the code of the
  nearest representable value -- random values in the normal range,
  multiples of 2^-33 in the subnormal range, exact midpoints between two
  codes, zeros of both signs and magnitudes beyond the largest value;
* stochastic rounding keeps the expectation: a body-force increment far
  below the unit in the last place still moves the FP64 momentum by
  mass * g per step;
* a value beyond the largest E3M12 value saturates, and the totals report
  it as divergence.
"""
import numpy as np
import pytest

import e3m12_ref as R
from paper_2409_16781_gb300 import Lattice, velocity_set
from paper_2409_16781_gb300 import workloads as W

pytestmark = pytest.mark.gpu

HEADER = 64
DIMS = (16, 16, 14)  # 3584 cells x 19 directions >= 65536 values
N = DIMS[0] * DIMS[1] * DIMS[2]


def _codes(lat):
    raw = np.frombuffer(lat.checkpoint(), dtype=np.uint8)[HEADER:]
    return raw.view(np.uint16).reshape(19, N)


def test_decode_every_code():
    lat = Lattice(*DIMS, 0.7, storage="e3m12s")
    snap = bytearray(lat.checkpoint())
    codes = np.zeros(19 * N, dtype=np.uint16)
    codes[:65536] = np.arange(65536, dtype=np.uint32).astype(np.uint16)
    codes[65536:] = np.arange(19 * N - 65536, dtype=np.uint16)
    snap[HEADER:] = codes.tobytes()
    lat.restore(bytes(snap))
    _, w = velocity_set()
    f = lat.populations().reshape(19, N)
    want = w[:, None] + R.decode(codes.reshape(19, N))
    assert np.array_equal(f, want)


def _import(values):
    """Store deviations `values` (float32, 19*N of them) through the FP64
    import; returns the stored codes."""
    _, w = velocity_set()
    d = np.asarray(values, dtype=np.float32).reshape(19, N)
    f = w[:, None] + d.astype(np.float64)
    lat = Lattice(*DIMS, 0.7, storage="e3m12s")
    lat.set_populations(f.reshape((19,) + DIMS[::-1]))
    # what the import rounds: the deviation f - w, as an FP32 value
    return _codes(lat), (f - w[:, None]).astype(np.float32)


def test_round_to_nearest_matches_the_definition():
    rng = np.random.default_rng(12)
    n = 19 * N
    vals = np.empty(n, dtype=np.float32)
    k = n // 4
    # normal range, both signs, log-uniform magnitudes in [2^-10, 0.124)
    vals[:k] = (np.exp2(rng.uniform(-10, np.log2(0.124), k)) * rng.choice([-1, 1], k)).astype(np.float32)
    # subnormal range: multiples of 2^-33 below 2^-10, none within 2^-32 of
    # a midpoint between two codes (the midpoints come next: a value that
    # near one is first rounded onto the 2^-33 grid of the scaled FP32 value)
    ks = rng.integers(-(2 ** 23) + 1, 2 ** 23, k)
    ks[np.abs(np.abs(ks) % 2048 - 1024) <= 1] += 4
    vals[k:2 * k] = (ks * 2.0 ** -33).astype(np.float32)
    # exact midpoints between neighbouring codes (ties), both signs
    c = rng.integers(0, 0x7FFE, k)
    mid = (R.decode(c) + R.decode(c + 1)) / 2
    vals[2 * k:3 * k] = (mid * rng.choice([-1, 1], k)).astype(np.float32)
    rest = n - 3 * k
    tail = np.concatenate([[0.0, -0.0, 0.124984, 0.13, -0.5, 2.0, 1e-30, -2.0 ** -22, 2.0 ** -23]],
                          axis=None)
    vals[3 * k:3 * k + tail.size] = tail
    vals[3 * k + tail.size:] = rng.uniform(-0.02, 0.02, rest - tail.size).astype(np.float32)
    got, imported = _import(vals)
    assert np.array_equal(np.asarray(imported).reshape(-1)[2 * k:3 * k], vals[2 * k:3 * k]), \
        "the midpoints must reach the conversion unchanged"
    want = R.encode_rn(imported.reshape(-1)).reshape(19, N)
    bad = np.nonzero(got != want)
    assert bad[0].size == 0, (f"{bad[0].size} codes differ, e.g. value {imported[bad][0]!r}: "
                              f"{got[bad][0]:#06x} vs {want[bad][0]:#06x}")


def test_stochastic_rounding_is_unbiased():
    """All-fluid periodic box in uniform motion (u = 0.1 along x) with a weak
    force: every stored value changes by less than a unit in the last place
    per step (near d = 0.02 the unit is 2^-18); the FP64 momentum must still
    grow by mass * g per step."""
    n, steps, g = 24, 1000, 3e-7
    lat = Lattice(n, n, n, 0.7, storage="e3m12s", force=(g, 0, 0), rounding="stochastic")
    rho = np.ones((n, n, n))
    u = np.zeros((3, n, n, n))
    u[0] = 0.1  # stored values far from zero
    lat.init_fields(rho, u)
    m0, p0 = lat.totals()
    lat.step(steps)
    m1, p1 = lat.totals()
    assert abs((p1[0] - p0[0]) / (m0 * g * steps) - 1) < 0.02
    assert abs(m1 - m0) / m0 < 1e-6


def test_saturation_is_reported_as_divergence():
    from paper_2409_16781_gb300 import LbDiverged
    flags = W.cavity_flags(12, 10, 8)
    lat = Lattice(12, 10, 8, 0.7, u_lid=(0.1, 0, 0), flags=flags, storage="e3m12s")
    _, w = velocity_set()
    f = np.broadcast_to(w[:, None, None, None], (19, 8, 10, 12)).copy()
    f[3, 4, 5, 6] = w[3] + 0.3  # beyond the largest E3M12 value
    lat.set_populations(f)
    with pytest.raises(LbDiverged):
        lat.totals()
