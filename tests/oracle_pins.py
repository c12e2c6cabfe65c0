"""Pins for the FP64 oracle: facts fixed by the paper and by the mathematics.

Each ``pin_*`` function takes an oracle shared library (``lib``; None = the
built oracle) and raises AssertionError when the oracle disagrees with a fact
that does not come from the oracle itself: closed-form moments, exact fixed
points and conservation laws, exact steady solutions of the discrete scheme
(Couette, Poiseuille at the published "magic" relaxation time), asymptotic
decay rates of exact Navier-Stokes solutions with their convergence order,
Galilean advection, mirror symmetry and a brute-force push stepper.
``tests/test_oracle_mutants.py`` plants plausible mistakes in copies of the
oracle's C source and checks that every mistake fails at least one pin.

Equations: arXiv 2409.16781 Sec. 2, Eq. 1 (BGK lattice equation with source),
Eq. 2-3 (second-order equilibrium); Sec. 3.1 (fused pull, two arrays);
Sec. 3.3 (lid-driven cavity: no-slip walls, lid moving at u0).
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np

import oracle as O
from paper_2409_16781_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
I3 = np.eye(3)


def _golden_velocity_set():
    rows = []
    with open(os.path.join(GOLDEN, "d3q19_velocity_set.txt")) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            cx, cy, cz, w = line.split()
            rows.append(((int(cx), int(cy), int(cz)), Fraction(w)))
    return rows


# ------------------------------------------------------------------ tables
def pin_lattice_tables(lib=None):
    """Velocity set = the published D3Q19 table; isotropy up to 4th order."""
    c, w = O.velocity_set(lib)
    gold = dict(_golden_velocity_set())
    got = {tuple(int(v) for v in c[i]): w[i] for i in range(19)}
    assert set(got) == set(gold), "velocity set differs from the D3Q19 table"
    for k, wv in gold.items():
        assert abs(got[k] - float(wv)) <= 1e-17, f"weight of {k}"
    cf = c.astype(np.float64)
    assert abs(w.sum() - 1.0) < 1e-15
    assert np.abs(np.einsum("i,ia->a", w, cf)).max() < 1e-16
    assert np.abs(np.einsum("i,ia,ib->ab", w, cf, cf) - I3 / 3).max() < 1e-15
    assert np.abs(np.einsum("i,ia,ib,ic->abc", w, cf, cf, cf)).max() < 1e-16
    d4 = (np.einsum("ab,cd->abcd", I3, I3) + np.einsum("ac,bd->abcd", I3, I3)
          + np.einsum("ad,bc->abcd", I3, I3)) / 9
    assert np.abs(np.einsum("i,ia,ib,ic,id->abcd", w, cf, cf, cf, cf) - d4).max() < 1e-15


# ------------------------------------------------------- closed-form moments
def pin_equilibrium_moments(lib=None):
    """Moments 0-3 of f^eq (Eq. 2-3) in closed form:
    sum f = rho, sum f c = rho u, sum f cc = rho (I/3 + uu),
    sum f c_a c_b c_g = rho/3 (u_a d_bg + u_b d_ag + u_g d_ab)."""
    c, _ = O.velocity_set(lib)
    cf = c.astype(np.float64)
    rng = np.random.default_rng(7)
    for _ in range(20):
        rho = 0.8 + 0.4 * rng.random()
        u = 0.2 * (rng.random(3) - 0.5)
        f = O.equilibrium(rho, u, lib)
        assert abs(f.sum() - rho) < 1e-14
        assert np.abs(f @ cf - rho * u).max() < 1e-15
        P = np.einsum("i,ia,ib->ab", f, cf, cf)
        assert np.abs(P - rho * (I3 / 3 + np.outer(u, u))).max() < 1e-15
        T = np.einsum("i,ia,ib,ic->abc", f, cf, cf, cf)
        T0 = rho / 3 * (np.einsum("a,bc->abc", u, I3) + np.einsum("b,ac->abc", u, I3)
                        + np.einsum("c,ab->abc", u, I3))
        assert np.abs(T - T0).max() < 1e-15


def pin_source_moments(lib=None):
    """Guo source: sum S = 0, sum S c = (1-1/2tau) F, sum S cc = (1-1/2tau)(uF+Fu),
    with F = rho g."""
    c, _ = O.velocity_set(lib)
    cf = c.astype(np.float64)
    rng = np.random.default_rng(11)
    for _ in range(20):
        tau = 0.51 + rng.random()
        rho = 0.8 + 0.4 * rng.random()
        u = 0.2 * (rng.random(3) - 0.5)
        g = 1e-3 * (rng.random(3) - 0.5)
        S = O.source(tau, rho, u, g, lib)
        F = rho * g
        pref = 1 - 0.5 / tau
        assert abs(S.sum()) < 1e-18
        assert np.abs(S @ cf - pref * F).max() < 1e-18
        P = np.einsum("i,ia,ib->ab", S, cf, cf)
        assert np.abs(P - pref * (np.outer(u, F) + np.outer(F, u))).max() < 1e-18


# ------------------------------------------------------------ exact dynamics
def pin_rest_fixed_point(lib=None):
    """f = w, no lid motion, no force, any flag field: a fixed point.  In the
    oracle's plain FP64 form sum(w) is 1 only to rounding, so the state may
    move by a couple of ulp once and must then stay put (no accumulation)."""
    fl = W.random_flags(6, 5, 7, seed=3, p_wall=0.3, p_lid=0.1)
    L = O.Lattice(6, 5, 7, 0.6, u_lid=(0, 0, 0), flags=fl, lib=lib)
    A0 = L.A.copy()
    L.step(7)
    assert np.abs(L.A - A0).max() <= 4e-16, "rest state is not a fixed point"
    L.step(1000)
    assert np.abs(L.A - A0).max() <= 4e-16, "rest state drifts"


def pin_pure_streaming(lib=None):
    """omega -> 0 (tau = 1e300): collision is the identity in FP64 and the
    step is pure transport, value A_i(x) lands at x + c_i (periodic), on a
    non-cubic grid so that any axis or sign mistake moves it elsewhere."""
    nx, ny, nz = 5, 6, 7
    c, w = O.velocity_set(lib)
    rng = np.random.default_rng(5)
    A = w[:, None, None, None] + 1e-3 * rng.random((19, nz, ny, nx))
    L = O.Lattice(nx, ny, nz, 1e300, lib=lib)
    L.set_populations(A)
    L.step(1)
    for i in range(19):
        expect = np.roll(A[i], shift=(c[i][2], c[i][1], c[i][0]), axis=(0, 1, 2))
        assert np.array_equal(L.A[i], expect), f"direction {c[i]} not transported by c_i"


def pin_single_cell_collision(lib=None):
    """On a 1x1x1 periodic lattice every direction pulls from the cell itself,
    so one step is the collision alone.  BGK with Guo forcing then fixes the
    moments: rho' = rho, j' = j + rho g, and the second moment
    Pi' = (1-w) Pi + w rho (I/3 + uu) + (1-w/2)(uF + Fu), u = j/rho + g/2."""
    c, w = O.velocity_set(lib)
    cf = c.astype(np.float64)
    rng = np.random.default_rng(13)
    for _ in range(10):
        tau = 0.52 + 1.5 * rng.random()
        om = 1.0 / tau
        g = 1e-3 * (rng.random(3) - 0.5)
        f = w + 0.01 * (rng.random(19) - 0.5)
        L = O.Lattice(1, 1, 1, tau, force=g, lib=lib)
        L.set_populations(f.reshape(19, 1, 1, 1))
        L.step(1)
        fp = L.A.reshape(19)
        rho = f.sum()
        j = f @ cf
        u = j / rho + g / 2
        F = rho * g
        assert abs(fp.sum() - rho) < 1e-15
        assert np.abs(fp @ cf - (j + F)).max() < 1e-16
        Pi = np.einsum("i,ia,ib->ab", f, cf, cf)
        Pi_p = np.einsum("i,ia,ib->ab", fp, cf, cf)
        expect = ((1 - om) * Pi + om * rho * (I3 / 3 + np.outer(u, u))
                  + (1 - om / 2) * (np.outer(u, F) + np.outer(F, u)))
        assert np.abs(Pi_p - expect).max() < 1e-15


def pin_mass_conservation_cavity(lib=None):
    """Lid-driven cavity (walls + lid, lid corrections cancel pairwise):
    total mass is conserved to rounding over 300 steps."""
    n = 14
    L = O.Lattice(n, n, n, 0.6, u_lid=(0.1, 0, 0), flags=W.cavity_flags(n, n, n), lib=lib)
    m0, _ = L.totals()
    assert abs(m0 - (n - 2) ** 3) < 1e-9
    L.step(300)
    m1, p1 = L.totals()
    assert abs(m1 - m0) / m0 < 1e-13, f"mass drift {abs(m1 - m0) / m0:.3e}"
    assert p1[0] > 1e-3 * m0 * 0.1 * 1e-3, "lid did not drive the flow"


def pin_periodic_momentum(lib=None):
    """Periodic box: momentum is conserved without force and grows by exactly
    (total mass) * g per step with a body force g."""
    nx, ny, nz = 8, 7, 6
    rho, u = W.random_fields(nx, ny, nz, seed=21, du=0.04, drho=0.02)
    L = O.Lattice(nx, ny, nz, 0.7, lib=lib)
    L.init_fields(rho, u)
    m0, p0 = L.totals()
    L.step(50)
    m1, p1 = L.totals()
    assert abs(m1 - m0) < 1e-13 * m0
    assert np.abs(p1 - p0).max() < 1e-13 * m0
    g = np.array([2e-5, -1e-5, 3e-5])
    L = O.Lattice(nx, ny, nz, 0.7, force=g, lib=lib)
    L.init_fields(rho, u)
    m0, p0 = L.totals()
    L.step(40)
    m1, p1 = L.totals()
    assert abs(m1 - m0) < 1e-13 * m0
    assert np.abs(p1 - (p0 + 40 * m0 * g)).max() < 1e-12 * m0 * np.abs(g).max() * 40


def _shear_wave_nu_error(n, tau, lib):
    """Fit the decay rate of u_x = u0 sin(kz) (exact NS solution; amplitude
    ~ exp(-nu k^2 t)) and return nu_fit / ((tau-1/2)/3) - 1."""
    nu = (tau - 0.5) / 3
    k = 2 * math.pi / n
    z = np.arange(n)
    u = np.zeros((3, n, 1, 1))
    u[0, :, 0, 0] = 1e-3 * np.sin(k * z)
    L = O.Lattice(1, 1, n, tau, lib=lib)
    L.init_fields(None, u)
    ts, amps = [], []
    for t in range(0, 2001, 100):
        _, uu = L.moments()
        if t >= 200:
            ts.append(t)
            amps.append(2 / n * np.sum(uu[0, :, 0, 0] * np.sin(k * z)))
        L.step(100)
    amps = np.array(amps)
    assert (amps > 0).all()
    slope = np.polyfit(np.array(ts), np.log(amps), 1)[0]
    return -slope / (k * k) / nu - 1


def pin_shear_wave(lib=None):
    """Shear-wave viscosity nu = (tau - 1/2)/3, approached at second order in
    the lattice spacing (error ratio ~4 per doubling)."""
    e32 = _shear_wave_nu_error(32, 0.8, lib)
    e64 = _shear_wave_nu_error(64, 0.8, lib)
    assert abs(e64) < 1e-3, f"nu error {e64:.3e} at n=64"
    assert 3.5 < e32 / e64 < 4.5, f"convergence ratio {e32 / e64:.3f}"


def pin_taylor_green_2d(lib=None):
    """2D Taylor-Green vortex (exact NS solution, initial pressure included):
    kinetic energy decays as exp(-4 nu k^2 t) = exp(-2 nu |k|^2 t)."""
    n, tau, u0 = 64, 0.6, 0.01
    nu = (tau - 0.5) / 3
    k = 2 * math.pi / n
    x = np.arange(n)[None, None, :]
    y = np.arange(n)[None, :, None]
    u = np.zeros((3, 1, n, n))
    u[0] = u0 * np.cos(k * x) * np.sin(k * y)
    u[1] = -u0 * np.sin(k * x) * np.cos(k * y)
    p = -u0 ** 2 / 4 * (np.cos(2 * k * x) + np.cos(2 * k * y))
    L = O.Lattice(n, n, 1, tau, lib=lib)
    L.init_fields((1 + 3 * p)[0], u)
    ts, E = [], []
    for t in range(0, 801, 50):
        r, uu = L.moments()
        if t >= 100:
            ts.append(t)
            E.append(0.5 * np.sum(r * (uu ** 2).sum(0)))
        L.step(50)
    slope = np.polyfit(np.array(ts), np.log(E), 1)[0]
    err = -slope / (4 * nu * k * k) - 1
    assert abs(err) < 1e-4, f"TGV decay-rate error {err:.3e}"


def pin_galilean_advection(lib=None):
    """A transverse wave u_y = eps sin(kx) on a uniform stream U x-hat is
    carried downstream at speed U (momentum flux rho u u of Eq. 2-3) while
    it decays at exp(-nu k^2 t)."""
    n, tau, U, eps = 64, 0.7, 0.05, 1e-4
    nu = (tau - 0.5) / 3
    k = 2 * math.pi / n
    x = np.arange(n)
    u = np.zeros((3, 1, 1, n))
    u[0] = U
    u[1, 0, 0, :] = eps * np.sin(k * x)
    L = O.Lattice(n, 1, 1, tau, lib=lib)
    L.init_fields(None, u)
    T = 160
    L.step(T)
    _, uu = L.moments()
    v = uu[1, 0, 0, :]
    C, S = np.sum(v * np.cos(k * x)), np.sum(v * np.sin(k * x))
    shift = math.atan2(-C, S) / k
    amp = math.hypot(C, S) * 2 / n / eps
    assert abs(shift - U * T) < 0.02 * U * T, f"advected {shift:.3f}, expected {U * T}"
    assert abs(amp / math.exp(-nu * k * k * T) - 1) < 0.01


def pin_couette(lib=None):
    """Plane Couette flow between a resting wall (z = 0) and the lid (top
    plane, u_lid along x): the steady state is the exact linear profile with
    both walls halfway between solid and fluid cells."""
    nz, U = 12, 0.05
    fl = np.zeros((nz, 1, 1), dtype=np.uint8)
    fl[0] = W.WALL
    fl[-1] = W.LID
    L = O.Lattice(1, 1, nz, 1.0, u_lid=(U, 0, 0), flags=fl, lib=lib)
    L.step(3000)
    rho, u = L.moments()
    z = np.arange(1, nz - 1)
    exact = U * (z - 0.5) / (nz - 2)
    assert np.abs(u[0, 1:-1, 0, 0] - exact).max() < 1e-12 * U
    assert np.abs(u[1:, 1:-1]).max() < 1e-13 * U


def pin_poiseuille(lib=None):
    """Force-driven channel (walls at y = 0, ny-1): the steady profile has
    the exact discrete curvature -g/nu, and at tau = 1/2 + sqrt(3/16) (the
    relaxation time at which halfway bounce-back is exact for BGK) it equals
    the analytic parabola g/(2 nu) (y - 1/2)(ny - 3/2 - y)."""
    ny, g = 18, 1e-6
    fl = np.zeros((1, ny, 1), dtype=np.uint8)
    fl[:, 0] = W.WALL
    fl[:, -1] = W.WALL
    for tau in (0.8, 0.5 + math.sqrt(3 / 16)):
        nu = (tau - 0.5) / 3
        L = O.Lattice(1, ny, 1, tau, flags=fl, force=(g, 0, 0), lib=lib)
        L.step(40000)
        _, u = L.moments()
        ux = u[0, 0, 1:-1, 0]
        curv = ux[2:] - 2 * ux[1:-1] + ux[:-2]
        assert np.abs(curv / (-g / nu) - 1).max() < 1e-9
        if tau != 0.8:
            y = np.arange(1, ny - 1)
            exact = g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
            assert np.abs(ux - exact).max() < 1e-9 * exact.max()


def pin_cavity_mirror(lib=None):
    """Cavity with the lid moving along x is symmetric under y -> ny-1-y:
    u_x, u_z, rho even and u_y odd."""
    nx, ny, nz = 12, 11, 10
    L = O.Lattice(nx, ny, nz, 0.6, u_lid=(0.1, 0, 0), flags=W.cavity_flags(nx, ny, nz),
                  lib=lib)
    L.step(120)
    rho, u = L.moments()
    m = slice(None, None, -1)
    assert np.abs(rho - rho[:, m, :]).max() < 1e-14
    assert np.abs(u[0] - u[0][:, m, :]).max() < 1e-15
    assert np.abs(u[2] - u[2][:, m, :]).max() < 1e-15
    assert np.abs(u[1] + u[1][:, m, :]).max() < 1e-15
    assert np.abs(u[0]).max() > 1e-3


def _to_brute_order(c_oracle):
    from brute_push import VEL
    return [VEL.index(tuple(int(v) for v in c_oracle[i])) for i in range(19)]


def pin_brute_force(lib=None):
    """Agreement with the push-form brute-force stepper on tiny grids:
    1x1x1 (pure collision), a 3x3x3 box with one fluid cell (pure
    bounce-back off walls and lid), a 3x5x7 random flag field with lid
    and force, and a 7x4x3 grid with far-field planes, walls and a lid."""
    from brute_push import Brute
    c, w = O.velocity_set(lib)
    perm = _to_brute_order(c)          # oracle index i -> brute index perm[i]
    cases = []
    cases.append((1, 1, 1, 0.7, (0, 0, 0), (1e-4, -2e-4, 3e-4), np.zeros((1, 1, 1), np.uint8)))
    box = np.full((3, 3, 3), W.WALL, np.uint8)
    box[2, :, :] = W.LID
    box[1, 1, 1] = W.FLUID
    cases.append((3, 3, 3, 0.9, (0.07, -0.03, 0.0), (0, 0, 0), box))
    cases.append((3, 5, 7, 0.65, (0.05, 0.02, 0.0), (1e-4, 0, -1e-4),
                  W.random_flags(3, 5, 7, seed=9, p_wall=0.25, p_lid=0.15)))
    # far-field planes (free stream at u_lid) at both x ends, walls and a lid
    ff = W.random_flags(7, 4, 3, seed=4, p_wall=0.2, p_lid=0.1)
    ff[:, :, 0] = W.FARFIELD
    ff[:, :, 6] = W.FARFIELD
    ff[1, 2, 3] = W.FARFIELD
    cases.append((7, 4, 3, 0.75, (0.06, -0.02, 0.01), (0, 2e-4, 0), ff))
    rng = np.random.default_rng(17)
    for nx, ny, nz, tau, ulid, g, fl in cases:
        A = w[:, None, None, None] + 0.01 * (rng.random((19, nz, ny, nx)) - 0.5)
        L = O.Lattice(nx, ny, nz, tau, u_lid=ulid, flags=fl, force=g, lib=lib)
        L.set_populations(A)
        B = Brute(nx, ny, nz, tau, ulid, g, lambda x, y, z: int(fl[z, y, x]))
        for cell in B.fluid:
            x, y, z = cell
            vals = [0.0] * 19
            for i in range(19):
                vals[perm[i]] = A[i, z, y, x]
            B.P[cell] = vals
        for _ in range(4):
            L.step(1)
            B.step()
        for (x, y, z) in B.fluid:
            for i in range(19):
                assert abs(L.A[i, z, y, x] - B.P[(x, y, z)][perm[i]]) < 1e-15, \
                    f"brute force disagrees at {(x, y, z)} dir {c[i]}"


# ------------------------------------------------------------------ far field
def _farfield_channel(nx, ny, nz, U, walls):
    fl = np.zeros((nz, ny, nx), np.uint8)
    if walls:
        fl[:, 0, :] = W.WALL
        fl[:, ny - 1, :] = W.WALL
    fl[:, :, 0] = np.where(fl[:, :, 0] == 0, W.FARFIELD, fl[:, :, 0])
    fl[:, :, nx - 1] = np.where(fl[:, :, nx - 1] == 0, W.FARFIELD, fl[:, :, nx - 1])
    return fl


def pin_farfield_free_stream(lib=None):
    """Far-field planes at both ends of a box periodic in y, z hold the free
    stream (rho = 1, u = U): the uniform flow is a fixed point (to rounding),
    and a fluid started at rest becomes exactly that uniform flow (the only
    steady state the two planes allow)."""
    U = (0.05, 0.01, -0.02)
    nx, ny, nz = 24, 3, 2
    fl = _farfield_channel(nx, ny, nz, U, walls=False)
    mask = fl == 0
    L = O.Lattice(nx, ny, nz, 0.7, u_lid=U, flags=fl, lib=lib)
    u0 = np.zeros((3, nz, ny, nx))
    for a in range(3):
        u0[a] = U[a]
    L.init_fields(None, u0)
    A0 = L.A.copy()
    L.step(100)
    assert np.abs(L.A[:, mask] - A0[:, mask]).max() < 1e-14, "uniform free stream is not a fixed point"
    L = O.Lattice(nx, ny, nz, 0.7, u_lid=U, flags=fl, lib=lib)
    L.step(4000)
    rho, u = L.moments()
    assert np.abs(rho[mask] - 1.0).max() < 1e-12, "density does not settle at 1"
    for a in range(3):
        assert np.abs(u[a][mask] - U[a]).max() < 1e-12, "velocity does not settle at U"


def pin_farfield_channel_flux(lib=None):
    """Walled channel (walls at y = 0, ny-1) between far-field planes: at
    the steady state the mass carried across every plane x + 1/2 (the
    populations that stream from column x to x + 1, minus those from x + 1
    to x) is the same for every x -- the discrete continuity equation."""
    U = (0.05, 0.0, 0.0)
    nx, ny, nz = 24, 9, 1
    fl = _farfield_channel(nx, ny, nz, U, walls=True)
    c, _ = O.velocity_set(lib)
    L = O.Lattice(nx, ny, nz, 0.8, u_lid=U, flags=fl, lib=lib)
    L.step(6000)
    J = []
    for x in range(1, nx - 2):
        s = 0.0
        for z in range(nz):
            for y in range(ny):
                for i in range(19):
                    cx, cy, cz = (int(v) for v in c[i])
                    ty, tz = (y + cy) % ny, (z + cz) % nz
                    if cx == 1 and fl[z, y, x] == 0 and fl[tz, ty, x + 1] == 0:
                        s += L.A[i, z, y, x]
                    if cx == -1 and fl[z, y, x + 1] == 0 and fl[tz, ty, x] == 0:
                        s -= L.A[i, z, y, x + 1]
        J.append(s)
    J = np.array(J)
    assert J.mean() > 0.1, "no flow through the channel"
    assert (J.max() - J.min()) / J.mean() < 1e-10, f"mass flux varies along the channel: {J}"


# ------------------------------------------------------------------ TRT
def pin_trt_reduces_to_bgk(lib=None):
    """TRT with omega- = omega+ is the BGK step (to rounding) on a grid with
    walls, lid and force."""
    nx, ny, nz = 7, 6, 5
    fl = W.random_flags(nx, ny, nz, seed=41, p_wall=0.2, p_lid=0.1)
    _, w = O.velocity_set(lib)
    A = W.random_populations(nx, ny, nz, seed=42, w=w, amp=0.02)
    tau, ulid, g = 0.7, (0.03, -0.02, 0.01), (1e-4, 0.0, -2e-4)
    b = O.step_array(nx, ny, nz, tau, ulid, g, fl, A, lib=lib)
    t = O.step_array(nx, ny, nz, tau, ulid, g, fl, A, lib=lib, omega_minus=1.0 / tau)
    assert np.abs(b - t).max() < 1e-16


def pin_trt_single_cell(lib=None):
    """TRT on a 1x1x1 periodic lattice (the collision alone) relaxes even
    moments at omega+ and odd ones at omega-.  Closed forms for D3Q19 with
    Guo forcing (F = rho g, u = j/rho + g/2): rho' = rho, j' = j + F,
    Pi' = (1-w+) Pi + w+ rho (I/3 + uu) + (1-w+/2)(uF + Fu), and the odd
    third moment Q_xyy = sum_i f_i c_ix c_iy^2, whose equilibrium value is
    rho u_x / 3 and whose forcing value is F_x / 3:
    Q' = (1-w-) Q + w- rho u_x / 3 + (1-w-/2) F_x / 3."""
    c, w = O.velocity_set(lib)
    cf = c.astype(np.float64)
    rng = np.random.default_rng(17)
    for _ in range(10):
        tau = 0.51 + 1.5 * rng.random()
        wp, wm = 1.0 / tau, 0.2 + 1.7 * rng.random()
        g = 1e-3 * (rng.random(3) - 0.5)
        f = w + 0.01 * (rng.random(19) - 0.5)
        L = O.Lattice(1, 1, 1, tau, force=g, lib=lib, omega_minus=wm)
        L.set_populations(f.reshape(19, 1, 1, 1))
        L.step(1)
        fp = L.A.reshape(19)
        rho = f.sum()
        j = f @ cf
        u = j / rho + g / 2
        F = rho * g
        assert abs(fp.sum() - rho) < 1e-15
        assert np.abs(fp @ cf - (j + F)).max() < 1e-16
        Pi = np.einsum("i,ia,ib->ab", f, cf, cf)
        Pi_p = np.einsum("i,ia,ib->ab", fp, cf, cf)
        expect = ((1 - wp) * Pi + wp * rho * (I3 / 3 + np.outer(u, u))
                  + (1 - wp / 2) * (np.outer(u, F) + np.outer(F, u)))
        assert np.abs(Pi_p - expect).max() < 1e-15
        phi = cf[:, 0] * cf[:, 1] ** 2
        Q, Qp = f @ phi, fp @ phi
        assert abs(Qp - ((1 - wm) * Q + wm * rho * u[0] / 3 + (1 - wm / 2) * F[0] / 3)) < 1e-16


def pin_trt_conservation(lib=None):
    """TRT conserves mass, and momentum grows by exactly mass * g per step in
    a periodic box, whatever omega- is."""
    nx, ny, nz = 8, 7, 6
    rho, u = W.random_fields(nx, ny, nz, seed=43, du=0.04, drho=0.02)
    g = np.array([2e-5, -1e-5, 3e-5])
    L = O.Lattice(nx, ny, nz, 0.6, force=g, lib=lib, omega_minus=1.3)
    L.init_fields(rho, u)
    m0, p0 = L.totals()
    L.step(30)
    m1, p1 = L.totals()
    assert abs(m1 - m0) < 1e-13 * m0
    assert np.abs(p1 - (p0 + 30 * m0 * g)).max() < 1e-12 * m0 * np.abs(g).max() * 30


def pin_trt_viscosity(lib=None):
    """The shear viscosity is (tau - 1/2)/3 whatever Lambda is: the decay of
    u0 sin(kz) with two different omega- agrees with nu to second order."""
    n, tau = 64, 0.8
    nu = (tau - 0.5) / 3
    k = 2 * math.pi / n
    z = np.arange(n)
    for wm in (O.trt_omega_minus(tau, 3.0 / 16.0), O.trt_omega_minus(tau, 1.0 / 4.0)):
        u = np.zeros((3, n, 1, 1))
        u[0, :, 0, 0] = 1e-3 * np.sin(k * z)
        L = O.Lattice(1, 1, n, tau, lib=lib, omega_minus=wm)
        L.init_fields(None, u)
        ts, amps = [], []
        for t in range(0, 2001, 100):
            _, uu = L.moments()
            if t >= 200:
                ts.append(t)
                amps.append(2 / n * np.sum(uu[0, :, 0, 0] * np.sin(k * z)))
            L.step(100)
        slope = np.polyfit(np.array(ts), np.log(np.array(amps)), 1)[0]
        assert abs(-slope / (k * k) / nu - 1) < 1e-3


def pin_trt_poiseuille_magic(lib=None):
    """With Lambda = 3/16 halfway bounce-back is exact for the Poiseuille
    flow at ANY tau: the steady profile is g/(2 nu)(y - 1/2)(ny - 3/2 - y)."""
    ny, g = 18, 1e-6
    fl = np.zeros((1, ny, 1), dtype=np.uint8)
    fl[:, 0] = W.WALL
    fl[:, -1] = W.WALL
    for tau in (0.55, 0.8, 1.7):
        nu = (tau - 0.5) / 3
        L = O.Lattice(1, ny, 1, tau, flags=fl, force=(g, 0, 0), lib=lib,
                      omega_minus=O.trt_omega_minus(tau, 3.0 / 16.0))
        L.step(60000 if tau < 0.6 else 30000)
        _, u = L.moments()
        ux = u[0, 0, 1:-1, 0]
        y = np.arange(1, ny - 1)
        exact = g / (2 * nu) * (y - 0.5) * (ny - 1.5 - y)
        assert np.abs(ux - exact).max() < 1e-9 * exact.max(), f"tau {tau}"


ALL_PINS = [
    pin_lattice_tables,
    pin_equilibrium_moments,
    pin_source_moments,
    pin_rest_fixed_point,
    pin_pure_streaming,
    pin_single_cell_collision,
    pin_mass_conservation_cavity,
    pin_periodic_momentum,
    pin_shear_wave,
    pin_taylor_green_2d,
    pin_galilean_advection,
    pin_couette,
    pin_poiseuille,
    pin_cavity_mirror,
    pin_brute_force,
    pin_farfield_free_stream,
    pin_farfield_channel_flux,
    pin_trt_reduces_to_bgk,
    pin_trt_single_cell,
    pin_trt_conservation,
    pin_trt_viscosity,
    pin_trt_poiseuille_magic,
]
