// lb_kernels.cuh -- device building blocks shared by the step, moment and
// batch kernels: the pull (streaming with bounce-back and moving lid) and
// the BGK collision with Guo forcing, both in deviation form d_i = f_i - w_i.
//
// arXiv 2409.16781: Eq. 1 (lattice BGK with source), Eq. 2-3 (equilibrium,
// read as the standard second-order form 1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u),
// Sec. 3.1 (fused approach: scattered read from f^pre, write f^post),
// Sec. 3.3 (lid-driven cavity: no-slip walls and a lid moving at u0).
#pragma once

#include <type_traits>

#include "lb_common.cuh"

namespace lbgb {

#ifdef LBGB_CHECKED
// Bounds-checked build (a test build, liblbgb_checked.so, never the
// product): every population load and store of the step kernels goes through
// ld_pop / st_pop, which check it against the current launch's windows --
// loads inside the array the step reads, stores inside the array it writes
// (19 planes of ps values each) -- set on the launch's stream by the
// launching translation unit (check_window_set).  An access outside is
// counted in g_violations and skipped (a load returns 0), so a bad index
// neither faults nor corrupts memory.  Per translation unit; zero (off) in
// the units that launch no step kernel.
struct CheckWindow {
    uintptr_t rlo, rhi, wlo, whi;
    int on;
};
static __constant__ CheckWindow g_check;
static __device__ unsigned long long g_violations;
static __device__ unsigned long long g_checks;  // accesses checked (shows the checks ran)
#endif

// Row-mapped launches: `xblocks` blocks along x for every row (y, z).  The
// grid is three-dimensional (blockIdx.y = y, blockIdx.z = z) whenever ny and
// nz fit its y and z limits, which spares every block the two integer
// divisions of a flat row index; otherwise it is one flat x dimension of
// xblocks * ny * nz blocks.  gridDim.x tells the kernel which: it equals
// xblocks only for the 3D grid (or for a single row, where both agree).
inline dim3 row_grid(int xblocks, int ny, int nz) {
    if (ny <= 65535 && nz <= 65535) return dim3((unsigned)xblocks, (unsigned)ny, (unsigned)nz);
    return dim3((unsigned)((int64_t)xblocks * ny * nz), 1u, 1u);
}
__device__ __forceinline__ void block_row(int xblocks, int ny, int& xb, int& y, int& z) {
    if (gridDim.x == (unsigned)xblocks) {
        xb = (int)blockIdx.x;
        y = (int)blockIdx.y;
        z = (int)blockIdx.z;
    } else {
        const int row = (int)blockIdx.x / xblocks;
        xb = (int)blockIdx.x - row * xblocks;
        y = row % ny;
        z = row / ny;
    }
}

// Global loads/stores of population values with a cache policy:
//   HINT 0: default (L1 + L2),  1: streaming (.cs, evict-first),
//   HINT 2: L2 only for loads (.cg), streaming stores,
//   HINT 3: loads through the read-only (non-coherent) path, default stores
//           -- for arrays that the launch also writes, valid only where
//           every location a thread loads is written by no other thread of
//           the launch and by this thread only after the load.
template <int HINT, class S>
__device__ __forceinline__ S ld_pop(const S* p) {
    if constexpr (std::is_same<S, f32d>::value) {
        return f32d{ld_pop<HINT>(reinterpret_cast<const float*>(p))};
    } else if constexpr (std::is_same<S, e3m12>::value) {
        return e3m12{ld_pop<HINT>(reinterpret_cast<const unsigned short*>(p))};
    } else {
#ifdef LBGB_CHECKED
        if (g_check.on) {
            const uintptr_t a = reinterpret_cast<uintptr_t>(p);
            atomicAdd(&g_checks, 1ull);
            if (a < g_check.rlo || a + sizeof(S) > g_check.rhi) {
                atomicAdd(&g_violations, 1ull);
                return S{};
            }
        }
#endif
        if constexpr (HINT == 1) return __ldcs(p);
        else if constexpr (HINT == 2) return __ldcg(p);
        else if constexpr (HINT == 3) return __ldg(p);
        else return *p;
    }
}
template <int HINT, class S>
__device__ __forceinline__ void st_pop(S* p, S v) {
    if constexpr (std::is_same<S, f32d>::value) {
        st_pop<HINT>(reinterpret_cast<float*>(p), v.v);
    } else if constexpr (std::is_same<S, e3m12>::value) {
        st_pop<HINT>(reinterpret_cast<unsigned short*>(p), (unsigned short)v.v);
    } else {
#ifdef LBGB_CHECKED
        if (g_check.on) {
            const uintptr_t a = reinterpret_cast<uintptr_t>(p);
            atomicAdd(&g_checks, 1ull);
            if (a < g_check.wlo || a + sizeof(S) > g_check.whi) {
                atomicAdd(&g_violations, 1ull);
                return;
            }
        }
#endif
        if constexpr (HINT == 0 || HINT == 3) *p = v;
        else __stcs(p, v);
    }
}

// Where the state between two steps keeps the post-collision value P_i(x)
// of direction i at cell x:
//   FORM_AB        plane i, cell x (the two-array scheme of Sec. 3.1: the
//                  step reads array A and writes array B);
//   FORM_SWAPPED   plane opp(i), cell x   (in-place "AA" scheme, after an
//   FORM_STREAMED  plane i, cell x + c_i   even / odd number of steps).
// The in-place scheme keeps one array: a step from FORM_SWAPPED reads the
// values streaming into cell x from plane opp(i) at x - c_i and writes its
// results to plane i at x + c_i (FORM_STREAMED); a step from FORM_STREAMED
// reads plane i at x and writes plane opp(i) at x (FORM_SWAPPED).  Either
// way a thread writes exactly the locations it read, so no two threads
// touch the same value.  A fluid cell's value streaming into a solid
// neighbour s = x + c_i lands in the solid cell's slot (plane i at s),
// where the bounce-back of the next step finds it.
enum { FORM_AB = 0, FORM_SWAPPED = 1, FORM_STREAMED = 2 };

// Streaming, pull form: d[i] <- P_i(x - c_i), with periodic wrap at the
// domain edges; if the source is a solid cell, halfway bounce-back takes the
// cell's own opposite post-collision value P_opp(i)(x), plus
// 6 w_i (c_i . u_lid) when the source is a moving-lid cell (wall density 1);
// a far-field source sends the free stream (p.ff, set_farfield), whatever
// the fluid sends out.  FORM says where P lives (above).
// MASK_FIRST changes only the order of work for cells next to a wall: all
// 18 neighbour codes are loaded first (independent loads) into a bit mask of
// solid sources, then every direction loads from its selected address (the
// fluid source or the cell's own opposite value), so the 19 value loads are
// in flight together instead of each waiting on its own code byte; lid and
// far-field terms follow for the directions that need them.  Same values.
template <class S, int HINT = 0, int FORM = FORM_AB, bool MASK_FIRST = false>
__device__ __forceinline__ void pull_cell(const S* __restrict__ A, const uint8_t* __restrict__ code,
                                          const LatticeParams& p, int x, int y, int z, int cell,
                                          uint8_t cc, typename Storage<S>::math (&d)[Q]) {
    using M = typename Storage<S>::math;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int nxy = nx * ny;
    // source coordinate for c = +1, 0, -1 along each axis: x - c
    const int xs[3] = {x == nx - 1 ? 0 : x + 1, x, x == 0 ? nx - 1 : x - 1};
    const int ys[3] = {(y == ny - 1 ? 0 : y + 1) * nx, y * nx, (y == 0 ? ny - 1 : y - 1) * nx};
    const int zs[3] = {(z == nz - 1 ? 0 : z + 1) * nxy, z * nxy, (z == 0 ? nz - 1 : z - 1) * nxy};
    // P_i at a fluid source src, and P_opp(i) at this cell (bounce-back)
    auto fluid_src = [&](int i, int src) -> M {
        if constexpr (FORM == FORM_AB) return Storage<S>::load(ld_pop<HINT>(A + (int64_t)i * p.ps + src));
        else if constexpr (FORM == FORM_SWAPPED)
            return Storage<S>::load(ld_pop<HINT>(A + (int64_t)D3Q19::opp(i) * p.ps + src));
        else return Storage<S>::load(ld_pop<HINT>(A + (int64_t)i * p.ps + cell));
    };
    auto own_opp = [&](int i, int src) -> M {
        if constexpr (FORM == FORM_AB) return Storage<S>::load(ld_pop<HINT>(A + (int64_t)D3Q19::opp(i) * p.ps + cell));
        else if constexpr (FORM == FORM_SWAPPED) return Storage<S>::load(ld_pop<HINT>(A + (int64_t)i * p.ps + cell));
        else return Storage<S>::load(ld_pop<HINT>(A + (int64_t)D3Q19::opp(i) * p.ps + src));
    };
    if (!(cc & CODE_NEAR_WALL)) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int src = xs[D3Q19::cx(i) + 1] + ys[D3Q19::cy(i) + 1] + zs[D3Q19::cz(i) + 1];
            d[i] = fluid_src(i, src);
        }
    } else if constexpr (MASK_FIRST) {
        // all neighbour codes first (independent loads), then all 19 values
        // from the selected addresses, then the rare lid / far-field terms
        uint32_t solid = 0, special = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const uint8_t t = code[xs[D3Q19::cx(i) + 1] + ys[D3Q19::cy(i) + 1] + zs[D3Q19::cz(i) + 1]] & CODE_TYPE;
            solid |= (uint32_t)(t != 0) << i;
            special |= (uint32_t)(t >= 2) << i;
        }
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int src = xs[D3Q19::cx(i) + 1] + ys[D3Q19::cy(i) + 1] + zs[D3Q19::cz(i) + 1];
            const bool b = (solid >> i) & 1u;
            int64_t off;
            if constexpr (FORM == FORM_AB)
                off = b ? (int64_t)D3Q19::opp(i) * p.ps + cell : (int64_t)i * p.ps + src;
            else if constexpr (FORM == FORM_SWAPPED)
                off = b ? (int64_t)i * p.ps + cell : (int64_t)D3Q19::opp(i) * p.ps + src;
            else
                off = b ? (int64_t)D3Q19::opp(i) * p.ps + src : (int64_t)i * p.ps + cell;
            d[i] = Storage<S>::load(ld_pop<HINT>(A + off));
        }
        if (special) {
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                if (!((special >> i) & 1u)) continue;
                const int src = xs[D3Q19::cx(i) + 1] + ys[D3Q19::cy(i) + 1] + zs[D3Q19::cz(i) + 1];
                const uint8_t t = code[src] & CODE_TYPE;
                if (t == CODE_FARFIELD) {
                    d[i] = (M)p.ff[i];
                } else {
                    const double cu = D3Q19::cx(i) * p.ulid[0] + D3Q19::cy(i) * p.ulid[1] +
                                      D3Q19::cz(i) * p.ulid[2];
                    d[i] += (M)(6.0 * D3Q19::w(i) * cu);
                }
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int src = xs[D3Q19::cx(i) + 1] + ys[D3Q19::cy(i) + 1] + zs[D3Q19::cz(i) + 1];
            const uint8_t t = (i == 0) ? 0 : (code[src] & CODE_TYPE);
            if (t == 0) {
                d[i] = fluid_src(i, src);
            } else if (t == CODE_FARFIELD) {
                d[i] = (M)p.ff[i];
            } else {
                M v = own_opp(i, src);
                if (t == 2) {
                    const double cu = D3Q19::cx(i) * p.ulid[0] + D3Q19::cy(i) * p.ulid[1] +
                                      D3Q19::cz(i) * p.ulid[2];
                    v += (M)(6.0 * D3Q19::w(i) * cu);
                }
                d[i] = v;
            }
        }
    }
}

// Bounce-back fix-up for a cell next to a wall: every direction whose pull
// source x - c_i is solid takes the cell's own opposite value instead, plus
// the moving-lid term for LID sources, or the free stream for far-field
// sources (same rules as pull_cell; FORM and MASK_FIRST as there).
template <class S, int HINT = 0, int FORM = FORM_AB, bool MASK_FIRST = false>
__device__ __forceinline__ void bounce_fix(const S* __restrict__ A, const uint8_t* __restrict__ code,
                                           const LatticeParams& p, int x, int y, int z, int cell,
                                           typename Storage<S>::math (&d)[Q]) {
    using M = typename Storage<S>::math;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int nxy = nx * ny;
    const int xs[3] = {x == nx - 1 ? 0 : x + 1, x, x == 0 ? nx - 1 : x - 1};
    const int ys[3] = {(y == ny - 1 ? 0 : y + 1) * nx, y * nx, (y == 0 ? ny - 1 : y - 1) * nx};
    const int zs[3] = {(z == nz - 1 ? 0 : z + 1) * nxy, z * nxy, (z == 0 ? nz - 1 : z - 1) * nxy};
    if constexpr (MASK_FIRST) {
        uint32_t solid = 0, special = 0;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            const uint8_t t = code[xs[D3Q19::cx(i) + 1] + ys[D3Q19::cy(i) + 1] + zs[D3Q19::cz(i) + 1]] & CODE_TYPE;
            solid |= (uint32_t)(t != 0) << i;
            special |= (uint32_t)(t >= 2) << i;
        }
        if (!solid) return;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if ((solid >> i) & 1u) {
                const int src = xs[D3Q19::cx(i) + 1] + ys[D3Q19::cy(i) + 1] + zs[D3Q19::cz(i) + 1];
                const S* q = FORM == FORM_AB         ? A + (int64_t)D3Q19::opp(i) * p.ps + cell
                             : FORM == FORM_SWAPPED ? A + (int64_t)i * p.ps + cell
                                                    : A + (int64_t)D3Q19::opp(i) * p.ps + src;
                d[i] = Storage<S>::load(ld_pop<HINT>(q));
            }
        }
        if (special) {
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                if (!((special >> i) & 1u)) continue;
                const int src = xs[D3Q19::cx(i) + 1] + ys[D3Q19::cy(i) + 1] + zs[D3Q19::cz(i) + 1];
                const uint8_t t = code[src] & CODE_TYPE;
                if (t == CODE_FARFIELD) {
                    d[i] = (M)p.ff[i];
                } else {
                    const double cu = D3Q19::cx(i) * p.ulid[0] + D3Q19::cy(i) * p.ulid[1] +
                                      D3Q19::cz(i) * p.ulid[2];
                    d[i] += (M)(6.0 * D3Q19::w(i) * cu);
                }
            }
        }
        return;
    }
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int src = xs[D3Q19::cx(i) + 1] + ys[D3Q19::cy(i) + 1] + zs[D3Q19::cz(i) + 1];
        const uint8_t t = code[src] & CODE_TYPE;
        if (t == CODE_FARFIELD) {
            d[i] = (M)p.ff[i];
        } else if (t != 0) {
            // the cell's own P_opp(i), wherever FORM keeps it
            const S* q = FORM == FORM_AB         ? A + (int64_t)D3Q19::opp(i) * p.ps + cell
                         : FORM == FORM_SWAPPED ? A + (int64_t)i * p.ps + cell
                                                : A + (int64_t)D3Q19::opp(i) * p.ps + src;
            M v = Storage<S>::load(ld_pop<HINT>(q));
            if (t == 2) {
                const double cu = D3Q19::cx(i) * p.ulid[0] + D3Q19::cy(i) * p.ulid[1] + D3Q19::cz(i) * p.ulid[2];
                v += (M)(6.0 * D3Q19::w(i) * cu);
            }
            d[i] = v;
        }
    }
}

// Zeroth and first moments of the deviations: drho = rho - 1 = sum d_i,
// j = sum d_i c_i (sum w_i c_i = 0).  Opposite directions (2k-1, 2k) enter
// j through their difference.
template <class M>
__device__ __forceinline__ void moment_sums(const M (&d)[Q], M& drho, M& jx, M& jy, M& jz) {
    M s = d[0];
    jx = 0;
    jy = 0;
    jz = 0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = 2 * k + 1;
        s += d[i] + d[i + 1];
        const M diff = d[i] - d[i + 1];
        if (D3Q19::cx(i) == 1) jx += diff;
        if (D3Q19::cx(i) == -1) jx -= diff;
        if (D3Q19::cy(i) == 1) jy += diff;
        if (D3Q19::cy(i) == -1) jy -= diff;
        if (D3Q19::cz(i) == 1) jz += diff;
        if (D3Q19::cz(i) == -1) jz -= diff;
    }
    drho = s;
}

// Two cells' FP32 values in one register pair.  Arithmetic on it maps to the
// packed FP32 instructions of sm_100-class GPUs (add / mul / fma on .f32x2:
// one instruction for both cells, each lane rounded exactly as the scalar
// instruction would round it).  The step kernels that keep two x-adjacent
// cells per register pair run the same collision template on it.
struct f32x2 {
    float2 v;
    f32x2() = default;
    __device__ __forceinline__ f32x2(int s) : v(make_float2((float)s, (float)s)) {}
    __device__ __forceinline__ f32x2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ explicit f32x2(double s) : v(make_float2((float)s, (float)s)) {}
    __device__ __forceinline__ f32x2(float a, float b) : v(make_float2(a, b)) {}
};
__device__ __forceinline__ f32x2 operator+(f32x2 a, f32x2 b) {
    f32x2 r;
    r.v = __fadd2_rn(a.v, b.v);
    return r;
}
__device__ __forceinline__ f32x2 operator-(f32x2 a) { return f32x2(-a.v.x, -a.v.y); }
// a - b as one packed subtraction (each lane rounded as the scalar
// subtraction), not as an addition of a separately negated pair
__device__ __forceinline__ f32x2 operator-(f32x2 a, f32x2 b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;"
        : "=l"(r)
        : "l"(*reinterpret_cast<const unsigned long long*>(&a.v)),
          "l"(*reinterpret_cast<const unsigned long long*>(&b.v)));
    f32x2 o;
    o.v = *reinterpret_cast<const float2*>(&r);
    return o;
}
__device__ __forceinline__ f32x2 operator*(f32x2 a, f32x2 b) {
    f32x2 r;
    r.v = __fmul2_rn(a.v, b.v);
    return r;
}
__device__ __forceinline__ f32x2& operator+=(f32x2& a, f32x2 b) { return a = a + b; }
__device__ __forceinline__ f32x2& operator-=(f32x2& a, f32x2 b) { return a = a - b; }

// Fused multiply-add a * b + c (one rounding) for every math type.
__device__ __forceinline__ double fmad(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float fmad(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ f32x2 fmad(f32x2 a, f32x2 b, f32x2 c) {
    f32x2 r;
    r.v = __ffma2_rn(a.v, b.v, c.v);
    return r;
}

// 1/rho.  FP32: correctly rounded -- the hardware approximation's error has
// a sign bias, so the equilibrium momentum rho u would fall short of j by a
// fixed fraction every step and the collision would drain momentum (an
// artificial dissipation that builds up over thousands of steps).  FP64:
// the hardware's approximate reciprocal refined by two Newton steps
// y <- y + y (1 - r y), each squaring the relative error, so the result is
// within about one unit in the last place of 1/r -- three orders of
// magnitude below the FP32 bias -- for a fraction of the FP64 instructions
// of the IEEE division (the FP64 pipe bounds the FP64 forms).  Densities
// are near 1, far from the approximation's subnormal and overflow limits.
__device__ __forceinline__ double recip(double r) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(r));
    double e = __fma_rn(-r, y, 1.0);
    y = __fma_rn(y, e, y);
    e = __fma_rn(-r, y, 1.0);
    return __fma_rn(y, e, y);
}
__device__ __forceinline__ float recip(float r) { return __frcp_rn(r); }
__device__ __forceinline__ f32x2 recip(f32x2 r) { return f32x2(__frcp_rn(r.v.x), __frcp_rn(r.v.y)); }

// Density and half-force-shifted velocity u = j/rho + g/2 from deviations.
template <class M>
__device__ __forceinline__ void macro_dev(const M (&d)[Q], const LatticeParams& p, M& drho, M& rho,
                                          M& ux, M& uy, M& uz) {
    M jx, jy, jz;
    moment_sums<M>(d, drho, jx, jy, jz);
    rho = M(1) + drho;
    const M inv = recip(rho);
    ux = fmad(jx, inv, param<M>(p.gh[0], p.gh_f[0]));
    uy = fmad(jy, inv, param<M>(p.gh[1], p.gh_f[1]));
    uz = fmad(jz, inv, param<M>(p.gh[2], p.gh_f[2]));
}

// BGK relaxation towards f^eq (Eq. 2-3) plus the Guo source term (the S_i
// of Eq. 1), in place, computing the moments itself:
//   d_i <- (1 - omega) d_i + omega deq_i + S_i,
//   deq_i = f^eq_i - w_i = w_i (drho + rho (3 cu + 4.5 cu^2 - 1.5 uu)),
//   S_i   = (1 - omega/2) w_i [3(c_i - u) + 9 (c_i.u) c_i] . F,  F = rho g,
//   u = j / rho + g / 2.
// It works on opposite pairs (i, i'), c_i' = -c_i: the pair sum relaxes with
// the part of deq + S even in c, the pair difference with the odd part.  In
// exact arithmetic this collision conserves mass and moves the momentum
// from j to j + F; in finite precision the rounded weights (1/18, 1/36 are
// not representable) would bias both by a fixed fraction every step.  So the
// three axis pairs take the difference that makes the momentum exactly
// j + F, and the rest population the value that keeps the mass: the same
// collision, with the conservation laws holding to rounding.
//
// Two-relaxation-time form (Ginzburg's TRT; not in the paper): the pair
// differences (odd part) relax at p.omega_m and take the odd Guo part scaled
// by (1 - omega_m/2); the pair sums (even part) keep omega.  omega_m = omega
// is the BGK collision above, evaluated by the same expressions.  The
// momentum j + F after the collision holds for any omega_m.
//
// M is double, float, or f32x2 (two cells at once); every multiply-add is an
// explicit fmad, so the packed form rounds each cell as the scalar form does.
//
// FP64 arithmetic (M = double) takes the axis pairs' differences and the
// rest population from the equilibrium directly, as the diagonal pairs do:
// there the rounded weights move mass and momentum by parts in 1e16 per
// step, far below anything the solutions resolve, while the closure's sums
// cost 12 instructions per cell on the FP64 pipe that bounds the FP64 forms.
//
// relax_emit hands each post-collision value to emit(i, value) as soon as it
// is final (FP32: the diagonal pairs first, then the axis pairs, then the
// rest population; FP64: the axis pairs, the diagonal pairs, the rest), so a
// kernel can store it at once instead of keeping all 19 in registers;
// relax_dev writes them back into d.
template <class M, bool FORCE, class Emit>
__device__ __forceinline__ void relax_emit(const M (&d)[Q], const LatticeParams& p, Emit&& emit) {
    constexpr bool DIRECT = std::is_same<M, double>::value;
    // pre-collision pair sums / differences and moments (the axis pairs
    // (1,2), (3,4), (5,6) start j along +x, +y, +z; the diagonal pairs add
    // to it, so no sum starts from a zero)
    M ps[9], pd[9];
    M drho = d[0];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = 2 * k + 1;
        ps[k] = d[i] + d[i + 1];
        pd[k] = d[i] - d[i + 1];
        drho += ps[k];
    }
    M jx = pd[0], jy = pd[1], jz = pd[2];
#pragma unroll
    for (int k = 3; k < 9; ++k) {
        const int i = 2 * k + 1;
        if (D3Q19::cx(i) == 1) jx += pd[k];
        if (D3Q19::cx(i) == -1) jx -= pd[k];
        if (D3Q19::cy(i) == 1) jy += pd[k];
        if (D3Q19::cy(i) == -1) jy -= pd[k];
        if (D3Q19::cz(i) == 1) jz += pd[k];
        if (D3Q19::cz(i) == -1) jz -= pd[k];
    }
    const M rho = M(1) + drho;
    const M inv = recip(rho);
    // u = j / rho + g / 2 (without a force: j / rho)
    M ux, uy, uz;
    if constexpr (FORCE) {
        ux = fmad(jx, inv, param<M>(p.gh[0], p.gh_f[0]));
        uy = fmad(jy, inv, param<M>(p.gh[1], p.gh_f[1]));
        uz = fmad(jz, inv, param<M>(p.gh[2], p.gh_f[2]));
    } else {
        ux = jx * inv;
        uy = jy * inv;
        uz = jz * inv;
    }
    const M om = param<M>(p.omega, p.omega_f);
    const M omm = param<M>(p.omega_m, p.omega_m_f);
    // -1.5 u.u (rounding is symmetric in sign, so this is exactly -(1.5 u.u),
    // and no operand below needs a negation)
    const M nuu15 = M(-1.5) * fmad(ux, ux, fmad(uy, uy, uz * uz));
    M Fx = 0, Fy = 0, Fz = 0, uF = 0, pref = 0, pref_m = 0;
    if (FORCE) {
        Fx = rho * param<M>(p.g[0], p.g_f[0]);
        Fy = rho * param<M>(p.g[1], p.g_f[1]);
        Fz = rho * param<M>(p.g[2], p.g_f[2]);
        uF = fmad(ux, Fx, fmad(uy, Fy, uz * Fz));
        pref = param<M>(p.pref, p.pref_f);
        pref_m = param<M>(p.pref_m, p.pref_m_f);
    }
    // Half the post-collision pair sums (hs) and differences (hd):
    //   hs = (1 - omega)/2 (d_i + d_i') + even,   hd = (1 - omega_m)/2 (d_i - d_i') + odd,
    //   d_i = hs + hd,  d_i' = hs - hd,  per weight class W:
    //   even = omega W (rho (4.5 cu^2 - 1.5 uu) + drho) [+ pref W (9 cu cF - 3 uF)]
    //   odd  = 3 omega_m W rho cu                       [+ 3 pref_m W cF]
    const M wa = (M)D3Q19::w(1), wb = (M)D3Q19::w(7);
    const M omh = param<M>(p.omh, p.omh_f);
    const M omh_m = param<M>(p.omh_m, p.omh_m_f);
    const M orho = om * rho;
    const M base = om * fmad(rho, nuu15, drho);
    const M a1 = M(4.5) * wa * orho, b1 = wa * base;
    const M omr = omm * rho;
    const M a2 = M(4.5) * wb * orho, b2 = wb * base, c2 = M(3) * wb * omr;
    M fa1 = 0, fb1 = 0, fa2 = 0, fb2 = 0, fc2 = 0;
    if (FORCE) {
        fa1 = M(9) * pref * wa;
        fb1 = M(-3) * pref * wa * uF;
        fa2 = M(9) * pref * wb;
        fb2 = M(-3) * pref * wb * uF;
        fc2 = M(3) * pref_m * wb;
    }
    // c_i . u and c_i . F of the pair (2k+1, 2k+2): a signed component for an
    // axis pair, the sum or difference of two components for a diagonal pair
    auto dot = [&](int i, M& cu, M& cF) {
        bool first = true;
        auto term = [&](int c, M u, M F) {
            if (c == 0) return;
            if (first) {
                cu = c > 0 ? u : -u;
                cF = c > 0 ? F : -F;
                first = false;
            } else if (c > 0) {
                cu = cu + u;
                cF = cF + F;
            } else {
                cu = cu - u;
                cF = cF - F;
            }
        };
        term(D3Q19::cx(i), ux, Fx);
        term(D3Q19::cy(i), uy, Fy);
        term(D3Q19::cz(i), uz, Fz);
    };
    // the even half-sums of the axis pairs (FP32: needed for the mass below;
    // FP64: the axis pairs are final here)
    M hsa[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        M cu = 0, cF = 0;
        dot(2 * k + 1, cu, cF);
        M even = fmad(a1, cu * cu, b1);
        if (FORCE) even = even + fmad(fa1, cu * cF, fb1);
        hsa[k] = fmad(omh, ps[k], even);
        if constexpr (DIRECT) {
            M odd = (M(3) * wa) * omr * cu;
            if (FORCE) odd = fmad(M(3) * pref_m * wa, cF, odd);
            const M hd = fmad(omh_m, pd[k], odd);
            emit(2 * k + 1, hsa[k] + hd);
            emit(2 * k + 2, hsa[k] - hd);
        }
    }
    M msum = 0;
    if constexpr (!DIRECT) msum = hsa[0] + hsa[1] + hsa[2];
    // half the momentum carried by the 12 diagonal directions; each sum
    // starts at its first term (the flags fold away once the loop is unrolled)
    M ox = 0, oy = 0, oz = 0;
    bool fx = true, fy = true, fz = true;
    auto acc = [](M& o, bool& first, int c, M v) {
        if (c == 0) return;
        if (first) o = c > 0 ? v : -v;
        else if (c > 0) o += v;
        else o -= v;
        first = false;
    };
#pragma unroll
    for (int k = 3; k < 9; ++k) {
        const int i = 2 * k + 1;
        M cu = 0, cF = 0;
        dot(i, cu, cF);
        M even = fmad(a2, cu * cu, b2);
        if (FORCE) even = even + fmad(fa2, cu * cF, fb2);
        const M hs = fmad(omh, ps[k], even);
        M odd = c2 * cu;
        if (FORCE) odd = fmad(fc2, cF, odd);
        const M hd = fmad(omh_m, pd[k], odd);
        if constexpr (!DIRECT) {
            acc(ox, fx, D3Q19::cx(i), hd);
            acc(oy, fy, D3Q19::cy(i), hd);
            acc(oz, fz, D3Q19::cz(i), hd);
            msum += hs;
        }
        emit(i, hs + hd);
        emit(i + 1, hs - hd);
    }
    if constexpr (DIRECT) {
        // rest population: (1 - omega) d_0 + omega deq_0 + S_0, c_0 = 0
        M e0 = M(D3Q19::w(0)) * base;
        if (FORCE) e0 = fmad(M(-3) * D3Q19::w(0) * pref, uF, e0);
        emit(0, fmad(M(p.om1), d[0], e0));
    } else {
        // axis pairs (1,2) x, (3,4) y, (5,6) z: post-collision momentum j + F;
        // nhd = o - (j [+ F]) / 2 is exactly minus the half difference
        // (j [+ F]) / 2 - o, so the pair is (hs - nhd, hs + nhd)
        const M nhdx = fmad(M(-0.5), FORCE ? jx + Fx : jx, ox);
        const M nhdy = fmad(M(-0.5), FORCE ? jy + Fy : jy, oy);
        const M nhdz = fmad(M(-0.5), FORCE ? jz + Fz : jz, oz);
        emit(1, hsa[0] - nhdx);
        emit(2, hsa[0] + nhdx);
        emit(3, hsa[1] - nhdy);
        emit(4, hsa[1] + nhdy);
        emit(5, hsa[2] - nhdz);
        emit(6, hsa[2] + nhdz);
        emit(0, fmad(M(-2), msum, drho));  // mass unchanged by the collision
    }
}

template <class M, bool FORCE>
__device__ __forceinline__ void relax_dev(M (&d)[Q], const LatticeParams& p) {
    M out[Q];
    relax_emit<M, FORCE>(d, p, [&](int i, M v) { out[i] = v; });
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = out[i];
}

// How a step kernel rounds a new value into the storage type S: to nearest
// even (SR = false: Storage<S>::store), or stochastically (SR = true, 16-bit
// storage only: sr_key / sr_bits / cvt_rs2 of lb_common.cuh, with the
// launch's seed).  `key` is the cell pair's hash (key(cell)); a value is
// rounded by the cell that computed it, wherever it is stored.
template <class S> __device__ __forceinline__ S from_bits16(uint32_t w);
template <> __device__ __forceinline__ __half from_bits16<__half>(uint32_t w) {
    return __ushort_as_half((unsigned short)w);
}
template <> __device__ __forceinline__ __nv_bfloat16 from_bits16<__nv_bfloat16>(uint32_t w) {
    return __ushort_as_bfloat16((unsigned short)w);
}
template <> __device__ __forceinline__ e3m12 from_bits16<e3m12>(uint32_t w) { return e3m12{(uint16_t)w}; }

template <class S, bool SR>
struct Rounder {
    static_assert(!SR || sizeof(S) == 2, "stochastic rounding is for 16-bit storage");
    uint32_t seed;
    __device__ __forceinline__ explicit Rounder(uint32_t step_seed) : seed(step_seed) {}
    __device__ __forceinline__ uint32_t key(int cell) const {
        if constexpr (SR) return sr_key(cell, seed);
        else return 0u;
    }
    // value v of direction i of cell `cell`
    __device__ __forceinline__ S one(typename Storage<S>::math v, uint32_t key, int cell, int i) const {
        if constexpr (SR) {
            const uint32_t b = sr_bits(key, i);
            return from_bits16<S>((cell & 1) ? cvt_rs2<S>(0.f, v, b) >> 16 : cvt_rs2<S>(v, 0.f, b));
        } else {
            return Storage<S>::store(v);
        }
    }
    // direction i of the even cell (lo) and the next one (hi), packed into
    // one 32-bit word (16-bit storage)
    __device__ __forceinline__ uint32_t two(float lo, float hi, uint32_t key, int i) const {
        static_assert(sizeof(S) == 2, "packed pairs are 16-bit");
        if constexpr (SR) {
            return cvt_rs2<S>(lo, hi, sr_bits(key, i));
        } else if constexpr (std::is_same<S, __half>::value) {
            const __half2 h = __floats2half2_rn(lo, hi);
            return *reinterpret_cast<const uint32_t*>(&h);
        } else if constexpr (std::is_same<S, e3m12>::value) {
            return e3m12_encode2(lo, hi, e3m12_rn_add(lo), e3m12_rn_add(hi));
        } else {
            const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
            return *reinterpret_cast<const uint32_t*>(&h);
        }
    }
};

// One in-place ("AA") update of fluid cell (x, y, z) whose state has layout
// FORM (FORM_SWAPPED or FORM_STREAMED): pull, collide, and store in the other
// layout -- from FORM_STREAMED into plane opp(i) at the cell, from
// FORM_SWAPPED into plane i at x + c_i (periodic wrap).  Ar and Aw are the
// same array (see step_kernel_inplace for why they are two pointers).
template <class S, bool FORCE, int FORM, bool SR = false>
__device__ __forceinline__ void inplace_update(const S* Ar, S* Aw, const uint8_t* __restrict__ code,
                                               const LatticeParams& p, int x, int y, int z, int cell, uint8_t cc,
                                               uint32_t seed = 0) {
    using M = typename Storage<S>::math;
    M d[Q];
    pull_cell<S, 0, FORM>(Ar, code, p, x, y, z, cell, cc, d);
    relax_dev<M, FORCE>(d, p);
    const Rounder<S, SR> R(seed);
    const uint32_t key = R.key(cell);
    if constexpr (FORM == FORM_STREAMED) {
#pragma unroll
        for (int i = 0; i < Q; ++i) st_pop<0>(Aw + (int64_t)D3Q19::opp(i) * p.ps + cell, R.one(d[i], key, cell, i));
    } else {
        const int nx = p.nx, ny = p.ny, nz = p.nz;
        const int nxy = nx * ny;
        const int xt[3] = {x == 0 ? nx - 1 : x - 1, x, x == nx - 1 ? 0 : x + 1};
        const int yt[3] = {(y == 0 ? ny - 1 : y - 1) * nx, y * nx, (y == ny - 1 ? 0 : y + 1) * nx};
        const int zt[3] = {(z == 0 ? nz - 1 : z - 1) * nxy, z * nxy, (z == nz - 1 ? 0 : z + 1) * nxy};
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int t = xt[D3Q19::cx(i) + 1] + yt[D3Q19::cy(i) + 1] + zt[D3Q19::cz(i) + 1];
            st_pop<0>(Aw + (int64_t)i * p.ps + t, R.one(d[i], key, cell, i));
        }
    }
}

}  // namespace lbgb
