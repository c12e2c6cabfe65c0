// lb_kernels.cuh -- device building blocks shared by the step, moment and
// batch kernels: the pull (streaming with bounce-back and moving lid) and
// the BGK collision with Guo forcing, both in deviation form d_i = f_i - w_i.
//
// arXiv 2409.16781: Eq. 1 (lattice BGK with source), Eq. 2-3 (equilibrium,
// read as the standard second-order form 1 + 3 c.u + 9/2 (c.u)^2 - 3/2 u.u),
// Sec. 3.1 (fused approach: scattered read from f^pre, write f^post),
// Sec. 3.3 (lid-driven cavity: no-slip walls and a lid moving at u0).
#pragma once

#include "lb_common.cuh"

namespace lbgb {

// Global loads/stores of population values with a cache policy:
//   HINT 0: default (L1 + L2),  1: streaming (.cs, evict-first),
//   HINT 2: L2 only for loads (.cg), streaming stores.
template <int HINT, class S>
__device__ __forceinline__ S ld_pop(const S* p) {
    if constexpr (HINT == 1) return __ldcs(p);
    else if constexpr (HINT == 2) return __ldcg(p);
    else return *p;
}
template <int HINT, class S>
__device__ __forceinline__ void st_pop(S* p, S v) {
    if constexpr (HINT == 0) *p = v;
    else __stcs(p, v);
}

// Streaming, pull form: d[i] <- A_i(x - c_i), with periodic wrap at the
// domain edges; if the source is a solid cell, halfway bounce-back takes the
// cell's own opposite post-collision value, plus 6 w_i (c_i . u_lid) when
// the source is a moving-lid cell (wall density 1).
template <class S, int HINT = 0>
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
    if (!(cc & CODE_NEAR_WALL)) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int src = xs[D3Q19::cx(i) + 1] + ys[D3Q19::cy(i) + 1] + zs[D3Q19::cz(i) + 1];
            d[i] = Storage<S>::load(ld_pop<HINT>(A + (int64_t)i * p.ps + src));
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int src = xs[D3Q19::cx(i) + 1] + ys[D3Q19::cy(i) + 1] + zs[D3Q19::cz(i) + 1];
            const uint8_t t = (i == 0) ? 0 : (code[src] & CODE_TYPE);
            if (t == 0) {
                d[i] = Storage<S>::load(ld_pop<HINT>(A + (int64_t)i * p.ps + src));
            } else {
                M v = Storage<S>::load(ld_pop<HINT>(A + (int64_t)D3Q19::opp(i) * p.ps + cell));
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
// the moving-lid term for LID sources (same rule as pull_cell).
template <class S, int HINT = 0>
__device__ __forceinline__ void bounce_fix(const S* __restrict__ A, const uint8_t* __restrict__ code,
                                           const LatticeParams& p, int x, int y, int z, int cell,
                                           typename Storage<S>::math (&d)[Q]) {
    using M = typename Storage<S>::math;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int nxy = nx * ny;
    const int xs[3] = {x == nx - 1 ? 0 : x + 1, x, x == 0 ? nx - 1 : x - 1};
    const int ys[3] = {(y == ny - 1 ? 0 : y + 1) * nx, y * nx, (y == 0 ? ny - 1 : y - 1) * nx};
    const int zs[3] = {(z == nz - 1 ? 0 : z + 1) * nxy, z * nxy, (z == 0 ? nz - 1 : z - 1) * nxy};
#pragma unroll
    for (int i = 1; i < Q; ++i) {
        const int src = xs[D3Q19::cx(i) + 1] + ys[D3Q19::cy(i) + 1] + zs[D3Q19::cz(i) + 1];
        const uint8_t t = code[src] & CODE_TYPE;
        if (t != 0) {
            M v = Storage<S>::load(ld_pop<HINT>(A + (int64_t)D3Q19::opp(i) * p.ps + cell));
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

// 1/rho: IEEE division in FP64; in FP32 the approximate reciprocal (about
// 2 ulp) -- far below the FP32 tolerance and several instructions shorter.
__device__ __forceinline__ double recip(double r) { return 1.0 / r; }
__device__ __forceinline__ float recip(float r) { return __fdividef(1.0f, r); }

// Density and half-force-shifted velocity u = j/rho + g/2 from deviations.
template <class M>
__device__ __forceinline__ void macro_dev(const M (&d)[Q], const LatticeParams& p, M& drho, M& rho,
                                          M& ux, M& uy, M& uz) {
    M jx, jy, jz;
    moment_sums<M>(d, drho, jx, jy, jz);
    rho = M(1) + drho;
    const M inv = recip(rho);
    ux = jx * inv + M(0.5) * (M)p.g[0];
    uy = jy * inv + M(0.5) * (M)p.g[1];
    uz = jz * inv + M(0.5) * (M)p.g[2];
}

// BGK relaxation towards f^eq (Eq. 2-3) plus the Guo source term, in place:
//   d_i <- (1 - omega) d_i + omega deq_i + S_i,
//   deq_i = f^eq_i - w_i = w_i (drho + rho (3 cu + 4.5 cu^2 - 1.5 uu)),
//   S_i   = (1 - omega/2) w_i [3(c_i - u) + 9 (c_i.u) c_i] . (rho g).
// For an opposite pair (i, i') c_i' = -c_i, so both terms split into a part
// even in c (shared) and a part odd in c (sign-flipped):
//   even: w (drho + rho (4.5 cu^2 - 1.5 uu)),  (1-omega/2) w (9 cu cF - 3 uF)
//   odd : 3 w rho cu,                          (1-omega/2) 3 w cF.
template <class M, bool FORCE>
__device__ __forceinline__ void collide_dev(M (&d)[Q], const LatticeParams& p, M drho, M rho, M ux,
                                            M uy, M uz) {
    const M om = (M)p.omega;
    const M omc = M(1) - om;
    const M uu15 = M(1.5) * (ux * ux + uy * uy + uz * uz);
    M Fx = 0, Fy = 0, Fz = 0, uF = 0, pref = 0;
    if (FORCE) {
        Fx = rho * (M)p.g[0];
        Fy = rho * (M)p.g[1];
        Fz = rho * (M)p.g[2];
        uF = ux * Fx + uy * Fy + uz * Fz;
        pref = M(1) - M(0.5) * om;
    }
    // per weight class W: even = aW cu^2 + bW (+ force), odd = cW cu (+ force)
    //   aW = 4.5 omega W rho, bW = omega W (drho - 1.5 rho uu), cW = 3 omega W rho
    const M wa = (M)D3Q19::w(1), wb = (M)D3Q19::w(7);
    const M orho = om * rho;
    const M base = om * (drho - rho * uu15);
    const M a1 = M(4.5) * wa * orho, b1 = wa * base, c1 = M(3) * wa * orho;
    const M a2 = M(4.5) * wb * orho, b2 = wb * base, c2 = M(3) * wb * orho;
    M fa1 = 0, fb1 = 0, fc1 = 0, fa2 = 0, fb2 = 0, fc2 = 0;
    if (FORCE) {  // Guo: even (1-omega/2) W (9 cu cF - 3 uF), odd (1-omega/2) 3 W cF
        fa1 = M(9) * pref * wa;
        fb1 = M(-3) * pref * wa * uF;
        fc1 = M(3) * pref * wa;
        fa2 = M(9) * pref * wb;
        fb2 = M(-3) * pref * wb * uF;
        fc2 = M(3) * pref * wb;
    }
    {
        const M w0 = (M)D3Q19::w(0);
        M e = w0 * base;
        if (FORCE) e += pref * w0 * (M(-3) * uF);
        d[0] = omc * d[0] + e;
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = 2 * k + 1;
        const bool axis = i <= 6;
        M cu = 0, cF = 0;
        if (D3Q19::cx(i) == 1) { cu += ux; cF += Fx; }
        if (D3Q19::cx(i) == -1) { cu -= ux; cF -= Fx; }
        if (D3Q19::cy(i) == 1) { cu += uy; cF += Fy; }
        if (D3Q19::cy(i) == -1) { cu -= uy; cF -= Fy; }
        if (D3Q19::cz(i) == 1) { cu += uz; cF += Fz; }
        if (D3Q19::cz(i) == -1) { cu -= uz; cF -= Fz; }
        M even = (axis ? a1 : a2) * (cu * cu) + (axis ? b1 : b2);
        M odd = (axis ? c1 : c2) * cu;
        if (FORCE) {
            even += (axis ? fa1 : fa2) * (cu * cF) + (axis ? fb1 : fb2);
            odd += (axis ? fc1 : fc2) * cF;
        }
        d[i] = omc * d[i] + (even + odd);
        d[i + 1] = omc * d[i + 1] + (even - odd);
    }
}

}  // namespace lbgb
