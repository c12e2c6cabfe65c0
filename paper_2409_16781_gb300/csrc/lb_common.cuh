// lb_common.cuh -- D3Q19 lattice constants and storage traits for the
// sm_103a kernels of liblbgb.
//
// The velocity set is the 3D extension of the paper's D2Q9 (arXiv 2409.16781
// Sec. 2; 3D named as future work in Sec. 6): rest, the 6 axis neighbours
// (w = 1/18) and the 12 edge neighbours (w = 1/36), c_s^2 = 1/3, in the order
// fixed by include/lbgb.h (opposites are 2k-1, 2k).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>
#include <type_traits>

#include "lb_fpconv.cuh"

namespace lbgb {

constexpr int Q = 19;

struct D3Q19 {
    __host__ __device__ static constexpr int cx(int i) {
        constexpr int t[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        return t[i];
    }
    __host__ __device__ static constexpr int cy(int i) {
        constexpr int t[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        return t[i];
    }
    __host__ __device__ static constexpr int cz(int i) {
        constexpr int t[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        return t[i];
    }
    // The same components for a run-time index, from 2-bit fields (c + 1) of
    // 64-bit constants (no table in local memory).
    __host__ __device__ static constexpr uint64_t pack_(int a) {
        uint64_t k = 0;
        for (int i = 0; i < Q; ++i)
            k |= (uint64_t)((a == 0 ? cx(i) : a == 1 ? cy(i) : cz(i)) + 1) << (2 * i);
        return k;
    }
    __host__ __device__ static int cx_rt(int i) { return (int)((pack_(0) >> (2 * i)) & 3u) - 1; }
    __host__ __device__ static int cy_rt(int i) { return (int)((pack_(1) >> (2 * i)) & 3u) - 1; }
    __host__ __device__ static int cz_rt(int i) { return (int)((pack_(2) >> (2 * i)) & 3u) - 1; }
    __host__ __device__ static constexpr int opp(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
    __host__ __device__ static constexpr double w(int i) {
        return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    }
};

// Internal per-cell code byte (built from the user's flags at create time):
//   bits 0-1: own type (0 fluid, 1 wall, 2 lid, 3 far field)
//   bit 7   : some pull source x - c_i of this cell is solid, so the cell
//             takes the bounce-back path (interior cells skip the 18
//             neighbour-flag reads).
constexpr uint8_t CODE_TYPE = 0x03;
constexpr uint8_t CODE_FARFIELD = 0x03;
constexpr uint8_t CODE_NEAR_WALL = 0x80;

// Storage traits: populations are stored as deviations d_i = f_i - w_i.
template <class S> struct Storage;

template <> struct Storage<double> {
    using math = double;
    static constexpr int id = 0;
    __device__ __forceinline__ static double load(double v) { return v; }
    __device__ __forceinline__ static double store(double v) { return v; }
};
template <> struct Storage<float> {
    using math = float;
    static constexpr int id = 1;
    __device__ __forceinline__ static float load(float v) { return v; }
    __device__ __forceinline__ static float store(float v) { return v; }
};
template <> struct Storage<__half> {
    using math = float;
    static constexpr int id = 2;
    __device__ __forceinline__ static float load(__half v) { return __half2float(v); }
    __device__ __forceinline__ static __half store(float v) { return __float2half_rn(v); }
};
template <> struct Storage<__nv_bfloat16> {
    using math = float;
    static constexpr int id = 3;
    __device__ __forceinline__ static float load(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ __forceinline__ static __nv_bfloat16 store(float v) { return __float2bfloat16_rn(v); }
};

// "Mixed2" (the paper's Sec. 3.1.1): FP32 storage, FP64 arithmetic.  A
// distinct 4-byte type so that the templates can tell it from FP32 math.
struct f32d {
    float v;
};
template <> struct Storage<f32d> {
    using math = double;
    static constexpr int id = 4;
    // integer-pipe conversions (lb_fpconv.cuh): the FP64 pipe bounds this form
    __device__ __forceinline__ static double load(f32d v) { return widen_f32(v.v); }
    __device__ __forceinline__ static f32d store(double v) { return f32d{narrow_f64(v)}; }
};

// Stochastic rounding (SR) of 16-bit stored deviations (lb_options.rounding
// = 1).  Round-to-nearest drops every change smaller than half a unit in the
// last place of the stored value, so a small body force, whose increment
// per step is below that, stalls the flow; SR rounds up with probability
// equal to the dropped fraction, which keeps every value's expectation and
// turns the rounding error into noise.  The random bits come from a
// counter-based hash of (cell pair, direction, step), the same whichever
// kernel shape stores the value, so every step variant gives the same
// bits:
//   key  = fmix32((cell >> 1) ^ seed(step))   (cells 2k and 2k+1 share it)
//   bits = lo32(key * C_i) ^ hi32(key * C_i)  (per direction i)
// fmix32 is the 32-bit finalizer of Appleby's MurmurHash3; C_i are odd
// constants from SplitMix64 (Steele, Lea & Flood 2014) of i + 1.  The
// hardware conversion (cvt.rs.f16x2 / .bf16x2, sm_100-class GPUs) adds the
// bits below the kept mantissa and truncates, taking the low half's bits
// from bits[15:0] and the high half's from bits[31:16] (FP16 the low 13 of
// each), so cell 2k is always converted in the low half and cell 2k+1 in
// the high half.
__host__ __device__ constexpr uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}
__host__ __device__ constexpr uint32_t sr_const(int i) {
    uint64_t z = (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return (uint32_t)z | 1u;
}
// Seed of the step that takes a lattice from `step` to step + 1 steps.
__host__ __device__ constexpr uint32_t sr_seed(int64_t step) {
    return fmix32((uint32_t)step * 0x9E3779B9u ^ fmix32((uint32_t)((uint64_t)step >> 32) + 0x632BE5ABu));
}
__device__ __forceinline__ uint32_t sr_key(int cell, uint32_t seed) { return fmix32(((uint32_t)cell >> 1) ^ seed); }
__device__ __forceinline__ uint32_t sr_bits(uint32_t key, int i) {
    const uint64_t m = (uint64_t)key * sr_const(i);
    return (uint32_t)m ^ (uint32_t)(m >> 32);
}
// The two values packed as (lo | hi << 16), stochastically rounded.
template <class S> __device__ __forceinline__ uint32_t cvt_rs2(float lo, float hi, uint32_t bits);
template <> __device__ __forceinline__ uint32_t cvt_rs2<__half>(float lo, float hi, uint32_t bits) {
    uint32_t r;
    asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(r) : "f"(hi), "f"(lo), "r"(bits));
    return r;
}
template <> __device__ __forceinline__ uint32_t cvt_rs2<__nv_bfloat16>(float lo, float hi, uint32_t bits) {
    uint32_t r;
    asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(r) : "f"(hi), "f"(lo), "r"(bits));
    return r;
}
struct e3m12;
template <> __device__ __forceinline__ uint32_t cvt_rs2<e3m12>(float lo, float hi, uint32_t bits);

// A 16-bit float format of the deviation, finer than FP16 where the
// deviations of a low-Mach flow are: 1 sign, 3 exponent and 12 mantissa
// bits (FP16 has 5 and 10).  |d| in [2^(e-11), 2^(e-10)) for exponent field
// e = 1..7, step 2^(e-23); e = 0 holds the subnormal range [0, 2^-10) in
// steps of 2^-22.  The largest value is (2 - 2^-12) 2^-4 ~ 0.125; larger
// magnitudes (and NaN) saturate to it, and the totals count a saturated
// value as a bad cell.  Above 2^-10 the unit in the last place is a quarter
// of FP16's, and no coarser below.  The conversions use the binary32 bit
// layout: a code placed in bits 26..11 (sign in bit 31) is the float value
// times 2^-116, so decoding is a shift and a multiplication by 2^116 (exact:
// FP32 subnormal inputs included), and encoding multiplies by 2^-116, adds
// the rounding increment below the 12th mantissa bit (half-even for
// rounding to nearest, 11 random bits for stochastic rounding) to the
// magnitude, clamps it, and shifts.
struct e3m12 {
    uint16_t v;
};
constexpr uint32_t E3M12_MAG_MAX = 0x03FFFFFFu;  // FP32 magnitude bits of the largest code (any low bits)
// FP32 bit pattern of a code held in the high half of a word: an arithmetic
// shift by 5 puts the magnitude at bits 25..11 and copies the sign into bits
// 31..26, of which the mask keeps bit 31.
__device__ __forceinline__ uint32_t e3m12_bits_hi(uint32_t w) {
    return (uint32_t)((int32_t)w >> 5) & 0x83FFF800u;
}
__device__ __forceinline__ float e3m12_decode(uint32_t code) {
    return __uint_as_float(e3m12_bits_hi(code << 16)) * 0x1p116f;
}
// the pair (low half, high half) of a 32-bit word as two FP32 values
__device__ __forceinline__ float2 e3m12_decode2(uint32_t w) {
    const float2 b = make_float2(__uint_as_float(e3m12_bits_hi(w << 16)), __uint_as_float(e3m12_bits_hi(w)));
    return __fmul2_rn(b, make_float2(0x1p116f, 0x1p116f));
}
// Magnitude bits of |x| 2^-116 plus `add` (the rounding increment below the
// kept 12 mantissa bits, 0 .. 0x7FF), clamped to the largest code.
__device__ __forceinline__ uint32_t e3m12_mag(float x, uint32_t add) {
    return min(__float_as_uint(fabsf(x) * 0x1p-116f) + add, E3M12_MAG_MAX);
}
__device__ __forceinline__ uint32_t e3m12_rn_add(float x) {
    return 0x3FFu + ((__float_as_uint(fabsf(x) * 0x1p-116f) >> 11) & 1u);  // ties to the even code
}
__device__ __forceinline__ uint32_t e3m12_encode_add(float x, uint32_t add) {
    return (e3m12_mag(x, add) >> 11) | ((__float_as_uint(x) >> 16) & 0x8000u);
}
__device__ __forceinline__ uint32_t e3m12_encode_rn(float x) { return e3m12_encode_add(x, e3m12_rn_add(x)); }
// two codes packed as (lo | hi << 16)
__device__ __forceinline__ uint32_t e3m12_encode2(float lo, float hi, uint32_t add_lo, uint32_t add_hi) {
    const uint32_t mag = (e3m12_mag(lo, add_lo) >> 11) | ((e3m12_mag(hi, add_hi) << 5) & 0x7FFF0000u);
    return mag | (__float_as_uint(hi) & 0x80000000u) | ((__float_as_uint(lo) >> 16) & 0x8000u);
}
template <> struct Storage<e3m12> {
    using math = float;
    static constexpr int id = 5;
    __device__ __forceinline__ static float load(e3m12 v) { return e3m12_decode(v.v); }
    __device__ __forceinline__ static e3m12 store(float v) { return e3m12{(uint16_t)e3m12_encode_rn(v)}; }
};
// The 16-bit IEEE storage types (FP16, BF16), which the kernels that work on
// packed 16-bit registers (variants 6-12 and 14) handle.
template <class S>
constexpr bool ieee16 = std::is_same<S, __half>::value || std::is_same<S, __nv_bfloat16>::value;
// stochastic rounding of an E3M12 pair: the low half takes bits[10:0], the
// high half bits[31:21] (each cell's own bits, as for the IEEE forms)
template <> __device__ __forceinline__ uint32_t cvt_rs2<e3m12>(float lo, float hi, uint32_t bits) {
    return e3m12_encode2(lo, hi, bits & 0x7FFu, bits >> 21);
}

// Parameters of one lattice as seen by the kernels.
struct LatticeParams {
    int nx, ny, nz;
    int64_t N;        // nx*ny*nz
    int64_t ps;       // plane stride between populations (elements), >= N
    double omega;     // 1/tau: rate of the part of f even under c -> -c
    double omega_m;   // rate of the odd part (two-relaxation-time); = omega for BGK
    double g[3];      // body force per unit mass
    double ulid[3];   // lid velocity (and free-stream velocity of far-field cells)
    double ff[19];    // far-field deviations f^eq_i(1, ulid) - w_i (set_farfield)
    int* err;         // device error word (bounded waits that gave up), or nullptr
    // z-planes [zlo, zhi) hold the lattice's own cells; the totals and the
    // moments cover only them.  A z-slab of a decomposed lattice keeps a
    // ghost plane below and above (zlo = 1, zhi = nz - 1) whose inward
    // populations are the neighbouring slabs' values; otherwise 0 and nz.
    int zlo, zhi;
    // rounding of 16-bit stored values: 0 nearest even, 1 stochastic with
    // the step's seed (sr_seed of the steps taken before this one)
    int sr;
    uint32_t sr_seed;
    // omega, omega_m and g rounded to FP32 on the host (set_farfield): the
    // FP32-arithmetic kernels read these instead of converting the FP64
    // fields in every thread (a GB300 runs that conversion on its narrow
    // FP64 pipe); the rounding is the same, so the results are too.
    float omega_f, omega_m_f, g_f[3];
    // per-lattice constants of the collision, also computed on the host
    // (set_farfield) so that no thread recomputes them: half the force
    // (the velocity shift), (1 - omega)/2 and (1 - omega_m)/2 (the pair
    // sums' and differences' own share), 1 - omega/2 and 1 - omega_m/2 (the
    // Guo prefactors), each exactly as a thread would round it
    double gh[3], omh, omh_m, pref, pref_m;
    float gh_f[3], omh_f, omh_m_f, pref_f, pref_m_f;
    double om1;  // 1 - omega (the FP64 rest population's own share)
};

// A lattice parameter in the arithmetic type M: the FP64 field for FP64
// arithmetic, its FP32 copy otherwise.
template <class M>
__host__ __device__ __forceinline__ M param(double d, float f) {
    if constexpr (sizeof(M) == sizeof(double) && !std::is_class<M>::value) return (M)d;
    else return M(f);
}

// The free stream seen from a far-field cell (the inflow and outflow planes
// of flow past an obstacle, the paper's von Karman street use case,
// Sec. 3.3): the deviations f^eq_i(1, U) - w_i = w_i (3 c.U + 9/2 (c.U)^2 -
// 3/2 U.U) of the equilibrium of Eq. 2-3 at density 1 and U = ulid, filled
// on the host once per lattice so that kernels only read them.
inline void set_farfield(LatticeParams& p) {
    p.omega_f = (float)p.omega;
    p.omega_m_f = (float)p.omega_m;
    for (int a = 0; a < 3; ++a) {
        p.g_f[a] = (float)p.g[a];
        p.gh[a] = 0.5 * p.g[a];      // exact
        p.gh_f[a] = 0.5f * p.g_f[a];  // exact
    }
    // each a product by 1/2 (exact) and one rounded sum, in the precision
    // that uses it
    p.omh = 0.5 - 0.5 * p.omega;
    p.omh_m = 0.5 - 0.5 * p.omega_m;
    p.om1 = 1.0 - p.omega;
    p.pref = 1.0 - 0.5 * p.omega;
    p.pref_m = 1.0 - 0.5 * p.omega_m;
    p.omh_f = 0.5f - 0.5f * p.omega_f;
    p.omh_m_f = 0.5f - 0.5f * p.omega_m_f;
    p.pref_f = 1.0f - 0.5f * p.omega_f;
    p.pref_m_f = 1.0f - 0.5f * p.omega_m_f;
    const double uu = p.ulid[0] * p.ulid[0] + p.ulid[1] * p.ulid[1] + p.ulid[2] * p.ulid[2];
    for (int i = 0; i < 19; ++i) {
        const double cu = D3Q19::cx(i) * p.ulid[0] + D3Q19::cy(i) * p.ulid[1] + D3Q19::cz(i) * p.ulid[2];
        p.ff[i] = D3Q19::w(i) * (3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
    }
}

// Error bits a kernel may set in LatticeParams::err.
constexpr int ERR_WAIT_TIMEOUT = 1;

}  // namespace lbgb
