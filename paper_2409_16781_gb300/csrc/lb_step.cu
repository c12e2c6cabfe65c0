// lb_step.cu -- the fused D3Q19 stream-and-collide step kernel (the hot path).
//
// arXiv 2409.16781 Sec. 3.1 ("fused approach"): one launch per time step
// reads the previous post-collision array A through a pull ("scattered read
// from f^pre"), relaxes towards the equilibrium of Eq. 2-3 with the BGK rate
// omega of Eq. 1 plus the source term S_i (Guo forcing), and writes array B;
// the host swaps A and B.  Populations are structure-of-arrays (one
// unit-stride plane per direction), x fastest.
//
// Mapping: one thread per cell; a block covers `blockDim.x` consecutive x of
// one (y, z) row, so each of the 19 gathers and 19 stores of a warp is one
// contiguous 32-element run (the y/z-shifted directions are row-aligned, the
// x-shifted ones are offset by one element and pick up one extra sector,
// served from L1/L2).  Interior cells read only their own code byte; cells
// next to a wall read the 18 neighbour codes (cached) for bounce-back --
// variants 16 and 17 read all 18 before any value (MASK_FIRST), so that the
// value loads of such a cell are in flight together.  The other launch
// shapes (two or four cells per thread, packed FP32 pairs, a TMA pipeline)
// are documented at their kernels below; lb_set_kernel numbers them.
#include <type_traits>

#include "lb_internal.h"
#include "lb_kernels.cuh"
#include "lb_pairs.cuh"
#include "lb_mbarrier.cuh"

namespace lbgb {

// Variants 1-3 (and 16 with MASK_FIRST: cells next to a wall gather their
// neighbour codes before any value, blocks of at most 128 threads capped at
// 48 registers).
template <class S, bool FORCE, int HINT, bool MASK_FIRST = false, bool SR = false>
__global__ void __launch_bounds__(MASK_FIRST ? 128 : 512, MASK_FIRST ? 10 : 0)
    step_kernel_rows(const S* __restrict__ A, S* __restrict__ B, const uint8_t* __restrict__ code, LatticeParams p,
                     int xblocks) {
    using M = typename Storage<S>::math;
    int xb, y, z;
    block_row(xblocks, p.ny, xb, y, z);
    const int row = y + p.ny * z;
    const int x = xb * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    const int cell = x + p.nx * row;
    const uint8_t cc = code[cell];
    if (cc & CODE_TYPE) return;  // solid cells are never written
    M d[Q];
    pull_cell<S, HINT, FORM_AB, MASK_FIRST>(A, code, p, x, y, z, cell, cc, d);
    relax_dev<M, FORCE>(d, p);
    const Rounder<S, SR> R(p.sr_seed);
    const uint32_t key = R.key(cell);
#pragma unroll
    for (int i = 0; i < Q; ++i) st_pop<HINT>(B + (int64_t)i * p.ps + cell, R.one(d[i], key, cell, i));
}

// ---------------------------------------------------------------------------
// Variant 4: two x-consecutive cells per thread (nx even).  Each direction is
// one aligned 2-element vector load from the source row; for c_x = +1 the
// value at x0-1 comes from the previous lane (shuffle), for c_x = -1 the
// value at x0+2 from the next lane, and the warp's edge lanes (or the row's
// last pair) load that single element themselves, wrapping periodically.
// Cells next to a wall then replace the directions with solid sources
// (bounce_fix); all lanes execute the shuffles, so the loads are uniform.
// ---------------------------------------------------------------------------
template <class S, bool FORCE, int HINT>
__global__ void __launch_bounds__(256) step_kernel_pairs(const S* __restrict__ A, S* __restrict__ B,
                                                         const uint8_t* __restrict__ code, LatticeParams p,
                                                         int xblocks) {
    using M = typename Storage<S>::math;
    using V = typename Vec2<S>::T;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    int xb, y, z;
    block_row(xblocks, ny, xb, y, z);
    const int row = y + ny * z;
    const int x0 = 2 * (xb * blockDim.x + threadIdx.x);
    const bool active = x0 < nx;
    const int xa = active ? x0 : 0;  // in-bounds address for idle lanes
    const int lane = threadIdx.x & 31;
    const int nxy = nx * ny;
    const int yo[3] = {(y == ny - 1 ? 0 : y + 1) * nx, y * nx, (y == 0 ? ny - 1 : y - 1) * nx};
    const int zo[3] = {(z == nz - 1 ? 0 : z + 1) * nxy, z * nxy, (z == 0 ? nz - 1 : z - 1) * nxy};
    const int cell0 = xa + nx * row;
    M d0[Q], d1[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const S* rowp = A + (int64_t)i * p.ps + yo[D3Q19::cy(i) + 1] + zo[D3Q19::cz(i) + 1];
        const V v = ld_pop<HINT>(reinterpret_cast<const V*>(rowp + xa));
        M a, b;
        split2<S>(v, a, b);
        if (D3Q19::cx(i) == 0) {
            d0[i] = a;
            d1[i] = b;
        } else if (D3Q19::cx(i) == 1) {  // source x - 1
            M prev = __shfl_up_sync(0xffffffffu, b, 1);
            if (lane == 0 && active) prev = Storage<S>::load(ld_pop<HINT>(rowp + (x0 == 0 ? nx - 1 : x0 - 1)));
            d0[i] = prev;
            d1[i] = a;
        } else {  // source x + 1
            M next = __shfl_down_sync(0xffffffffu, a, 1);
            if (active && (lane == 31 || x0 + 2 >= nx))
                next = Storage<S>::load(ld_pop<HINT>(rowp + (x0 + 2 >= nx ? x0 + 2 - nx : x0 + 2)));
            d0[i] = b;
            d1[i] = next;
        }
    }
    if (!active) return;
    const uint8_t c0 = code[cell0], c1 = code[cell0 + 1];
    if (c0 & CODE_NEAR_WALL) bounce_fix<S, HINT>(A, code, p, x0, y, z, cell0, d0);
    if (c1 & CODE_NEAR_WALL) bounce_fix<S, HINT>(A, code, p, x0 + 1, y, z, cell0 + 1, d1);
    {
        relax_dev<M, FORCE>(d0, p);
    }
    {
        relax_dev<M, FORCE>(d1, p);
    }
    const bool f0 = !(c0 & CODE_TYPE), f1 = !(c1 & CODE_TYPE);
    if (f0 && f1) {
#pragma unroll
        for (int i = 0; i < Q; ++i)
            st_pop<HINT>(reinterpret_cast<V*>(B + (int64_t)i * p.ps + cell0), pack2<S>(d0[i], d1[i]));
    } else {  // solid cells are never written
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (f0) st_pop<HINT>(B + (int64_t)i * p.ps + cell0, Storage<S>::store(d0[i]));
            if (f1) st_pop<HINT>(B + (int64_t)i * p.ps + cell0 + 1, Storage<S>::store(d1[i]));
        }
    }
}

template <class S, int HINT>
static cudaError_t step_pairs_t(const void* A, void* B, const uint8_t* code, const LatticeParams& p, int block,
                                cudaStream_t st) {
    int bx = block > 0 ? (block / 32) * 32 : 128;  // whole warps (the shuffles need all 32 lanes)
    if (bx < 32) bx = 32;
    if (bx > 256) bx = 256;
    const int pairs = p.nx / 2;
    const int need = ((pairs + 31) / 32) * 32;
    if (bx > need) bx = need;
    const int xblocks = (pairs + bx - 1) / bx;
    const bool force = p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    if (force)
        step_kernel_pairs<S, true, HINT><<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    else
        step_kernel_pairs<S, false, HINT><<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Variant 6 (16-bit storage): two x-consecutive cells per thread with the
// loaded values kept packed, one 32-bit register per direction (low half =
// cell x0, high half = x0+1).  The x-shifted directions are rebuilt with a
// lane shuffle and a byte permute: for c_x = +1 the pair (x0-1, x0) is
// (previous lane's high half, own low half); for c_x = -1 the pair
// (x0+1, x0+2) is (own high half, next lane's low half).  Each cell is then
// unpacked to FP32, collided and repacked into a 32-bit store.
// ---------------------------------------------------------------------------
template <class S> __device__ __forceinline__ float lo16(uint32_t v);
template <class S> __device__ __forceinline__ float hi16(uint32_t v);
template <class S> __device__ __forceinline__ uint32_t to16(float f);
template <> __device__ __forceinline__ float lo16<__half>(uint32_t v) {
    return __half2float(__ushort_as_half((unsigned short)(v & 0xffffu)));
}
template <> __device__ __forceinline__ float hi16<__half>(uint32_t v) {
    return __half2float(__ushort_as_half((unsigned short)(v >> 16)));
}
template <> __device__ __forceinline__ uint32_t to16<__half>(float f) {
    return (uint32_t)__half_as_ushort(__float2half_rn(f));
}
// a bf16 value is the upper 16 bits of the FP32 value it stands for
template <> __device__ __forceinline__ float lo16<__nv_bfloat16>(uint32_t v) { return __uint_as_float(v << 16); }
template <> __device__ __forceinline__ float hi16<__nv_bfloat16>(uint32_t v) {
    return __uint_as_float(v & 0xffff0000u);
}
template <> __device__ __forceinline__ uint32_t to16<__nv_bfloat16>(float f) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(f));
}

template <class S, bool FORCE, int HINT>
__global__ void __launch_bounds__(256, 3) step_kernel_pairs16(const S* __restrict__ A, S* __restrict__ B,
                                                           const uint8_t* __restrict__ code, LatticeParams p,
                                                           int xblocks) {
    static_assert(sizeof(S) == 2, "16-bit storage only");
    const uint16_t* __restrict__ A16 = reinterpret_cast<const uint16_t*>(A);
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    int xb, y, z;
    block_row(xblocks, ny, xb, y, z);
    const int row = y + ny * z;
    const int x0 = 2 * (xb * blockDim.x + threadIdx.x);
    const bool active = x0 < nx;
    const int xa = active ? x0 : 0;  // in-bounds address for idle lanes
    const int lane = threadIdx.x & 31;
    const int nxy = nx * ny;
    const int yo[3] = {(y == ny - 1 ? 0 : y + 1) * nx, y * nx, (y == 0 ? ny - 1 : y - 1) * nx};
    const int zo[3] = {(z == nz - 1 ? 0 : z + 1) * nxy, z * nxy, (z == 0 ? nz - 1 : z - 1) * nxy};
    const int cell0 = xa + nx * row;
    uint32_t v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const uint16_t* rowp = A16 + (int64_t)i * p.ps + yo[D3Q19::cy(i) + 1] + zo[D3Q19::cz(i) + 1];
        const uint32_t raw = ld_pop<HINT>(reinterpret_cast<const uint32_t*>(rowp + xa));
        if (D3Q19::cx(i) == 0) {
            v[i] = raw;
        } else if (D3Q19::cx(i) == 1) {  // source x - 1: (prev.hi, own.lo)
            uint32_t prev = __shfl_up_sync(0xffffffffu, raw, 1);
            if (lane == 0 && active)
                prev = (uint32_t)ld_pop<HINT>(rowp + (x0 == 0 ? nx - 1 : x0 - 1)) << 16;
            v[i] = __byte_perm(prev, raw, 0x5432);
        } else {  // source x + 1: (own.hi, next.lo)
            uint32_t next = __shfl_down_sync(0xffffffffu, raw, 1);
            if (active && (lane == 31 || x0 + 2 >= nx))
                next = (uint32_t)ld_pop<HINT>(rowp + (x0 + 2 >= nx ? x0 + 2 - nx : x0 + 2));
            v[i] = __byte_perm(raw, next, 0x5432);
        }
    }
    if (!active) return;
    const uint8_t c0 = code[cell0], c1 = code[cell0 + 1];
    uint32_t out[Q];
    {
        float d[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = lo16<S>(v[i]);
        if (c0 & CODE_NEAR_WALL) bounce_fix<S, HINT>(A, code, p, x0, y, z, cell0, d);
        relax_dev<float, FORCE>(d, p);
#pragma unroll
        for (int i = 0; i < Q; ++i) out[i] = to16<S>(d[i]);
    }
    {
        float d[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = hi16<S>(v[i]);
        if (c1 & CODE_NEAR_WALL) bounce_fix<S, HINT>(A, code, p, x0 + 1, y, z, cell0 + 1, d);
        relax_dev<float, FORCE>(d, p);
#pragma unroll
        for (int i = 0; i < Q; ++i) out[i] |= to16<S>(d[i]) << 16;
    }
    uint16_t* B16 = reinterpret_cast<uint16_t*>(B);
    const bool f0 = !(c0 & CODE_TYPE), f1 = !(c1 & CODE_TYPE);
    if (f0 && f1) {
#pragma unroll
        for (int i = 0; i < Q; ++i) st_pop<HINT>(reinterpret_cast<uint32_t*>(B16 + (int64_t)i * p.ps + cell0), out[i]);
    } else {  // solid cells are never written
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (f0) st_pop<HINT>(B16 + (int64_t)i * p.ps + cell0, (uint16_t)(out[i] & 0xffffu));
            if (f1) st_pop<HINT>(B16 + (int64_t)i * p.ps + cell0 + 1, (uint16_t)(out[i] >> 16));
        }
    }
}

template <class S, int HINT>
static cudaError_t step_pairs16_t(const void* A, void* B, const uint8_t* code, const LatticeParams& p, int block,
                                  cudaStream_t st) {
    int bx = block > 0 ? (block / 32) * 32 : 128;  // whole warps (the shuffles need all 32 lanes)
    if (bx < 32) bx = 32;
    if (bx > 256) bx = 256;
    const int pairs = p.nx / 2;
    const int need = ((pairs + 31) / 32) * 32;
    if (bx > need) bx = need;
    const int xblocks = (pairs + bx - 1) / bx;
    const bool force = p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    if (force)
        step_kernel_pairs16<S, true, HINT><<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    else
        step_kernel_pairs16<S, false, HINT><<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Variant 8 (16-bit storage, nx % 4 == 0): four x-consecutive cells per
// thread, loaded as one 8-byte word per direction (cells x0..x0+3), which
// doubles the bytes each thread keeps in flight.  x-shifts as in variant 6:
// c_x = +1 needs (x0-1 .. x0+2), the first from the previous lane's top
// half; c_x = -1 needs (x0+1 .. x0+4), the last from the next lane's bottom
// half; warp and row edges load that element themselves.
// ---------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ float get16(const uint2& v, int k) {
    return k == 0 ? lo16<S>(v.x) : k == 1 ? hi16<S>(v.x) : k == 2 ? lo16<S>(v.y) : hi16<S>(v.y);
}

template <class S, bool FORCE, int HINT>
__global__ void __launch_bounds__(128, 4) step_kernel_quads16(const S* __restrict__ A, S* __restrict__ B,
                                                              const uint8_t* __restrict__ code, LatticeParams p,
                                                              int xblocks) {
    static_assert(sizeof(S) == 2, "16-bit storage only");
    const uint16_t* __restrict__ A16 = reinterpret_cast<const uint16_t*>(A);
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    int xb, y, z;
    block_row(xblocks, ny, xb, y, z);
    const int row = y + ny * z;
    const int x0 = 4 * (xb * blockDim.x + threadIdx.x);
    const bool active = x0 < nx;
    const int xa = active ? x0 : 0;  // in-bounds address for idle lanes
    const int lane = threadIdx.x & 31;
    const int nxy = nx * ny;
    const int yo[3] = {(y == ny - 1 ? 0 : y + 1) * nx, y * nx, (y == 0 ? ny - 1 : y - 1) * nx};
    const int zo[3] = {(z == nz - 1 ? 0 : z + 1) * nxy, z * nxy, (z == 0 ? nz - 1 : z - 1) * nxy};
    const int cell0 = xa + nx * row;
    uint2 v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const uint16_t* rowp = A16 + (int64_t)i * p.ps + yo[D3Q19::cy(i) + 1] + zo[D3Q19::cz(i) + 1];
        const uint2 raw = ld_pop<HINT>(reinterpret_cast<const uint2*>(rowp + xa));
        if (D3Q19::cx(i) == 0) {
            v[i] = raw;
        } else if (D3Q19::cx(i) == 1) {  // source x - 1: (prev top, x0, x0+1, x0+2)
            uint32_t prev = __shfl_up_sync(0xffffffffu, raw.y, 1);
            if (lane == 0 && active)
                prev = (uint32_t)ld_pop<HINT>(rowp + (x0 == 0 ? nx - 1 : x0 - 1)) << 16;
            v[i] = make_uint2(__byte_perm(prev, raw.x, 0x5432), __byte_perm(raw.x, raw.y, 0x5432));
        } else {  // source x + 1: (x0+1, x0+2, x0+3, next bottom)
            uint32_t next = __shfl_down_sync(0xffffffffu, raw.x, 1);
            if (active && (lane == 31 || x0 + 4 >= nx))
                next = (uint32_t)ld_pop<HINT>(rowp + (x0 + 4 >= nx ? x0 + 4 - nx : x0 + 4));
            v[i] = make_uint2(__byte_perm(raw.x, raw.y, 0x5432), __byte_perm(raw.y, next, 0x5432));
        }
    }
    if (!active) return;
    const uint32_t codes = *reinterpret_cast<const uint32_t*>(code + cell0);  // 4 code bytes
    uint2 out[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) out[i] = make_uint2(0u, 0u);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float d[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = get16<S>(v[i], k);
        const uint8_t ck = (uint8_t)(codes >> (8 * k));
        if (ck & CODE_NEAR_WALL) bounce_fix<S, HINT>(A, code, p, x0 + k, y, z, cell0 + k, d);
        relax_dev<float, FORCE>(d, p);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const uint32_t h = to16<S>(d[i]) << (16 * (k & 1));
            if (k < 2) out[i].x |= h;
            else out[i].y |= h;
        }
    }
    uint16_t* B16 = reinterpret_cast<uint16_t*>(B);
    const uint32_t solid = codes & 0x03030303u;
    if (solid == 0) {
#pragma unroll
        for (int i = 0; i < Q; ++i) st_pop<HINT>(reinterpret_cast<uint2*>(B16 + (int64_t)i * p.ps + cell0), out[i]);
    } else {  // solid cells are never written
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if ((codes >> (8 * k)) & CODE_TYPE) continue;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const uint32_t word = k < 2 ? out[i].x : out[i].y;
                st_pop<HINT>(B16 + (int64_t)i * p.ps + cell0 + k, (uint16_t)(word >> (16 * (k & 1))));
            }
        }
    }
}

template <class S, int HINT>
static cudaError_t step_quads16_t(const void* A, void* B, const uint8_t* code, const LatticeParams& p, int block,
                                  cudaStream_t st) {
    int bx = block > 0 ? (block / 32) * 32 : 64;  // whole warps (the shuffles need all 32 lanes)
    if (bx < 32) bx = 32;
    if (bx > 128) bx = 128;
    const int quads = p.nx / 4;
    const int need = ((quads + 31) / 32) * 32;
    if (bx > need) bx = need;
    const int xblocks = (quads + bx - 1) / bx;
    const bool force = p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    if (force)
        step_kernel_quads16<S, true, HINT><<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    else
        step_kernel_quads16<S, false, HINT><<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Variants 13 and 14: the collision of two x-adjacent cells at once in packed
// FP32 (f32x2: one add/mul/fma instruction for both cells), which halves the
// arithmetic instructions per cell -- the bound of the 16-bit kernels, whose
// bytes per cell are half those of FP32 storage.
//   13: two cells per thread (float, FP16 or BF16 storage, nx even); each
//       direction is one aligned 2-vector load, x-shifts by lane shuffles as
//       in variant 4.
//   14: four cells per thread (16-bit storage, nx % 4 == 0); one 8-byte load
//       per direction as in variant 8, the cells collided as two pairs.
//   15: variant 13 in blocks of at most 128 threads capped at 64 registers
//       (32 warps per SM; a few values spill to L1-backed local memory).
//   17: variant 15 with the mask-first bounce-back fix-up (MASK_FIRST:
//       neighbour codes first, then the wall values together).
// Cells next to a wall leave the packed form for the bounce-back fix-up of
// each cell and re-enter it.
// ---------------------------------------------------------------------------
//   18: variant 15 with whole-row blocks (nx a multiple of 64, at most 1024;
//       else variant 15): the values that cross a warp edge come from the
//       neighbouring warp through shared memory (ROW of pair_x2_update).
//   19: variant 18 with the mask-first bounce-back fix-up (17 where the row
//       does not fit).
template <class S, bool FORCE, int HINT, int MINB, bool MASK_FIRST = false, bool SR = false, bool ROW = false>
__global__ void __launch_bounds__(ROW ? 512 : 256 / MINB, ROW ? 2 : (MINB == 1 ? 0 : 4 * MINB))
    step_kernel_pairs_x2(const S* __restrict__ A, S* __restrict__ B, const uint8_t* __restrict__ code, LatticeParams p,
                         int xblocks) {
    int xb, y, z;
    block_row(xblocks, p.ny, xb, y, z);
    const int x0 = 2 * (xb * blockDim.x + threadIdx.x);
    const bool active = ROW || x0 < p.nx;
    const int xa = active ? x0 : 0;  // in-bounds address for idle lanes
    pair_x2_update<S, FORCE, HINT, MASK_FIRST, SR, ROW>(A, B, code, p, xa, y, z, xa + p.nx * (y + p.ny * z),
                                                        threadIdx.x & 31, active);
}

template <class S, int HINT, int MINB, bool MASK_FIRST = false, bool SR = false>
static cudaError_t step_pairs_x2_t(const void* A, void* B, const uint8_t* code, const LatticeParams& p, int block,
                                   cudaStream_t st) {
    int bx = block > 0 ? (block / 32) * 32 : 64;  // whole warps (the shuffles need all 32 lanes)
    if (bx < 32) bx = 32;
    if (bx > 256 / MINB) bx = 256 / MINB;
    const int pairs = p.nx / 2;
    const int need = ((pairs + 31) / 32) * 32;
    if (bx > need) bx = need;
    const int xblocks = (pairs + bx - 1) / bx;
    const bool force = p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    if (force)
        step_kernel_pairs_x2<S, true, HINT, MINB, MASK_FIRST, SR>
            <<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    else
        step_kernel_pairs_x2<S, false, HINT, MINB, MASK_FIRST, SR>
            <<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    return cudaGetLastError();
}

// Variants 18 and 19 (19: with MASK_FIRST): one block per row, nx / 2
// threads (variant 15, or 17, where the row does not fit whole warps or one
// block).
template <class S, int HINT, bool SR = false, bool MASK_FIRST = false>
static cudaError_t step_pairs_x2_row_t(const void* A, void* B, const uint8_t* code, const LatticeParams& p,
                                       cudaStream_t st) {
    if (p.nx % 64 != 0 || p.nx > 1024)
        return step_pairs_x2_t<S, HINT, 2, MASK_FIRST, SR>(A, B, code, p, 64, st);
    const bool force = p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    if (force)
        step_kernel_pairs_x2<S, true, HINT, 2, MASK_FIRST, SR, true>
            <<<row_grid(1, p.ny, p.nz), p.nx / 2, 0, st>>>((const S*)A, (S*)B, code, p, 1);
    else
        step_kernel_pairs_x2<S, false, HINT, 2, MASK_FIRST, SR, true>
            <<<row_grid(1, p.ny, p.nz), p.nx / 2, 0, st>>>((const S*)A, (S*)B, code, p, 1);
    return cudaGetLastError();
}

template <class S, bool FORCE, int HINT>
__global__ void __launch_bounds__(128, 4) step_kernel_quads16_x2(const S* __restrict__ A, S* __restrict__ B,
                                                                 const uint8_t* __restrict__ code, LatticeParams p,
                                                                 int xblocks) {
    static_assert(sizeof(S) == 2, "16-bit storage only");
    const uint16_t* __restrict__ A16 = reinterpret_cast<const uint16_t*>(A);
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    int xb, y, z;
    block_row(xblocks, ny, xb, y, z);
    const int row = y + ny * z;
    const int x0 = 4 * (xb * blockDim.x + threadIdx.x);
    const bool active = x0 < nx;
    const int xa = active ? x0 : 0;  // in-bounds address for idle lanes
    const int lane = threadIdx.x & 31;
    const int nxy = nx * ny;
    const int yo[3] = {(y == ny - 1 ? 0 : y + 1) * nx, y * nx, (y == 0 ? ny - 1 : y - 1) * nx};
    const int zo[3] = {(z == nz - 1 ? 0 : z + 1) * nxy, z * nxy, (z == 0 ? nz - 1 : z - 1) * nxy};
    const int cell0 = xa + nx * row;
    uint2 v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const uint16_t* rowp = A16 + (int64_t)i * p.ps + yo[D3Q19::cy(i) + 1] + zo[D3Q19::cz(i) + 1];
        const uint2 raw = ld_pop<HINT>(reinterpret_cast<const uint2*>(rowp + xa));
        if (D3Q19::cx(i) == 0) {
            v[i] = raw;
        } else if (D3Q19::cx(i) == 1) {  // source x - 1: (prev top, x0, x0+1, x0+2)
            uint32_t prev = __shfl_up_sync(0xffffffffu, raw.y, 1);
            if (lane == 0 && active)
                prev = (uint32_t)ld_pop<HINT>(rowp + (x0 == 0 ? nx - 1 : x0 - 1)) << 16;
            v[i] = make_uint2(__byte_perm(prev, raw.x, 0x5432), __byte_perm(raw.x, raw.y, 0x5432));
        } else {  // source x + 1: (x0+1, x0+2, x0+3, next bottom)
            uint32_t next = __shfl_down_sync(0xffffffffu, raw.x, 1);
            if (active && (lane == 31 || x0 + 4 >= nx))
                next = (uint32_t)ld_pop<HINT>(rowp + (x0 + 4 >= nx ? x0 + 4 - nx : x0 + 4));
            v[i] = make_uint2(__byte_perm(raw.x, raw.y, 0x5432), __byte_perm(raw.y, next, 0x5432));
        }
    }
    if (!active) return;
    const uint32_t codes = *reinterpret_cast<const uint32_t*>(code + cell0);  // 4 code bytes
    uint16_t* B16 = reinterpret_cast<uint16_t*>(B);
#pragma unroll
    for (int h = 0; h < 2; ++h) {  // cells (x0, x0+1), then (x0+2, x0+3)
        const uint8_t ca = (uint8_t)(codes >> (16 * h)), cb = (uint8_t)(codes >> (16 * h + 8));
        f32x2 d[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) d[i] = to_x2<S>(h == 0 ? v[i].x : v[i].y);
        bounce_fix_x2<S, HINT>(A, code, p, x0 + 2 * h, y, z, cell0 + 2 * h, ca, cb, d);
        relax_dev<f32x2, FORCE>(d, p);
        // each pair is stored as soon as it is done (one 4-byte word per
        // direction), so no packed results are held across the second pair.
        // (Storing each value from inside the collision, as it becomes
        // final, measured slower here.)
        uint16_t* cp = B16 + cell0 + 2 * h;
        if (!((ca | cb) & CODE_TYPE)) {
#pragma unroll
            for (int i = 0; i < Q; ++i) st_pop<HINT>(reinterpret_cast<uint32_t*>(cp + (int64_t)i * p.ps), from_x2<S>(d[i]));
        } else {  // solid cells are never written
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const uint32_t word = from_x2<S>(d[i]);
                if (!(ca & CODE_TYPE)) st_pop<HINT>(cp + (int64_t)i * p.ps, (uint16_t)(word & 0xffffu));
                if (!(cb & CODE_TYPE)) st_pop<HINT>(cp + (int64_t)i * p.ps + 1, (uint16_t)(word >> 16));
            }
        }
    }
}

template <class S, int HINT>
static cudaError_t step_quads16_x2_t(const void* A, void* B, const uint8_t* code, const LatticeParams& p, int block,
                                     cudaStream_t st) {
    int bx = block > 0 ? (block / 32) * 32 : 64;  // whole warps (the shuffles need all 32 lanes)
    if (bx < 32) bx = 32;
    if (bx > 128) bx = 128;
    const int quads = p.nx / 4;
    const int need = ((quads + 31) / 32) * 32;
    if (bx > need) bx = need;
    const int xblocks = (quads + bx - 1) / bx;
    const bool force = p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    if (force)
        step_kernel_quads16_x2<S, true, HINT><<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    else
        step_kernel_quads16_x2<S, false, HINT><<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    return cudaGetLastError();
}

template <class S, int HINT, bool MASK_FIRST = false, bool SR = false>
static cudaError_t step_rows_t(const void* A, void* B, const uint8_t* code, const LatticeParams& p, int block,
                               cudaStream_t st);

// ---------------------------------------------------------------------------
// Variant 10 (16-bit storage, nx % 16 == 0): TMA bulk-copy pipeline.
// A tile is R rows x TX cells (R * TX = 512).  One producer warp copies, for
// every row of the tile and every direction i, the source run of plane i at
// row (y - c_y, z - c_z), x in [x0, x0 + TX), into shared memory with
// cp.async.bulk, plus a 16-byte halo before it (c_x = +1) or after it
// (c_x = -1), wrapped periodically, and the tile's code bytes; the copies
// complete on the stage's "full" mbarrier.  Four consumer warps wait on it,
// compute four cells per thread from shared memory (x-shifts are aligned
// 4- and 8-byte loads plus byte permutes) and store to B directly, then
// release the stage on its "empty" mbarrier.  Bytes in flight live in the
// STAGES-deep shared-memory ring, not in registers.  Every wait is bounded
// (iteration cap and a 2 s %globaltimer deadline); a wait that gives up sets
// ERR_WAIT_TIMEOUT in p.err and the block stops, after the producer has
// waited (again bounded) for the copies it issued.
// ---------------------------------------------------------------------------
constexpr int TMA_STAGES = 4;
// consumer warps per block and threads per block for G cells per consumer
// thread: four-cell and two-cell threads use 4 consumer warps, one-cell
// threads 8 (fewer registers each, so more warps hide shared-memory latency)
__host__ __device__ constexpr int tma_consumer_warps(int G) { return G == 1 ? 8 : 4; }
__host__ __device__ constexpr int tma_threads(int G) { return 32 * (1 + tma_consumer_warps(G)); }
constexpr int TMA_HALO = 8;  // 16 bytes of 16-bit values
// cells per tile with G cells per consumer thread
__host__ __device__ constexpr int tma_tile_cells(int G) { return G * 32 * tma_consumer_warps(G); }
// largest stage ring: TX = 16 -> R = tile/16 rows of 19 * (16 + 16) * 2 + 16 bytes
__host__ __device__ constexpr int tma_max_smem(int G) {
    return TMA_STAGES * (tma_tile_cells(G) / 16) * (19 * (16 + 2 * TMA_HALO) * 2 + 16);
}

struct TmaGeom {
    int TX;          // tile width in cells (divides nx, multiple of 16)
    int R;           // rows per tile
    int xchunks;     // nx / TX
    int nrows;       // ny * nz
    int64_t ntiles;  // xchunks * ceil(nrows / R)
    int rb;          // bytes of one (row, direction) buffer: (TX + 2 halo) * 2
    int row_bytes;   // 19 * rb + TX (codes)
    int stage_bytes; // R * row_bytes
};

template <class S, bool FORCE, int G>
__global__ void __launch_bounds__(tma_threads(G), G == 4 ? 2 : (G == 2 ? 4 : 3)) step_kernel_tma16(const S* __restrict__ A, S* __restrict__ B,
                                                                 const uint8_t* __restrict__ code, LatticeParams p,
                                                                 TmaGeom g) {
    static_assert(sizeof(S) == 2, "16-bit storage only");
    extern __shared__ __align__(128) uint8_t smem[];
    __shared__ __align__(8) uint64_t full_bar[TMA_STAGES];
    __shared__ __align__(8) uint64_t empty_bar[TMA_STAGES];
    __shared__ int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    if (threadIdx.x == 0) {
        for (int s = 0; s < TMA_STAGES; ++s) {
            mbar_init(smem_addr(&full_bar[s]), 1);
            mbar_init(smem_addr(&empty_bar[s]), tma_consumer_warps(G));
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    const uint16_t* A16 = reinterpret_cast<const uint16_t*>(A);

    if (warp == 0) {
        // ------------------------------ producer ------------------------------
        int64_t k = 0;
        for (int64_t t = blockIdx.x; t < g.ntiles; t += gridDim.x, ++k) {
            const int s = (int)(k % TMA_STAGES);
            const uint32_t n = (uint32_t)(k / TMA_STAGES);
            bool ok = true;
            if (lane == 0) {
                if (k >= TMA_STAGES) ok = mbar_wait(smem_addr(&empty_bar[s]), (n - 1) & 1);
                if (ok && *(volatile int*)&abort_flag) ok = false;
            }
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) {
                if (lane == 0) {
                    atomicOr(p.err, ERR_WAIT_TIMEOUT);
                    *(volatile int*)&abort_flag = 1;
                }
                break;
            }
            const int xc = (int)(t % g.xchunks);
            const int row0 = (int)(t / g.xchunks) * g.R;
            const int rows = min(g.R, g.nrows - row0);
            const int x0 = xc * g.TX;
            const uint32_t fb = smem_addr(&full_bar[s]);
            if (lane == 0) mbar_expect_tx(fb, (uint32_t)rows * (19u * g.TX * 2u + 10u * 16u + (uint32_t)g.TX));
            __syncwarp();
            const uint32_t stage = smem_addr(smem) + (uint32_t)s * g.stage_bytes;
            for (int idx = lane; idx < rows * 20; idx += 32) {
                const int r = idx / 20, i = idx % 20;
                const int row = row0 + r;
                const uint32_t rbase = stage + (uint32_t)r * g.row_bytes;
                if (i == 19) {  // the tile's code bytes
                    bulk_g2s(rbase + 19u * g.rb, code + (int64_t)row * nx + x0, (uint32_t)g.TX, fb);
                    continue;
                }
                const int y = row % ny, z = row / ny;
                int sy = y - D3Q19::cy_rt(i), sz = z - D3Q19::cz_rt(i);
                sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
                sz = sz < 0 ? sz + nz : (sz >= nz ? sz - nz : sz);
                const uint16_t* srow = A16 + (int64_t)i * p.ps + ((int64_t)sz * ny + sy) * nx;
                const uint32_t buf = rbase + (uint32_t)i * g.rb;
                bulk_g2s(buf + 2u * TMA_HALO, srow + x0, 2u * g.TX, fb);
                const int cxi = D3Q19::cx_rt(i);
                if (cxi == 1)  // needs x0 - 1: halo before, wrapping at x = 0
                    bulk_g2s(buf, srow + (x0 == 0 ? nx - TMA_HALO : x0 - TMA_HALO), 16u, fb);
                else if (cxi == -1)  // needs x0 + TX: halo after, wrapping at x = nx
                    bulk_g2s(buf + 2u * (TMA_HALO + g.TX), srow + (x0 + g.TX == nx ? 0 : x0 + g.TX), 16u, fb);
            }
        }
        // do not leave while copies into this block's shared memory are in flight
        if (lane == 0) {
            const int64_t used = k < TMA_STAGES ? k : TMA_STAGES;
            for (int64_t q = k - used; q < k; ++q) {
                const int s = (int)(q % TMA_STAGES);
                if (!mbar_wait(smem_addr(&full_bar[s]), (uint32_t)(q / TMA_STAGES) & 1)) atomicOr(p.err, ERR_WAIT_TIMEOUT);
            }
        }
        return;
    }

    // -------------------------------- consumers --------------------------------
    const int ct = (warp - 1) * 32 + lane;  // 0 .. 32 * consumer warps - 1
    const int groups_per_row = g.TX / G;
    const int r = ct / groups_per_row, j = ct % groups_per_row;
    // G packed 16-bit values per direction
    using W = typename std::conditional<G == 4, uint2, typename std::conditional<G == 2, uint32_t, uint16_t>::type>::type;
    int64_t k = 0;
    for (int64_t t = blockIdx.x; t < g.ntiles; t += gridDim.x, ++k) {
        const int s = (int)(k % TMA_STAGES);
        const uint32_t n = (uint32_t)(k / TMA_STAGES);
        bool ok = true;
        if (lane == 0) {
            ok = mbar_wait(smem_addr(&full_bar[s]), n & 1);
            if (ok && *(volatile int*)&abort_flag) ok = false;
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) {
            if (lane == 0) {
                atomicOr(p.err, ERR_WAIT_TIMEOUT);
                *(volatile int*)&abort_flag = 1;
            }
            break;
        }
        const int xc = (int)(t % g.xchunks);
        const int row0 = (int)(t / g.xchunks) * g.R;
        const int rows = min(g.R, g.nrows - row0);
        const bool mine = r < rows;
        // a thread without a row in this (last, partial) tile reads row 0 and discards it
        const uint8_t* rb8 = smem + (size_t)s * g.stage_bytes + (size_t)(mine ? r : 0) * g.row_bytes;
        W v[Q];
        uint32_t codes;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const uint8_t* b = rb8 + i * g.rb + 2 * (TMA_HALO + G * j);
            if constexpr (G == 1) {
                v[i] = *reinterpret_cast<const uint16_t*>(b - 2 * D3Q19::cx(i));  // the value at x - c_x
            } else if constexpr (G == 4) {
                const uint2 q = *reinterpret_cast<const uint2*>(b);
                if (D3Q19::cx(i) == 0) {
                    v[i] = q;
                } else if (D3Q19::cx(i) == 1) {  // (x-1, x, x+1, x+2)
                    const uint32_t pr = *reinterpret_cast<const uint32_t*>(b - 4);
                    v[i] = make_uint2(__byte_perm(pr, q.x, 0x5432), __byte_perm(q.x, q.y, 0x5432));
                } else {  // (x+1, x+2, x+3, x+4)
                    const uint32_t nw = *reinterpret_cast<const uint32_t*>(b + 8);
                    v[i] = make_uint2(__byte_perm(q.x, q.y, 0x5432), __byte_perm(q.y, nw, 0x5432));
                }
            } else {
                const uint32_t q = *reinterpret_cast<const uint32_t*>(b);
                if (D3Q19::cx(i) == 0) {
                    v[i] = q;
                } else if (D3Q19::cx(i) == 1) {  // (x-1, x)
                    v[i] = __byte_perm(*reinterpret_cast<const uint32_t*>(b - 4), q, 0x5432);
                } else {  // (x+1, x+2)
                    v[i] = __byte_perm(q, *reinterpret_cast<const uint32_t*>(b + 4), 0x5432);
                }
            }
        }
        if constexpr (G == 4)
            codes = *reinterpret_cast<const uint32_t*>(rb8 + 19 * g.rb + 4 * j);
        else if constexpr (G == 2)
            codes = *reinterpret_cast<const uint16_t*>(rb8 + 19 * g.rb + 2 * j);
        else
            codes = rb8[19 * g.rb + j];
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_addr(&empty_bar[s]));  // this warp's shared-memory reads are done
        if (!mine) continue;
        const int row = row0 + r;
        const int y = row % ny, z = row / ny;
        const int xq = xc * g.TX + G * j;
        const int cell0 = xq + nx * row;
        W out[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if constexpr (G == 4) out[i] = make_uint2(0u, 0u);
            else out[i] = 0;
        }
#pragma unroll
        for (int kk = 0; kk < G; ++kk) {
            float d[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if constexpr (G == 4) d[i] = get16<S>(v[i], kk);
                else if constexpr (G == 2) d[i] = kk == 0 ? lo16<S>(v[i]) : hi16<S>(v[i]);
                else d[i] = lo16<S>((uint32_t)v[i]);
            }
            const uint8_t ck = (uint8_t)(codes >> (8 * kk));
            if (ck & CODE_NEAR_WALL) bounce_fix<S, 0>(A, code, p, xq + kk, y, z, cell0 + kk, d);
            relax_dev<float, FORCE>(d, p);
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const uint32_t h = to16<S>(d[i]) << (16 * (kk & 1));
                if constexpr (G == 4) {
                    if (kk < 2) out[i].x |= h;
                    else out[i].y |= h;
                } else {
                    out[i] |= (W)h;
                }
            }
        }
        uint16_t* B16 = reinterpret_cast<uint16_t*>(B);
        const uint32_t solid_mask = G == 4 ? 0x03030303u : (G == 2 ? 0x0303u : 0x03u);
        if ((codes & solid_mask) == 0) {
#pragma unroll
            for (int i = 0; i < Q; ++i) st_pop<0>(reinterpret_cast<W*>(B16 + (int64_t)i * p.ps + cell0), out[i]);
        } else {  // solid cells are never written
#pragma unroll
            for (int kk = 0; kk < G; ++kk) {
                if ((codes >> (8 * kk)) & CODE_TYPE) continue;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    uint32_t word;
                    if constexpr (G == 4) word = kk < 2 ? out[i].x : out[i].y;
                    else word = out[i];
                    st_pop<0>(B16 + (int64_t)i * p.ps + cell0 + kk, (uint16_t)(word >> (16 * (kk & 1))));
                }
            }
        }
    }
}

static bool tma_geometry(const LatticeParams& p, int G, TmaGeom& g) {
    if (p.nx % 16 != 0) return false;
    const int tile = tma_tile_cells(G);
    int TX = 0;
    for (int c : {512, 256, 128, 64, 32, 16})
        if (c <= tile && p.nx % c == 0) {
            TX = c;
            break;
        }
    if (TX == 0) return false;
    g.TX = TX;
    g.R = tile / TX;
    g.xchunks = p.nx / TX;
    g.nrows = p.ny * p.nz;
    g.ntiles = (int64_t)g.xchunks * ((g.nrows + g.R - 1) / g.R);
    g.rb = (TX + 2 * TMA_HALO) * 2;
    g.row_bytes = 19 * g.rb + TX;
    g.stage_bytes = g.R * g.row_bytes;
    return TMA_STAGES * g.stage_bytes <= tma_max_smem(G);
}

template <class S, bool FORCE, int G>
static cudaError_t launch_tma16(const void* A, void* B, const uint8_t* code, const LatticeParams& p, const TmaGeom& g,
                                cudaStream_t st) {
    const size_t smem = (size_t)TMA_STAGES * g.stage_bytes;
    auto kern = step_kernel_tma16<S, FORCE, G>;
    // launch shape per (device, shared-memory size), computed once
    struct Shape {
        int dev;
        size_t smem;
        int sms, per_sm;
    };
    static thread_local Shape cache[8];
    static thread_local int ncache = 0;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    int sms = 0, per_sm = 0;
    for (int c = 0; c < ncache; ++c)
        if (cache[c].dev == dev && cache[c].smem == smem) {
            sms = cache[c].sms;
            per_sm = cache[c].per_sm;
        }
    if (per_sm == 0) {
        // The attribute is the kernel's maximum for every later launch, so it is
        // set to the largest ring any tile geometry needs (TX = 16, R = 32),
        // never lowered to the current one.
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, tma_max_smem(G))) != cudaSuccess)
            return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, tma_threads(G), smem)) != cudaSuccess)
            return e;
        if (per_sm < 1) return cudaErrorInvalidConfiguration;
        cache[ncache % 8] = Shape{dev, smem, sms, per_sm};
        ++ncache;
    }
    int64_t grid = (int64_t)sms * per_sm;
    if (grid > g.ntiles) grid = g.ntiles;
    kern<<<(unsigned)grid, tma_threads(G), smem, st>>>((const S*)A, (S*)B, code, p, g);
    return cudaGetLastError();
}

template <class S, int G>
static cudaError_t step_tma16_t(const void* A, void* B, const uint8_t* code, const LatticeParams& p, int block,
                                cudaStream_t st) {
    TmaGeom g;
    if (!tma_geometry(p, G, g) || p.err == nullptr) return step_rows_t<S, 0>(A, B, code, p, block, st);
    const bool force = p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    return force ? launch_tma16<S, true, G>(A, B, code, p, g, st) : launch_tma16<S, false, G>(A, B, code, p, g, st);
}

template <class S, int HINT, bool MASK_FIRST, bool SR>
static cudaError_t step_rows_t(const void* A, void* B, const uint8_t* code, const LatticeParams& p, int block,
                               cudaStream_t st) {
    int bx = block > 0 ? (block / 32) * 32 : 256;
    if (bx < 32) bx = 32;
    if (bx > (MASK_FIRST ? 128 : 512)) bx = MASK_FIRST ? 128 : 512;
    // shrink the block for narrow rows (multiple of 32)
    const int need = ((p.nx + 31) / 32) * 32;
    if (bx > need) bx = need;
    const int xblocks = (p.nx + bx - 1) / bx;
    const bool force = p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    if (force)
        step_kernel_rows<S, true, HINT, MASK_FIRST, SR>
            <<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    else
        step_kernel_rows<S, false, HINT, MASK_FIRST, SR>
            <<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    return cudaGetLastError();
}

// Stochastic rounding (16-bit storage, p.sr): the one-cell kernels (1-3, and
// 16 with the mask-first bounce-back) and the packed two-cell kernels (13,
// 15, 17, 18, 19) have a stochastically rounding form; the default (0) runs 18,
// every other variant 15 (or 1 where the two-cell kernels do not apply).
template <class S>
static cudaError_t step_sr_t(int variant, const void* A, void* B, const uint8_t* code, const LatticeParams& p,
                             int block, cudaStream_t st) {
    const bool pairs_ok = (p.nx % 2) == 0;
    switch (variant) {
        case 1: return step_rows_t<S, 0, false, true>(A, B, code, p, block, st);
        case 2: return step_rows_t<S, 1, false, true>(A, B, code, p, block, st);
        case 3: return step_rows_t<S, 2, false, true>(A, B, code, p, block, st);
        case 16: return step_rows_t<S, 0, true, true>(A, B, code, p, block, st);
        case 13:
            if (pairs_ok) return step_pairs_x2_t<S, 0, 1, false, true>(A, B, code, p, block, st);
            return step_rows_t<S, 0, false, true>(A, B, code, p, block, st);
        case 17:
            if (pairs_ok) return step_pairs_x2_t<S, 0, 2, true, true>(A, B, code, p, block, st);
            return step_rows_t<S, 0, false, true>(A, B, code, p, block, st);
        case 18:
            if (pairs_ok) return step_pairs_x2_row_t<S, 0, true>(A, B, code, p, st);
            return step_rows_t<S, 0, false, true>(A, B, code, p, block, st);
        case 19:
            if (pairs_ok) return step_pairs_x2_row_t<S, 0, true, true>(A, B, code, p, st);
            return step_rows_t<S, 0, false, true>(A, B, code, p, block, st);
        case 0:
            if (pairs_ok && block == 0) return step_pairs_x2_row_t<S, 0, true>(A, B, code, p, st);
            [[fallthrough]];
        default:
            if (pairs_ok)
                return step_pairs_x2_t<S, 0, 2, false, true>(A, B, code, p, variant == 15 || block > 0 ? block : 64,
                                                             st);
            return step_rows_t<S, 0, false, true>(A, B, code, p, block > 0 ? block : 64, st);
    }
}

template <class S>
static cudaError_t step_t(int variant, const void* A, void* B, const uint8_t* code, const LatticeParams& p,
                          int block, cudaStream_t st) {
    if constexpr (sizeof(S) == 2) {
        if (p.sr) return step_sr_t<S>(variant, A, B, code, p, block, st);
    }
    // the two-cell FP32/FP64 kernels have no FP32-storage/FP64-math form
    const bool pairs_ok = (p.nx % 2) == 0 && !std::is_same<S, f32d>::value;
    switch (variant) {
        case 1: return step_rows_t<S, 0>(A, B, code, p, block, st);
        case 2: return step_rows_t<S, 1>(A, B, code, p, block, st);
        case 3: return step_rows_t<S, 2>(A, B, code, p, block, st);
        case 4:
        case 5:
            if constexpr (!std::is_same<S, f32d>::value) {
                if (pairs_ok)
                    return variant == 4 ? step_pairs_t<S, 0>(A, B, code, p, block, st)
                                        : step_pairs_t<S, 1>(A, B, code, p, block, st);
            }
            return variant == 4 ? step_rows_t<S, 0>(A, B, code, p, block, st)
                                : step_rows_t<S, 1>(A, B, code, p, block, st);
        case 6:
        case 7:
            if constexpr (ieee16<S>) {
                if (pairs_ok)
                    return variant == 6 ? step_pairs16_t<S, 0>(A, B, code, p, block, st)
                                        : step_pairs16_t<S, 1>(A, B, code, p, block, st);
            }
            return step_rows_t<S, 0>(A, B, code, p, block, st);
        case 8:
        case 9:
            if constexpr (ieee16<S>) {
                if (p.nx % 4 == 0)
                    return variant == 8 ? step_quads16_t<S, 0>(A, B, code, p, block, st)
                                        : step_quads16_t<S, 1>(A, B, code, p, block, st);
            }
            return step_rows_t<S, 0>(A, B, code, p, block, st);
        case 10:
        case 11:
        case 12:
            if constexpr (ieee16<S>)
                return variant == 10 ? step_tma16_t<S, 4>(A, B, code, p, block, st)
                       : variant == 11 ? step_tma16_t<S, 2>(A, B, code, p, block, st)
                                       : step_tma16_t<S, 1>(A, B, code, p, block, st);
            return step_rows_t<S, 0>(A, B, code, p, block, st);
        case 13:
        case 15:
            if constexpr (std::is_same<S, float>::value || sizeof(S) == 2) {
                if (pairs_ok)
                    return variant == 13 ? step_pairs_x2_t<S, 0, 1>(A, B, code, p, block, st)
                                         : step_pairs_x2_t<S, 0, 2>(A, B, code, p, block, st);
            }
            return step_rows_t<S, 0>(A, B, code, p, block, st);
        case 14:
            if constexpr (ieee16<S>) {
                if (p.nx % 4 == 0) return step_quads16_x2_t<S, 0>(A, B, code, p, block, st);
            }
            return step_rows_t<S, 0>(A, B, code, p, block, st);
        case 16: return step_rows_t<S, 0, true>(A, B, code, p, block, st);
        case 17:
            if constexpr (std::is_same<S, float>::value || sizeof(S) == 2) {
                if (pairs_ok) return step_pairs_x2_t<S, 0, 2, true>(A, B, code, p, block, st);
            }
            return step_rows_t<S, 0>(A, B, code, p, block, st);
        case 18:
        case 19:
            if constexpr (std::is_same<S, float>::value || sizeof(S) == 2) {
                if (pairs_ok)
                    return variant == 18 ? step_pairs_x2_row_t<S, 0>(A, B, code, p, st)
                                         : step_pairs_x2_row_t<S, 0, false, true>(A, B, code, p, st);
            }
            return step_rows_t<S, 0>(A, B, code, p, block, st);
        case 0:
            // measured defaults on GB300 (256^3): FP32 one cell per thread in
            // 64-thread blocks; FP64 two cells per thread; 16-bit storage two
            // cells per thread collided as a packed FP32 pair, 64 registers,
            // one block per row where the row fits (variant 18, else 15)
            if constexpr (sizeof(S) == 2) {
                if (pairs_ok) {
                    if (block > 0) return step_pairs_x2_t<S, 0, 2>(A, B, code, p, block, st);
                    return step_pairs_x2_row_t<S, 0>(A, B, code, p, st);
                }
            }
            if constexpr (ieee16<S>) {
                if (p.nx % 4 == 0) return step_quads16_x2_t<S, 0>(A, B, code, p, block > 0 ? block : 32, st);
            }
            if constexpr (sizeof(S) == 8) {
                if (pairs_ok) return step_pairs_t<S, 0>(A, B, code, p, block > 0 ? block : 128, st);
            }
            return step_rows_t<S, 0>(A, B, code, p, block > 0 ? block : 64, st);
        default: return cudaErrorInvalidValue;
    }
}

#ifdef LBGB_CHECKED
LBGB_CHECKED_UNIT(lbgb_checked_violations_step)
#endif

cudaError_t launch_step(int storage, int variant, const void* A, void* B, const uint8_t* code,
                        const LatticeParams& p, int block, cudaStream_t st) {
#ifdef LBGB_CHECKED
    const cudaError_t ce = check_window_set(A, B, p, storage, st);
    if (ce != cudaSuccess) return ce;
#endif
    LBGB_DISPATCH(storage, step_t<S>(variant, A, B, code, p, block, st));
}

}  // namespace lbgb
