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
// next to a wall read the 18 neighbour codes (cached) for bounce-back.
#include "lb_internal.h"
#include "lb_kernels.cuh"

namespace lbgb {

template <class S, bool FORCE, int HINT>
__global__ void __launch_bounds__(512) step_kernel_rows(const S* __restrict__ A, S* __restrict__ B,
                                                        const uint8_t* __restrict__ code, LatticeParams p,
                                                        int xblocks) {
    using M = typename Storage<S>::math;
    const int xb = blockIdx.x % xblocks;
    const int row = blockIdx.x / xblocks;
    const int x = xb * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    const int y = row % p.ny;
    const int z = row / p.ny;
    const int cell = x + p.nx * row;
    const uint8_t cc = code[cell];
    if (cc & CODE_TYPE) return;  // solid cells are never written
    M d[Q];
    pull_cell<S, HINT>(A, code, p, x, y, z, cell, cc, d);
    M drho, rho, ux, uy, uz;
    macro_dev<M>(d, p, drho, rho, ux, uy, uz);
    collide_dev<M, FORCE>(d, p, drho, rho, ux, uy, uz);
#pragma unroll
    for (int i = 0; i < Q; ++i) st_pop<HINT>(B + (int64_t)i * p.ps + cell, Storage<S>::store(d[i]));
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
template <class S> struct Vec2;
template <> struct Vec2<double> { using T = double2; };
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<__half> { using T = __half2; };
template <> struct Vec2<__nv_bfloat16> { using T = __nv_bfloat162; };

template <class S> __device__ __forceinline__ void split2(const typename Vec2<S>::T& v, typename Storage<S>::math& a,
                                                          typename Storage<S>::math& b);
template <> __device__ __forceinline__ void split2<double>(const double2& v, double& a, double& b) { a = v.x; b = v.y; }
template <> __device__ __forceinline__ void split2<float>(const float2& v, float& a, float& b) { a = v.x; b = v.y; }
template <> __device__ __forceinline__ void split2<__half>(const __half2& v, float& a, float& b) {
    const float2 f = __half22float2(v);
    a = f.x;
    b = f.y;
}
template <> __device__ __forceinline__ void split2<__nv_bfloat16>(const __nv_bfloat162& v, float& a, float& b) {
    const float2 f = __bfloat1622float2(v);
    a = f.x;
    b = f.y;
}
template <class S> __device__ __forceinline__ typename Vec2<S>::T pack2(typename Storage<S>::math a,
                                                                        typename Storage<S>::math b);
template <> __device__ __forceinline__ double2 pack2<double>(double a, double b) { return make_double2(a, b); }
template <> __device__ __forceinline__ float2 pack2<float>(float a, float b) { return make_float2(a, b); }
template <> __device__ __forceinline__ __half2 pack2<__half>(float a, float b) { return __floats2half2_rn(a, b); }
template <> __device__ __forceinline__ __nv_bfloat162 pack2<__nv_bfloat16>(float a, float b) {
    return __floats2bfloat162_rn(a, b);
}

template <class S, bool FORCE, int HINT>
__global__ void __launch_bounds__(256) step_kernel_pairs(const S* __restrict__ A, S* __restrict__ B,
                                                         const uint8_t* __restrict__ code, LatticeParams p,
                                                         int xblocks) {
    using M = typename Storage<S>::math;
    using V = typename Vec2<S>::T;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int xb = blockIdx.x % xblocks;
    const int row = blockIdx.x / xblocks;
    const int y = row % ny;
    const int z = row / ny;
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
        M drho, rho, ux, uy, uz;
        macro_dev<M>(d0, p, drho, rho, ux, uy, uz);
        collide_dev<M, FORCE>(d0, p, drho, rho, ux, uy, uz);
    }
    {
        M drho, rho, ux, uy, uz;
        macro_dev<M>(d1, p, drho, rho, ux, uy, uz);
        collide_dev<M, FORCE>(d1, p, drho, rho, ux, uy, uz);
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
    const int64_t blocks = (int64_t)xblocks * p.ny * p.nz;
    const bool force = p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    if (force)
        step_kernel_pairs<S, true, HINT><<<(unsigned)blocks, bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    else
        step_kernel_pairs<S, false, HINT><<<(unsigned)blocks, bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    return cudaGetLastError();
}

template <class S, int HINT>
static cudaError_t step_rows_t(const void* A, void* B, const uint8_t* code, const LatticeParams& p, int block,
                               cudaStream_t st) {
    int bx = block > 0 ? (block / 32) * 32 : 256;
    if (bx < 32) bx = 32;
    if (bx > 512) bx = 512;
    // shrink the block for narrow rows (multiple of 32)
    const int need = ((p.nx + 31) / 32) * 32;
    if (bx > need) bx = need;
    const int xblocks = (p.nx + bx - 1) / bx;
    const int64_t blocks = (int64_t)xblocks * p.ny * p.nz;
    const bool force = p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    if (force)
        step_kernel_rows<S, true, HINT><<<(unsigned)blocks, bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    else
        step_kernel_rows<S, false, HINT><<<(unsigned)blocks, bx, 0, st>>>((const S*)A, (S*)B, code, p, xblocks);
    return cudaGetLastError();
}

template <class S>
static cudaError_t step_t(int variant, const void* A, void* B, const uint8_t* code, const LatticeParams& p,
                          int block, cudaStream_t st) {
    const bool pairs_ok = (p.nx % 2) == 0;
    switch (variant) {
        case 1: return step_rows_t<S, 0>(A, B, code, p, block, st);
        case 2: return step_rows_t<S, 1>(A, B, code, p, block, st);
        case 3: return step_rows_t<S, 2>(A, B, code, p, block, st);
        case 4:
            return pairs_ok ? step_pairs_t<S, 0>(A, B, code, p, block, st) : step_rows_t<S, 0>(A, B, code, p, block, st);
        case 5:
            return pairs_ok ? step_pairs_t<S, 1>(A, B, code, p, block, st) : step_rows_t<S, 1>(A, B, code, p, block, st);
        case 0: return step_rows_t<S, 0>(A, B, code, p, block > 0 ? block : 128, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_step(int storage, int variant, const void* A, void* B, const uint8_t* code,
                        const LatticeParams& p, int block, cudaStream_t st) {
    LBGB_DISPATCH(storage, step_t<S>(variant, A, B, code, p, block, st));
}

}  // namespace lbgb
