// lb_pairs.cuh -- two x-adjacent cells per thread: loading both cells' 19
// pulled values with one aligned 2-vector per direction (the x-shifted
// directions completed by lane shuffles), and the packed-FP32 (f32x2)
// collision and store of the pair.  Shared by the single-lattice step
// kernels (lb_step.cu) and the batched step (lb_batch.cu).
//
// arXiv 2409.16781 Sec. 3.1 (fused pull: scattered read from f^pre, write
// f^post), Eq. 1-3 (collision); the boundary rules of Sec. 3.3 via
// bounce_fix.
#pragma once

#include "lb_kernels.cuh"

namespace lbgb {

template <class S> struct Vec2;
template <> struct Vec2<double> { using T = double2; };
template <> struct Vec2<float> { using T = float2; };
template <> struct Vec2<__half> { using T = __half2; };
template <> struct Vec2<__nv_bfloat16> { using T = __nv_bfloat162; };
template <> struct Vec2<e3m12> { using T = uint32_t; };  // low half: the first cell

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
template <> __device__ __forceinline__ void split2<e3m12>(const uint32_t& v, float& a, float& b) {
    const float2 f = e3m12_decode2(v);
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

template <> __device__ __forceinline__ uint32_t pack2<e3m12>(float a, float b) {
    return e3m12_encode2(a, b, e3m12_rn_add(a), e3m12_rn_add(b));
}

template <class S> __device__ __forceinline__ f32x2 to_x2(uint32_t w);  // two packed 16-bit values
template <> __device__ __forceinline__ f32x2 to_x2<__half>(uint32_t w) {
    f32x2 r;
    r.v = __half22float2(*reinterpret_cast<const __half2*>(&w));
    return r;
}
template <> __device__ __forceinline__ f32x2 to_x2<__nv_bfloat16>(uint32_t w) {
    return f32x2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
template <class S> __device__ __forceinline__ uint32_t from_x2(f32x2 d);
template <> __device__ __forceinline__ uint32_t from_x2<__half>(f32x2 d) {
    const __half2 h = __float22half2_rn(d.v);
    return *reinterpret_cast<const uint32_t*>(&h);
}
template <> __device__ __forceinline__ uint32_t from_x2<__nv_bfloat16>(f32x2 d) {
    const __nv_bfloat162 h = __float22bfloat162_rn(d.v);
    return *reinterpret_cast<const uint32_t*>(&h);
}

// Bounce-back fix-up of the cells of a packed pair whose codes say so.
template <class S, int HINT, int FORM = FORM_AB, bool MASK_FIRST = false>
__device__ __forceinline__ void bounce_fix_x2(const S* __restrict__ A, const uint8_t* __restrict__ code,
                                              const LatticeParams& p, int x0, int y, int z, int cell0, uint8_t c0,
                                              uint8_t c1, f32x2 (&d)[Q]) {
    if (!((c0 | c1) & CODE_NEAR_WALL)) return;
    float a[Q], b[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        a[i] = d[i].v.x;
        b[i] = d[i].v.y;
    }
    if (c0 & CODE_NEAR_WALL) bounce_fix<S, HINT, FORM, MASK_FIRST>(A, code, p, x0, y, z, cell0, a);
    if (c1 & CODE_NEAR_WALL) bounce_fix<S, HINT, FORM, MASK_FIRST>(A, code, p, x0 + 1, y, z, cell0 + 1, b);
#pragma unroll
    for (int i = 0; i < Q; ++i) d[i] = f32x2(a[i], b[i]);
}

// Pull, collide and store the pair of cells (x0, x0+1) of row (y, z), x0
// even, nx even (cell0 = x0 + nx (y + ny z)).  Every lane of the warp must
// call it (the x-shifts are shuffles); lanes that are not `active` pass any
// in-bounds coordinates and store nothing.  The value at x0-1 (for c_x = +1)
// comes from the previous lane's second cell and the value at x0+2 (c_x =
// -1) from the next lane's first cell when that lane holds the same row;
// otherwise (warp edge, row edge, periodic wrap) the lane loads it itself.
//
// ROW: the block is the whole row (nx / 2 threads, nx a multiple of 64 and at
// most 1024, every lane active).  The values that cross a warp edge, and the
// periodic wrap at the row's ends, then pass through shared memory after one
// block barrier instead of being loaded again by the edge lanes.
template <class S, bool FORCE, int HINT, bool MASK_FIRST = false, bool SR = false, bool ROW = false>
__device__ __forceinline__ void pair_x2_update(const S* __restrict__ A, S* __restrict__ B,
                                               const uint8_t* __restrict__ code, const LatticeParams& p, int x0,
                                               int y, int z, int cell0, int lane, bool active) {
    using V = typename Vec2<S>::T;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int nxy = nx * ny;
    const int yo[3] = {(y == ny - 1 ? 0 : y + 1) * nx, y * nx, (y == 0 ? ny - 1 : y - 1) * nx};
    const int zo[3] = {(z == nz - 1 ? 0 : z + 1) * nxy, z * nxy, (z == 0 ? nz - 1 : z - 1) * nxy};
    const bool own_prev = lane == 0 || x0 == 0;        // x0-1 not in the previous lane
    const bool own_next = lane == 31 || x0 + 2 >= nx;  // x0+2 not in the next lane
    f32x2 d[Q];
    if constexpr (ROW) {
        // every pair load first; then lane 31 of each warp publishes its
        // second cell's values of the c_x = +1 directions and lane 0 its
        // first cell's values of the c_x = -1 directions (at most 16 warps)
        __shared__ float edge[2][5][16];
        const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
        V v[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i)
            v[i] = ld_pop<HINT>(reinterpret_cast<const V*>(A + (int64_t)i * p.ps + yo[D3Q19::cy(i) + 1] +
                                                           zo[D3Q19::cz(i) + 1] + x0));
        int kp = 0, km = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float a, b;
            split2<S>(v[i], a, b);
            d[i] = f32x2(a, b);
            if (D3Q19::cx(i) == 1) {
                if (lane == 31) edge[0][kp][warp] = b;
                ++kp;
            } else if (D3Q19::cx(i) == -1) {
                if (lane == 0) edge[1][km][warp] = a;
                ++km;
            }
        }
        __syncthreads();
        const int wprev = warp == 0 ? nwarps - 1 : warp - 1;
        const int wnext = warp == nwarps - 1 ? 0 : warp + 1;
        kp = km = 0;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (D3Q19::cx(i) == 1) {  // (x0 - 1, x0) <- (previous lane's x0 - 1, own x0)
                float prev = __shfl_up_sync(0xffffffffu, d[i].v.y, 1);
                if (lane == 0) prev = edge[0][kp][wprev];
                ++kp;
                d[i] = f32x2(prev, d[i].v.x);
            } else if (D3Q19::cx(i) == -1) {  // (x0 + 1, x0 + 2) <- (own x0 + 1, next lane's x0 + 2)
                float next = __shfl_down_sync(0xffffffffu, d[i].v.x, 1);
                if (lane == 31) next = edge[1][km][wnext];
                ++km;
                d[i] = f32x2(d[i].v.y, next);
            }
        }
    } else {
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const S* rowp = A + (int64_t)i * p.ps + yo[D3Q19::cy(i) + 1] + zo[D3Q19::cz(i) + 1];
        const V v = ld_pop<HINT>(reinterpret_cast<const V*>(rowp + x0));
        float a, b;
        split2<S>(v, a, b);
        if (D3Q19::cx(i) == 0) {
            d[i] = f32x2(a, b);
        } else if (D3Q19::cx(i) == 1) {  // source x - 1
            float prev = __shfl_up_sync(0xffffffffu, b, 1);
            if (own_prev && active) prev = Storage<S>::load(ld_pop<HINT>(rowp + (x0 == 0 ? nx - 1 : x0 - 1)));
            d[i] = f32x2(prev, a);
        } else {  // source x + 1
            float next = __shfl_down_sync(0xffffffffu, a, 1);
            if (own_next && active)
                next = Storage<S>::load(ld_pop<HINT>(rowp + (x0 + 2 >= nx ? x0 + 2 - nx : x0 + 2)));
            d[i] = f32x2(b, next);
        }
    }
    }
    if (!active) return;
    const uint8_t c0 = code[cell0], c1 = code[cell0 + 1];
    bounce_fix_x2<S, HINT, FORM_AB, MASK_FIRST>(A, code, p, x0, y, z, cell0, c0, c1, d);
    relax_dev<f32x2, FORCE>(d, p);
    const bool f0 = !(c0 & CODE_TYPE), f1 = !(c1 & CODE_TYPE);
    const Rounder<S, SR> R(p.sr_seed);
    const uint32_t key = R.key(cell0);
    if (f0 && f1) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if constexpr (SR)
                st_pop<HINT>(reinterpret_cast<uint32_t*>(B + (int64_t)i * p.ps + cell0),
                             R.two(d[i].v.x, d[i].v.y, key, i));
            else
                st_pop<HINT>(reinterpret_cast<V*>(B + (int64_t)i * p.ps + cell0), pack2<S>(d[i].v.x, d[i].v.y));
        }
    } else {  // solid cells are never written
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            if (f0) st_pop<HINT>(B + (int64_t)i * p.ps + cell0, R.one(d[i].v.x, key, cell0, i));
            if (f1) st_pop<HINT>(B + (int64_t)i * p.ps + cell0 + 1, R.one(d[i].v.y, key, cell0 + 1, i));
        }
    }
}

}  // namespace lbgb
