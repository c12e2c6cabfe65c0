// lb_inplace.cu -- the fused D3Q19 stream-and-collide step on ONE population
// array (the in-place "AA" access pattern), for lattices created with
// lb_options.inplace = 1.
//
// Same update as lb_step.cu (arXiv 2409.16781 Eq. 1-3 with the boundary
// rules of Sec. 3.3, collision relax_dev), but the state keeps no second
// array: the paper's fused scheme (Sec. 3.1) alternates two arrays f^pre and
// f^post, which doubles the memory; here the two steps of a pair alternate
// two layouts of the same array (FORM_SWAPPED, FORM_STREAMED in
// lb_kernels.cuh) and every thread writes exactly the values it read.
// Bytes per update are the same 2*19*sizeof(pop) + 1.
//   from FORM_STREAMED: read plane i at the cell itself, write plane opp(i)
//       at the cell: every access is aligned and local;
//   from FORM_SWAPPED: read plane opp(i) at x - c_i, write plane i at
//       x + c_i: both shifted by the velocity (x-shifts are one element off
//       the warp's 128-byte segment, as in the two-array pull).
// Mapping: one thread per cell, a block covers consecutive x of one row.
#include <type_traits>

#include "lb_internal.h"
#include "lb_kernels.cuh"
#include "lb_pairs.cuh"

namespace lbgb {

// One stored value of the neighbouring lane (up: lane - 1, else lane + 1),
// and the helpers that pack two stored values into one aligned store.
template <class S>
__device__ __forceinline__ uint16_t bits16(S v) {
    static_assert(sizeof(S) == 2, "16-bit storage");
    return *reinterpret_cast<const uint16_t*>(&v);
}
template <class S>
__device__ __forceinline__ S shfl_val(S v, bool up) {
    if constexpr (sizeof(S) == 2) {
        const uint32_t w = bits16(v);
        const uint32_t r = up ? __shfl_up_sync(0xffffffffu, w, 1) : __shfl_down_sync(0xffffffffu, w, 1);
        return from_bits16<S>(r);
    } else {
        return up ? __shfl_up_sync(0xffffffffu, v, 1) : __shfl_down_sync(0xffffffffu, v, 1);
    }
}
template <class S>
__device__ __forceinline__ typename Vec2<S>::T pack_vals(S a, S b) {
    return typename Vec2<S>::T{a, b};
}

// Ar and Aw are the same array.  They come in as two pointers (neither
// restrict-qualified, so the compiler keeps every load before the stores that
// follow it) only so that the compiler does not keep the 19 load addresses
// live through the collision to reuse them for the stores: it recomputes the
// store addresses instead, which leaves more registers for more warps.
// Every slot of the array is loaded and then stored by one thread only (the
// 19 values a thread reads are the 19 slots it writes), so the two-cell
// kernel loads through the read-only path (ld_pop HINT 3).
template <class S, bool FORCE, int FORM, bool SR>
__global__ void __launch_bounds__(512) step_kernel_inplace(const S* Ar, S* Aw, const uint8_t* __restrict__ code,
                                                           LatticeParams p, int xblocks) {
    int xb, y, z;
    block_row(xblocks, p.ny, xb, y, z);
    const int row = y + p.ny * z;
    const int x = xb * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    const int cell = x + p.nx * row;
    const uint8_t cc = code[cell];
    if (cc & CODE_TYPE) return;  // solid cells hold no values of their own
    inplace_update<S, FORCE, FORM, SR>(Ar, Aw, code, p, x, y, z, cell, cc, p.sr_seed);
}

// ---------------------------------------------------------------------------
// Two x-adjacent cells per thread (nx even; FP32 or 16-bit storage), the
// pair collided in packed FP32 (f32x2), capped at 64 registers (blocks of at
// most 128 threads, 8 per SM) like the two-array variant 15.
//   from FORM_STREAMED: one aligned 2-vector load of plane i at the pair
//     and one aligned 2-vector store into plane opp(i) at the pair;
//   from FORM_SWAPPED: the pair's pulled values from plane opp(i) at
//     x - c_i (aligned 2-vector loads, x-shifts by lane shuffles, as in the
//     two-array pair kernel); each cell's result goes to plane i at x + c_i:
//     one aligned 2-vector store where c_x = 0, one store per cell where the
//     x-shift would break the alignment.
// Solid cells of a pair store nothing (as in the one-cell kernel).
//
// ROW (16-bit storage from FORM_SWAPPED, nx a multiple of 64 and at most
// 1024): one block holds a whole row, nx/2 threads.  The values that cross a
// warp edge (and the periodic wrap at the row's ends) then pass through
// shared memory, so that every lane issues one aligned pair store per
// direction and no lane stores a single value: after the block barrier no
// thread of the row still has to read, and no other block touches the row's
// slots.  A row with a solid cell takes the general stores below.
// ---------------------------------------------------------------------------
//
// OFF32 (ROW only; the launch chooses it when 19 planes of ps values fit
// 32-bit element offsets): the load and store addresses of the whole-row
// path are 32-bit offsets from the array's base, fewer instructions than the
// 64-bit row pointers.
//
// The stores of the all-fluid paths are streaming stores (.cs, evict first):
// the next step reads the array from its first plane again, long after
// these lines could still be in L2.
template <class S, bool FORCE, int FORM, bool SR, bool ROW = false, bool OFF32 = false>
__global__ void __launch_bounds__(ROW ? 512 : 128, ROW ? 2 : 8)
    step_kernel_inplace_pairs(const S* Ar, S* Aw, const uint8_t* __restrict__ code, LatticeParams p,
                              int xblocks) {
    using V = typename Vec2<S>::T;
    static_assert(!OFF32 || ROW, "32-bit offsets are a form of the whole-row path");
    // element i of plane `plane`, row offset `rowoff`, x = `x`
    auto at = [&](int plane, int rowoff, int x) -> int64_t {
        if constexpr (OFF32) return (int64_t)(uint32_t)((uint32_t)plane * (uint32_t)p.ps + (uint32_t)(rowoff + x));
        else return (int64_t)plane * p.ps + rowoff + x;
    };
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    int xb, y, z;
    block_row(xblocks, ny, xb, y, z);
    const int row = y + ny * z;
    const int x0r = 2 * (xb * blockDim.x + threadIdx.x);
    const bool active = x0r < nx;
    const int x0 = active ? x0r : 0;  // in-bounds address for idle lanes
    const int lane = threadIdx.x & 31;
    const int nxy = nx * ny;
    const int cell0 = x0 + nx * row;
    f32x2 d[Q];
    if constexpr (FORM == FORM_STREAMED) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float a, b;
            split2<S>(ld_pop<3>(reinterpret_cast<const V*>(Ar + (int64_t)i * p.ps + cell0)), a, b);
            d[i] = f32x2(a, b);
        }
    } else {
        // pull from plane opp(i) at x - c_i
        const int yo[3] = {(y == ny - 1 ? 0 : y + 1) * nx, y * nx, (y == 0 ? ny - 1 : y - 1) * nx};
        const int zo[3] = {(z == nz - 1 ? 0 : z + 1) * nxy, z * nxy, (z == 0 ? nz - 1 : z - 1) * nxy};
        const bool own_prev = lane == 0 || x0 == 0;
        const bool own_next = lane == 31 || x0 + 2 >= nx;
        // every load first, then the unpacking and the shuffles (as in the
        // two-array pair kernel)
        const int xprev = x0 == 0 ? nx - 1 : x0 - 1, xnext = x0 + 2 >= nx ? x0 + 2 - nx : x0 + 2;
        V v[Q];
        S e[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const S* rowp = Ar + (int64_t)D3Q19::opp(i) * p.ps + yo[D3Q19::cy(i) + 1] + zo[D3Q19::cz(i) + 1];
            v[i] = ld_pop<3>(reinterpret_cast<const V*>(Ar + at(D3Q19::opp(i), yo[D3Q19::cy(i) + 1] + zo[D3Q19::cz(i) + 1], x0)));
            if constexpr (!ROW) {
                if (D3Q19::cx(i) == 1 && own_prev && active) e[i] = ld_pop<3>(rowp + xprev);
                if (D3Q19::cx(i) == -1 && own_next && active) e[i] = ld_pop<3>(rowp + xnext);
            }
        }
        if constexpr (ROW) {
            // whole-row block: the values that cross a warp edge (and the
            // periodic wrap) come from the neighbouring warp through shared
            // memory -- lane 31's second cell for c_x = +1, lane 0's first
            // cell for c_x = -1 -- instead of a second load by the edge lane
            __shared__ float edge_in[2][5][16];
            const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
            int kp = 0, km = 0;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                float a, b;
                split2<S>(v[i], a, b);
                d[i] = f32x2(a, b);
                if (D3Q19::cx(i) == 1) {
                    if (lane == 31) edge_in[0][kp][warp] = b;
                    ++kp;
                } else if (D3Q19::cx(i) == -1) {
                    if (lane == 0) edge_in[1][km][warp] = a;
                    ++km;
                }
            }
            __syncthreads();
            const int wprev = warp == 0 ? nwarps - 1 : warp - 1;
            const int wnext = warp == nwarps - 1 ? 0 : warp + 1;
            kp = km = 0;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (D3Q19::cx(i) == 1) {  // source x - 1
                    float prev = __shfl_up_sync(0xffffffffu, d[i].v.y, 1);
                    if (lane == 0) prev = edge_in[0][kp][wprev];
                    ++kp;
                    d[i] = f32x2(prev, d[i].v.x);
                } else if (D3Q19::cx(i) == -1) {  // source x + 1
                    float next = __shfl_down_sync(0xffffffffu, d[i].v.x, 1);
                    if (lane == 31) next = edge_in[1][km][wnext];
                    ++km;
                    d[i] = f32x2(d[i].v.y, next);
                }
            }
        } else {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float a, b;
            split2<S>(v[i], a, b);
            if (D3Q19::cx(i) == 0) {
                d[i] = f32x2(a, b);
            } else if (D3Q19::cx(i) == 1) {  // source x - 1
                float prev = __shfl_up_sync(0xffffffffu, b, 1);
                if (own_prev && active) prev = Storage<S>::load(e[i]);
                d[i] = f32x2(prev, a);
            } else {  // source x + 1
                float next = __shfl_down_sync(0xffffffffu, a, 1);
                if (own_next && active) next = Storage<S>::load(e[i]);
                d[i] = f32x2(b, next);
            }
        }
        }
    }
    const uint8_t c0 = code[cell0], c1 = code[cell0 + 1];
    // what this lane stores: solid cells hold no values of their own, idle
    // lanes nothing
    const bool f0 = active && !(c0 & CODE_TYPE), f1 = active && !(c1 & CODE_TYPE);
    if constexpr (FORM == FORM_STREAMED) {
        if (!f0 && !f1) return;
    }
    // (from the swapped layout every lane goes on: its stores below trade
    // values with the neighbouring lanes)
    bounce_fix_x2<S, 0, FORM>(Ar, code, p, x0, y, z, cell0, c0, c1, d);
    relax_dev<f32x2, FORCE>(d, p);
    // each value is rounded by the cell that computed it (cell0 or
    // cell0 + 1), wherever it is stored
    const Rounder<S, SR> R(p.sr_seed);
    const uint32_t key = R.key(cell0);
    auto pair_word = [&](int i) {
        if constexpr (SR) return R.two(d[i].v.x, d[i].v.y, key, i);
        else return pack2<S>(d[i].v.x, d[i].v.y);
    };
    auto pair_store = [&](S* q, int i) {  // all-fluid pairs only: streaming stores
        if constexpr (SR) st_pop<1>(reinterpret_cast<uint32_t*>(q), pair_word(i));
        else st_pop<1>(reinterpret_cast<V*>(q), pair_word(i));
    };
    if constexpr (FORM == FORM_STREAMED) {
        // -> FORM_SWAPPED: P_i(x) into plane opp(i) at x (the pair test
        // once, outside the loop over directions)
        if (f0 && f1) {
#pragma unroll
            for (int i = 0; i < Q; ++i) pair_store(Aw + (int64_t)D3Q19::opp(i) * p.ps + cell0, i);
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                S* q = Aw + (int64_t)D3Q19::opp(i) * p.ps + cell0;
                if (f0) st_pop<0>(q, R.one(d[i].v.x, key, cell0, i));
                if (f1) st_pop<0>(q + 1, R.one(d[i].v.y, key, cell0 + 1, i));
            }
        }
    } else {
        // -> FORM_STREAMED: P_i(x) into plane i at x + c_i (periodic wrap).
        // A direction with c_x = +-1 moves both values of the pair one slot
        // along x, out of the pair's alignment: the aligned slots (x0, x0+1)
        // then take one value of this lane and one of the neighbouring lane
        // (a shuffle), so each lane still issues one aligned pair store; at
        // a warp or row edge a lane stores its outgoing value on its own.
        const int yt[3] = {(y == 0 ? ny - 1 : y - 1) * nx, y * nx, (y == ny - 1 ? 0 : y + 1) * nx};
        const int zt[3] = {(z == 0 ? nz - 1 : z - 1) * nxy, z * nxy, (z == nz - 1 ? 0 : z + 1) * nxy};
        const bool has_prev = lane != 0 && x0 != 0;      // the previous lane holds pair x0 - 2
        const bool has_next = lane != 31 && x0 + 2 < nx;  // the next lane holds pair x0 + 2
        const bool p1 = __shfl_up_sync(0xffffffffu, f1, 1);
        const bool n0 = __shfl_down_sync(0xffffffffu, f0, 1);
        // the two values of slots (x0, x0+1), written where each is fluid
        auto put = [&](S* q, S a, S b, bool fa, bool fb) {
            if (fa && fb) {
                if constexpr (sizeof(S) == 2)
                    st_pop<0>(reinterpret_cast<uint32_t*>(q), (uint32_t)bits16(a) | ((uint32_t)bits16(b) << 16));
                else
                    st_pop<0>(reinterpret_cast<V*>(q), pack_vals<S>(a, b));
            } else {
                if (fa) st_pop<0>(q, a);
                if (fb) st_pop<0>(q + 1, b);
            }
        };
        if constexpr (sizeof(S) == 2) {
            // each pair's two values rounded into one word (low half: cell
            // x0), which then travels between lanes as a whole
            uint32_t w[Q];
#pragma unroll
            for (int i = 0; i < Q; ++i) w[i] = R.two(d[i].v.x, d[i].v.y, key, i);
            if constexpr (ROW) {
                // lane 31's words of the c_x = +1 directions and lane 0's of
                // the c_x = -1 directions, per warp (at most 16 warps)
                __shared__ uint32_t edge[2][5][16];
                const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
                int kp = 0, km = 0;
#pragma unroll
                for (int i = 0; i < Q; ++i) {
                    if (D3Q19::cx(i) == 1) {
                        if (lane == 31) edge[0][kp][warp] = w[i];
                        ++kp;
                    } else if (D3Q19::cx(i) == -1) {
                        if (lane == 0) edge[1][km][warp] = w[i];
                        ++km;
                    }
                }
                if (__syncthreads_and(f0 && f1)) {
                    const int wprev = warp == 0 ? nwarps - 1 : warp - 1;
                    const int wnext = warp == nwarps - 1 ? 0 : warp + 1;
                    kp = km = 0;
#pragma unroll
                    for (int i = 0; i < Q; ++i) {
                        uint32_t* q = reinterpret_cast<uint32_t*>(Aw + at(i, yt[D3Q19::cy(i) + 1] + zt[D3Q19::cz(i) + 1], x0));
                        uint32_t v = w[i];
                        if (D3Q19::cx(i) == 1) {  // slots (x0, x0 + 1) <- (x0 - 1, x0)
                            uint32_t pw = __shfl_up_sync(0xffffffffu, w[i], 1);
                            if (lane == 0) pw = edge[0][kp][wprev];
                            ++kp;
                            v = __byte_perm(pw, w[i], 0x5432);
                        } else if (D3Q19::cx(i) == -1) {  // slots (x0, x0 + 1) <- (x0 + 1, x0 + 2)
                            uint32_t nw = __shfl_down_sync(0xffffffffu, w[i], 1);
                            if (lane == 31) nw = edge[1][km][wnext];
                            ++km;
                            v = __byte_perm(w[i], nw, 0x5432);
                        }
                        st_pop<1>(q, v);
                    }
                    return;
                }
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                S* rowt = Aw + (int64_t)i * p.ps + yt[D3Q19::cy(i) + 1] + zt[D3Q19::cz(i) + 1];
                const uint32_t wi = w[i];
                const S v0 = from_bits16<S>(wi & 0xffffu), v1 = from_bits16<S>(wi >> 16);
                if (D3Q19::cx(i) == 0) {
                    put(rowt + x0, v0, v1, f0, f1);
                } else if (D3Q19::cx(i) == 1) {  // x0 -> x0 + 1, x0 + 1 -> x0 + 2
                    const uint32_t pw = __shfl_up_sync(0xffffffffu, wi, 1);
                    if (has_prev) {  // slots (x0, x0 + 1) <- (previous lane's x0 - 1, x0)
                        if (p1 && f0) st_pop<0>(reinterpret_cast<uint32_t*>(rowt + x0), __byte_perm(pw, wi, 0x5432));
                        else put(rowt + x0, from_bits16<S>(pw >> 16), v0, p1, f0);
                    } else if (f0) {
                        st_pop<0>(rowt + x0 + 1, v0);
                    }
                    if (!has_next && f1) st_pop<0>(rowt + (x0 + 2 >= nx ? x0 + 2 - nx : x0 + 2), v1);
                } else {  // x0 -> x0 - 1, x0 + 1 -> x0
                    const uint32_t nw = __shfl_down_sync(0xffffffffu, wi, 1);
                    if (has_next) {  // slots (x0, x0 + 1) <- (x0 + 1, next lane's x0 + 2)
                        if (f1 && n0) st_pop<0>(reinterpret_cast<uint32_t*>(rowt + x0), __byte_perm(wi, nw, 0x5432));
                        else put(rowt + x0, v1, from_bits16<S>(nw & 0xffffu), f1, n0);
                    } else if (f1) {
                        st_pop<0>(rowt + x0, v1);
                    }
                    if (!has_prev && f0) st_pop<0>(rowt + (x0 == 0 ? nx - 1 : x0 - 1), v0);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                S* rowt = Aw + (int64_t)i * p.ps + yt[D3Q19::cy(i) + 1] + zt[D3Q19::cz(i) + 1];
                const S v0 = R.one(d[i].v.x, key, cell0, i), v1 = R.one(d[i].v.y, key, cell0 + 1, i);
                if (D3Q19::cx(i) == 0) {
                    put(rowt + x0, v0, v1, f0, f1);
                } else if (D3Q19::cx(i) == 1) {  // x0 -> x0 + 1, x0 + 1 -> x0 + 2
                    const S pv = shfl_val<S>(v1, true);  // the previous lane's x0 - 1 -> x0
                    if (has_prev) put(rowt + x0, pv, v0, p1, f0);
                    else if (f0) st_pop<0>(rowt + x0 + 1, v0);
                    if (!has_next && f1) st_pop<0>(rowt + (x0 + 2 >= nx ? x0 + 2 - nx : x0 + 2), v1);
                } else {  // x0 -> x0 - 1, x0 + 1 -> x0
                    const S nv = shfl_val<S>(v0, false);  // the next lane's x0 + 2 -> x0 + 1
                    if (has_next) put(rowt + x0, v1, nv, f1, n0);
                    else if (f1) st_pop<0>(rowt + x0, v1);
                    if (!has_prev && f0) st_pop<0>(rowt + (x0 == 0 ? nx - 1 : x0 - 1), v0);
                }
            }
        }
    }
}

template <class S, int FORM, bool SR>
static cudaError_t step_inplace_pairs_form(void* A, const uint8_t* code, const LatticeParams& p, int block,
                                           cudaStream_t st) {
    const bool force = p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    if constexpr (sizeof(S) == 2 && FORM == FORM_SWAPPED) {
        if (p.nx % 64 == 0 && p.nx <= 1024) {  // one block per row, nx/2 threads
            const dim3 g = row_grid(1, p.ny, p.nz);
            const bool off32 = (uint64_t)Q * (uint64_t)p.ps <= 0xFFFFFFFFull;
            if (force && off32)
                step_kernel_inplace_pairs<S, true, FORM, SR, true, true><<<g, p.nx / 2, 0, st>>>((const S*)A, (S*)A, code, p, 1);
            else if (force)
                step_kernel_inplace_pairs<S, true, FORM, SR, true><<<g, p.nx / 2, 0, st>>>((const S*)A, (S*)A, code, p, 1);
            else if (off32)
                step_kernel_inplace_pairs<S, false, FORM, SR, true, true><<<g, p.nx / 2, 0, st>>>((const S*)A, (S*)A, code, p, 1);
            else
                step_kernel_inplace_pairs<S, false, FORM, SR, true><<<g, p.nx / 2, 0, st>>>((const S*)A, (S*)A, code, p, 1);
            return cudaGetLastError();
        }
    }
    int bx = block > 0 ? (block / 32) * 32 : 64;  // whole warps (the shuffles need all 32 lanes)
    if (bx < 32) bx = 32;
    if (bx > 128) bx = 128;
    const int pairs = p.nx / 2;
    const int need = ((pairs + 31) / 32) * 32;
    if (bx > need) bx = need;
    const int xblocks = (pairs + bx - 1) / bx;
    if (force)
        step_kernel_inplace_pairs<S, true, FORM, SR>
            <<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)A, code, p, xblocks);
    else
        step_kernel_inplace_pairs<S, false, FORM, SR>
            <<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)A, code, p, xblocks);
    return cudaGetLastError();
}

template <class S, int FORM, bool SR>
static cudaError_t step_inplace_form(void* A, const uint8_t* code, const LatticeParams& p, int block,
                                     cudaStream_t st) {
    int bx = block > 0 ? (block / 32) * 32 : 128;
    if (bx < 32) bx = 32;
    if (bx > 512) bx = 512;
    const int need = ((p.nx + 31) / 32) * 32;  // shrink the block for narrow rows
    if (bx > need) bx = need;
    const int xblocks = (p.nx + bx - 1) / bx;
    const bool force = p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    if (force)
        step_kernel_inplace<S, true, FORM, SR><<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)A, code, p, xblocks);
    else
        step_kernel_inplace<S, false, FORM, SR><<<row_grid(xblocks, p.ny, p.nz), bx, 0, st>>>((const S*)A, (S*)A, code, p, xblocks);
    return cudaGetLastError();
}

// Variants of an in-place lattice: 2 = two cells per thread in packed FP32
// (FP32 or 16-bit storage, nx even); anything else one cell per thread.
// SR: the stochastically rounding form (16-bit storage, p.sr).
template <class S, bool SR>
static cudaError_t step_inplace_r(int variant, void* A, const uint8_t* code, const LatticeParams& p, int form,
                                  int block, cudaStream_t st) {
    if constexpr (std::is_same<S, float>::value || sizeof(S) == 2) {
        if (variant == 2 && p.nx % 2 == 0) {
            if (form == FORM_SWAPPED) return step_inplace_pairs_form<S, FORM_SWAPPED, SR>(A, code, p, block, st);
            if (form == FORM_STREAMED) return step_inplace_pairs_form<S, FORM_STREAMED, SR>(A, code, p, block, st);
            return cudaErrorInvalidValue;
        }
    }
    if (form == FORM_SWAPPED) return step_inplace_form<S, FORM_SWAPPED, SR>(A, code, p, block, st);
    if (form == FORM_STREAMED) return step_inplace_form<S, FORM_STREAMED, SR>(A, code, p, block, st);
    return cudaErrorInvalidValue;
}

template <class S>
static cudaError_t step_inplace_t(int variant, void* A, const uint8_t* code, const LatticeParams& p, int form,
                                  int block, cudaStream_t st) {
    if constexpr (sizeof(S) == 2) {
        if (p.sr) return step_inplace_r<S, true>(variant, A, code, p, form, block, st);
    }
    return step_inplace_r<S, false>(variant, A, code, p, form, block, st);
}

#ifdef LBGB_CHECKED
LBGB_CHECKED_UNIT(lbgb_checked_violations_inplace)
#endif

cudaError_t launch_step_inplace(int storage, int variant, void* A, const uint8_t* code, const LatticeParams& p,
                                int form, int block, cudaStream_t st) {
#ifdef LBGB_CHECKED
    const cudaError_t ce = check_window_set(A, A, p, storage, st);
    if (ce != cudaSuccess) return ce;
#endif
    LBGB_DISPATCH(storage, step_inplace_t<S>(variant, A, code, p, form, block, st));
}

}  // namespace lbgb
