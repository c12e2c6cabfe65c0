// lb_kernels.cu -- sm_103a kernels of liblbgb: cell classification, the
// fused D3Q19 stream-collide step, equilibrium initialisation, moments,
// FP64 totals and population import/export.
//
// Hot path (arXiv 2409.16781 Sec. 3.1 "fused approach", Eq. 1-3): one launch
// of step_kernel per time step reads array A (post-collision values of the
// previous step) with a pull gather and writes array B.  Populations are
// structure-of-arrays (Sec. 3.1), one unit-stride plane per direction, x
// fastest (Sec. 4.2 column-major default).
#include <type_traits>

#include "lb_internal.h"
#include "lb_kernels.cuh"

namespace lbgb {

// ---------------------------------------------------------------------------
// Cell classification: code = own type | NEAR_WALL if any pull source is solid.
// ---------------------------------------------------------------------------
__global__ void classify_kernel(const uint8_t* __restrict__ flags, uint8_t* __restrict__ code, int nx,
                                int ny, int nz) {
    const int64_t N = (int64_t)nx * ny * nz;
    for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < N;
         cell += (int64_t)gridDim.x * blockDim.x) {
        const int x = (int)(cell % nx);
        const int y = (int)((cell / nx) % ny);
        const int z = (int)(cell / ((int64_t)nx * ny));
        uint8_t own = flags[cell] & CODE_TYPE;
        uint8_t near = 0;
        if (own == 0) {
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                int sx = x - D3Q19::cx(i), sy = y - D3Q19::cy(i), sz = z - D3Q19::cz(i);
                sx = sx < 0 ? sx + nx : (sx >= nx ? sx - nx : sx);
                sy = sy < 0 ? sy + ny : (sy >= ny ? sy - ny : sy);
                sz = sz < 0 ? sz + nz : (sz >= nz ? sz - nz : sz);
                if (flags[sx + (int64_t)nx * (sy + (int64_t)ny * sz)] & CODE_TYPE) near = CODE_NEAR_WALL;
            }
        }
        code[cell] = own | near;
    }
}

// ---------------------------------------------------------------------------
// Equilibrium initialisation of cells [c0, c0+count): d_i = f^eq_i - w_i.
// rho/u are chunk-local (index cell - c0; u SoA with stride ustride), NULL =
// rho 1 / u 0.  Both arrays are written (the same array for the in-place
// scheme, whose state then has the swapped layout: direction i in plane
// opp(i)).
// ---------------------------------------------------------------------------
template <class S>
__global__ void init_kernel(S* A, S* B, int64_t ps, const double* __restrict__ rho,
                            const double* __restrict__ u, int64_t ustride, int64_t c0, int64_t count,
                            int swapped) {
    using M = typename Storage<S>::math;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
        const M r = rho ? (M)rho[k] : M(1);
        const M ux = u ? (M)u[k] : M(0);
        const M uy = u ? (M)u[ustride + k] : M(0);
        const M uz = u ? (M)u[2 * ustride + k] : M(0);
        const M uu15 = M(1.5) * (ux * ux + uy * uy + uz * uz);
        const M drho = r - M(1);
        const int64_t cell = c0 + k;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const M cu = D3Q19::cx(i) * ux + D3Q19::cy(i) * uy + D3Q19::cz(i) * uz;
            const M dv = (M)D3Q19::w(i) * (drho + r * (M(3) * cu + M(4.5) * cu * cu - uu15));
            const S s = Storage<S>::store(dv);
            const int plane = swapped ? D3Q19::opp(i) : i;
            A[plane * ps + cell] = s;
            B[plane * ps + cell] = s;
        }
    }
}

// ---------------------------------------------------------------------------
// Moments of cells [c0, c0+count) into chunk-local rho (count) and u (SoA,
// stride ustride).  Solid cells: 0.
// ---------------------------------------------------------------------------
template <class S, int FORM>
__global__ void moments_kernel(const S* __restrict__ A, const uint8_t* __restrict__ code, LatticeParams p,
                               double* __restrict__ rho, double* __restrict__ u, int64_t ustride, int64_t c0,
                               int64_t count) {
    using M = typename Storage<S>::math;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int cell = (int)(c0 + k);
        const uint8_t cc = code[cell];
        double r = 0, vx = 0, vy = 0, vz = 0;
        const int z = cell / (p.nx * p.ny);
        if (!(cc & CODE_TYPE) && z >= p.zlo && z < p.zhi) {
            const int x = cell % p.nx, y = (cell / p.nx) % p.ny;
            M d[Q];
            pull_cell<S, 0, FORM>(A, code, p, x, y, z, cell, cc, d);
            M drho, mr, ux, uy, uz;
            macro_dev<M>(d, p, drho, mr, ux, uy, uz);
            r = mr;
            vx = ux;
            vy = uy;
            vz = uz;
        }
        if (rho) rho[k] = r;
        if (u) {
            u[k] = vx;
            u[ustride + k] = vy;
            u[2 * ustride + k] = vz;
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 totals.  Each block walks (row, x-chunk) items of TOT_THREADS cells;
// a thread adds drho = rho - 1 and j = sum f c of its fluid cells in the
// math type for up to TOT_FOLD items, then folds them into FP64
// accumulators.  Per-block partials (sum drho, sum j, fluid count, bad
// count) are reduced warp -> block in a fixed order; a second single-block
// kernel adds the partials in a fixed order, so the result is reproducible.
//   mass = n_fluid + sum drho,  momentum = sum j + (g/2) mass
// (rho u = j + rho g/2 with the half-force shift).
// FLAGS: `code` is a plain flag field (values 0-3, no "next to a wall" bit,
// as lb_totals_static receives it), so every fluid cell checks its 18 pull
// sources for bounce-back.
// ---------------------------------------------------------------------------
constexpr int TOT_THREADS = 256;
constexpr int TOT_FOLD = 8;
constexpr int TOT_PARTS = 6;

// At most 64 registers (4 blocks of TOT_THREADS per SM): uncapped, the 19
// pulled values, the sums and the FP64 accumulators took 97 registers, two
// blocks per SM, and the reduction ran at well under half the bandwidth.
template <class S, int FORM, bool FLAGS = false>
__global__ void __launch_bounds__(TOT_THREADS, 4) totals_kernel(const S* __restrict__ A,
                                                             const uint8_t* __restrict__ code,
                                                             LatticeParams p, double* __restrict__ partials) {
    using M = typename Storage<S>::math;
    double acc[TOT_PARTS] = {0, 0, 0, 0, 0, 0};
    const int xblocks = (p.nx + TOT_THREADS - 1) / TOT_THREADS;
    const int64_t items = (int64_t)xblocks * p.ny * (p.zhi - p.zlo);
    M sd = 0, sx = 0, sy = 0, sz = 0;
    int nf = 0, nbad = 0, pending = 0;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int xb = (int)(it % xblocks);
        const int row = p.zlo * p.ny + (int)(it / xblocks);
        const int x = xb * TOT_THREADS + threadIdx.x;
        if (x < p.nx) {
            const int cell = x + p.nx * row;
            const uint8_t cc = FLAGS ? (uint8_t)(code[cell] | CODE_NEAR_WALL) : code[cell];
            if (!(cc & CODE_TYPE)) {
                M d[Q];
                pull_cell<S, 0, FORM>(A, code, p, x, row % p.ny, row / p.ny, cell, cc, d);
                M drho, jx, jy, jz;
                moment_sums<M>(d, drho, jx, jy, jz);
                sd += drho;
                sx += jx;
                sy += jy;
                sz += jz;
                nf += 1;
                bool bad = !(M(1) + drho > M(0)) || !isfinite(drho) || !isfinite(jx) || !isfinite(jy) || !isfinite(jz);
                if constexpr (std::is_same<S, e3m12>::value) {
                    // a saturated E3M12 value (its range is |d| < 1/8) counts as divergence
#pragma unroll
                    for (int i = 0; i < Q; ++i) bad |= fabsf(d[i]) >= 0x1.fffp-4f;
                }
                if (bad) nbad += 1;
            }
        }
        if (++pending == TOT_FOLD) {
            acc[0] += (double)sd;
            acc[1] += (double)sx;
            acc[2] += (double)sy;
            acc[3] += (double)sz;
            sd = sx = sy = sz = 0;
            pending = 0;
        }
    }
    acc[0] += (double)sd;
    acc[1] += (double)sx;
    acc[2] += (double)sy;
    acc[3] += (double)sz;
    acc[4] = (double)nf;
    acc[5] = (double)nbad;
#pragma unroll
    for (int k = 0; k < TOT_PARTS; ++k)
        for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], off);
    __shared__ double sm[TOT_THREADS / 32][TOT_PARTS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < TOT_PARTS; ++k) sm[warp][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < TOT_PARTS) {
        double s = 0;
        for (int wi = 0; wi < TOT_THREADS / 32; ++wi) s += sm[wi][threadIdx.x];
        partials[(int64_t)blockIdx.x * TOT_PARTS + threadIdx.x] = s;
    }
}

// out[0] = mass, out[1..3] = momentum, out[4] = bad-cell count.
__global__ void __launch_bounds__(TOT_THREADS) totals_finalize_kernel(const double* __restrict__ partials,
                                                                      int nblocks, LatticeParams p,
                                                                      double* __restrict__ out) {
    double acc[TOT_PARTS] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += TOT_THREADS)
        for (int k = 0; k < TOT_PARTS; ++k) acc[k] += partials[(int64_t)b * TOT_PARTS + k];
    __shared__ double sm[TOT_THREADS][TOT_PARTS];
    for (int k = 0; k < TOT_PARTS; ++k) sm[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int half = TOT_THREADS / 2; half > 0; half >>= 1) {
        if (threadIdx.x < half)
            for (int k = 0; k < TOT_PARTS; ++k) sm[threadIdx.x][k] += sm[threadIdx.x + half][k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double mass = sm[0][4] + sm[0][0];
        out[0] = mass;
        for (int a = 0; a < 3; ++a) out[1 + a] = sm[0][1 + a] + 0.5 * p.g[a] * mass;
        out[4] = sm[0][5];
    }
}

// ---------------------------------------------------------------------------
// Population import / export (FP64 f = w + d), cells [c0, c0+count).
// Chunk buffer layout: buf[i*count + k].  `form` is where the state keeps
// P_i(x) (FORM_AB, FORM_SWAPPED, FORM_STREAMED); in the streamed layout a
// solid cell has no values of its own and exports the rest state f = w.
// ---------------------------------------------------------------------------
template <class S>
__device__ __forceinline__ double export_pop(const S* __restrict__ A, const uint8_t* __restrict__ code,
                                             const LatticeParams& p, int form, int64_t cell, int i) {
    if (form == FORM_AB) return D3Q19::w(i) + (double)Storage<S>::load(A[i * p.ps + cell]);
    if (form == FORM_SWAPPED) return D3Q19::w(i) + (double)Storage<S>::load(A[D3Q19::opp(i) * p.ps + cell]);
    if (code[cell] & CODE_TYPE) return D3Q19::w(i);
    const int x = (int)(cell % p.nx), y = (int)((cell / p.nx) % p.ny), z = (int)(cell / ((int64_t)p.nx * p.ny));
    int tx = x + D3Q19::cx_rt(i), ty = y + D3Q19::cy_rt(i), tz = z + D3Q19::cz_rt(i);
    tx = tx < 0 ? tx + p.nx : (tx >= p.nx ? tx - p.nx : tx);
    ty = ty < 0 ? ty + p.ny : (ty >= p.ny ? ty - p.ny : ty);
    tz = tz < 0 ? tz + p.nz : (tz >= p.nz ? tz - p.nz : tz);
    const int64_t t = tx + (int64_t)p.nx * (ty + (int64_t)p.ny * tz);
    return D3Q19::w(i) + (double)Storage<S>::load(A[i * p.ps + t]);
}

template <class S>
__global__ void get_pops_kernel(const S* __restrict__ A, const uint8_t* __restrict__ code, LatticeParams p, int form,
                                int64_t c0, int64_t count, double* __restrict__ buf) {
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < Q; ++i) buf[i * count + k] = export_pop<S>(A, code, p, form, c0 + k, i);
    }
}

// Import: writes both arrays (two-array scheme) or, with `swapped`, the one
// array of the in-place scheme in the swapped layout.
template <class S>
__global__ void set_pops_kernel(S* A, S* B, int64_t ps, int64_t c0, int64_t count,
                                const double* __restrict__ buf, int swapped) {
    using M = typename Storage<S>::math;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < count;
         k += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const double dv = buf[i * count + k] - D3Q19::w(i);
            const S s = Storage<S>::store((M)dv);
            const int plane = swapped ? D3Q19::opp(i) : i;
            A[plane * ps + c0 + k] = s;
            B[plane * ps + c0 + k] = s;
        }
    }
}

template <class S>
__global__ void gather_pops_kernel(const S* __restrict__ A, const uint8_t* __restrict__ code, LatticeParams p,
                                   int form, const int64_t* __restrict__ cells, int n, double* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    const int64_t cell = cells[k];
#pragma unroll
    for (int i = 0; i < Q; ++i) out[(int64_t)k * Q + i] = export_pop<S>(A, code, p, form, cell, i);
}

// ---------------------------------------------------------------------------
// Host-side launchers
// ---------------------------------------------------------------------------
static inline int grid_for(int64_t n, int threads) {
    int64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 64) b = 152 * 64;
    return (int)b;
}

cudaError_t launch_classify(const uint8_t* flags, uint8_t* code, int nx, int ny, int nz, cudaStream_t st) {
    const int64_t N = (int64_t)nx * ny * nz;
    classify_kernel<<<grid_for(N, 256), 256, 0, st>>>(flags, code, nx, ny, nz);
    return cudaGetLastError();
}

template <class S>
static cudaError_t init_t(void* A, void* B, int64_t ps, const double* rho, const double* u, int64_t ustride,
                          int64_t c0, int64_t count, int swapped, cudaStream_t st) {
    init_kernel<S><<<grid_for(count, 256), 256, 0, st>>>((S*)A, (S*)B, ps, rho, u, ustride, c0, count, swapped);
    return cudaGetLastError();
}

cudaError_t launch_init(int storage, void* A, void* B, int64_t ps, const double* rho, const double* u,
                        int64_t ustride, int64_t c0, int64_t count, cudaStream_t st, int swapped) {
    LBGB_DISPATCH(storage, init_t<S>(A, B, ps, rho, u, ustride, c0, count, swapped, st));
}

template <class S>
static cudaError_t moments_t(const void* A, const uint8_t* code, const LatticeParams& p, double* rho, double* u,
                             int64_t ustride, int64_t c0, int64_t count, int form, cudaStream_t st) {
    const int g = grid_for(count, 256);
    const S* a = (const S*)A;
    if (form == FORM_SWAPPED)
        moments_kernel<S, FORM_SWAPPED><<<g, 256, 0, st>>>(a, code, p, rho, u, ustride, c0, count);
    else if (form == FORM_STREAMED)
        moments_kernel<S, FORM_STREAMED><<<g, 256, 0, st>>>(a, code, p, rho, u, ustride, c0, count);
    else
        moments_kernel<S, FORM_AB><<<g, 256, 0, st>>>(a, code, p, rho, u, ustride, c0, count);
    return cudaGetLastError();
}

cudaError_t launch_moments(int storage, const void* A, const uint8_t* code, const LatticeParams& p, double* rho,
                           double* u, int64_t ustride, int64_t c0, int64_t count, cudaStream_t st, int form) {
    LBGB_DISPATCH(storage, moments_t<S>(A, code, p, rho, u, ustride, c0, count, form, st));
}

int totals_blocks(int64_t N) {
    // about 4 items of TOT_THREADS cells per block, at most 152*16 blocks
    int64_t b = (N + 4 * TOT_THREADS - 1) / (4 * TOT_THREADS);
    if (b < 1) b = 1;
    if (b > 152 * 16) b = 152 * 16;
    return (int)b;
}

template <class S>
static cudaError_t totals_t(const void* A, const uint8_t* code, const LatticeParams& p, double* partials,
                            double* out5, int form, cudaStream_t st) {
    const int nb = totals_blocks(p.N);
    const S* a = (const S*)A;
    if (form == FORM_SWAPPED)
        totals_kernel<S, FORM_SWAPPED><<<nb, TOT_THREADS, 0, st>>>(a, code, p, partials);
    else if (form == FORM_STREAMED)
        totals_kernel<S, FORM_STREAMED><<<nb, TOT_THREADS, 0, st>>>(a, code, p, partials);
    else
        totals_kernel<S, FORM_AB><<<nb, TOT_THREADS, 0, st>>>(a, code, p, partials);
    totals_finalize_kernel<<<1, TOT_THREADS, 0, st>>>(partials, nb, p, out5);
    return cudaGetLastError();
}

cudaError_t launch_totals(int storage, const void* A, const uint8_t* code, const LatticeParams& p,
                          double* partials, double* out5, cudaStream_t st, int form) {
    LBGB_DISPATCH(storage, totals_t<S>(A, code, p, partials, out5, form, st));
}

template <class S>
static cudaError_t totals_flags_t(const void* A, const uint8_t* flags, const LatticeParams& p, double* partials,
                                  int max_blocks, double* out5, cudaStream_t st) {
    int nb = totals_blocks(p.N);
    if (nb > max_blocks) nb = max_blocks;
    totals_kernel<S, FORM_AB, true><<<nb, TOT_THREADS, 0, st>>>((const S*)A, flags, p, partials);
    totals_finalize_kernel<<<1, TOT_THREADS, 0, st>>>(partials, nb, p, out5);
    return cudaGetLastError();
}

cudaError_t launch_totals_flags(int storage, const void* A, const uint8_t* flags, const LatticeParams& p,
                                double* partials, int max_blocks, double* out5, cudaStream_t st) {
    if (max_blocks < 1) return cudaErrorInvalidValue;
    LBGB_DISPATCH(storage, totals_flags_t<S>(A, flags, p, partials, max_blocks, out5, st));
}

template <class S>
static cudaError_t get_pops_t(const void* A, const uint8_t* code, const LatticeParams& p, int form, int64_t c0,
                              int64_t count, double* buf, cudaStream_t st) {
    get_pops_kernel<S><<<grid_for(count, 256), 256, 0, st>>>((const S*)A, code, p, form, c0, count, buf);
    return cudaGetLastError();
}

cudaError_t launch_get_pops(int storage, const void* A, const uint8_t* code, const LatticeParams& p, int form,
                            int64_t c0, int64_t count, double* buf, cudaStream_t st) {
    LBGB_DISPATCH(storage, get_pops_t<S>(A, code, p, form, c0, count, buf, st));
}

template <class S>
static cudaError_t set_pops_t(void* A, void* B, int64_t ps, int64_t c0, int64_t count, const double* buf,
                              int swapped, cudaStream_t st) {
    set_pops_kernel<S><<<grid_for(count, 256), 256, 0, st>>>((S*)A, (S*)B, ps, c0, count, buf, swapped);
    return cudaGetLastError();
}

cudaError_t launch_set_pops(int storage, void* A, void* B, int64_t ps, int64_t c0, int64_t count,
                            const double* buf, cudaStream_t st, int swapped) {
    LBGB_DISPATCH(storage, set_pops_t<S>(A, B, ps, c0, count, buf, swapped, st));
}

template <class S>
static cudaError_t gather_t(const void* A, const uint8_t* code, const LatticeParams& p, int form,
                            const int64_t* cells, int n, double* out, cudaStream_t st) {
    gather_pops_kernel<S><<<(n + 127) / 128, 128, 0, st>>>((const S*)A, code, p, form, cells, n, out);
    return cudaGetLastError();
}

cudaError_t launch_gather_pops(int storage, const void* A, const uint8_t* code, const LatticeParams& p, int form,
                               const int64_t* cells, int n, double* out, cudaStream_t st) {
    LBGB_DISPATCH(storage, gather_t<S>(A, code, p, form, cells, n, out, st));
}

}  // namespace lbgb
