// lb_static.cu -- FP64 mass/momentum totals that allocate nothing.
//
// Some callers cannot call cudaMalloc at all: code that runs inside another
// framework's memory pool or a fixed device-memory budget, real-time loops
// where an allocation may block or fail at the worst moment, or callers
// that hold the populations in their own buffers and have no lattice
// object.  lb_totals_static serves them: the caller passes the population
// array, the flag field and the output, and the per-block partial sums of
// the reduction go to a fixed array in this file's static device memory.
//
// Scratch: lb_static_partials below, LB_STATIC_MAX_BLOCKS * 6 + 8 doubles
// (about 58 KB), placed in every GPU that loads the library and kept until
// the process exits.  The kernel never launches more blocks than the array
// holds (it strides over the lattice), so every lattice the library accepts
// (fewer than 2^31 cells) fits; larger sizes are rejected.
//
// All calls share the one array and it keeps the last call's values; each
// call overwrites every partial it reads, so nothing needs clearing, but
// two calls whose work overlaps on the GPU (different streams, or one
// stream from two threads) race on it and must be serialised by the caller.
#include <cmath>
#include <mutex>

#include "lbgb.h"
#include "lb_internal.h"
#include "lb_kernels.cuh"

namespace lbgb {
namespace {

constexpr int STATIC_THREADS = 256;
constexpr int STATIC_PARTS = 6;    // sum drho, sum j (3), fluid count, bad count
constexpr int STATIC_FOLD = 8;     // cells per thread summed in the math type before FP64
constexpr int STATIC_MAX_BLOCKS = LB_STATIC_MAX_BLOCKS;

__device__ __align__(256) double lb_static_partials[STATIC_MAX_BLOCKS * STATIC_PARTS + 8];

// Device address of lb_static_partials, looked up once per device.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch[kMaxDevices] = {nullptr};

cudaError_t scratch_for_current_device(double** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, lb_static_partials);
        if (e != cudaSuccess) return e;
        g_scratch[dev] = static_cast<double*>(p);
    }
    *out = g_scratch[dev];
    return cudaSuccess;
}

// Same sums as the lattice's totals kernel, from the caller's flag field:
// the flags carry no "next to a wall" bit, so every fluid cell checks its
// 18 pull sources for bounce-back.
template <class S>
__global__ void __launch_bounds__(STATIC_THREADS) totals_static_kernel(const S* __restrict__ A,
                                                                       const uint8_t* __restrict__ flags,
                                                                       LatticeParams p,
                                                                       double* __restrict__ partials) {
    using M = typename Storage<S>::math;
    double acc[STATIC_PARTS] = {0, 0, 0, 0, 0, 0};
    const int xblocks = (p.nx + STATIC_THREADS - 1) / STATIC_THREADS;
    const int64_t items = (int64_t)xblocks * p.ny * p.nz;
    M sd = 0, sx = 0, sy = 0, sz = 0;
    int nf = 0, nbad = 0, pending = 0;
    for (int64_t it = blockIdx.x; it < items; it += gridDim.x) {
        const int xb = (int)(it % xblocks);
        const int row = (int)(it / xblocks);
        const int x = xb * STATIC_THREADS + threadIdx.x;
        if (x < p.nx) {
            const int cell = x + p.nx * row;
            if (!(flags[cell] & CODE_TYPE)) {
                M d[Q];
                pull_cell<S>(A, flags, p, x, row % p.ny, row / p.ny, cell, CODE_NEAR_WALL, d);
                M drho, jx, jy, jz;
                moment_sums<M>(d, drho, jx, jy, jz);
                sd += drho;
                sx += jx;
                sy += jy;
                sz += jz;
                nf += 1;
                if (!(M(1) + drho > M(0)) || !isfinite(drho) || !isfinite(jx) || !isfinite(jy) || !isfinite(jz))
                    nbad += 1;
            }
        }
        if (++pending == STATIC_FOLD) {
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
    for (int k = 0; k < STATIC_PARTS; ++k)
        for (int off = 16; off > 0; off >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], off);
    __shared__ double sm[STATIC_THREADS / 32][STATIC_PARTS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < STATIC_PARTS; ++k) sm[warp][k] = acc[k];
    __syncthreads();
    if (threadIdx.x < STATIC_PARTS) {
        double s = 0;
        for (int wi = 0; wi < STATIC_THREADS / 32; ++wi) s += sm[wi][threadIdx.x];
        partials[(int64_t)blockIdx.x * STATIC_PARTS + threadIdx.x] = s;
    }
}

// One block adds the partials in a fixed order; result after the partials:
// mass, momentum (3), bad-cell count.
__global__ void __launch_bounds__(STATIC_THREADS) totals_static_finalize(double* __restrict__ partials,
                                                                         int nblocks, LatticeParams p) {
    double acc[STATIC_PARTS] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += STATIC_THREADS)
        for (int k = 0; k < STATIC_PARTS; ++k) acc[k] += partials[(int64_t)b * STATIC_PARTS + k];
    __shared__ double sm[STATIC_THREADS][STATIC_PARTS];
    for (int k = 0; k < STATIC_PARTS; ++k) sm[threadIdx.x][k] = acc[k];
    __syncthreads();
    for (int half = STATIC_THREADS / 2; half > 0; half >>= 1) {
        if (threadIdx.x < half)
            for (int k = 0; k < STATIC_PARTS; ++k) sm[threadIdx.x][k] += sm[threadIdx.x + half][k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        double* out = partials + STATIC_MAX_BLOCKS * STATIC_PARTS;
        const double mass = sm[0][4] + sm[0][0];
        out[0] = mass;
        for (int a = 0; a < 3; ++a) out[1 + a] = sm[0][1 + a] + 0.5 * p.g[a] * mass;
        out[4] = sm[0][5];
    }
}

template <class S>
cudaError_t launch_totals_static(const void* A, const uint8_t* flags, const LatticeParams& p, double* scratch,
                                 cudaStream_t st) {
    const int xblocks = (p.nx + STATIC_THREADS - 1) / STATIC_THREADS;
    const int64_t items = (int64_t)xblocks * p.ny * p.nz;
    int64_t nb = (items + 3) / 4;
    if (nb < 1) nb = 1;
    if (nb > STATIC_MAX_BLOCKS) nb = STATIC_MAX_BLOCKS;
    totals_static_kernel<S><<<(int)nb, STATIC_THREADS, 0, st>>>((const S*)A, flags, p, scratch);
    totals_static_finalize<<<1, STATIC_THREADS, 0, st>>>(scratch, (int)nb, p);
    return cudaGetLastError();
}

cudaError_t dispatch_totals_static(int storage, const void* A, const uint8_t* flags, const LatticeParams& p,
                                   double* scratch, cudaStream_t st) {
    LBGB_DISPATCH(storage, launch_totals_static<S>(A, flags, p, scratch, st));
}

}  // namespace
}  // namespace lbgb

extern "C" int lb_totals_static(const void* populations, int64_t plane_stride, const uint8_t* flags, int nx, int ny,
                                int nz, int storage, const double* force, const double* u_lid, void* stream,
                                double* out) {
    using namespace lbgb;
    if (!populations || !flags || !out) return LB_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1) return LB_EINVAL;
    const int64_t N = (int64_t)nx * ny * nz;
    if (N >= (int64_t(1) << 31)) return LB_EINVAL;  // beyond the library's cell limit
    if (plane_stride < N || storage < LB_F64 || storage > LB_F32D) return LB_EINVAL;
    LatticeParams p;
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    p.N = N;
    p.ps = plane_stride;
    p.omega = 1.0;  // not used by the totals
    p.omega_m = 1.0;
    p.err = nullptr;
    for (int a = 0; a < 3; ++a) {
        p.g[a] = force ? force[a] : 0.0;
        p.ulid[a] = u_lid ? u_lid[a] : 0.0;
        if (!std::isfinite(p.g[a]) || !std::isfinite(p.ulid[a])) return LB_EINVAL;
    }
    set_farfield(p);
    double* scratch = nullptr;
    cudaError_t e = scratch_for_current_device(&scratch);
    if (e != cudaSuccess) return LB_ECUDA;
    cudaStream_t st = (cudaStream_t)stream;
    e = dispatch_totals_static(storage, populations, flags, p, scratch, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(out, scratch + STATIC_MAX_BLOCKS * STATIC_PARTS, 5 * sizeof(double),
                            cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LB_ECUDA;
    if (out[4] != 0.0 || !std::isfinite(out[0])) return LB_EDIVERGED;
    return LB_OK;
}
