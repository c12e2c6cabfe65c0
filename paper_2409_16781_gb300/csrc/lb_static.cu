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
// The reduction is the lattice's own totals kernel (lb_kernels.cu), run on
// the caller's flag field instead of the lattice's cell codes.
//
// All calls share the one array and it keeps the last call's values; each
// call overwrites every partial it reads, so nothing needs clearing, but
// two calls whose work overlaps on the GPU (different streams, or one
// stream from two threads) race on it and must be serialised by the caller.
#include <cmath>

#include "lbgb.h"
#include "lb_internal.h"

namespace lbgb {
namespace {

constexpr int STATIC_PARTS = 6;  // sum drho, sum j (3), fluid count, bad count
constexpr int STATIC_MAX_BLOCKS = LB_STATIC_MAX_BLOCKS;

__device__ __align__(256) double lb_static_partials[STATIC_MAX_BLOCKS * STATIC_PARTS + 8];

// Device address of lb_static_partials in the current device's context.
// Looked up on every call: the lookup is a host-side query (no device work),
// and a cached address would go stale if the caller reset the device or
// switched contexts, after which the kernel would write to unmapped memory.
cudaError_t scratch_for_current_device(double** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, lb_static_partials);
    if (e != cudaSuccess) return e;
    *out = static_cast<double*>(p);
    return cudaSuccess;
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
    if (plane_stride < N || storage < LB_F64 || storage > LB_E3M12S) return LB_EINVAL;
    LatticeParams p{};
    p.nx = nx;
    p.ny = ny;
    p.nz = nz;
    p.N = N;
    p.ps = plane_stride;
    p.zlo = 0;
    p.zhi = nz;
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
    double* result = scratch + STATIC_MAX_BLOCKS * STATIC_PARTS;
    cudaStream_t st = (cudaStream_t)stream;
    e = launch_totals_flags(storage, populations, flags, p, scratch, STATIC_MAX_BLOCKS, result, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, result, 5 * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return LB_ECUDA;
    if (out[4] != 0.0 || !std::isfinite(out[0])) return LB_EDIVERGED;
    return LB_OK;
}
