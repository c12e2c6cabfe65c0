// lb_halo.cu -- halo planes of a z-slab lattice (the multi-GPU domain
// decomposition that arXiv 2409.16781 names as future work in Sec. 6).
//
// A lattice split into z-slabs keeps, on each rank, its own planes plus one
// ghost plane below (z = 0) and one above (z = nz - 1).  A step pulls the
// populations with c_z = +1 into the lowest own plane from the ghost plane
// below, and those with c_z = -1 into the highest own plane from the ghost
// plane above; no other value of a ghost plane is ever read.  So after each
// step a rank sends its lowest own plane's five c_z = -1 populations to the
// rank below and its highest own plane's five c_z = +1 populations to the
// rank above, and writes what it receives into its ghost planes.  Each of
// those is a contiguous run of nx*ny values in its population plane, so a
// message is five runs back to back: 5 * nx * ny values of the storage type.
#include "lb_internal.h"

namespace lbgb {
namespace {

// The directions with c_z = +1 and c_z = -1, in library order.
struct HaloDirs {
    int up[5], dn[5];
};
constexpr HaloDirs halo_dirs() {
    HaloDirs h{};
    int nu = 0, nd = 0;
    for (int i = 0; i < Q; ++i) {
        if (D3Q19::cz(i) == 1) h.up[nu++] = i;
        if (D3Q19::cz(i) == -1) h.dn[nd++] = i;
    }
    return h;
}
__constant__ HaloDirs c_halo = halo_dirs();

// pack != 0: lo[k] <- plane dn[k] at z = 1, hi[k] <- plane up[k] at z = nz-2.
// pack == 0: plane up[k] at z = 0 <- lo[k], plane dn[k] at z = nz-1 <- hi[k].
// blockIdx.y: k + 5 * side (side 0: lo, side 1: hi).
template <class T>
__global__ void halo_kernel(T* __restrict__ A, int64_t ps, int64_t nxy, int nz, T* __restrict__ lo,
                            T* __restrict__ hi, int pack) {
    const int k = blockIdx.y % 5, side = blockIdx.y / 5;
    T* msg = (side == 0 ? lo : hi) + (int64_t)k * nxy;
    int dir, z;
    if (pack) {
        dir = side == 0 ? c_halo.dn[k] : c_halo.up[k];
        z = side == 0 ? 1 : nz - 2;
    } else {
        dir = side == 0 ? c_halo.up[k] : c_halo.dn[k];
        z = side == 0 ? 0 : nz - 1;
    }
    T* plane = A + (int64_t)dir * ps + (int64_t)z * nxy;
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nxy; c += (int64_t)gridDim.x * blockDim.x) {
        if (pack) msg[c] = plane[c];
        else plane[c] = msg[c];
    }
}

template <class T>
cudaError_t halo_t(void* A, int64_t ps, int64_t nxy, int nz, void* lo, void* hi, int pack, cudaStream_t st) {
    int64_t bx = (nxy + 255) / 256;
    if (bx > 152 * 4) bx = 152 * 4;
    if (bx < 1) bx = 1;
    halo_kernel<T><<<dim3((unsigned)bx, 10), 256, 0, st>>>((T*)A, ps, nxy, nz, (T*)lo, (T*)hi, pack);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_halo(int sbytes, void* A, int64_t ps, int nx, int ny, int nz, void* lo, void* hi, int pack,
                        cudaStream_t st) {
    const int64_t nxy = (int64_t)nx * ny;
    switch (sbytes) {
        case 2: return halo_t<uint16_t>(A, ps, nxy, nz, lo, hi, pack, st);
        case 4: return halo_t<uint32_t>(A, ps, nxy, nz, lo, hi, pack, st);
        case 8: return halo_t<uint64_t>(A, ps, nxy, nz, lo, hi, pack, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbgb
