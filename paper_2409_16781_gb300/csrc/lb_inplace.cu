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
#include "lb_internal.h"
#include "lb_kernels.cuh"

namespace lbgb {

// Ar and Aw are the same array.  They come in as two pointers (neither
// restrict-qualified, so the compiler keeps every load before the stores that
// follow it) only so that the compiler does not keep the 19 load addresses
// live through the collision to reuse them for the stores: it recomputes the
// store addresses instead, which leaves more registers for more warps.
template <class S, bool FORCE, int FORM>
__global__ void __launch_bounds__(512) step_kernel_inplace(const S* Ar, S* Aw, const uint8_t* __restrict__ code,
                                                           LatticeParams p, int xblocks) {
    const int xb = blockIdx.x % xblocks;
    const int row = blockIdx.x / xblocks;
    const int x = xb * blockDim.x + threadIdx.x;
    if (x >= p.nx) return;
    const int y = row % p.ny;
    const int z = row / p.ny;
    const int cell = x + p.nx * row;
    const uint8_t cc = code[cell];
    if (cc & CODE_TYPE) return;  // solid cells hold no values of their own
    inplace_update<S, FORCE, FORM>(Ar, Aw, code, p, x, y, z, cell, cc);
}

template <class S, int FORM>
static cudaError_t step_inplace_form(void* A, const uint8_t* code, const LatticeParams& p, int block,
                                     cudaStream_t st) {
    int bx = block > 0 ? (block / 32) * 32 : 128;
    if (bx < 32) bx = 32;
    if (bx > 512) bx = 512;
    const int need = ((p.nx + 31) / 32) * 32;  // shrink the block for narrow rows
    if (bx > need) bx = need;
    const int xblocks = (p.nx + bx - 1) / bx;
    const int64_t blocks = (int64_t)xblocks * p.ny * p.nz;
    const bool force = p.g[0] != 0.0 || p.g[1] != 0.0 || p.g[2] != 0.0;
    if (force)
        step_kernel_inplace<S, true, FORM><<<(unsigned)blocks, bx, 0, st>>>((const S*)A, (S*)A, code, p, xblocks);
    else
        step_kernel_inplace<S, false, FORM><<<(unsigned)blocks, bx, 0, st>>>((const S*)A, (S*)A, code, p, xblocks);
    return cudaGetLastError();
}

template <class S>
static cudaError_t step_inplace_t(int variant, void* A, const uint8_t* code, const LatticeParams& p, int form,
                                  int block, cudaStream_t st) {
    (void)variant;  // one kernel family so far: one cell per thread
    if (form == FORM_SWAPPED) return step_inplace_form<S, FORM_SWAPPED>(A, code, p, block, st);
    if (form == FORM_STREAMED) return step_inplace_form<S, FORM_STREAMED>(A, code, p, block, st);
    return cudaErrorInvalidValue;
}

cudaError_t launch_step_inplace(int storage, int variant, void* A, const uint8_t* code, const LatticeParams& p,
                                int form, int block, cudaStream_t st) {
    LBGB_DISPATCH(storage, step_inplace_t<S>(variant, A, code, p, form, block, st));
}

}  // namespace lbgb
