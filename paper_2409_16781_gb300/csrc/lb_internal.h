// lb_internal.h -- private declarations shared by the C-ABI layer and the
// kernel launchers of liblbgb (not installed, not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lb_common.cuh"

namespace lbgb {

cudaError_t launch_classify(const uint8_t* flags, uint8_t* code, int nx, int ny, int nz, cudaStream_t st);
cudaError_t launch_step(int storage, int variant, const void* A, void* B, const uint8_t* code,
                        const LatticeParams& p, int block, cudaStream_t st);
cudaError_t launch_init(int storage, void* A, void* B, int64_t ps, const double* rho, const double* u,
                        int64_t ustride, int64_t c0, int64_t count, cudaStream_t st);
cudaError_t launch_moments(int storage, const void* A, const uint8_t* code, const LatticeParams& p, double* rho,
                           double* u, int64_t ustride, int64_t c0, int64_t count, cudaStream_t st);
int totals_blocks(int64_t N);
cudaError_t launch_totals(int storage, const void* A, const uint8_t* code, const LatticeParams& p,
                          double* partials, double* out5, cudaStream_t st);
cudaError_t launch_get_pops(int storage, const void* A, int64_t ps, int64_t c0, int64_t count, double* buf,
                            cudaStream_t st);
cudaError_t launch_set_pops(int storage, void* A, void* B, int64_t ps, int64_t c0, int64_t count,
                            const double* buf, cudaStream_t st);
cudaError_t launch_gather_pops(int storage, const void* A, int64_t ps, const int64_t* cells, int n, double* out,
                               cudaStream_t st);

// Instantiate CALL with S = the storage type of `storage` and return it.
#define LBGB_DISPATCH(storage, CALL)                      \
    switch (storage) {                                    \
        case 0: { using S = double; return CALL; }        \
        case 1: { using S = float; return CALL; }         \
        case 2: { using S = __half; return CALL; }        \
        case 3: { using S = __nv_bfloat16; return CALL; } \
        case 4: { using S = f32d; return CALL; }          \
        default: return cudaErrorInvalidValue;            \
    }

inline int storage_bytes(int storage) {
    switch (storage) {
        case 0: return 8;
        case 1: return 4;
        case 2: return 2;
        case 3: return 2;
        case 4: return 4;
        default: return 0;
    }
}

}  // namespace lbgb
