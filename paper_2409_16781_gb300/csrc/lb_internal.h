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
                        int64_t ustride, int64_t c0, int64_t count, cudaStream_t st, int swapped = 0);
// `form` (FORM_AB, FORM_SWAPPED, FORM_STREAMED of lb_kernels.cuh): where
// the state keeps its post-collision values.
cudaError_t launch_moments(int storage, const void* A, const uint8_t* code, const LatticeParams& p, double* rho,
                           double* u, int64_t ustride, int64_t c0, int64_t count, cudaStream_t st, int form = 0);
int totals_blocks(int64_t N);
cudaError_t launch_totals(int storage, const void* A, const uint8_t* code, const LatticeParams& p,
                          double* partials, double* out5, cudaStream_t st, int form = 0);
// The same totals from a plain flag field (no cell codes) over populations
// in the two-array layout, with at most max_blocks partial sums (6 doubles
// each) in `partials`: every fluid cell checks its pull sources.
cudaError_t launch_totals_flags(int storage, const void* A, const uint8_t* flags, const LatticeParams& p,
                                double* partials, int max_blocks, double* out5, cudaStream_t st);
cudaError_t launch_get_pops(int storage, const void* A, const uint8_t* code, const LatticeParams& p, int form,
                            int64_t c0, int64_t count, double* buf, cudaStream_t st);
cudaError_t launch_set_pops(int storage, void* A, void* B, int64_t ps, int64_t c0, int64_t count,
                            const double* buf, cudaStream_t st, int swapped = 0);
cudaError_t launch_gather_pops(int storage, const void* A, const uint8_t* code, const LatticeParams& p, int form,
                               const int64_t* cells, int n, double* out, cudaStream_t st);
// In-place (AA) step: from the state in layout `form` (FORM_SWAPPED or
// FORM_STREAMED) to the other layout, one array.
cudaError_t launch_step_inplace(int storage, int variant, void* A, const uint8_t* code, const LatticeParams& p,
                                int form, int block, cudaStream_t st);

// Halo planes of a z-slab (lb_halo.cu): pack != 0 copies the lowest own
// plane's c_z = -1 populations (z = 1) to lo and the highest own plane's
// c_z = +1 populations (z = nz - 2) to hi; pack == 0 copies lo into the
// c_z = +1 populations of the ghost plane z = 0 and hi into the c_z = -1
// populations of the ghost plane z = nz - 1.  lo and hi hold 5 * nx * ny
// values of sbytes bytes each.
cudaError_t launch_halo(int sbytes, void* A, int64_t ps, int nx, int ny, int nz, void* lo, void* hi, int pack,
                        cudaStream_t st);

// Instantiate CALL with S = the storage type of `storage` and return it.
#ifdef LBGB_CHECKED
// Bounds-checked build: each launching translation unit sets its own
// windows (see CheckWindow in lb_kernels.cuh) before every step launch and
// reports the accesses that fell outside them.
#define LBGB_CHECKED_UNIT(NAME)                                                                          \
    static cudaError_t check_window_set(const void* A, const void* B, const LatticeParams& p, int storage, \
                                        cudaStream_t st) {                                             \
        CheckWindow w;                                                                                 \
        const uintptr_t plane = (uintptr_t)Q * (uintptr_t)p.ps * (uintptr_t)storage_bytes(storage);    \
        w.rlo = reinterpret_cast<uintptr_t>(A);                                                        \
        w.rhi = w.rlo + plane;                                                                         \
        w.wlo = reinterpret_cast<uintptr_t>(B);                                                        \
        w.whi = w.wlo + plane;                                                                         \
        w.on = 1;                                                                                      \
        return cudaMemcpyToSymbolAsync(g_check, &w, sizeof w, 0, cudaMemcpyHostToDevice, st);         \
    }                                                                                                  \
    extern "C" unsigned long long NAME(int reset, unsigned long long* checks) {                        \
        unsigned long long v = 0, c = 0;                                                               \
        if (cudaDeviceSynchronize() != cudaSuccess) return ~0ull;                                      \
        if (cudaMemcpyFromSymbol(&v, g_violations, sizeof v) != cudaSuccess) return ~0ull;             \
        if (cudaMemcpyFromSymbol(&c, g_checks, sizeof c) != cudaSuccess) return ~0ull;                 \
        if (checks) *checks = c;                                                                       \
        if (reset) {                                                                                   \
            const unsigned long long z = 0;                                                            \
            if (cudaMemcpyToSymbol(g_violations, &z, sizeof z) != cudaSuccess) return ~0ull;           \
            if (cudaMemcpyToSymbol(g_checks, &z, sizeof z) != cudaSuccess) return ~0ull;               \
        }                                                                                              \
        return v;                                                                                      \
    }
#endif

#define LBGB_DISPATCH(storage, CALL)                      \
    switch (storage) {                                    \
        case 0: { using S = double; return CALL; }        \
        case 1: { using S = float; return CALL; }         \
        case 2: { using S = __half; return CALL; }        \
        case 3: { using S = __nv_bfloat16; return CALL; } \
        case 4: { using S = f32d; return CALL; }          \
        case 5: { using S = e3m12; return CALL; }         \
        default: return cudaErrorInvalidValue;            \
    }

// Rate of the odd part of the populations.  magic = 0: BGK (omega_m =
// 1/tau).  magic > 0: two-relaxation-time collision with the parameter
// Lambda = (tau - 1/2)(1/omega_m - 1/2) = magic held fixed, so that wall
// positions and the steady solution depend on Lambda only (Ginzburg's
// TRT; Lambda = 3/16 puts halfway bounce-back walls exactly halfway for the
// Poiseuille profile).
inline double trt_omega_minus(double tau, double magic) {
    if (magic == 0.0) return 1.0 / tau;
    return 1.0 / (magic / (tau - 0.5) + 0.5);
}

inline int storage_bytes(int storage) {
    switch (storage) {
        case 0: return 8;
        case 1: return 4;
        case 2: return 2;
        case 3: return 2;
        case 4: return 4;
        case 5: return 2;
        default: return 0;
    }
}

}  // namespace lbgb
