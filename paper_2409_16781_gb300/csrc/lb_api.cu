// lb_api.cu -- the C ABI of liblbgb (declared in include/lbgb.h): argument
// validation, device-memory layout of a lattice, chunked host transfers and
// the time-step loop.  All arithmetic runs in the kernels of lb_kernels.cu.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "lbgb.h"
#include "lb_internal.h"
#include "lb_kernels.cuh"

using namespace lbgb;

struct lb_lattice {
    int nx, ny, nz;
    int64_t N, ps;
    int storage, sbytes;
    double tau, omega_m, ulid[3], g[3];
    void* base;
    bool owns;
    size_t bytes;
    void* pop[2];  // pop[cur] holds the current post-collision array A (in
                   // place: pop[0] == pop[1], the one array)
    int cur;
    int inplace;   // one population array, AA access pattern
    int form;      // layout of the state: FORM_AB, or FORM_SWAPPED / FORM_STREAMED in place
    uint8_t* code;
    double* partials;
    double* tot_out;
    int* err;  // device error word set by kernels whose bounded waits gave up
    void* staging;
    size_t staging_bytes;
    cudaStream_t stream;
    int kernel, block;
    int64_t steps;
    bool walls;  // some flag is not LB_FLUID: cells next to a wall exist
    int halo_z;  // z-slab: planes 0 and nz-1 are ghost planes (lb_options.halo_z)
    int rounding;  // 16-bit storage: 0 nearest even, 1 stochastic (lb_options.rounding)
};

namespace {

thread_local std::string g_err;

int fail(int status, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int fail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return status;
}

int cuda_fail(cudaError_t e, const char* what) {
    return fail(LB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

constexpr size_t ALIGN = 256;
inline size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

struct Layout {
    int64_t N, ps;
    size_t pop_bytes, code_off, part_off, tot_off, stage_off, stage_bytes, total;
};

bool valid_dims(int nx, int ny, int nz) {
    if (nx < 1 || ny < 1 || nz < 1) return false;
    const int64_t N = (int64_t)nx * ny * nz;
    return N < (int64_t(1) << 31);
}

Layout layout_for(int nx, int ny, int nz, int storage, int inplace) {
    Layout L{};
    L.N = (int64_t)nx * ny * nz;
    L.ps = (int64_t)round_up((size_t)L.N, 128);
    L.pop_bytes = round_up((size_t)Q * L.ps * storage_bytes(storage), ALIGN);
    size_t off = (inplace ? 1 : 2) * L.pop_bytes;
    L.code_off = off;
    off += round_up((size_t)L.N, ALIGN);
    L.part_off = off;
    off += round_up((size_t)totals_blocks(L.N) * 6 * sizeof(double), ALIGN);
    L.tot_off = off;
    off += ALIGN;
    // staging for host transfers: FP64 populations of up to the whole lattice,
    // capped at 32 MiB, at least 64 KiB (one cell of populations is 152 B).
    size_t want = (size_t)L.N * Q * sizeof(double);
    if (want > (size_t(32) << 20)) want = size_t(32) << 20;
    if (want < (size_t(64) << 10)) want = size_t(64) << 10;
    L.stage_off = off;
    L.stage_bytes = round_up(want, ALIGN);
    off += L.stage_bytes;
    L.total = off;
    return L;
}

lb_options defaults() {
    lb_options o;
    memset(&o, 0, sizeof o);
    o.storage = LB_F32;
    return o;
}

LatticeParams params_of(const lb_lattice* h) {
    LatticeParams p;
    p.nx = h->nx;
    p.ny = h->ny;
    p.nz = h->nz;
    p.N = h->N;
    p.ps = h->ps;
    p.omega = 1.0 / h->tau;
    p.omega_m = h->omega_m;
    for (int a = 0; a < 3; ++a) {
        p.g[a] = h->g[a];
        p.ulid[a] = h->ulid[a];
    }
    set_farfield(p);
    p.err = h->err;
    p.zlo = h->halo_z ? 1 : 0;
    p.zhi = h->halo_z ? h->nz - 1 : h->nz;
    p.sr = h->rounding;
    p.sr_seed = sr_seed(h->steps);
    return p;
}

int64_t chunk_cells(const lb_lattice* h, size_t bytes_per_cell) {
    int64_t c = (int64_t)(h->staging_bytes / bytes_per_cell);
    return c < 1 ? 1 : c;
}

// Read (and clear) the device error word after the stream has drained.
int check_device_error(lb_lattice* h, const char* what) {
    int err = 0;
    cudaError_t e = cudaMemcpyAsync(&err, h->err, sizeof(int), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, what);
    if (err != 0) {
        const int zero = 0;
        e = cudaMemcpyAsync(h->err, &zero, sizeof(int), cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        return fail(LB_ETIMEOUT, "%s: a bounded device-side wait gave up (error word 0x%x)", what, err);
    }
    return LB_OK;
}

int create_common(lb_lattice** out, int nx, int ny, int nz, double tau, const double* u_lid, const uint8_t* flags,
                  const lb_options* opt, void* buffer, size_t bytes) {
    if (!out) return fail(LB_EINVAL, "lb_create: out is NULL");
    *out = nullptr;
    lb_options o = opt ? *opt : defaults();
    if (!valid_dims(nx, ny, nz)) return fail(LB_EINVAL, "lb_create: bad dims %d x %d x %d", nx, ny, nz);
    if (!(tau > 0.5) || !std::isfinite(tau)) return fail(LB_EINVAL, "lb_create: tau must be > 1/2 (got %g)", tau);
    if (o.storage < LB_F64 || o.storage > LB_E3M12S) return fail(LB_EINVAL, "lb_create: bad storage %d", o.storage);
    if (!(o.trt_magic >= 0.0) || !std::isfinite(o.trt_magic))
        return fail(LB_EINVAL, "lb_create: trt_magic must be >= 0 (got %g)", o.trt_magic);
    if (o.inplace != 0 && o.inplace != 1) return fail(LB_EINVAL, "lb_create: inplace must be 0 or 1 (got %d)", o.inplace);
    if (o.halo_z != 0 && o.halo_z != 1) return fail(LB_EINVAL, "lb_create: halo_z must be 0 or 1 (got %d)", o.halo_z);
    if (o.rounding != 0 && o.rounding != 1) return fail(LB_EINVAL, "lb_create: rounding must be 0 or 1 (got %d)", o.rounding);
    if (o.rounding && storage_bytes(o.storage) != 2)
        return fail(LB_EINVAL, "lb_create: stochastic rounding needs 16-bit storage (got storage %d)", o.storage);
    if (o.halo_z && (o.inplace || nz < 3))
        return fail(LB_EINVAL, "lb_create: a z-slab (halo_z) needs two population arrays and nz >= 3 (got inplace %d, "
                    "nz %d)", o.inplace, nz);
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(o.force[a])) return fail(LB_EINVAL, "lb_create: non-finite force");
        if (u_lid && !std::isfinite(u_lid[a])) return fail(LB_EINVAL, "lb_create: non-finite u_lid");
    }
    const Layout L = layout_for(nx, ny, nz, o.storage, o.inplace);
    bool walls = false;
    if (flags) {
        for (int64_t c = 0; c < L.N; ++c) {
            if (flags[c] > LB_FARFIELD) return fail(LB_EINVAL, "lb_create: flag %d at cell %lld", flags[c], (long long)c);
            walls |= flags[c] != LB_FLUID;
        }
    }
    if (buffer) {
        if (bytes < L.total) return fail(LB_ENOMEM, "lb_create_in: buffer %zu < required %zu", bytes, L.total);
        if ((uintptr_t)buffer % ALIGN) return fail(LB_EINVAL, "lb_create_in: buffer not 256-byte aligned");
    }
    lb_lattice* h = new (std::nothrow) lb_lattice();
    if (!h) return fail(LB_ENOMEM, "lb_create: host allocation failed");
    h->nx = nx;
    h->ny = ny;
    h->nz = nz;
    h->N = L.N;
    h->ps = L.ps;
    h->storage = o.storage;
    h->sbytes = storage_bytes(o.storage);
    h->tau = tau;
    h->omega_m = trt_omega_minus(tau, o.trt_magic);
    for (int a = 0; a < 3; ++a) {
        h->ulid[a] = u_lid ? u_lid[a] : 0.0;
        h->g[a] = o.force[a];
    }
    h->stream = (cudaStream_t)o.stream;
    h->kernel = o.kernel;
    h->block = o.block;
    h->bytes = L.total;
    if (buffer) {
        h->base = buffer;
        h->owns = false;
    } else {
        cudaError_t e = cudaMalloc(&h->base, L.total);
        if (e != cudaSuccess) {
            cudaGetLastError();
            delete h;
            return fail(LB_ENOMEM, "lb_create: cudaMalloc(%zu): %s", L.total, cudaGetErrorString(e));
        }
        h->owns = true;
    }
    char* b = (char*)h->base;
    h->inplace = o.inplace;
    h->halo_z = o.halo_z;
    h->rounding = o.rounding;
    h->walls = walls;
    h->form = o.inplace ? FORM_SWAPPED : FORM_AB;
    h->pop[0] = b;
    h->pop[1] = o.inplace ? b : b + L.pop_bytes;
    h->cur = 0;
    h->code = (uint8_t*)(b + L.code_off);
    h->partials = (double*)(b + L.part_off);
    h->tot_out = (double*)(b + L.tot_off);
    h->err = (int*)(b + L.tot_off + 128);
    h->staging = b + L.stage_off;
    h->staging_bytes = L.stage_bytes;
    h->steps = 0;

    // flags -> codes (through the staging area, in chunks of whole lattice)
    int rc = LB_OK;
    cudaError_t e = cudaSuccess;
    if (flags) {
        // the classifier needs the whole flag field; stage it in the B array
        // (not yet initialised) when it does not fit the staging area
        uint8_t* dflags = (size_t)L.N <= h->staging_bytes ? (uint8_t*)h->staging : (uint8_t*)h->pop[1];
        e = cudaMemcpyAsync(dflags, flags, (size_t)L.N, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = launch_classify(dflags, h->code, nx, ny, nz, h->stream);
    } else {
        e = cudaMemsetAsync(h->code, 0, (size_t)L.N, h->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(int), h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "lb_create: flags");
    if (rc == LB_OK) {
        e = launch_init(h->storage, h->pop[0], h->pop[1], h->ps, nullptr, nullptr, 0, 0, h->N, h->stream,
                        h->inplace);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) rc = cuda_fail(e, "lb_create: init");
    }
    if (rc != LB_OK) {
        if (h->owns) cudaFree(h->base);
        delete h;
        return rc;
    }
    *out = h;
    return LB_OK;
}

}  // namespace

extern "C" {

void lb_default_options(lb_options* opt) {
    if (opt) *opt = defaults();
}

int lb_velocity_set(int* c, double* w) {
    for (int i = 0; i < Q; ++i) {
        if (c) {
            c[3 * i + 0] = D3Q19::cx(i);
            c[3 * i + 1] = D3Q19::cy(i);
            c[3 * i + 2] = D3Q19::cz(i);
        }
        if (w) w[i] = D3Q19::w(i);
    }
    return Q;
}

size_t lb_bytes_required(int nx, int ny, int nz, const lb_options* opt) {
    const int storage = opt ? opt->storage : LB_F32;
    const int inplace = opt ? opt->inplace : 0;
    if (!valid_dims(nx, ny, nz) || storage < LB_F64 || storage > LB_E3M12S || (inplace != 0 && inplace != 1)) return 0;
    return layout_for(nx, ny, nz, storage, inplace).total;
}

int lb_create(lb_lattice** out, int nx, int ny, int nz, double tau, const double* u_lid, const uint8_t* flags,
              const lb_options* opt) {
    return create_common(out, nx, ny, nz, tau, u_lid, flags, opt, nullptr, 0);
}

int lb_create_in(lb_lattice** out, int nx, int ny, int nz, double tau, const double* u_lid, const uint8_t* flags,
                 const lb_options* opt, void* device_buffer, size_t bytes) {
    if (!device_buffer) return fail(LB_EINVAL, "lb_create_in: device_buffer is NULL");
    return create_common(out, nx, ny, nz, tau, u_lid, flags, opt, device_buffer, bytes);
}

// Device address of a host buffer of `bytes` bytes that the GPU can read and
// write directly -- page-locked host memory mapped into the device's address
// space (cudaHostAlloc / cudaMallocHost, or registered as mapped) -- or
// nullptr for anything else (pageable memory, or a range whose first and last
// bytes are not one contiguous mapping).  The kernels then move the fields
// between host memory and HBM themselves, in one launch over the lattice,
// instead of staging them chunk by chunk.
static void* mapped_host(const void* ptr, size_t bytes) {
    if (!ptr || bytes == 0) return nullptr;
    cudaPointerAttributes first{}, last{};
    if (cudaPointerGetAttributes(&first, ptr) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (first.type != cudaMemoryTypeHost || !first.devicePointer) return nullptr;
    const char* end = static_cast<const char*>(ptr) + (bytes - 1);
    if (cudaPointerGetAttributes(&last, end) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (last.type != cudaMemoryTypeHost || static_cast<char*>(last.devicePointer) !=
                                               static_cast<char*>(first.devicePointer) + (bytes - 1))
        return nullptr;
    return first.devicePointer;
}

int lb_init_fields(lb_lattice* h, const double* rho, const double* u) {
    if (!h) return fail(LB_EINVAL, "lb_init_fields: NULL handle");
    const size_t per_cell = (rho ? 8 : 0) + (u ? 24 : 0);
    if (per_cell == 0) {
        cudaError_t e = launch_init(h->storage, h->pop[0], h->pop[1], h->ps, nullptr, nullptr, 0, 0, h->N, h->stream,
                                    h->inplace);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (h->inplace) h->form = FORM_SWAPPED;
        return e == cudaSuccess ? LB_OK : cuda_fail(e, "lb_init_fields");
    }
    {
        // mapped host buffers: one launch reads them in place
        const double* mrho = rho ? (const double*)mapped_host(rho, (size_t)h->N * 8) : nullptr;
        const double* mu = u ? (const double*)mapped_host(u, (size_t)h->N * 24) : nullptr;
        if ((!rho || mrho) && (!u || mu)) {
            cudaError_t e = launch_init(h->storage, h->pop[h->cur], h->pop[1 - h->cur], h->ps, mrho, mu, h->N, 0,
                                        h->N, h->stream, h->inplace);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (h->inplace) h->form = FORM_SWAPPED;
            return e == cudaSuccess ? LB_OK : cuda_fail(e, "lb_init_fields");
        }
    }
    const int64_t chunk = chunk_cells(h, per_cell);
    double* st = (double*)h->staging;
    for (int64_t c0 = 0; c0 < h->N; c0 += chunk) {
        const int64_t cnt = (h->N - c0 < chunk) ? h->N - c0 : chunk;
        double* drho = rho ? st : nullptr;
        double* du = u ? st + (rho ? cnt : 0) : nullptr;
        cudaError_t e = cudaSuccess;
        if (rho) e = cudaMemcpyAsync(drho, rho + c0, cnt * 8, cudaMemcpyHostToDevice, h->stream);
        for (int a = 0; a < 3 && u && e == cudaSuccess; ++a)
            e = cudaMemcpyAsync(du + a * cnt, u + a * h->N + c0, cnt * 8, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = launch_init(h->storage, h->pop[h->cur], h->pop[1 - h->cur], h->ps, drho, du, cnt, c0, cnt, h->stream,
                            h->inplace);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (h->inplace) h->form = FORM_SWAPPED;  // cells already written are in that layout
        if (e != cudaSuccess) return cuda_fail(e, "lb_init_fields");
    }
    return LB_OK;
}

int lb_step(lb_lattice* h, int n) {
    if (!h) return fail(LB_EINVAL, "lb_step: NULL handle");
    if (n < 0) return fail(LB_EINVAL, "lb_step: n < 0");
    LatticeParams p = params_of(h);
    for (int t = 0; t < n; ++t) {
        p.sr_seed = sr_seed(h->steps);
        if (h->inplace) {
            cudaError_t e = launch_step_inplace(h->storage, h->kernel, h->pop[0], h->code, p, h->form, h->block,
                                                h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "lb_step");
            h->form = h->form == FORM_SWAPPED ? FORM_STREAMED : FORM_SWAPPED;
        } else {
            cudaError_t e = launch_step(h->storage, h->kernel, h->pop[h->cur], h->pop[1 - h->cur], h->code, p,
                                        h->block, h->stream);
            if (e != cudaSuccess) return cuda_fail(e, "lb_step");
            h->cur = 1 - h->cur;
        }
        h->steps++;
    }
    return LB_OK;
}

int lb_moments_device(lb_lattice* h, double* rho_dev, double* u_dev) {
    if (!h) return fail(LB_EINVAL, "lb_moments_device: NULL handle");
    cudaError_t e = launch_moments(h->storage, h->pop[h->cur], h->code, params_of(h), rho_dev, u_dev, h->N, 0, h->N,
                                   h->stream, h->form);
    return e == cudaSuccess ? LB_OK : cuda_fail(e, "lb_moments_device");
}

int lb_moments(lb_lattice* h, double* rho, double* u) {
    if (!h) return fail(LB_EINVAL, "lb_moments: NULL handle");
    if (!rho && !u) return LB_OK;
    const LatticeParams p = params_of(h);
    {
        // mapped host buffers: one launch writes them in place
        double* mrho = rho ? (double*)mapped_host(rho, (size_t)h->N * 8) : nullptr;
        double* mu = u ? (double*)mapped_host(u, (size_t)h->N * 24) : nullptr;
        if ((!rho || mrho) && (!u || mu)) {
            cudaError_t e = launch_moments(h->storage, h->pop[h->cur], h->code, p, mrho, mu, h->N, 0, h->N,
                                           h->stream, h->form);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            return e == cudaSuccess ? LB_OK : cuda_fail(e, "lb_moments");
        }
    }
    const int64_t chunk = chunk_cells(h, 32);
    double* st = (double*)h->staging;
    for (int64_t c0 = 0; c0 < h->N; c0 += chunk) {
        const int64_t cnt = (h->N - c0 < chunk) ? h->N - c0 : chunk;
        cudaError_t e =
            launch_moments(h->storage, h->pop[h->cur], h->code, p, st, st + cnt, cnt, c0, cnt, h->stream, h->form);
        if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho + c0, st, cnt * 8, cudaMemcpyDeviceToHost, h->stream);
        for (int a = 0; a < 3 && u && e == cudaSuccess; ++a)
            e = cudaMemcpyAsync(u + a * h->N + c0, st + (1 + a) * cnt, cnt * 8, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "lb_moments");
    }
    return LB_OK;
}

int lb_totals(lb_lattice* h, double* mass, double* mom) {
    if (!h) return fail(LB_EINVAL, "lb_totals: NULL handle");
    double out[5];
    cudaError_t e = launch_totals(h->storage, h->pop[h->cur], h->code, params_of(h), h->partials, h->tot_out,
                                  h->stream, h->form);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, h->tot_out, sizeof out, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lb_totals");
    const int rc = check_device_error(h, "lb_totals");
    if (rc != LB_OK) return rc;
    if (mass) *mass = out[0];
    if (mom)
        for (int a = 0; a < 3; ++a) mom[a] = out[1 + a];
    if (out[4] != 0.0 || !std::isfinite(out[0]))
        return fail(LB_EDIVERGED, "lb_totals: %.0f fluid cells with non-finite or non-positive density", out[4]);
    return LB_OK;
}

int lb_get_populations(lb_lattice* h, double* f) {
    if (!h || !f) return fail(LB_EINVAL, "lb_get_populations: NULL argument");
    const int64_t chunk = chunk_cells(h, Q * 8);
    double* st = (double*)h->staging;
    for (int64_t c0 = 0; c0 < h->N; c0 += chunk) {
        const int64_t cnt = (h->N - c0 < chunk) ? h->N - c0 : chunk;
        cudaError_t e = launch_get_pops(h->storage, h->pop[h->cur], h->code, params_of(h), h->form, c0, cnt, st,
                                        h->stream);
        for (int i = 0; i < Q && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(f + i * h->N + c0, st + i * cnt, cnt * 8, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "lb_get_populations");
    }
    return LB_OK;
}

int lb_set_populations(lb_lattice* h, const double* f) {
    if (!h || !f) return fail(LB_EINVAL, "lb_set_populations: NULL argument");
    const int64_t chunk = chunk_cells(h, Q * 8);
    double* st = (double*)h->staging;
    for (int64_t c0 = 0; c0 < h->N; c0 += chunk) {
        const int64_t cnt = (h->N - c0 < chunk) ? h->N - c0 : chunk;
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < Q && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(st + i * cnt, f + i * h->N + c0, cnt * 8, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = launch_set_pops(h->storage, h->pop[h->cur], h->pop[1 - h->cur], h->ps, c0, cnt, st, h->stream,
                                h->inplace);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (h->inplace) h->form = FORM_SWAPPED;  // cells already written are in that layout
        if (e != cudaSuccess) return cuda_fail(e, "lb_set_populations");
    }
    return LB_OK;
}

int lb_get_populations_at(lb_lattice* h, const int64_t* cells, int n, double* out) {
    if (!h || (n > 0 && (!cells || !out))) return fail(LB_EINVAL, "lb_get_populations_at: NULL argument");
    if (n < 0) return fail(LB_EINVAL, "lb_get_populations_at: n < 0");
    for (int k = 0; k < n; ++k)
        if (cells[k] < 0 || cells[k] >= h->N)
            return fail(LB_EINVAL, "lb_get_populations_at: cell %lld out of range", (long long)cells[k]);
    // cell indices (rounded up to ALIGN) followed by the gathered values
    int64_t chunk = (int64_t)((h->staging_bytes - ALIGN) / (8 + Q * 8));
    if (chunk < 1) chunk = 1;
    char* st = (char*)h->staging;
    for (int64_t k0 = 0; k0 < n; k0 += chunk) {
        const int cnt = (int)((n - k0 < chunk) ? n - k0 : chunk);
        int64_t* dcells = (int64_t*)st;
        double* dout = (double*)(st + round_up((size_t)cnt * 8, ALIGN));
        cudaError_t e = cudaMemcpyAsync(dcells, cells + k0, (size_t)cnt * 8, cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess)
            e = launch_gather_pops(h->storage, h->pop[h->cur], h->code, params_of(h), h->form, dcells, cnt, dout,
                                   h->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out + k0 * Q, dout, (size_t)cnt * Q * 8, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        if (e != cudaSuccess) return cuda_fail(e, "lb_get_populations_at");
    }
    return LB_OK;
}

// Checkpoint: a 64-byte header, then the stored values of the current
// population array verbatim, plane by plane (19 planes of N values).
struct CheckpointHeader {
    char magic[8];
    int32_t nx, ny, nz, storage, inplace, form;
    int64_t steps;
    int32_t sbytes, reserved[5];
};
static_assert(sizeof(CheckpointHeader) == 64, "checkpoint header layout");

size_t lb_checkpoint_bytes(lb_lattice* h) {
    if (!h) return 0;
    return sizeof(CheckpointHeader) + (size_t)Q * h->N * h->sbytes;
}

int lb_checkpoint_save(lb_lattice* h, void* host, size_t bytes) {
    if (!h || !host) return fail(LB_EINVAL, "lb_checkpoint_save: NULL argument");
    if (bytes < lb_checkpoint_bytes(h)) return fail(LB_EINVAL, "lb_checkpoint_save: buffer too small");
    CheckpointHeader hd;
    memset(&hd, 0, sizeof hd);
    memcpy(hd.magic, "LBGBCKP1", 8);
    hd.nx = h->nx;
    hd.ny = h->ny;
    hd.nz = h->nz;
    hd.storage = h->storage;
    hd.inplace = h->inplace;
    hd.form = h->form;
    hd.steps = h->steps;
    hd.sbytes = h->sbytes;
    memcpy(host, &hd, sizeof hd);
    const size_t row = (size_t)h->N * h->sbytes;
    cudaError_t e = cudaMemcpy2DAsync((char*)host + sizeof hd, row, h->pop[h->cur], (size_t)h->ps * h->sbytes, row, Q,
                                      cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    return e == cudaSuccess ? LB_OK : cuda_fail(e, "lb_checkpoint_save");
}

int lb_checkpoint_load(lb_lattice* h, const void* host, size_t bytes) {
    if (!h || !host) return fail(LB_EINVAL, "lb_checkpoint_load: NULL argument");
    if (bytes < lb_checkpoint_bytes(h)) return fail(LB_EINVAL, "lb_checkpoint_load: buffer too small");
    CheckpointHeader hd;
    memcpy(&hd, host, sizeof hd);
    if (memcmp(hd.magic, "LBGBCKP1", 8) != 0) return fail(LB_EINVAL, "lb_checkpoint_load: not a checkpoint");
    if (hd.nx != h->nx || hd.ny != h->ny || hd.nz != h->nz || hd.storage != h->storage || hd.inplace != h->inplace ||
        hd.sbytes != h->sbytes)
        return fail(LB_EINVAL, "lb_checkpoint_load: checkpoint of a %d x %d x %d lattice (storage %d, inplace %d) "
                    "does not fit this one", hd.nx, hd.ny, hd.nz, hd.storage, hd.inplace);
    if (h->inplace && hd.form != FORM_SWAPPED && hd.form != FORM_STREAMED)
        return fail(LB_EINVAL, "lb_checkpoint_load: bad layout");
    const size_t row = (size_t)h->N * h->sbytes;
    cudaError_t e = cudaMemcpy2DAsync(h->pop[h->cur], (size_t)h->ps * h->sbytes, (const char*)host + sizeof hd, row,
                                      row, Q, cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lb_checkpoint_load");
    if (h->inplace) h->form = hd.form;
    h->steps = hd.steps;
    return LB_OK;
}

int lb_set_kernel(lb_lattice* h, int variant, int block) {
    if (!h) return fail(LB_EINVAL, "lb_set_kernel: NULL handle");
    if (variant < 0 || variant > 19 || block < 0 || block > 1024)
        return fail(LB_EINVAL, "lb_set_kernel: bad variant %d / block %d", variant, block);
    h->kernel = variant;
    h->block = block;
    return LB_OK;
}

// Autotuning an in-place lattice: its steps rewrite the one array, so the
// populations are copied to host memory first and copied back (with the
// layout) after the timed steps.
static int autotune_inplace(lb_lattice* h, int reps, int* variant, int* block, float* ms_per_step) {
    const size_t bytes = (size_t)Q * h->ps * h->sbytes;
    char* snap = new (std::nothrow) char[bytes];
    if (!snap) return fail(LB_ENOMEM, "lb_autotune: no host memory for the %zu-byte snapshot", bytes);
    const int form0 = h->form;
    cudaError_t e = cudaMemcpyAsync(snap, h->pop[0], bytes, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const LatticeParams p = params_of(h);
    struct Cand {
        int v, b;
    };
    Cand cands[8];
    int nc = 0;
    for (int b : {32, 64, 128, 256, 512}) cands[nc++] = {1, b};
    if (h->nx % 2 == 0 && (h->sbytes == 2 || h->storage == LB_F32))
        for (int b : {32, 64, 128}) cands[nc++] = {2, b};
    int best = -1;
    float best_ms = 0.f;
    int form = h->form;
    auto one = [&](const Cand& c) {
        cudaError_t r = launch_step_inplace(h->storage, c.v, h->pop[0], h->code, p, form, c.b, h->stream);
        form = form == FORM_SWAPPED ? FORM_STREAMED : FORM_SWAPPED;
        return r;
    };
    for (int c = 0; c < nc && e == cudaSuccess; ++c) {
        e = one(cands[c]);
        if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r) e = one(cands[c]);
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (best < 0 || ms < best_ms)) {
            best = c;
            best_ms = ms;
        }
    }
    // restore the state whatever happened above
    cudaError_t er = cudaMemcpyAsync(h->pop[0], snap, bytes, cudaMemcpyHostToDevice, h->stream);
    if (er == cudaSuccess) er = cudaStreamSynchronize(h->stream);
    h->form = form0;
    delete[] snap;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "lb_autotune");
    if (er != cudaSuccess) return cuda_fail(er, "lb_autotune: restore");
    h->kernel = cands[best].v;
    h->block = cands[best].b;
    if (variant) *variant = h->kernel;
    if (block) *block = h->block;
    if (ms_per_step) *ms_per_step = best_ms / reps;
    return LB_OK;
}

int lb_autotune(lb_lattice* h, int reps, int* variant, int* block, float* ms_per_step) {
    if (!h) return fail(LB_EINVAL, "lb_autotune: NULL handle");
    if (reps < 1) reps = 1;
    struct Cand {
        int v, b;
    };
    Cand cands[32];
    int nc = 0;
    auto add = [&](int v, int b) {
        if (nc < 32) cands[nc++] = {v, b};
    };
    const bool sixteen = h->sbytes == 2;
    // stochastic rounding, and the E3M12 form: only the variants that have
    // that form (the others would run variant 15 or 1)
    const bool all = !h->rounding && h->storage != LB_E3M12S;
    if (h->inplace) return autotune_inplace(h, reps, variant, block, ms_per_step);
    for (int b : {32, 64, 128, 256}) add(1, b);
    if (h->nx % 2 == 0 && all) {
        for (int b : {64, 128}) add(sixteen ? 6 : 4, b);
    }
    if (sixteen && h->nx % 4 == 0 && all) {
        for (int b : {32, 64, 128}) add(8, b);
        for (int b : {32, 64, 128}) add(14, b);
    }
    if ((sixteen || h->storage == LB_F32) && h->nx % 2 == 0) {
        for (int b : {32, 64, 128}) add(13, b);
        for (int b : {64, 128}) add(15, b);
        if (h->nx % 64 == 0 && h->nx <= 1024) add(18, 0);
        if (h->walls) add(17, 64);
        if (h->walls && h->nx % 64 == 0 && h->nx <= 1024) add(19, 0);
    }
    if (h->walls) {
        for (int b : {64, 128}) add(16, b);
    }
    // (the TMA pipeline variants 10-12 are not tried: slower than the
    // register kernels on every lattice measured on GB300)
    const LatticeParams p = params_of(h);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return cuda_fail(cudaGetLastError(), "lb_autotune: event");
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return cuda_fail(cudaGetLastError(), "lb_autotune: event");
    }
    int best = -1;
    float best_ms = 0.f;
    cudaError_t e = cudaSuccess;
    const void* A = h->pop[h->cur];
    void* B = h->pop[1 - h->cur];
    for (int c = 0; c < nc && e == cudaSuccess; ++c) {
        e = launch_step(h->storage, cands[c].v, A, B, h->code, p, cands[c].b, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
        for (int r = 0; r < reps && e == cudaSuccess; ++r)
            e = launch_step(h->storage, cands[c].v, A, B, h->code, p, cands[c].b, h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e == cudaSuccess && (best < 0 || ms < best_ms)) {
            best = c;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return cuda_fail(e, "lb_autotune");
    h->kernel = cands[best].v;
    h->block = cands[best].b;
    if (variant) *variant = h->kernel;
    if (block) *block = h->block;
    if (ms_per_step) *ms_per_step = best_ms / reps;
    return LB_OK;
}

size_t lb_halo_bytes(lb_lattice* h) {
    if (!h || !h->halo_z) return 0;
    return (size_t)5 * h->nx * h->ny * h->sbytes;
}

int lb_halo_pack(lb_lattice* h, void* send_lo, void* send_hi) {
    if (!h || !send_lo || !send_hi) return fail(LB_EINVAL, "lb_halo_pack: NULL argument");
    if (!h->halo_z) return fail(LB_EINVAL, "lb_halo_pack: the lattice has no ghost planes (lb_options.halo_z)");
    cudaError_t e = launch_halo(h->sbytes, h->pop[h->cur], h->ps, h->nx, h->ny, h->nz, send_lo, send_hi, 1, h->stream);
    return e == cudaSuccess ? LB_OK : cuda_fail(e, "lb_halo_pack");
}

int lb_halo_unpack(lb_lattice* h, const void* recv_lo, const void* recv_hi) {
    if (!h || !recv_lo || !recv_hi) return fail(LB_EINVAL, "lb_halo_unpack: NULL argument");
    if (!h->halo_z) return fail(LB_EINVAL, "lb_halo_unpack: the lattice has no ghost planes (lb_options.halo_z)");
    cudaError_t e = launch_halo(h->sbytes, h->pop[h->cur], h->ps, h->nx, h->ny, h->nz, const_cast<void*>(recv_lo),
                                const_cast<void*>(recv_hi), 0, h->stream);
    return e == cudaSuccess ? LB_OK : cuda_fail(e, "lb_halo_unpack");
}

int lb_sync(lb_lattice* h) {
    if (!h) return fail(LB_EINVAL, "lb_sync: NULL handle");
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_fail(e, "lb_sync");
    return check_device_error(h, "lb_sync");
}

int lb_query(lb_lattice* h, int* dims, int* storage, int64_t* steps) {
    if (!h) return fail(LB_EINVAL, "lb_query: NULL handle");
    if (dims) {
        dims[0] = h->nx;
        dims[1] = h->ny;
        dims[2] = h->nz;
    }
    if (storage) *storage = h->storage;
    if (steps) *steps = h->steps;
    return LB_OK;
}

int lb_destroy(lb_lattice* h) {
    if (!h) return LB_OK;
    int rc = LB_OK;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_fail(e, "lb_destroy: sync");
    if (h->owns) {
        e = cudaFree(h->base);
        if (e != cudaSuccess && rc == LB_OK) rc = cuda_fail(e, "lb_destroy: cudaFree");
    }
    delete h;
    return rc;
}

const char* lb_status_string(int status) {
    switch (status) {
        case LB_OK: return "ok";
        case LB_EINVAL: return "invalid argument";
        case LB_ENOMEM: return "out of device memory";
        case LB_ECUDA: return "CUDA error";
        case LB_EDIVERGED: return "simulation diverged";
        case LB_ETIMEOUT: return "device wait timed out";
        case LB_EBUSY: return "resource busy";
        default: return "unknown status";
    }
}

const char* lb_last_error(void) { return g_err.c_str(); }

}  // extern "C"
