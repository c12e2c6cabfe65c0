// lb_batch.cu -- many independent lattices advanced by shared launches.
//
// Each lattice (a "slot") keeps its populations resident in one device
// pool; a batched time step is one persistent, grid-stride kernel per
// storage type that walks a work list of 128-cell items over every active
// slot of that type (the fused pull-collide update of arXiv 2409.16781
// Sec. 3.1 / Eq. 1-3, one thread per cell), followed by a one-block kernel
// that flips each slot's A/B parity and counts its remaining steps down.
// Slot membership, parities and step counters live in device memory, so a
// captured CUDA graph of several batched steps stays valid while lattices
// are admitted and retired between replays.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <new>
#include <string>
#include <vector>

#include "lbgb.h"
#include "lb_internal.h"
#include "lb_kernels.cuh"
#include "lb_pool.h"

namespace lbgb {
namespace {

constexpr int BATCH_THREADS = 128;   // cells per work item = threads per block
constexpr int BATCH_STORAGES = 6;    // storage types
constexpr int BATCH_TYPES = 12;      // kernel types: storage x (two arrays, in place)
constexpr int GRAPH_STEPS = 8;       // batched steps per captured graph
constexpr size_t BALIGN = 256;

// Division by a run-time invariant d < 2^31 for dividends n < 2^31 with one
// 64-bit multiply (Granlund & Montgomery, "Division by invariant integers
// using multiplication", PLDI 1994, Thm. 4.2 with N = 31): l = ceil(log2 d),
// m = ceil(2^(31+l) / d) < 2^32, n / d = (n * m) >> (31 + l).
struct FastDiv {
    uint32_t m;
    uint32_t shift;
    int d;
};
FastDiv make_fastdiv(int d) {
    FastDiv f;
    f.d = d;
    int l = 0;
    while ((1LL << l) < d) ++l;
    const unsigned __int128 one = 1;
    const unsigned __int128 num = one << (31 + l);
    f.m = (uint32_t)((num + (unsigned)d - 1) / (unsigned)d);
    f.shift = 31 + l;
    return f;
}
__device__ __forceinline__ int fdiv(int n, const FastDiv& f) {
    return (int)(((uint64_t)(uint32_t)n * f.m) >> f.shift);
}

struct SlotDev {
    void* pop[2];    // A/B arrays; an in-place slot has one array (pop[0] == pop[1])
    const uint8_t* code;
    LatticeParams p;
    FastDiv div_x;   // nx
    FastDiv div_xy;  // nx * ny
    int storage;
    int force;
    int inplace;     // parity 0: swapped layout, 1: streamed layout
};

// SR: stochastic rounding of a 16-bit slot (lb_options.rounding), seeded by
// the slot's step count exactly as a lattice stepped alone is.
template <class S, bool FORCE, bool INPLACE, bool SR>
__device__ __forceinline__ void update_cell(const SlotDev& sd, int parity, int cell, int x, int y, int z, uint8_t cc,
                                            uint32_t seed) {
    using M = typename Storage<S>::math;
    if constexpr (INPLACE) {  // pop[0] and pop[1] are the one array
        const S* Ar = static_cast<const S*>(sd.pop[0]);
        S* Aw = static_cast<S*>(sd.pop[1]);
        if (parity == 0) inplace_update<S, FORCE, FORM_SWAPPED, SR>(Ar, Aw, sd.code, sd.p, x, y, z, cell, cc, seed);
        else inplace_update<S, FORCE, FORM_STREAMED, SR>(Ar, Aw, sd.code, sd.p, x, y, z, cell, cc, seed);
        return;
    }
    const S* A = static_cast<const S*>(sd.pop[parity]);
    S* B = static_cast<S*>(sd.pop[parity ^ 1]);
    M d[Q];
    // mask-first bounce-back: served requests are small walled boxes, where a
    // large share of the cells is next to a wall (72 instead of 56 registers,
    // still faster on the seeded serving mix)
    pull_cell<S, 0, FORM_AB, true>(A, sd.code, sd.p, x, y, z, cell, cc, d);
    relax_dev<M, FORCE>(d, sd.p);
    const Rounder<S, SR> R(seed);
    const uint32_t key = R.key(cell);
#pragma unroll
    for (int i = 0; i < Q; ++i) B[(int64_t)i * sd.p.ps + cell] = R.one(d[i], key, cell, i);
}

template <class S, bool INPLACE, bool SR>
__device__ __forceinline__ void update_cell_f(const SlotDev& sd, int parity, int cell, int x, int y, int z,
                                              uint8_t cc, uint32_t seed) {
    if (sd.force)
        update_cell<S, true, INPLACE, SR>(sd, parity, cell, x, y, z, cc, seed);
    else
        update_cell<S, false, INPLACE, SR>(sd, parity, cell, x, y, z, cc, seed);
}

// One batched step for every active slot of storage type S and one
// population layout (two arrays, or in place -- separate kernels, so that the
// two-array kernel keeps its register count).
//   act[0..n)  slot ids, off[0..n]  cumulative 128-cell item counts,
//   n = *nact.  Slots whose remaining count is 0 are skipped.
template <class S, bool INPLACE>
__global__ void __launch_bounds__(BATCH_THREADS) batch_step_kernel(const SlotDev* __restrict__ slots,
                                                                   const int* __restrict__ parity,
                                                                   const int64_t* __restrict__ remaining,
                                                                   const int64_t* __restrict__ done,
                                                                   const int* __restrict__ act,
                                                                   const int* __restrict__ off,
                                                                   const int* __restrict__ nact) {
    const int n = *nact;
    if (n <= 0) return;
    const int total = off[n];
    const int G = gridDim.x;
    int k = 0;
    for (int item = blockIdx.x; item < total; item += G) {
        // the item's slot: largest k with off[k] <= item (items only grow)
        if (off[k + 1] <= item) {
            int lo = k + 1, hi = n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (off[mid] <= item) lo = mid;
                else hi = mid - 1;
            }
            k = lo;
        }
        const int slot = act[k];
        if (remaining[slot] <= 0) {
            // a paused or finished slot: jump to this block's first item past
            // its range (schedulers keep many admitted slots paused, and
            // walking their items one by one would cost every block a global
            // load per item)
            const int end = off[k + 1];
            item = end + ((blockIdx.x - end) % G + G) % G - G;  // the loop adds G
            continue;
        }
        const SlotDev& sd = slots[slot];
        const int cell = (item - off[k]) * BATCH_THREADS + threadIdx.x;
        if (cell >= (int)sd.p.N) continue;
        const int z = fdiv(cell, sd.div_xy);
        const int rem = cell - z * sd.div_xy.d;
        const int y = fdiv(rem, sd.div_x);
        const int x = rem - y * sd.div_x.d;
        const uint8_t cc = sd.code[cell];
        if (cc & CODE_TYPE) continue;
        const int par = parity[slot];
        if constexpr (sizeof(S) == 2) {
            if (sd.p.sr) {
                update_cell_f<S, INPLACE, true>(sd, par, cell, x, y, z, cc, sr_seed(done[slot]));
                continue;
            }
        }
        update_cell_f<S, INPLACE, false>(sd, par, cell, x, y, z, cc, 0u);
    }
}

// After a batched step: every listed slot that stepped flips its parity and
// counts down.
__global__ void batch_advance_kernel(int* __restrict__ parity, int64_t* __restrict__ remaining,
                                     int64_t* __restrict__ done, const int* __restrict__ list,
                                     const int* __restrict__ nlist) {
    const int n = *nlist;
    for (int k = threadIdx.x + blockIdx.x * blockDim.x; k < n; k += blockDim.x * gridDim.x) {
        const int s = list[k];
        if (remaining[s] > 0) {
            parity[s] ^= 1;
            remaining[s] -= 1;
            done[s] += 1;
        }
    }
}

// Set the step counters of n slots (quota grants from the host).
__global__ void batch_set_steps_kernel(int64_t* __restrict__ remaining, const int* __restrict__ slots,
                                       const int64_t* __restrict__ steps, int n) {
    for (int k = threadIdx.x + blockIdx.x * blockDim.x; k < n; k += blockDim.x * gridDim.x)
        remaining[slots[k]] = steps[k];
}

thread_local std::string g_berr;
int bfail(int status, const char* fmt, ...) __attribute__((format(printf, 2, 3)));
int bfail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_berr = buf;
    return status;
}
int bcuda(cudaError_t e, const char* what) { return bfail(LB_ECUDA, "%s: %s", what, cudaGetErrorString(e)); }
inline size_t rup(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Kernel type of a slot: its storage, plus BATCH_STORAGES if it is in place.
inline int kernel_type(int storage, int inplace) { return storage + (inplace ? BATCH_STORAGES : 0); }

size_t slot_bytes(int nx, int ny, int nz, int storage, int inplace) {
    const int64_t N = (int64_t)nx * ny * nz;
    const int64_t ps = (int64_t)rup((size_t)N, 128);
    return (inplace ? 1 : 2) * rup((size_t)Q * ps * storage_bytes(storage), BALIGN) + rup((size_t)N, BALIGN);
}

// Layout of a slot's state for the readers: the parity of an in-place slot
// names its layout; a two-array slot's current array is pop[parity].
inline int slot_form(const SlotDev& d, int par) {
    return d.inplace ? (par ? FORM_STREAMED : FORM_SWAPPED) : FORM_AB;
}

struct SlotHost {
    bool used = false;
    int storage = 0;
    size_t off = 0, bytes = 0;
    SlotDev dev;
};

}  // namespace
}  // namespace lbgb

using namespace lbgb;

// Host-side pipelining: a batched step never waits for the device.  Each
// lb_batch_step ends with an asynchronous copy of the per-slot step counters
// and parities into a pinned snapshot (event-tracked ring); lb_batch_poll
// waits only for the oldest pending snapshot, so the caller can keep the
// next chunk of steps queued while it retires finished slots.  Work lists
// and slot descriptors are uploaded from a pinned ring without
// synchronising.  Admission set-up (flag upload, classification,
// equilibrium initialisation) and the read-back of finished slots run on a
// second "io" stream: a finished slot has no steps left, so steps already
// queued skip it and never touch its memory.
constexpr int NSNAP = 4;  // pending counter snapshots
constexpr int NUP = 8;    // pinned upload-ring entries

struct Snapshot {
    int64_t* rem = nullptr;  // pinned, max_slots
    int* par = nullptr;      // pinned, max_slots
    cudaEvent_t ev = nullptr;
    int64_t seq = 0;
};

struct lb_batch {
    void* base = nullptr;
    size_t bytes = 0;
    bool owns = false;
    int max_slots = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t io = nullptr;
    cudaEvent_t io_ev = nullptr;
    cudaStream_t side[BATCH_TYPES] = {};
    cudaEvent_t fork = nullptr, join[BATCH_TYPES] = {};
    // device arrays (fixed area)
    SlotDev* d_slots = nullptr;
    int* d_parity = nullptr;
    int64_t* d_remaining = nullptr;
    int64_t* d_done = nullptr;
    int* d_act[BATCH_TYPES] = {};
    int* d_off[BATCH_TYPES] = {};
    int* d_nact = nullptr;  // BATCH_TYPES counts, then the advance-list count
    int* d_adv = nullptr;   // all admitted slots
    double* partials = nullptr;
    double* tot_out = nullptr;
    int* err = nullptr;
    void* staging = nullptr;     // main-stream host transfers
    void* io_staging = nullptr;  // io-stream host transfers
    size_t staging_bytes = 0;
    char* pool_base = nullptr;
    size_t pool_bytes = 0;
    Pool<BALIGN> pool;  // slot placement in the pool buffer (lb_pool.h)
    std::vector<SlotHost> slots;
    // host view of each slot's counters: the latest snapshot applied
    std::vector<int64_t> last_rem;
    std::vector<int> last_par;
    std::vector<int64_t> added_seq;  // snapshots with seq >= this describe the slot
    std::vector<cudaEvent_t> fetch_ev;  // per slot: an asynchronous fetch completed
    std::vector<char> fetching;         // per slot: a fetch was issued
    Snapshot snap[NSNAP];
    int64_t snap_head = 0, snap_tail = 0;  // issued / consumed snapshots
    char* up_buf = nullptr;  // pinned upload ring
    size_t up_entry = 0;
    cudaEvent_t up_ev[NUP] = {};
    int up_next = 0;
    bool dirty = true;
    int grid[BATCH_TYPES] = {};
    unsigned types_used = 0;  // kernel types that have had a slot: the ones a step launches
    cudaGraphExec_t graph = nullptr;
};

namespace {

struct BatchLayout {
    size_t slots_off, parity_off, rem_off, done_off, act_off, offs_off, nact_off, adv_off, part_off, tot_off, stage_off,
        stage_bytes, fixed;
};

BatchLayout batch_layout(int max_slots) {
    BatchLayout L{};
    size_t o = 0;
    auto take = [&](size_t n) {
        const size_t at = o;
        o += rup(n, BALIGN);
        return at;
    };
    L.slots_off = take(sizeof(SlotDev) * max_slots);
    L.parity_off = take(sizeof(int) * max_slots);
    L.rem_off = take(sizeof(int64_t) * max_slots);
    L.done_off = take(sizeof(int64_t) * max_slots);
    L.act_off = take(sizeof(int) * max_slots * BATCH_TYPES);
    L.offs_off = take(sizeof(int) * (max_slots + 1) * BATCH_TYPES);
    L.nact_off = take(sizeof(int) * (BATCH_TYPES + 1));
    L.adv_off = take(sizeof(int) * max_slots);
    L.part_off = take((size_t)totals_blocks(int64_t(1) << 31) * 6 * sizeof(double));
    L.tot_off = take(256);
    L.stage_bytes = size_t(16) << 20;  // two halves: main and io
    L.stage_off = take(L.stage_bytes);
    L.fixed = o;
    return L;
}

int64_t bchunk(const lb_batch* b, size_t per_cell) {
    const int64_t c = (int64_t)(b->staging_bytes / per_cell);
    return c < 1 ? 1 : c;
}

int slot_ok(lb_batch* b, int slot) {
    if (!b) return bfail(LB_EINVAL, "NULL batch");
    if (slot < 0 || slot >= b->max_slots || !b->slots[slot].used) return bfail(LB_EINVAL, "bad slot %d", slot);
    return LB_OK;
}

// A pinned upload-ring entry whose previous copy has completed.
char* up_acquire(lb_batch* b, cudaError_t* e) {
    *e = cudaEventSynchronize(b->up_ev[b->up_next]);
    return b->up_buf + (size_t)b->up_next * b->up_entry;
}
cudaError_t up_release(lb_batch* b, cudaStream_t st) {
    const cudaError_t e = cudaEventRecord(b->up_ev[b->up_next], st);
    b->up_next = (b->up_next + 1) % NUP;
    return e;
}

void apply_snapshot(lb_batch* b, const Snapshot& sn) {
    for (int s = 0; s < b->max_slots; ++s)
        if (b->slots[s].used && sn.seq >= b->added_seq[s]) {
            b->last_rem[s] = sn.rem[s];
            b->last_par[s] = sn.par[s];
        }
}

// Wait for the main stream and read every slot's counters directly.
int refresh_counters(lb_batch* b) {
    Snapshot& sn = b->snap[b->snap_head % NSNAP];
    cudaError_t e = cudaStreamSynchronize(b->stream);
    // any pending snapshots are complete now
    while (e == cudaSuccess && b->snap_tail < b->snap_head) {
        apply_snapshot(b, b->snap[b->snap_tail % NSNAP]);
        ++b->snap_tail;
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sn.rem, b->d_remaining, sizeof(int64_t) * b->max_slots, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sn.par, b->d_parity, sizeof(int) * b->max_slots, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(e, "batch: counters");
    Snapshot now = sn;
    now.seq = b->snap_head;  // describes every slot added so far
    apply_snapshot(b, now);
    return LB_OK;
}

bool finished_known(const lb_batch* b, int slot) { return b->last_rem[slot] == 0; }

// Rebuild the per-type work lists and the advance list (asynchronous).
int rebuild_lists(lb_batch* b) {
    cudaError_t e;
    char* up = up_acquire(b, &e);
    if (e != cudaSuccess) return bcuda(e, "batch: upload ring");
    const int M = b->max_slots;
    int* counts = (int*)up;                         // BATCH_TYPES + 1
    int* act = counts + (BATCH_TYPES + 1);          // BATCH_TYPES * M
    int* offs = act + (size_t)BATCH_TYPES * M;      // BATCH_TYPES * (M + 1)
    int* adv = offs + (size_t)BATCH_TYPES * (M + 1);  // M
    int nadv = 0;
    for (int t = 0; t < BATCH_TYPES; ++t) {
        counts[t] = 0;
        offs[(size_t)t * (M + 1)] = 0;
    }
    for (int s = 0; s < M; ++s) {
        const SlotHost& h = b->slots[s];
        if (!h.used) continue;
        const int t = kernel_type(h.storage, h.dev.inplace);
        const int64_t items = (h.dev.p.N + BATCH_THREADS - 1) / BATCH_THREADS;
        int* o = offs + (size_t)t * (M + 1);
        if ((int64_t)o[counts[t]] + items >= (int64_t(1) << 31)) return bfail(LB_ENOMEM, "batch: too many cells");
        act[(size_t)t * M + counts[t]] = s;
        o[counts[t] + 1] = o[counts[t]] + (int)items;
        ++counts[t];
        adv[nadv++] = s;
    }
    counts[BATCH_TYPES] = nadv;
    e = cudaSuccess;
    for (int t = 0; t < BATCH_TYPES && e == cudaSuccess; ++t) {
        if (counts[t] > 0)
            e = cudaMemcpyAsync(b->d_act[t], act + (size_t)t * M, counts[t] * sizeof(int), cudaMemcpyHostToDevice,
                                b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_off[t], offs + (size_t)t * (M + 1), (counts[t] + 1) * sizeof(int),
                                cudaMemcpyHostToDevice, b->stream);
    }
    if (e == cudaSuccess && nadv > 0)
        e = cudaMemcpyAsync(b->d_adv, adv, nadv * sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_nact, counts, (BATCH_TYPES + 1) * sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = up_release(b, b->stream);
    if (e != cudaSuccess) return bcuda(e, "batch: work lists");
    b->dirty = false;
    return LB_OK;
}

template <class S, bool INPLACE>
static void launch_typed(lb_batch* b, int t, cudaStream_t st) {
    batch_step_kernel<S, INPLACE><<<b->grid[t], BATCH_THREADS, 0, st>>>(b->d_slots, b->d_parity, b->d_remaining,
                                                                         b->d_done,
                                                                         b->d_act[t], b->d_off[t], b->d_nact + t);
}

cudaError_t launch_type(lb_batch* b, int t, cudaStream_t st) {
    switch (t) {
        case 0: launch_typed<double, false>(b, t, st); break;
        case 1: launch_typed<float, false>(b, t, st); break;
        case 2: launch_typed<__half, false>(b, t, st); break;
        case 3: launch_typed<__nv_bfloat16, false>(b, t, st); break;
        case 4: launch_typed<f32d, false>(b, t, st); break;
        case 5: launch_typed<e3m12, false>(b, t, st); break;
        case 6: launch_typed<double, true>(b, t, st); break;
        case 7: launch_typed<float, true>(b, t, st); break;
        case 8: launch_typed<__half, true>(b, t, st); break;
        case 9: launch_typed<__nv_bfloat16, true>(b, t, st); break;
        case 10: launch_typed<f32d, true>(b, t, st); break;
        default: launch_typed<e3m12, true>(b, t, st); break;
    }
    return cudaGetLastError();
}

template <class S, bool INPLACE>
static cudaError_t occupancy_of(int* per) {
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, batch_step_kernel<S, INPLACE>, BATCH_THREADS, 0);
}


// One batched step: the kernels of the types in use run concurrently on side
// streams forked from the batch stream, then the advance kernel.
cudaError_t issue_step(lb_batch* b) {
    cudaError_t e = cudaEventRecord(b->fork, b->stream);
    for (int t = 0; t < BATCH_TYPES && e == cudaSuccess; ++t) {
        if (!((b->types_used >> t) & 1u)) continue;
        e = cudaStreamWaitEvent(b->side[t], b->fork, 0);
        if (e == cudaSuccess) e = launch_type(b, t, b->side[t]);
        if (e == cudaSuccess) e = cudaEventRecord(b->join[t], b->side[t]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->join[t], 0);
    }
    if (e == cudaSuccess) {
        batch_advance_kernel<<<1, 256, 0, b->stream>>>(b->d_parity, b->d_remaining, b->d_done, b->d_adv,
                                                        b->d_nact + BATCH_TYPES);
        e = cudaGetLastError();
    }
    return e;
}

int ensure_graph(lb_batch* b) {
    if (b->graph) return LB_OK;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(e, "batch: begin capture");
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < GRAPH_STEPS && le == cudaSuccess; ++k) le = issue_step(b);
    e = cudaStreamEndCapture(b->stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bcuda(le, "batch: capture");
    }
    if (e != cudaSuccess) return bcuda(e, "batch: end capture");
    e = cudaGraphInstantiate(&b->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->graph = nullptr;
        return bcuda(e, "batch: instantiate");
    }
    return LB_OK;
}

void release_host(lb_batch* b) {
    for (int k = 0; k < NSNAP; ++k) {
        if (b->snap[k].rem) cudaFreeHost(b->snap[k].rem);
        if (b->snap[k].par) cudaFreeHost(b->snap[k].par);
        if (b->snap[k].ev) cudaEventDestroy(b->snap[k].ev);
    }
    for (int k = 0; k < NUP; ++k)
        if (b->up_ev[k]) cudaEventDestroy(b->up_ev[k]);
    for (auto ev : b->fetch_ev)
        if (ev) cudaEventDestroy(ev);
    if (b->up_buf) cudaFreeHost(b->up_buf);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    for (int t = 0; t < BATCH_TYPES; ++t) {
        if (b->side[t]) cudaStreamDestroy(b->side[t]);
        if (b->join[t]) cudaEventDestroy(b->join[t]);
    }
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->io_ev) cudaEventDestroy(b->io_ev);
    if (b->io) cudaStreamDestroy(b->io);
    if (b->owns && b->base) cudaFree(b->base);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

int batch_create_common(lb_batch** out, size_t capacity, int max_slots, void* stream, void* buffer, size_t bytes) {
    if (!out) return bfail(LB_EINVAL, "lb_batch_create: out is NULL");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 65536) return bfail(LB_EINVAL, "lb_batch_create: max_slots %d", max_slots);
    const BatchLayout L = batch_layout(max_slots);
    if (buffer) {
        if ((uintptr_t)buffer % BALIGN) return bfail(LB_EINVAL, "lb_batch_create_in: buffer not 256-byte aligned");
        if (bytes < L.fixed + BALIGN)
            return bfail(LB_ENOMEM, "lb_batch_create_in: buffer %zu < fixed area %zu", bytes, L.fixed);
    }
    lb_batch* b = new (std::nothrow) lb_batch();
    if (!b) return bfail(LB_ENOMEM, "lb_batch_create: host allocation");
    b->max_slots = max_slots;
    b->stream = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (!b->stream) {
        // graphs cannot be captured on the legacy default stream: use our own
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = (e == cudaSuccess);
    }
    if (e == cudaSuccess) {
        if (buffer) {
            b->base = buffer;
            b->bytes = bytes;
        } else {
            b->bytes = L.fixed + rup(capacity, BALIGN);
            e = cudaMalloc(&b->base, b->bytes);
            if (e != cudaSuccess) {
                cudaGetLastError();
                b->base = nullptr;
                release_host(b);
                delete b;
                return bfail(LB_ENOMEM, "lb_batch_create: cudaMalloc(%zu): %s", L.fixed + rup(capacity, BALIGN),
                             cudaGetErrorString(e));
            }
            b->owns = true;
        }
    }
    if (e != cudaSuccess) {
        release_host(b);
        delete b;
        return bcuda(e, "lb_batch_create");
    }
    char* c = (char*)b->base;
    b->d_slots = (SlotDev*)(c + L.slots_off);
    b->d_parity = (int*)(c + L.parity_off);
    b->d_remaining = (int64_t*)(c + L.rem_off);
    b->d_done = (int64_t*)(c + L.done_off);
    for (int t = 0; t < BATCH_TYPES; ++t) {
        b->d_act[t] = (int*)(c + L.act_off) + (size_t)t * max_slots;
        b->d_off[t] = (int*)(c + L.offs_off) + (size_t)t * (max_slots + 1);
    }
    b->d_nact = (int*)(c + L.nact_off);
    b->d_adv = (int*)(c + L.adv_off);
    b->partials = (double*)(c + L.part_off);
    b->tot_out = (double*)(c + L.tot_off);
    b->err = (int*)(c + L.tot_off + 128);
    b->staging_bytes = L.stage_bytes / 2;
    b->staging = c + L.stage_off;
    b->io_staging = c + L.stage_off + b->staging_bytes;
    b->pool_base = c + L.fixed;
    b->pool_bytes = b->bytes - L.fixed;
    b->pool.reset(b->pool_bytes);
    b->slots.assign(max_slots, SlotHost());
    b->last_rem.assign(max_slots, -1);
    b->last_par.assign(max_slots, 0);
    b->added_seq.assign(max_slots, 0);
    b->fetch_ev.assign(max_slots, nullptr);
    b->fetching.assign(max_slots, 0);
    b->up_entry = rup(sizeof(int) * ((size_t)(BATCH_TYPES + 1) + (size_t)BATCH_TYPES * max_slots +
                                     (size_t)BATCH_TYPES * (max_slots + 1) + max_slots) + sizeof(SlotDev) + 64,
                      BALIGN);
    int rc = LB_OK;
    e = cudaMemsetAsync(c, 0, L.stage_off, b->stream);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->io, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->io_ev, cudaEventDisableTiming);
    for (int t = 0; t < BATCH_TYPES && e == cudaSuccess; ++t) {
        e = cudaStreamCreateWithFlags(&b->side[t], cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->join[t], cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int k = 0; k < NSNAP && e == cudaSuccess; ++k) {
        e = cudaHostAlloc((void**)&b->snap[k].rem, sizeof(int64_t) * max_slots, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaHostAlloc((void**)&b->snap[k].par, sizeof(int) * max_slots, cudaHostAllocDefault);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->snap[k].ev, cudaEventDisableTiming);
    }
    if (e == cudaSuccess) e = cudaHostAlloc((void**)&b->up_buf, b->up_entry * NUP, cudaHostAllocDefault);
    for (int k = 0; k < NUP && e == cudaSuccess; ++k) {
        e = cudaEventCreateWithFlags(&b->up_ev[k], cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventRecord(b->up_ev[k], b->stream);
    }
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        int per[BATCH_TYPES] = {};
        e = occupancy_of<double, false>(&per[0]);
        if (e == cudaSuccess) e = occupancy_of<float, false>(&per[1]);
        if (e == cudaSuccess) e = occupancy_of<__half, false>(&per[2]);
        if (e == cudaSuccess) e = occupancy_of<__nv_bfloat16, false>(&per[3]);
        if (e == cudaSuccess) e = occupancy_of<f32d, false>(&per[4]);
        if (e == cudaSuccess) e = occupancy_of<e3m12, false>(&per[5]);
        if (e == cudaSuccess) e = occupancy_of<double, true>(&per[6]);
        if (e == cudaSuccess) e = occupancy_of<float, true>(&per[7]);
        if (e == cudaSuccess) e = occupancy_of<__half, true>(&per[8]);
        if (e == cudaSuccess) e = occupancy_of<__nv_bfloat16, true>(&per[9]);
        if (e == cudaSuccess) e = occupancy_of<f32d, true>(&per[10]);
        if (e == cudaSuccess) e = occupancy_of<e3m12, true>(&per[11]);
        for (int t = 0; t < BATCH_TYPES; ++t) b->grid[t] = sms * (per[t] > 0 ? per[t] : 1);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) rc = bcuda(e, "lb_batch_create");
    if (rc != LB_OK) {
        release_host(b);
        delete b;
        return rc;
    }
    *out = b;
    return LB_OK;
}

// The stream, staging area and parity to read a slot on: the io stream
// without waiting when the slot is known to be finished, otherwise the main
// stream after it has drained.
int reader_for(lb_batch* b, int slot, cudaStream_t* st, double** staging, int* par) {
    if (!finished_known(b, slot)) {
        const int rc = refresh_counters(b);
        if (rc != LB_OK) return rc;
    }
    if (finished_known(b, slot)) {
        *st = b->io;
        *staging = (double*)b->io_staging;
    } else {
        *st = b->stream;  // drained by refresh_counters
        *staging = (double*)b->staging;
    }
    *par = b->last_par[slot];
    return LB_OK;
}

}  // namespace

extern "C" {

size_t lb_batch_slot_bytes(int nx, int ny, int nz, int storage, int inplace) {
    if (nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny * nz >= (int64_t(1) << 31)) return 0;
    if (storage < LB_F64 || storage > LB_E3M12S || (inplace != 0 && inplace != 1)) return 0;
    return slot_bytes(nx, ny, nz, storage, inplace);
}

size_t lb_batch_fixed_bytes(int max_slots) {
    if (max_slots < 1 || max_slots > 65536) return 0;
    return batch_layout(max_slots).fixed;
}

int lb_batch_create(lb_batch** out, size_t capacity_bytes, int max_slots, void* stream) {
    return batch_create_common(out, capacity_bytes, max_slots, stream, nullptr, 0);
}

int lb_batch_create_in(lb_batch** out, void* device_buffer, size_t bytes, int max_slots, void* stream) {
    if (!device_buffer) return bfail(LB_EINVAL, "lb_batch_create_in: NULL buffer");
    return batch_create_common(out, 0, max_slots, stream, device_buffer, bytes);
}

int lb_batch_add(lb_batch* b, int nx, int ny, int nz, double tau, const double* u_lid, const uint8_t* flags,
                 const lb_options* opt, int64_t steps, int* slot_out) {
    if (!b || !slot_out) return bfail(LB_EINVAL, "lb_batch_add: NULL argument");
    *slot_out = -1;
    lb_options o;
    lb_default_options(&o);
    if (opt) o = *opt;
    if (nx < 1 || ny < 1 || nz < 1 || (int64_t)nx * ny * nz >= (int64_t(1) << 31))
        return bfail(LB_EINVAL, "lb_batch_add: bad dims %d x %d x %d", nx, ny, nz);
    if (!(tau > 0.5) || !std::isfinite(tau)) return bfail(LB_EINVAL, "lb_batch_add: tau must be > 1/2");
    if (o.storage < LB_F64 || o.storage > LB_E3M12S) return bfail(LB_EINVAL, "lb_batch_add: bad storage");
    if (!(o.trt_magic >= 0.0) || !std::isfinite(o.trt_magic))
        return bfail(LB_EINVAL, "lb_batch_add: trt_magic must be >= 0");
    if (o.inplace != 0 && o.inplace != 1) return bfail(LB_EINVAL, "lb_batch_add: inplace must be 0 or 1");
    if (o.rounding != 0 && o.rounding != 1) return bfail(LB_EINVAL, "lb_batch_add: rounding must be 0 or 1");
    if (o.rounding && storage_bytes(o.storage) != 2)
        return bfail(LB_EINVAL, "lb_batch_add: stochastic rounding needs 16-bit storage");
    if (o.halo_z) return bfail(LB_EINVAL, "lb_batch_add: batch slots have no ghost planes (halo_z)");
    if (steps < 0) return bfail(LB_EINVAL, "lb_batch_add: steps < 0");
    for (int a = 0; a < 3; ++a)
        if (!std::isfinite(o.force[a]) || (u_lid && !std::isfinite(u_lid[a])))
            return bfail(LB_EINVAL, "lb_batch_add: non-finite force or lid velocity");
    const int64_t N = (int64_t)nx * ny * nz;
    if (flags)
        for (int64_t c = 0; c < N; ++c)
            if (flags[c] > LB_FARFIELD) return bfail(LB_EINVAL, "lb_batch_add: flag %d at cell %lld", flags[c], (long long)c);
    int slot = -1;
    for (int s = 0; s < b->max_slots; ++s)
        if (!b->slots[s].used) {
            slot = s;
            break;
        }
    if (slot < 0) return bfail(LB_EBUSY, "lb_batch_add: all %d slots in use", b->max_slots);
    const size_t need = slot_bytes(nx, ny, nz, o.storage, o.inplace);
    size_t off = 0;
    if (!b->pool.alloc(need, &off))
        return bfail(LB_ENOMEM, "lb_batch_add: %zu bytes do not fit the pool (%zu free)", need, b->pool.free_bytes());
    SlotHost& h = b->slots[slot];
    const int64_t ps = (int64_t)rup((size_t)N, 128);
    const size_t popb = rup((size_t)Q * ps * storage_bytes(o.storage), BALIGN);
    char* base = b->pool_base + off;
    SlotDev d;
    d.pop[0] = base;
    d.pop[1] = o.inplace ? base : base + popb;
    d.code = (const uint8_t*)(base + (o.inplace ? 1 : 2) * popb);
    d.inplace = o.inplace;
    d.p.nx = nx;
    d.p.ny = ny;
    d.p.nz = nz;
    d.p.N = N;
    d.p.ps = ps;
    d.p.zlo = 0;
    d.p.zhi = nz;
    d.p.sr = o.rounding;
    d.p.sr_seed = 0;  // per step from the slot's step count
    d.p.omega = 1.0 / tau;
    d.p.omega_m = trt_omega_minus(tau, o.trt_magic);
    for (int a = 0; a < 3; ++a) {
        d.p.g[a] = o.force[a];
        d.p.ulid[a] = u_lid ? u_lid[a] : 0.0;
    }
    set_farfield(d.p);
    d.p.err = b->err;
    d.div_x = make_fastdiv(nx);
    d.div_xy = make_fastdiv(nx * ny);
    d.storage = o.storage;
    d.force = (o.force[0] != 0.0 || o.force[1] != 0.0 || o.force[2] != 0.0) ? 1 : 0;
    // set-up on the io stream: the slot is in no work list yet
    cudaError_t e = cudaSuccess;
    uint8_t* code = (uint8_t*)d.code;
    if (flags) {
        // stage the flags in the slot's B array (not yet initialised)
        e = cudaMemcpyAsync(d.pop[1], flags, (size_t)N, cudaMemcpyHostToDevice, b->io);
        if (e == cudaSuccess) e = launch_classify((const uint8_t*)d.pop[1], code, nx, ny, nz, b->io);
    } else {
        e = cudaMemsetAsync(code, 0, (size_t)N, b->io);
    }
    if (e == cudaSuccess)
        e = launch_init(o.storage, d.pop[0], d.pop[1], ps, nullptr, nullptr, 0, 0, N, b->io, o.inplace);
    if (e == cudaSuccess) e = cudaEventRecord(b->io_ev, b->io);
    // descriptor and counters on the main stream, after the set-up
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->io_ev, 0);
    char* up = nullptr;
    if (e == cudaSuccess) up = up_acquire(b, &e);
    if (e == cudaSuccess) {
        memcpy(up, &d, sizeof(SlotDev));
        int64_t* cnt = (int64_t*)(up + rup(sizeof(SlotDev), 16));
        cnt[0] = steps;  // remaining
        cnt[1] = 0;      // done
        int* par = (int*)(cnt + 2);
        *par = 0;
        e = cudaMemcpyAsync(b->d_slots + slot, up, sizeof(SlotDev), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_remaining + slot, &cnt[0], sizeof(int64_t), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_done + slot, &cnt[1], sizeof(int64_t), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(b->d_parity + slot, par, sizeof(int), cudaMemcpyHostToDevice, b->stream);
        const cudaError_t e2 = up_release(b, b->stream);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) {
        b->pool.release(off, need);
        return bcuda(e, "lb_batch_add");
    }
    const unsigned tbit = 1u << kernel_type(o.storage, o.inplace);
    if (!(b->types_used & tbit)) {
        // a kernel type not launched so far: the captured step graph lacks its
        // kernel, so it is re-captured at the next lb_batch_step (after the
        // replays already queued have finished)
        if (b->graph) {
            cudaError_t eg = cudaStreamSynchronize(b->stream);
            if (eg == cudaSuccess) eg = cudaGraphExecDestroy(b->graph);
            b->graph = nullptr;
            if (eg != cudaSuccess) return bcuda(eg, "lb_batch_add: graph");
        }
        b->types_used |= tbit;
    }
    h.used = true;
    h.storage = o.storage;
    h.off = off;
    h.bytes = need;
    h.dev = d;
    b->last_rem[slot] = steps;
    b->last_par[slot] = 0;
    b->added_seq[slot] = b->snap_head;  // later snapshots describe it
    b->dirty = true;
    *slot_out = slot;
    return LB_OK;
}

int lb_batch_set_steps(lb_batch* b, int slot, int64_t steps) {
    int rc = slot_ok(b, slot);
    if (rc != LB_OK) return rc;
    if (steps < 0) return bfail(LB_EINVAL, "lb_batch_set_steps: steps < 0");
    cudaError_t e;
    char* up = up_acquire(b, &e);
    if (e == cudaSuccess) {
        memcpy(up, &steps, sizeof steps);
        e = cudaMemcpyAsync(b->d_remaining + slot, up, sizeof(int64_t), cudaMemcpyHostToDevice, b->stream);
        const cudaError_t e2 = up_release(b, b->stream);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return bcuda(e, "lb_batch_set_steps");
    b->last_rem[slot] = steps;
    b->added_seq[slot] = b->snap_head;
    return LB_OK;
}

int lb_batch_set_steps_many(lb_batch* b, int n, const int* slots, const int64_t* steps) {
    if (!b || n < 0 || (n > 0 && (!slots || !steps))) return bfail(LB_EINVAL, "lb_batch_set_steps_many: bad arguments");
    if (n == 0) return LB_OK;
    if (n > b->max_slots) return bfail(LB_EINVAL, "lb_batch_set_steps_many: n > max_slots");
    for (int k = 0; k < n; ++k) {
        const int rc = slot_ok(b, slots[k]);
        if (rc != LB_OK) return rc;
        if (steps[k] < 0) return bfail(LB_EINVAL, "lb_batch_set_steps_many: steps < 0");
    }
    cudaError_t e;
    char* up = up_acquire(b, &e);
    if (e == cudaSuccess) {
        // the entry holds (5 + 9 * max_slots) ints: room for n slots and n counts
        int64_t* cnt = (int64_t*)up;
        int* ids = (int*)(cnt + n);
        memcpy(cnt, steps, sizeof(int64_t) * n);
        memcpy(ids, slots, sizeof(int) * n);
        int64_t* dcnt = (int64_t*)b->staging;  // main-stream staging: ordered after queued work
        int* dids = (int*)(dcnt + n);
        e = cudaMemcpyAsync(dcnt, up, sizeof(int64_t) * n + sizeof(int) * n, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) {
            batch_set_steps_kernel<<<(n + 255) / 256, 256, 0, b->stream>>>(b->d_remaining, dids, dcnt, n);
            e = cudaGetLastError();
        }
        const cudaError_t e2 = up_release(b, b->stream);
        if (e == cudaSuccess) e = e2;
    }
    if (e != cudaSuccess) return bcuda(e, "lb_batch_set_steps_many");
    for (int k = 0; k < n; ++k) {
        b->last_rem[slots[k]] = steps[k];
        b->added_seq[slots[k]] = b->snap_head;
    }
    return LB_OK;
}

int lb_batch_init_fields(lb_batch* b, int slot, const double* rho, const double* u) {
    int rc = slot_ok(b, slot);
    if (rc != LB_OK) return rc;
    if ((rc = refresh_counters(b)) != LB_OK) return rc;  // drains the main stream
    const SlotDev& d = b->slots[slot].dev;
    const int par = b->last_par[slot];
    const size_t per_cell = (rho ? 8 : 0) + (u ? 24 : 0);
    const int64_t N = d.p.N;
    const int64_t chunk = per_cell ? bchunk(b, per_cell) : N;
    double* st = (double*)b->staging;
    for (int64_t c0 = 0; c0 < N; c0 += chunk) {
        const int64_t cnt = (N - c0 < chunk) ? N - c0 : chunk;
        double* drho = rho ? st : nullptr;
        double* du = u ? st + (rho ? cnt : 0) : nullptr;
        cudaError_t e = cudaSuccess;
        if (rho) e = cudaMemcpyAsync(drho, rho + c0, cnt * 8, cudaMemcpyHostToDevice, b->stream);
        for (int a = 0; a < 3 && u && e == cudaSuccess; ++a)
            e = cudaMemcpyAsync(du + a * cnt, u + a * N + c0, cnt * 8, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = launch_init(d.storage, d.pop[par], d.pop[par ^ 1], d.p.ps, drho, du, cnt, c0, cnt, b->stream,
                            d.inplace);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bcuda(e, "lb_batch_init_fields");
    }
    if (d.inplace && par != 0) {  // the initialised state has the swapped layout: parity 0
        const int zero = 0;
        cudaError_t e = cudaMemcpyAsync(b->d_parity + slot, &zero, sizeof zero, cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
        if (e != cudaSuccess) return bcuda(e, "lb_batch_init_fields: parity");
        b->last_par[slot] = 0;
        b->added_seq[slot] = b->snap_head;  // snapshots taken from now on describe it
    }
    return LB_OK;
}

int lb_batch_step(lb_batch* b, int n) {
    if (!b) return bfail(LB_EINVAL, "lb_batch_step: NULL batch");
    if (n < 0) return bfail(LB_EINVAL, "lb_batch_step: n < 0");
    if (b->dirty) {
        const int rc = rebuild_lists(b);
        if (rc != LB_OK) return rc;
    }
    int done = 0;
    if (n >= GRAPH_STEPS) {
        const int rc = ensure_graph(b);
        if (rc != LB_OK) return rc;
        for (; done + GRAPH_STEPS <= n; done += GRAPH_STEPS) {
            cudaError_t e = cudaGraphLaunch(b->graph, b->stream);
            if (e != cudaSuccess) return bcuda(e, "lb_batch_step: graph launch");
        }
    }
    for (; done < n; ++done) {
        cudaError_t e = issue_step(b);
        if (e != cudaSuccess) return bcuda(e, "lb_batch_step");
    }
    // snapshot of the counters after these steps (asynchronous)
    if (b->snap_head - b->snap_tail == NSNAP) {  // ring full: absorb the oldest
        Snapshot& old = b->snap[b->snap_tail % NSNAP];
        cudaError_t e = cudaEventSynchronize(old.ev);
        if (e != cudaSuccess) return bcuda(e, "lb_batch_step: snapshot");
        apply_snapshot(b, old);
        ++b->snap_tail;
    }
    Snapshot& sn = b->snap[b->snap_head % NSNAP];
    cudaError_t e =
        cudaMemcpyAsync(sn.rem, b->d_remaining, sizeof(int64_t) * b->max_slots, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(sn.par, b->d_parity, sizeof(int) * b->max_slots, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaEventRecord(sn.ev, b->stream);
    if (e != cudaSuccess) return bcuda(e, "lb_batch_step: snapshot");
    sn.seq = b->snap_head;
    ++b->snap_head;
    return LB_OK;
}

int lb_batch_poll(lb_batch* b, int* done_slots, int max, int* ndone) {
    if (!b || !ndone || (max > 0 && !done_slots)) return bfail(LB_EINVAL, "lb_batch_poll: NULL argument");
    if (b->snap_tail < b->snap_head) {
        Snapshot& sn = b->snap[b->snap_tail % NSNAP];
        cudaError_t e = cudaEventSynchronize(sn.ev);
        if (e != cudaSuccess) return bcuda(e, "lb_batch_poll");
        apply_snapshot(b, sn);
        ++b->snap_tail;
    } else {
        const int rc = refresh_counters(b);
        if (rc != LB_OK) return rc;
    }
    int k = 0;
    for (int s = 0; s < b->max_slots; ++s)
        if (b->slots[s].used && finished_known(b, s)) {
            if (k < max) done_slots[k] = s;
            ++k;
        }
    *ndone = k;
    return LB_OK;
}

int lb_batch_query(lb_batch* b, int slot, int64_t* remaining, int64_t* done, int* dims, int* storage) {
    int rc = slot_ok(b, slot);
    if (rc != LB_OK) return rc;
    if ((rc = refresh_counters(b)) != LB_OK) return rc;
    int64_t d = 0;
    cudaError_t e = cudaMemcpyAsync(&d, b->d_done + slot, 8, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(e, "lb_batch_query");
    if (remaining) *remaining = b->last_rem[slot];
    if (done) *done = d;
    const SlotDev& sd = b->slots[slot].dev;
    if (dims) {
        dims[0] = sd.p.nx;
        dims[1] = sd.p.ny;
        dims[2] = sd.p.nz;
    }
    if (storage) *storage = sd.storage;
    return LB_OK;
}

int lb_batch_moments(lb_batch* b, int slot, double* rho, double* u) {
    int rc = slot_ok(b, slot);
    if (rc != LB_OK) return rc;
    if (!rho && !u) return LB_OK;
    cudaStream_t st;
    double* stg;
    int par;
    if ((rc = reader_for(b, slot, &st, &stg, &par)) != LB_OK) return rc;
    const SlotDev& d = b->slots[slot].dev;
    const int64_t N = d.p.N;
    const int64_t chunk = bchunk(b, 32);
    for (int64_t c0 = 0; c0 < N; c0 += chunk) {
        const int64_t cnt = (N - c0 < chunk) ? N - c0 : chunk;
        cudaError_t e =
            launch_moments(d.storage, d.pop[par], d.code, d.p, stg, stg + cnt, cnt, c0, cnt, st, slot_form(d, par));
        if (e == cudaSuccess && rho) e = cudaMemcpyAsync(rho + c0, stg, cnt * 8, cudaMemcpyDeviceToHost, st);
        for (int a = 0; a < 3 && u && e == cudaSuccess; ++a)
            e = cudaMemcpyAsync(u + a * N + c0, stg + (1 + a) * cnt, cnt * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return bcuda(e, "lb_batch_moments");
    }
    return LB_OK;
}

int lb_batch_totals(lb_batch* b, int slot, double* mass, double* mom) {
    int rc = slot_ok(b, slot);
    if (rc != LB_OK) return rc;
    cudaStream_t st;
    double* stg;
    int par;
    if ((rc = reader_for(b, slot, &st, &stg, &par)) != LB_OK) return rc;
    const SlotDev& d = b->slots[slot].dev;
    double out[5];
    cudaError_t e = launch_totals(d.storage, d.pop[par], d.code, d.p, b->partials, b->tot_out, st, slot_form(d, par));
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, b->tot_out, sizeof out, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return bcuda(e, "lb_batch_totals");
    if (mass) *mass = out[0];
    if (mom)
        for (int a = 0; a < 3; ++a) mom[a] = out[1 + a];
    if (out[4] != 0.0 || !std::isfinite(out[0]))
        return bfail(LB_EDIVERGED, "lb_batch_totals: %.0f fluid cells with non-finite or non-positive density", out[4]);
    return LB_OK;
}

int lb_batch_get_populations(lb_batch* b, int slot, double* f) {
    int rc = slot_ok(b, slot);
    if (rc != LB_OK) return rc;
    if (!f) return bfail(LB_EINVAL, "lb_batch_get_populations: NULL f");
    cudaStream_t st;
    double* stg;
    int par;
    if ((rc = reader_for(b, slot, &st, &stg, &par)) != LB_OK) return rc;
    const SlotDev& d = b->slots[slot].dev;
    const int64_t N = d.p.N;
    const int64_t chunk = bchunk(b, Q * 8);
    for (int64_t c0 = 0; c0 < N; c0 += chunk) {
        const int64_t cnt = (N - c0 < chunk) ? N - c0 : chunk;
        cudaError_t e = launch_get_pops(d.storage, d.pop[par], d.code, d.p, slot_form(d, par), c0, cnt, stg, st);
        for (int i = 0; i < Q && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync(f + i * N + c0, stg + i * cnt, cnt * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return bcuda(e, "lb_batch_get_populations");
    }
    return LB_OK;
}

int lb_batch_fetch(lb_batch* b, int slot, double* rho, double* u) {
    int rc = slot_ok(b, slot);
    if (rc != LB_OK) return rc;
    if (!rho || !u) return bfail(LB_EINVAL, "lb_batch_fetch: NULL buffer");
    if (!finished_known(b, slot)) {
        if ((rc = refresh_counters(b)) != LB_OK) return rc;
        if (!finished_known(b, slot)) return bfail(LB_EBUSY, "lb_batch_fetch: slot %d still has steps", slot);
    }
    const SlotDev& d = b->slots[slot].dev;
    const int par = b->last_par[slot];
    const int64_t N = d.p.N;
    cudaError_t e = cudaSuccess;
    if (!b->fetch_ev[slot]) e = cudaEventCreateWithFlags(&b->fetch_ev[slot], cudaEventDisableTiming);
    if (!d.inplace) {
        // the finished slot's B array (>= 38 bytes per cell) holds rho and u
        double* dr = (double*)d.pop[par ^ 1];
        double* du = dr + N;
        if (e == cudaSuccess) e = launch_moments(d.storage, d.pop[par], d.code, d.p, dr, du, N, 0, N, b->io);
        if (e == cudaSuccess) e = cudaMemcpyAsync(rho, dr, (size_t)N * 8, cudaMemcpyDeviceToHost, b->io);
        if (e == cudaSuccess) e = cudaMemcpyAsync(u, du, (size_t)N * 24, cudaMemcpyDeviceToHost, b->io);
    } else {
        // no spare array: chunks through the io staging area, each chunk's
        // moments kernel ordered after the previous chunk's copies on the
        // io stream (so the host never waits here)
        const int64_t chunk = bchunk(b, 32);
        double* stg = (double*)b->io_staging;
        for (int64_t c0 = 0; c0 < N && e == cudaSuccess; c0 += chunk) {
            const int64_t cnt = (N - c0 < chunk) ? N - c0 : chunk;
            e = launch_moments(d.storage, d.pop[par], d.code, d.p, stg, stg + cnt, cnt, c0, cnt, b->io,
                               slot_form(d, par));
            if (e == cudaSuccess) e = cudaMemcpyAsync(rho + c0, stg, cnt * 8, cudaMemcpyDeviceToHost, b->io);
            for (int a = 0; a < 3 && e == cudaSuccess; ++a)
                e = cudaMemcpyAsync(u + a * N + c0, stg + (1 + a) * cnt, cnt * 8, cudaMemcpyDeviceToHost, b->io);
        }
    }
    if (e == cudaSuccess) e = cudaEventRecord(b->fetch_ev[slot], b->io);
    if (e != cudaSuccess) return bcuda(e, "lb_batch_fetch");
    b->fetching[slot] = 1;
    return LB_OK;
}

int lb_batch_fetch_done(lb_batch* b, int slot) {
    int rc = slot_ok(b, slot);
    if (rc != LB_OK) return rc;
    if (!b->fetching[slot]) return bfail(LB_EINVAL, "lb_batch_fetch_done: no fetch issued for slot %d", slot);
    const cudaError_t e = cudaEventQuery(b->fetch_ev[slot]);
    if (e == cudaSuccess) return 1;
    if (e == cudaErrorNotReady) return 0;
    return bcuda(e, "lb_batch_fetch_done");
}

int lb_batch_remove(lb_batch* b, int slot) {
    int rc = slot_ok(b, slot);
    if (rc != LB_OK) return rc;
    if (b->fetching[slot]) {  // its memory is being read back
        const cudaError_t e = cudaEventSynchronize(b->fetch_ev[slot]);
        if (e != cudaSuccess) return bcuda(e, "lb_batch_remove: fetch");
        b->fetching[slot] = 0;
    }
    if (!finished_known(b, slot)) {
        // still stepping: drain the queued work, then stop it
        if ((rc = refresh_counters(b)) != LB_OK) return rc;
        if (!finished_known(b, slot)) {
            const int64_t z = 0;
            cudaError_t e = cudaMemcpyAsync(b->d_remaining + slot, &z, sizeof z, cudaMemcpyHostToDevice, b->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
            if (e != cudaSuccess) return bcuda(e, "lb_batch_remove");
            b->last_rem[slot] = 0;
        }
    }
    // the io stream may still read it (moments issued by this thread have
    // returned, but be safe for other threads' readers)
    cudaError_t e = cudaStreamSynchronize(b->io);
    if (e != cudaSuccess) return bcuda(e, "lb_batch_remove");
    SlotHost& h = b->slots[slot];
    b->pool.release(h.off, h.bytes);
    h.used = false;
    b->dirty = true;
    return LB_OK;
}

int lb_batch_free_bytes(lb_batch* b, size_t* free_bytes, int* free_slots) {
    if (!b) return bfail(LB_EINVAL, "lb_batch_free_bytes: NULL batch");
    if (free_bytes) *free_bytes = b->pool.free_bytes();
    if (free_slots) {
        int n = 0;
        for (auto& s : b->slots) n += s.used ? 0 : 1;
        *free_slots = n;
    }
    return LB_OK;
}

int lb_batch_sync(lb_batch* b) {
    if (!b) return bfail(LB_EINVAL, "lb_batch_sync: NULL batch");
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->io);
    return e == cudaSuccess ? LB_OK : bcuda(e, "lb_batch_sync");
}

int lb_batch_destroy(lb_batch* b) {
    if (!b) return LB_OK;
    int rc = LB_OK;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e == cudaSuccess && b->io) e = cudaStreamSynchronize(b->io);
    if (e != cudaSuccess) rc = bcuda(e, "lb_batch_destroy: sync");
    release_host(b);
    delete b;
    return rc;
}

const char* lb_batch_last_error(void) { return g_berr.c_str(); }

}  // extern "C"
