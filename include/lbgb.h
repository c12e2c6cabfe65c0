/*
 * lbgb.h -- C ABI of the GB300 D3Q19 lattice-Boltzmann library (liblbgb.so).
 *
 * The library advances a 3D lattice with the fused stream-and-collide BGK
 * update of arXiv 2409.16781 (Sec. 2, Eq. 1-3; fused pull with two
 * population arrays, Sec. 3.1; structure-of-arrays populations, Sec. 3.1;
 * lid-driven cavity walls and moving lid, Sec. 3.3), extended from the
 * paper's D2Q9 to the D3Q19 velocity set (the paper's Sec. 6 names the 3D
 * extension and mixed precision as future work).
 *
 * Conventions shared by every call
 *  - Every call returns an lb_status value (0 = LB_OK, negative = error).
 *    A failed call leaves the handle valid (except lb_destroy, which always
 *    releases it).  lb_last_error() gives a one-line description of the most
 *    recent failure on this thread.
 *  - Host buffers passed in are owned by the caller and are only read or
 *    written during the call.  Device buffers passed in (lb_create_in,
 *    lb_moments_device) are owned by the caller and must outlive their use.
 *  - Grid: nx, ny, nz >= 1, nx*ny*nz < 2^31 cells.  A scalar field has N =
 *    nx*ny*nz entries with cell index x + nx*(y + ny*z) (x fastest, the
 *    column-major order of Sec. 4.2).  A vector field u is SoA: u[a*N + cell],
 *    a = 0,1,2 for x,y,z.  Populations are q-major: f[i*N + cell].
 *  - The domain wraps periodically on all six faces; walls are cells
 *    flagged LB_WALL or LB_LID, open boundaries cells flagged LB_FARFIELD.
 *  - Velocity order (fixed): i = 0 rest; 1..6 = +x,-x,+y,-y,+z,-z;
 *    7..18 = (1,1,0),(-1,-1,0),(1,-1,0),(-1,1,0),(1,0,1),(-1,0,-1),
 *    (1,0,-1),(-1,0,1),(0,1,1),(0,-1,-1),(0,1,-1),(0,-1,1).  Directions
 *    2k-1 and 2k are opposite.  Weights 1/3, 1/18 (axes), 1/36 (diagonals).
 *  - Work is issued asynchronously on the lattice's stream; calls that
 *    return data to host memory synchronise that stream before returning.
 */
#ifndef LBGB_H
#define LBGB_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LB_Q 19

typedef struct lb_lattice lb_lattice; /* opaque */

typedef enum {
    LB_OK = 0,
    LB_EINVAL = -1,    /* bad argument (sizes, tau <= 1/2, flag values, NULL) */
    LB_ENOMEM = -2,    /* device allocation failed or buffer too small */
    LB_ECUDA = -3,     /* a CUDA runtime call or kernel launch failed */
    LB_EDIVERGED = -4, /* non-finite or non-positive density found */
    LB_ETIMEOUT = -5,  /* a bounded device-side wait gave up */
    LB_EBUSY = -6      /* resource in use (batch capacity reached) */
} lb_status;

/* Population storage (the paper's precision modes, Sec. 3.1.1).  Every
 * form stores the deviation f_i - w_i; the math is FP32 except for LB_F64
 * (FP64 storage and math) and LB_F32D (FP32 storage, FP64 math).
 * LB_E3M12S (not in the paper) is a 16-bit float of the deviation with 1
 * sign, 3 exponent and 12 mantissa bits: |d| in [2^(e-11), 2^(e-10)) for
 * exponent field e = 1..7, steps of 2^-22 below 2^-10; largest value
 * (2 - 2^-12) 2^-4 ~ 0.125 (larger magnitudes saturate, and lb_totals
 * then reports LB_EDIVERGED).  Where the deviations of a low-Mach flow lie
 * (|d| > 2^-10) its resolution is four times FP16's, for the same bytes. */
typedef enum {
    LB_F64 = 0,   /* "Double": FP64 storage, FP64 math            */
    LB_F32 = 1,   /* "Single": FP32 storage, FP32 math            */
    LB_F16S = 2,  /* "Mixed1": FP16 storage of f - w, FP32 math   */
    LB_BF16S = 3, /* BF16 storage of f - w, FP32 math             */
    LB_F32D = 4,  /* "Mixed2": FP32 storage of f - w, FP64 math   */
    LB_E3M12S = 5 /* E3M12 16-bit storage of f - w, FP32 math     */
} lb_storage;

/* Cell flags (uint8 per cell).  LB_WALL: no-slip wall (halfway
 * bounce-back).  LB_LID: wall moving at u_lid (Sec. 3.3, lid-driven cavity).
 * LB_FARFIELD: the free stream -- a fluid cell pulling from it receives the
 * equilibrium f^eq(rho = 1, u = u_lid) of Eq. 2-3 whatever it sent out;
 * planes of far-field cells are the inflow and outflow of flow past an
 * obstacle (the von Karman street use case of Sec. 3.3, whose boundary
 * conditions the paper does not give).  Solid and far-field cells are
 * never updated and report rho = 0, u = 0. */
enum { LB_FLUID = 0, LB_WALL = 1, LB_LID = 2, LB_FARFIELD = 3 };

typedef struct lb_options {
    int storage;       /* lb_storage; default LB_F32 */
    int kernel;        /* step kernel variant: 0 = library's choice */
    int block;         /* threads per block of the step kernel; 0 = choice */
    int rounding;      /* how a step rounds the new 16-bit stored values
                          (LB_F16S, LB_BF16S, LB_E3M12S; must be 0 for
                          other storage):
                          0 (default) to nearest even; 1 stochastically --
                          up with probability equal to the dropped fraction,
                          so each stored value is unbiased and changes far
                          below the 16-bit resolution (a weak body force)
                          are kept on average instead of lost.  The random
                          bits are a hash of (cell, direction, steps taken),
                          so a run is reproducible, every step variant and
                          batch slot gives bitwise the same result, and a
                          checkpoint restores the stream with the step
                          count.  Supported by step variants 1-3, 13, 15-19
                          and the in-place kernels; the default runs 18 (15
                          where the row does not fit it), other variants
                          run 15 (1 where it does not apply).  Equilibrium
                          initialisation and population import round to
                          nearest even. */
    double force[3];   /* body force per unit mass g (Guo forcing, the S_i
                          of Eq. 1); default 0 */
    void *stream;      /* cudaStream_t to issue work on; NULL = default */
    double trt_magic;  /* collision: 0 = BGK (Eq. 1, one rate omega = 1/tau,
                          the default); > 0 = two-relaxation-time collision
                          (Ginzburg's TRT, not in the paper): the part of f
                          even under c -> -c relaxes at 1/tau, the odd part
                          at omega_m with (tau - 1/2)(1/omega_m - 1/2) =
                          trt_magic, and the Guo source splits the same way.
                          3/16 makes halfway bounce-back walls exact for
                          Poiseuille flow at any tau.  Must be >= 0. */
    int inplace;       /* 0 (default): two population arrays, the paper's
                          fused scheme (Sec. 3.1: read f^pre, write f^post,
                          swap).  1: ONE array, updated in place with the
                          "AA" access pattern (not in the paper): the steps
                          alternate between two layouts of the same array,
                          each thread writing exactly the values it read, so
                          the lattice needs half the population memory for
                          the same bytes per update.  Its step kernels:
                          variant 2, two cells per thread collided in
                          packed FP32 (FP32 or 16-bit storage, nx even);
                          any other variant one cell per thread.  Values
                          that lb_get_populations reports for solid cells
                          are the rest state f = w. */
    int halo_z;        /* 0 (default): an ordinary lattice.  1: one z-slab
                          of a lattice decomposed along z over several GPUs
                          (the multi-GPU extension that Sec. 6 names as
                          future work): planes z = 0 and z = nz - 1 are
                          ghost planes holding the neighbouring slabs'
                          boundary planes (their flags are the neighbours'
                          flags; see lb_halo_pack).  The own planes are
                          1 .. nz-2; lb_totals sums only them and
                          lb_moments reports 0 on the ghost planes.  Needs
                          two population arrays (inplace = 0) and nz >= 3. */
    int reserved[4];
} lb_options;

/* Fill *opt with the defaults (FP32, no force, default stream). */
void lb_default_options(lb_options *opt);

/* The library's velocity set: c[3*i + a], w[i], i in the order above.
 * Returns LB_Q. */
int lb_velocity_set(int *c, double *w);

/* Bytes of device memory one lattice needs (populations A and B, cell
 * codes, host-transfer staging and reduction scratch).  0 on bad sizes. */
size_t lb_bytes_required(int nx, int ny, int nz, const lb_options *opt);

/* Create a lattice of nx x ny x nz cells for one of the use cases of
 * Sec. 3.3 (lid-driven cavity, Taylor-Green vortex, flow past an obstacle).
 *   tau    BGK relaxation time, omega = 1/tau of Eq. 1; must be > 1/2.
 *   u_lid  velocity of LB_LID cells and of the free stream of LB_FARFIELD
 *          cells (NULL = 0); halfway bounce-back off a LID source adds
 *          6 w_i (c_i . u_lid) (wall density 1).
 *   flags  host, N bytes, values LB_FLUID/LB_WALL/LB_LID/LB_FARFIELD,
 *          copied at create; NULL = all fluid.
 *   opt    NULL = defaults.
 * The library allocates lb_bytes_required() bytes of device memory with
 * cudaMalloc; the populations start at rest, f = w (rho = 1, u = 0).
 * Errors: LB_EINVAL, LB_ENOMEM, LB_ECUDA; *out is NULL on error. */
int lb_create(lb_lattice **out, int nx, int ny, int nz, double tau,
              const double *u_lid, const uint8_t *flags, const lb_options *opt);

/* As lb_create, but all device memory comes from the caller's buffer
 * (device pointer, 256-byte aligned, at least lb_bytes_required() bytes),
 * which must stay valid until lb_destroy.  Used by the Python binding so
 * that PyTorch owns the allocation. */
int lb_create_in(lb_lattice **out, int nx, int ny, int nz, double tau,
                 const double *u_lid, const uint8_t *flags, const lb_options *opt,
                 void *device_buffer, size_t bytes);

/* Set every cell to the equilibrium f^eq(rho, u) of Eq. 2-3.
 *   rho  host, N doubles (NULL = 1);  u  host, 3N doubles SoA (NULL = 0).
 * Buffers in page-locked host memory that is mapped into the device's
 * address space (cudaHostAlloc / cudaMallocHost, or registered as mapped;
 * both ends of each buffer are checked) are read by the kernel in place, in
 * one launch; other host memory goes through the library's staging area in
 * chunks.  Same result either way; synchronises the lattice's stream. */
int lb_init_fields(lb_lattice *h, const double *rho, const double *u);

/* Advance n >= 0 time steps: each is one fused pull-collide launch
 * (Eq. 1 with the boundary rules) from array A into B, then A <-> B.
 * Asynchronous on the lattice's stream. */
int lb_step(lb_lattice *h, int n);

/* Macroscopic fields of the current state: rho and u (half-force shifted,
 * u = (sum_i f_i c_i)/rho + g/2) of the streamed populations at every fluid
 * cell; solid cells report rho = 0, u = 0.
 *   rho  host, N doubles;  u  host, 3N doubles SoA.  Either may be NULL.
 * Mapped page-locked host buffers (as for lb_init_fields) are written by the
 * kernel in place, in one launch; other host memory through the staging
 * area in chunks.  Synchronises the lattice's stream. */
int lb_moments(lb_lattice *h, double *rho, double *u);

/* As lb_moments, into device buffers (N and 3N doubles), asynchronous. */
int lb_moments_device(lb_lattice *h, double *rho_dev, double *u_dev);

/* FP64 totals over fluid cells: mass = sum rho, mom = sum rho u.  Computed
 * on the device with FP64 accumulators and a fixed reduction order (the
 * result is bitwise reproducible).  Returns LB_EDIVERGED (after filling
 * the outputs) when a fluid cell has a non-finite or non-positive rho. */
int lb_totals(lb_lattice *h, double *mass, double *mom);

/* Copy the post-collision populations (array A: the state after the last
 * step) to/from host FP64, q-major f[i*N + cell], library velocity order.
 * get: f = w_i + d_i of the stored deviation d_i, rounded to FP64 (exact
 * unless d_i carries bits below FP64's resolution at w_i, which only FP64
 * storage does); set: d_i = f - w_i rounded to the storage type, to nearest
 * even.  So set(get()) reproduces FP32 and 16-bit states exactly and FP64
 * states to within one FP64 rounding; lb_checkpoint_* below is exact for
 * every form. */
int lb_get_populations(lb_lattice *h, double *f);
int lb_set_populations(lb_lattice *h, const double *f);

/* Checkpoint / restart, bit-exact: the stored values of the current
 * population array verbatim (19 planes of N values of the storage type),
 * behind a 64-byte header with the dims, storage, layout (in place) and
 * step count.  lb_checkpoint_bytes gives the buffer size (0 for NULL);
 * save fills a host buffer of at least that size; load restores it into a
 * lattice of the same dims, storage and population scheme (LB_EINVAL
 * otherwise), layout and step count included.  Both synchronise the
 * lattice's stream. */
size_t lb_checkpoint_bytes(lb_lattice *h);
int lb_checkpoint_save(lb_lattice *h, void *host, size_t bytes);
int lb_checkpoint_load(lb_lattice *h, const void *host, size_t bytes);

/* Populations of n listed cells (cell indices in [0, N)): out[k*19 + i].
 * For sampled checks on lattices too large to copy whole. */
int lb_get_populations_at(lb_lattice *h, const int64_t *cells, int n, double *out);

/* Step-kernel choice.  Variants: 0 library default (measured on GB300:
 * FP32 and Mixed2 one cell per thread, FP64 two cells per thread, 16-bit
 * storage variant 18, or 15 where the row does not fit it); 1 one cell per
 * thread;
 * 2, 3 as 1 with streaming / L2-only cache policies; 4, 5 two cells per
 * thread (even nx); 6, 7 two cells per thread, packed 16-bit registers
 * (16-bit storage, even nx); 8, 9 four cells per thread, packed 16-bit
 * (16-bit storage, nx % 4 == 0); 10, 11, 12 TMA bulk-copy pipeline
 * through shared memory, four / two / one cells per thread (16-bit storage,
 * nx % 16 == 0; block size fixed); 13 two cells per thread collided together
 * in packed FP32 (f32x2) arithmetic (FP32 or 16-bit storage, even nx); 14
 * four cells per thread, collided as two packed pairs (16-bit storage,
 * nx % 4 == 0); 15 as 13 with fewer registers per thread and more warps;
 * 16 as 1 and 17 as 15, each with the bounce-back of cells next to a wall
 * reordered (all neighbour flags read first, then every value load issued
 * together): same results, faster on lattices with many wall cells (porous
 * media), a little slower elsewhere; 16 caps blocks at 128 threads;
 * 18 as 15 with one block per row, the values crossing a warp edge passed
 * through shared memory (nx % 64 == 0 and nx <= 1024, else 15; block size
 * fixed at nx / 2); 19 as 18 with the reordered bounce-back of 17 (else 17).
 * A variant that does not apply to the lattice runs
 * variant 1.  In-place lattices have their own two kernels (see
 * lb_options.inplace: variant 2 two cells per thread, others one).
 * block = threads per block (0 = default; rounded down to whole warps). */
int lb_set_kernel(lb_lattice *h, int variant, int block);

/* Autotuner: time every applicable (variant, block) pair on this lattice
 * (the TMA pipeline variants 10-12 excepted: slower than the register
 * kernels on every lattice measured on GB300; lb_set_kernel still selects
 * them) with `reps` launches each (CUDA events on the lattice's stream), keep the
 * fastest for later lb_step calls and report it (outputs may be NULL).
 * The timed launches read array A and write array B only, so the lattice
 * state is unchanged.  An in-place lattice has no second array: its
 * populations are copied to host memory (malloc'd here, 19*N*sizeof(pop)
 * bytes) before the timed steps and copied back after them, so its state is
 * unchanged too (LB_ENOMEM if the host buffer cannot be had).  Synchronises
 * the stream. */
int lb_autotune(lb_lattice *h, int reps, int *variant, int *block, float *ms_per_step);

/* Totals without any allocation (the paper has no counterpart: it is a
 * service for callers that cannot allocate device memory -- code running
 * inside another framework's memory pool or a fixed memory budget, or a
 * real-time loop where an allocation may block or fail -- and that hold the
 * populations in their own buffers).  Same result as lb_totals.
 *   populations  device, 19 planes of plane_stride >= N elements of the
 *                storage type, each value the deviation f_i - w_i, library
 *                velocity order, plane i holding direction i (the
 *                two-array layout of a lattice with lb_options.inplace = 0).
 *                The arrays of an in-place lattice keep their values in
 *                other places and are not accepted: the totals would be
 *                wrong without any error;
 *   flags        device, N bytes, LB_FLUID/LB_WALL/LB_LID/LB_FARFIELD (the
 *                two low bits are read);
 *   force, u_lid host, 3 doubles each or NULL (= 0);
 *   stream       cudaStream_t or NULL; the call copies the result to host
 *                memory and synchronises the stream, so it must never be
 *                called on a stream that is being captured;
 *   out          host, 5 doubles: mass, momentum x/y/z, count of fluid
 *                cells with non-finite or non-positive density.
 * The reduction's scratch is a static device array of
 * LB_STATIC_MAX_BLOCKS * 6 + 8 doubles (about 58 KB) that every GPU loading
 * the library holds until exit; the kernel strides over the lattice with at
 * most LB_STATIC_MAX_BLOCKS blocks, so any lattice below 2^31 cells fits and
 * larger ones are rejected (LB_EINVAL).  Every call looks up the array's
 * device address (cudaGetSymbolAddress) in the current device's context,
 * so a device reset or a context switch between calls is harmless.  The
 * array is shared by all calls and keeps the last call's values: calls
 * that overlap on the GPU race on it and must be serialised by the caller.
 * Calls no cudaMalloc or cudaFree.  Returns LB_OK, LB_EINVAL, LB_ECUDA, or
 * LB_EDIVERGED (after filling out). */
#define LB_STATIC_MAX_BLOCKS 1216
int lb_totals_static(const void *populations, int64_t plane_stride, const uint8_t *flags,
                     int nx, int ny, int nz, int storage, const double *force,
                     const double *u_lid, void *stream, double *out);

/* ---------------------------------------------------------------------
 * Batches: many independent lattices advanced by shared launches (no
 * counterpart in the paper, which runs one lattice; this is the serving
 * form of the same update).  A batch owns one device pool; each admitted
 * lattice ("slot") keeps its populations resident there with its own
 * size, tau, storage, force, lid and step budget.  lb_batch_step(b, n)
 * advances every slot that still has steps left by up to n steps: per step,
 * one persistent kernel per storage type over all such slots (one thread
 * per cell, the same pull-collide update as lb_step), then a one-block
 * kernel that swaps each slot's A/B arrays and counts its steps down.
 * Groups of 8 steps are replayed from a captured CUDA graph; membership
 * lives in device memory, so the graph stays valid as slots come and go.
 * ------------------------------------------------------------------- */
typedef struct lb_batch lb_batch; /* opaque */

/* Pool bytes one slot of this size, storage and population layout
 * (inplace 0: two arrays, 1: one array, as lb_options.inplace) takes (0 on
 * bad arguments). */
size_t lb_batch_slot_bytes(int nx, int ny, int nz, int storage, int inplace);
/* Device bytes of a batch's fixed area (slot table, work lists, reduction
 * scratch, 16 MiB host-transfer staging) for max_slots slots. */
size_t lb_batch_fixed_bytes(int max_slots);

/* Create a batch with a pool of capacity_bytes (the HBM budget for slots)
 * and up to max_slots (1..65536) slots; the library allocates fixed area +
 * pool with cudaMalloc.  stream: cudaStream_t to issue work on; NULL makes
 * the batch create and own a non-blocking stream (CUDA graphs cannot be
 * captured on the legacy default stream). */
int lb_batch_create(lb_batch **out, size_t capacity_bytes, int max_slots, void *stream);
/* As lb_batch_create, with all device memory from the caller's buffer
 * (256-byte aligned; the pool is what remains after the fixed area). */
int lb_batch_create_in(lb_batch **out, void *device_buffer, size_t bytes, int max_slots, void *stream);

/* Admit a lattice: arguments as lb_create (opt: storage, force, trt_magic
 * and inplace -- an in-place slot keeps one population array, so the pool
 * holds about twice as many; its lb_batch_fetch reads back through the
 * batch's staging area instead of the slot's spare array), plus the number
 * of steps it is to take.  Starts at rest (f = w).  Returns the
 * slot id in *slot.  LB_ENOMEM: it does not fit the pool's free space;
 * LB_EBUSY: all slots in use; LB_EINVAL: bad arguments.  Synchronises. */
int lb_batch_add(lb_batch *b, int nx, int ny, int nz, double tau, const double *u_lid,
                 const uint8_t *flags, const lb_options *opt, int64_t steps, int *slot);
/* Set a slot's remaining step count. */
int lb_batch_set_steps(lb_batch *b, int slot, int64_t steps);
/* Set the step counters of n slots at once (one upload, ordered after the
 * work already queued): used by schedulers that grant step quotas per
 * chunk.  A slot whose counter is 0 is skipped by lb_batch_step.  A slot
 * reported finished by lb_batch_poll may be read back (lb_batch_fetch) or
 * removed only if the caller grants it no further steps. */
int lb_batch_set_steps_many(lb_batch *b, int n, const int *slots, const int64_t *steps);
/* As lb_init_fields, for one slot. */
int lb_batch_init_fields(lb_batch *b, int slot, const double *rho, const double *u);
/* Advance every slot with steps left by up to n steps (asynchronous). */
int lb_batch_step(lb_batch *b, int n);
/* Slots that have taken all their steps and are still admitted: up to max
 * ids into done_slots, their total count in *ndone.  Synchronises. */
int lb_batch_poll(lb_batch *b, int *done_slots, int max, int *ndone);
/* Remaining and taken steps, dims[3], storage of a slot (outputs may be NULL). */
int lb_batch_query(lb_batch *b, int slot, int64_t *remaining, int64_t *done, int *dims, int *storage);
/* As lb_moments / lb_totals / lb_get_populations, for one slot. */
int lb_batch_moments(lb_batch *b, int slot, double *rho, double *u);
int lb_batch_totals(lb_batch *b, int slot, double *mass, double *mom);
int lb_batch_get_populations(lb_batch *b, int slot, double *f);
/* Asynchronous read-back of a finished slot (no steps left): rho (N) and u
 * (3N SoA) into caller host buffers, which must stay valid until
 * lb_batch_fetch_done reports 1 (pinned buffers make the copy truly
 * asynchronous).  Runs on the batch's io stream while queued steps go on;
 * the slot's spare population array is the device-side scratch.
 * LB_EBUSY if the slot still has steps. */
int lb_batch_fetch(lb_batch *b, int slot, double *rho, double *u);
/* 1 when the slot's fetch has completed, 0 while pending, <0 on error. */
int lb_batch_fetch_done(lb_batch *b, int slot);
/* Retire a slot and return its memory to the pool (waits for its fetch;
 * drains queued work only if the slot still had steps). */
int lb_batch_remove(lb_batch *b, int slot);
/* Free pool bytes and free slots (either may be NULL). */
int lb_batch_free_bytes(lb_batch *b, size_t *free_bytes, int *free_slots);
/* Wait for the batch's stream. */
int lb_batch_sync(lb_batch *b);
/* Release the batch (and its memory if the library allocated it). */
int lb_batch_destroy(lb_batch *b);
/* Description of the last batch failure on the calling thread. */
const char *lb_batch_last_error(void);

/* Self-test of the bounded device-side wait (no counterpart in the paper):
 * the TMA pipeline step kernels (variants 10-12) wait on shared-memory
 * barriers for their bulk copies, and each wait gives up after a deadline
 * and reports (LB_ETIMEOUT from lb_sync) rather than hang the GPU.  This
 * call runs that same wait on a barrier that nothing signals, with a
 * deadline of `seconds` (0 < seconds <= 5), on `stream` (cudaStream_t or
 * NULL), and synchronises it.  Returns LB_ETIMEOUT when the wait gave up
 * as designed (the expected result), LB_EINVAL for a bad deadline,
 * LB_ENOMEM / LB_ECUDA on CUDA failures.  The device context stays usable. */
int lb_selftest_wait(double seconds, void *stream);

/* Halo exchange of a z-slab lattice (lb_options.halo_z = 1).  A step pulls
 * the five populations with c_z = +1 into the lowest own plane (z = 1)
 * from the ghost plane z = 0, and the five with c_z = -1 into the highest
 * own plane (z = nz - 2) from the ghost plane z = nz - 1; nothing else of
 * a ghost plane is read.  So between steps each slab sends the rank below
 * its lowest own plane's c_z = -1 populations and the rank above its
 * highest own plane's c_z = +1 populations (periodic in z: the last rank's
 * "above" is rank 0), and writes what it receives into its ghost planes.
 * A message is those five populations' planes back to back, in the
 * library's velocity order: 5 * nx * ny values of the storage type,
 * lb_halo_bytes() bytes (0 for a lattice without ghost planes).
 *   lb_halo_pack    send_lo <- z = 1, c_z = -1 (for the rank below);
 *                   send_hi <- z = nz - 2, c_z = +1 (for the rank above);
 *   lb_halo_unpack  ghost z = 0, c_z = +1 <- recv_lo (the rank below's
 *                   send_hi); ghost z = nz - 1, c_z = -1 <- recv_hi (the
 *                   rank above's send_lo).
 * Buffers are device pointers owned by the caller (suitably aligned for the
 * storage type).  Both calls are asynchronous on the lattice's stream and
 * act on the current state (after the last lb_step).  Done after every
 * step, the slabs together take bitwise the steps of the whole lattice.
 * Errors: LB_EINVAL (NULL, or no ghost planes), LB_ECUDA. */
size_t lb_halo_bytes(lb_lattice *h);
int lb_halo_pack(lb_lattice *h, void *send_lo, void *send_hi);
int lb_halo_unpack(lb_lattice *h, const void *recv_lo, const void *recv_hi);

/* Wait for all work issued on the lattice's stream.  Returns LB_ETIMEOUT
 * (and clears the condition) if a kernel's bounded wait on an asynchronous
 * copy gave up since the last check. */
int lb_sync(lb_lattice *h);

/* Query: dims[3], storage, steps taken since create. */
int lb_query(lb_lattice *h, int *dims, int *storage, int64_t *steps);

/* Release the lattice (frees library-allocated device memory).  Safe on
 * NULL. */
int lb_destroy(lb_lattice *h);

/* Static description of a status code. */
const char *lb_status_string(int status);

/* Description of the last failure on the calling thread ("" if none). */
const char *lb_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* LBGB_H */
