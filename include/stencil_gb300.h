/*
 * stencil_gb300.h -- C ABI of the GB300 (sm_103a) stencil sweep library.
 *
 * The operations are those of Malas, Ltaief, Hager, Keyes, "Towards energy
 * efficiency and maximum computational intensity for stencil algorithms using
 * wavefront diamond temporal blocking" (arXiv:1410.5561):
 *   - Section I (problem statement): a sweep updates every interior point of a
 *     3D grid from its neighbours' previous values; sweeps repeat over many
 *     time steps, Jacobi-style, with two domain-sized arrays (Section I-A).
 *   - Listing 1: 7-point constant-coefficient stencil (scalars c0, c1).
 *   - Listing 2: 7-point variable-coefficient stencil (7 arrays C0..C6;
 *     C1 +x, C2 -x, C3 +y, C4 -y, C5 +z, C6 -z).
 *   - Listing 3: 25-point (radius 4) axis-symmetric variable-coefficient
 *     stencil (13 arrays; C00 centre, C(3(d-1)+a+1) weighs the pair at
 *     distance d on axis a = x, y, z).
 *   - Section II-A / III: the temporally blocked (wavefront diamond) schedule,
 *     selected with stencil_set_tuning(STENCIL_BLOCKED, ...).
 *
 * Conventions shared by every entry point:
 *   - Return value: STENCIL_OK (0) or a negative stencil_status. Nothing
 *     throws across the ABI. stencil_strerror() names a status.
 *   - Streams: every device operation is enqueued on the cudaStream_t given
 *     to stencil_create (0 = legacy default stream) and is asynchronous with
 *     respect to the host unless stated otherwise.
 *   - Memory: the library never allocates device memory. The caller allocates
 *     the two field arrays, the coefficient arrays and the workspace (sizes
 *     from stencil_layout_of / stencil_workspace_bytes) and keeps them alive
 *     until the work enqueued on them has finished. Device pointers must be
 *     16-byte aligned.
 *   - Grid layout (element index, shared by the field and coefficient arrays
 *     of one grid; R = halo width = stencil radius):
 *       interior point (i, j, k), 0 <= i < nx, 0 <= j < ny, 0 <= k < nz, is at
 *       ((k + R) * pitch_y + (j + R)) * pitch_x + x_offset + i
 *     with pitch_y = ny + 2R and planes = nz + 2R. Cells that are not interior
 *     form the Dirichlet halo (plus row padding); stencil_set_field fills them.
 *   - Dense arrays passed to set_field / set_coeffs / get_field hold the
 *     interior only, shaped (nz, ny, nx), x fastest, in the array's dtype.
 */
#ifndef STENCIL_GB300_H
#define STENCIL_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct stencil_grid* stencil_t; /* opaque, owned by the library */

enum stencil_kind { STENCIL_7PT_CONST = 0, STENCIL_7PT_VAR = 1, STENCIL_25PT_VAR = 2 };
enum stencil_dtype { STENCIL_F32 = 0, STENCIL_F64 = 1, STENCIL_BF16 = 2 };
enum stencil_scheme { STENCIL_PLAIN = 0, STENCIL_BLOCKED = 1, STENCIL_AUTO = 2, STENCIL_WAVEFRONT = 3 };
/* Where a dense array passed to set_coeffs / set_field / get_field lives.
 * STENCIL_HOST: host memory; the call waits for its copy when the caller needs
 * the data back (page-locked memory is moved by the library's copy kernel,
 * pageable memory by a pitched DMA). STENCIL_DEVICE: device memory.
 * STENCIL_HOST_ASYNC (set_field / get_field only): page-locked host memory,
 * moved by the copy engines (a pitched DMA) on the handle's stream without
 * waiting and without occupying SMs, so that the transfer can overlap a sweep
 * running on another stream; the caller keeps the host array alive and
 * unchanged (set_field) or unread (get_field) until the stream has passed the
 * copy. Pageable memory is rejected with STENCIL_EINVAL. */
enum stencil_where { STENCIL_HOST = 0, STENCIL_DEVICE = 1, STENCIL_HOST_ASYNC = 2 };
enum stencil_array { STENCIL_FIELD_ARRAY = 0, STENCIL_COEF_ARRAY = 1, STENCIL_GRAD_ARRAY = 2 };

enum stencil_status {
    STENCIL_OK = 0,
    STENCIL_EINVAL = -1,   /* bad argument: shape, dtype, pointer alignment, tuning */
    STENCIL_ENOSMEM = -2,  /* blocked tuning needs more shared memory than one CTA may have */
    STENCIL_ETIMEOUT = -3, /* a bounded device-side wait gave up (see stencil_status) */
    STENCIL_ECUDA = -4,    /* a CUDA runtime call failed */
    STENCIL_EUNBOUND = -5, /* arrays not bound yet */
    STENCIL_ENOTSUP = -6   /* combination not implemented */
};

/* Blocked-schedule tunables (Section II-A, III-A): dw = diamond width D_w
 * along y (a multiple of 2R with D_w/R - 1 <= 64 time levels), nf = frontlines
 * N_F (z planes per time level per wavefront step: 1 or 2), warps = warps per
 * CTA (1..16; the CTA is the thread group that shares one extruded diamond),
 * xtile = x columns one CTA owns (a multiple of 16 bytes' worth of field
 * elements, at most 4096; the leading-dimension tile of Section III-A). A row
 * wider than xtile is split into tiles that run as one thread-block cluster
 * (at most 16); for the 7-point stencils the first and last tiles of a row
 * are wider by the trapezoid overlap they need on one side only. Tunings whose
 * rings exceed the shared memory of one CTA, whose items exceed 4 per warp, or
 * whose diamonds hold more than 256 computed or loaded rows per x-tile chunk,
 * are rejected (STENCIL_ENOSMEM / STENCIL_EINVAL). */
typedef struct {
    int dw;
    int nf;
    int warps;
    int xtile;
} stencil_tuning;

typedef struct {
    int radius;        /* R */
    int elem_bytes;    /* bytes per element of this array */
    int x_offset;      /* elements before interior x = 0 in each row */
    int pitch_x;       /* elements per row */
    int pitch_y;       /* rows per plane (ny + 2R) */
    int planes;        /* nz + 2R */
    size_t bytes;      /* pitch_x * pitch_y * planes * elem_bytes */
} stencil_layout;

/* Create a grid handle. kind: stencil_kind. nx, ny, nz >= 1 interior sizes.
 * field_dtype: STENCIL_F32 or STENCIL_F64. coef_dtype: equal to field_dtype,
 * or STENCIL_BF16 with an FP32 field (coefficients stored in BF16, widened
 * exactly to FP32 in registers); ignored for STENCIL_7PT_CONST. cuda_stream:
 * a cudaStream_t (may be NULL). *out receives the handle. */
int stencil_create(stencil_t* out, int kind, int nx, int ny, int nz, int field_dtype, int coef_dtype,
                   void* cuda_stream);

/* Layout of the field (which = STENCIL_FIELD_ARRAY), of one coefficient array
 * (STENCIL_COEF_ARRAY) or of one FP64 coefficient-gradient array
 * (STENCIL_GRAD_ARRAY, same element index, 8-byte elements) of this grid. */
int stencil_layout_of(stencil_t h, int which, stencil_layout* out);

/* Bytes of device workspace the handle can use (caller-allocated, passed to
 * bind). With a workspace bound, the blocked schedule runs as one persistent
 * launch whose thread-block clusters walk the dependency-ordered list of
 * diamond tiles (Section II-A's queue of ready diamonds; the tiles are derived
 * on the device, the workspace holds their completion counters and the
 * status word read by stencil_status); without one (NULL) it runs one launch
 * per diamond row and has nothing to wait on. */
size_t stencil_workspace_bytes(stencil_t h);

/* Bind caller-owned device arrays: field_a, field_b (field layout; ping-pong
 * pair), coef[0..n_c-1] (coefficient layout; NULL for 7PT_CONST), workspace
 * (stencil_workspace_bytes, may be NULL when that is 0). Borrowed, not owned. */
int stencil_bind(stencil_t h, void* field_a, void* field_b, void* const* coef, void* workspace);

/* Coefficients. 7PT_CONST: scalars = {c0, c1} (host), arrays ignored.
 * Variable kinds: arrays[m] = dense interior array m (coef dtype), on the host
 * (where = STENCIL_HOST) or device (STENCIL_DEVICE); copied into the bound
 * coefficient arrays, whose halo is set to 0. */
int stencil_set_coeffs(stencil_t h, const double* scalars, const void* const* arrays, int where);

/* Initial field u_0: dense interior src (field dtype, host or device). Both
 * field arrays get every non-interior cell set to halo_value (the Dirichlet
 * value, never written again by a sweep: the fill is skipped when the bound
 * arrays already hold this value there from an earlier set_field); src goes to
 * the interior of field_a, which becomes the current array (time 0). */
int stencil_set_field(stencil_t h, const void* src, double halo_value, int where);

/* Select the schedule used by run(): STENCIL_PLAIN (one launch per step;
 * tuning->nf = 2 makes every thread copy the loads of its next two planes
 * into shared memory ahead of use, 0 loads each plane when it is updated,
 * NULL: 2 for the 25-point stencil with BF16 coefficients, where it measured
 * faster, else 0; other tuning fields ignored),
 * STENCIL_WAVEFRONT (wavefront temporal blocking through L2: Section II-A's
 * thread group sharing one cache block, here every CTA of the GPU sharing the
 * L2; each launch advances h = dw / (2R) steps: time level l of the pass
 * sweeps z chunks of nf planes (nf >= R) two chunks behind level l-1, on xy
 * tiles of 32 vectors by `warps` rows (4, 8 or 16, >= R), the CTAs waiting on
 * bounded completion flags; xtile = 2 copies every load two planes ahead into
 * shared memory where nf >= R + 2 and it fits, 0 does not; xtile = 4 (25-point
 * stencil, FP32 field, 8 rows) stages the field's tile planes with their halos
 * in shared memory by tensor copies issued by one producer warp, and each
 * thread's coefficient vectors by its own asynchronous copies a plane or more
 * ahead, where every (level, tile) CTA fits on the GPU at once (else the
 * column walk runs); NULL: h = 2,
 * 8-plane chunks, 8 rows, no copies ahead; needs a bound workspace, else
 * STENCIL_EINVAL; bit-identical to the plain sweep), or
 * STENCIL_BLOCKED with *tuning (NULL: library default: D_w = 8R, N_F = 2 where it
 * fits (1 for the 7-point variable stencil with FP32 coefficients), 16 warps for
 * R = 1, the widest x tile whose rows fit one warp of vectors), or
 * STENCIL_AUTO (plain for FP64 fields and the 25-point stencil, where the plain sweep
 * measured faster on GB300; else the default blocked tuning when it fits, else plain).
 * Returns STENCIL_ENOSMEM / STENCIL_EINVAL for an infeasible blocked tuning. */
int stencil_set_tuning(stencil_t h, int scheme, const stencil_tuning* tuning);

/* Advance the current field by T >= 0 Jacobi steps (Listings 1-3 applied T
 * times). Asynchronous on the handle's stream: it only enqueues kernels and
 * memsets (no host copy, no wait), so it can be captured in a CUDA graph.
 * Afterwards field_a holds u_T if (initial parity + T) is even, field_b
 * otherwise (see stencil_parity). A persistent blocked launch whose dependency
 * wait runs out of its limit cannot hang: it sets the status word (see
 * stencil_status) and the field is then undefined. */
int stencil_run(stencil_t h, int T);

/* Device error/timeout word of the handle (synchronous: waits for the
 * handle's stream). Returns STENCIL_OK, STENCIL_ETIMEOUT if a persistent
 * blocked launch since the last stencil_set_field (or stencil_bind) gave up a
 * dependency wait (the field is then undefined until the next set_field),
 * STENCIL_ECUDA on an asynchronous CUDA error, or STENCIL_EINVAL. */
int stencil_status(stencil_t h);

/* Bound on the spin iterations of one dependency wait of the persistent
 * blocked schedule (about 0.15 us each; default 2^24, a few seconds). */
int stencil_set_wait_limit(stencil_t h, unsigned spins);

/* Test hook: in later persistent blocked launches, tile `tile` of the plan
 * also waits on a flag that no tile sets, so that its wait runs out and
 * stencil_status reports STENCIL_ETIMEOUT; -1 removes the stall. A tile index
 * beyond the plan's tiles has no effect. */
int stencil_inject_stall(stencil_t h, int tile);

/* 0 if field_a holds the current time level, 1 if field_b does. */
int stencil_parity(stencil_t h);

/* Copy the current field's interior to dense dst (host or device). With
 * where = STENCIL_HOST the call waits for the stream. */
int stencil_get_field(stencil_t h, void* dst, int where);

/* ---- Adjoint (reverse mode) of the variable-coefficient sweeps (Listings 2, 3).
 * For a cotangent lambda_T of u_T (for L = 0.5 ||u_T - target||^2 it is
 * u_T - target): lambda_t = A^T lambda_{t+1}, dL/du_0 = lambda_0 and
 * dL/dC_m(p) = sum_t lambda_{t+1}(p) x (the field value multiplying C_m(p) in
 * step t). States are kept at every k-th step (k = ckpt_every, or ceil(sqrt(T))
 * when ckpt_every <= 0) and the steps in between are recomputed during the
 * backward pass. The coefficient gradients accumulate in FP64. */

/* Workspace bytes both calls below need for (T, ckpt_every): (ceil(T/k) + 2k + 1)
 * field arrays (the checkpoints, one segment's states and its k + 1 cotangents). */
size_t stencil_adjoint_workspace_bytes(stencil_t h, int T, int ckpt_every);

/* Like stencil_run(h, T), and stores the checkpoints u_0, u_k, u_2k, ... in
 * workspace (device, stencil_adjoint_workspace_bytes long). Uses the schedule
 * chosen by stencil_set_tuning for the forward steps. STENCIL_ENOTSUP for the
 * 7-point constant-coefficient stencil. */
int stencil_run_checkpointed(stencil_t h, int T, int ckpt_every, void* workspace, size_t workspace_bytes);

/* Backward pass after stencil_run_checkpointed(h, T, ckpt_every, workspace, ...)
 * with the same coefficients. Per checkpoint segment (k steps): the states are
 * recomputed from the checkpoint (with STENCIL_WAVEFRONT tuned: by one
 * temporally blocked pass whose time levels each write their own state array;
 * otherwise one plain step per state), the k cotangents lambda_t follow (with
 * STENCIL_WAVEFRONT tuned: by one temporally blocked pass of transposed steps,
 * each level writing its own cotangent array; otherwise one transposed step
 * each), and the coefficient gradients of all k steps are then
 * accumulated in one pass (each FP64 gradient array read and written once per
 * segment, not once per step; the FP64 fma sequence per element is unchanged). lambda_T: device, field layout, the cotangent of
 * u_T on the interior (its halo is ignored). g_u0: device, field layout; gets
 * dL/du_0 on the interior and 0 elsewhere. g_coef[m], m < n_c: device, gradient
 * layout (STENCIL_GRAD_ARRAY, FP64); overwritten with dL/dC_m on the interior and
 * 0 elsewhere. Asynchronous on the handle's stream; the workspace's checkpoints
 * are read, its other buffers overwritten. */
int stencil_run_adjoint(stencil_t h, int T, int ckpt_every, const void* lambda_T, void* g_u0, void* const* g_coef,
                        void* workspace, size_t workspace_bytes);

/* Shared-memory bytes per CTA the blocked kernel needs for a tuning (0 if the
 * tuning is malformed); the device limit is cudaDevAttrMaxSharedMemoryPerBlockOptin. */
size_t stencil_blocked_smem_bytes(stencil_t h, const stencil_tuning* tuning);

/* Number of kernels this handle has launched so far (sweeps, fills), into *out. */
int stencil_launch_count(stencil_t h, long long* out);

/* Number of STENCIL_WAVEFRONT passes (Section II-A's thread group, see
 * stencil_set_tuning) this handle has run with tile copies into shared memory
 * (tuning xtile = 4), into *out; the passes that fell back to the column walk
 * are not counted. */
int stencil_tile_copy_passes(stencil_t h, long long* out);

/* Host transfers, no counterpart in the paper: copy `bytes` from src to dst with
 * the SMs' own 16-byte loads and stores, by `ctas` CTAs (1..1024) of 1024 threads,
 * asynchronously on cuda_stream. Either pointer may be device memory of the
 * current device, managed memory or page-locked host memory mapped for it;
 * anything else (pageable host memory, another device's memory) is refused
 * with STENCIL_EINVAL before any access. With few CTAs the
 * copy streams host memory over the link on the SMs a running sweep leaves free,
 * instead of on the copy engines. Both pointers 16-byte aligned and bytes a
 * multiple of 16, else STENCIL_EINVAL; the caller keeps both buffers alive and
 * untouched until the stream has passed the copy. */
int stencil_copy(void* dst, const void* src, size_t bytes, int ctas, void* cuda_stream);

/* Measurement support, no counterpart in the paper: time a grid-filling kernel
 * of independent dependent-FMA chains in dtype (STENCIL_F32 or STENCIL_F64) on
 * cuda_stream and return its duration (*seconds) and flop count (*flops, two
 * per FMA). scratch: device buffer of at least 65536 bytes. Synchronous. */
int stencil_probe_fma(int dtype, int iters, void* scratch, void* cuda_stream, double* seconds, double* flops);

/* ---- Batch: many independent grids advanced by one persistent launch.
 * Every grid runs the blocked schedule (Section II-A) with one tile covering
 * its whole x extent; tiles of all grids sit in one dependency-ordered list
 * and the CTAs of one persistent kernel pop them from an atomic counter, each
 * waiting (with a bounded spin) until the diamonds below it have published
 * their results: the GPU form of the paper's queue of ready diamond tiles. */
typedef struct stencil_batch* stencil_batch_t; /* opaque, owned by the library */

/* Plan a batch: grids[q] (bound, same kind and dtypes) advances by T[q] >= 0 steps
 * per launch. tuning: dw, nf (1 or 2) and warps are used for every grid; xtile is
 * ignored. STENCIL_EINVAL if a grid cannot use the tuning. */
int stencil_batch_create(stencil_batch_t* out, const stencil_t* grids, const int* T, int n,
                         const stencil_tuning* tuning);

/* Device workspace bytes the batch needs (descriptors, tile list, counters). */
size_t stencil_batch_workspace_bytes(stencil_batch_t b);

/* Number of tiles one launch processes. */
int stencil_batch_item_count(stencil_batch_t b);

/* Upload the plan into workspace (device, caller-owned, 16-byte aligned,
 * stencil_batch_workspace_bytes long); synchronous on cuda_stream, so it must
 * not be called on a capturing stream (STENCIL_EINVAL). The grids' current
 * parities are recorded here. */
int stencil_batch_bind(stencil_batch_t b, void* workspace, void* cuda_stream);

/* Enqueue one launch (a counter reset and the persistent kernel) on cuda_stream;
 * it can be captured in a CUDA graph. Each grid advances by its T; the handles'
 * parities are updated by this call. Replays of a captured graph advance the
 * grids again without passing through this call: afterwards call
 * stencil_batch_sync_parity before using the grids. */
int stencil_batch_launch(stencil_batch_t b, void* cuda_stream);

/* Kernels this batch has enqueued so far. */
int stencil_batch_launch_count(stencil_batch_t b, long long* out);

/* Status of the last launch (synchronous): *status = STENCIL_OK, or
 * STENCIL_ETIMEOUT when a dependency wait gave up (the grids' contents are then
 * undefined). */
int stencil_batch_status(stencil_batch_t b, int* status);

/* Copy the device-side parities (which array holds each grid's current time
 * level) into the grid handles. Synchronous. */
int stencil_batch_sync_parity(stencil_batch_t b);

/* Bound on the spin iterations of a dependency wait (about 0.2 us each; the
 * default, 2^24, is a few seconds). */
int stencil_batch_set_wait_limit(stencil_batch_t b, unsigned spins);

/* Test hook: make tile `item` wait on a completion flag that no tile ever sets,
 * so that its wait runs out and the launch reports STENCIL_ETIMEOUT. */
int stencil_batch_inject_stall(stencil_batch_t b, int item);

int stencil_batch_destroy(stencil_batch_t b);

/* Run a batch once without any device allocation by the caller or the library.
 * The paper has no counterpart: this serves callers that cannot allocate device
 * memory for a workspace, for example code whose device memory is all owned by
 * another allocator (a framework's caching allocator, a pre-sized arena), or a
 * latency-critical loop that must not call cudaMalloc because it can
 * synchronise the device.
 * Same meaning as stencil_batch_create + stencil_batch_bind + stencil_batch_launch
 * with the same arguments (grids, T, n, tuning), but the batch's scratch (grid
 * descriptors, tile list, dependency flags, status) lives in a fixed 4 MiB
 * array in device memory owned by the library, which every GPU that loads the
 * library holds until the process exits. A batch whose scratch would exceed
 * 4 MiB is rejected with STENCIL_EINVAL before anything is launched. The
 * grids' arrays are the caller's, as usual, and must be on the current device,
 * as must cuda_stream (else STENCIL_EINVAL). The call is synchronous: it
 * uploads the plan (waiting for cuda_stream), enqueues the launch on
 * cuda_stream and updates the grids' parities; if status_out is not NULL it
 * also waits for the launch and stores STENCIL_OK or STENCIL_ETIMEOUT there.
 * It must never be called on a stream that is capturing a CUDA graph (it
 * returns STENCIL_EINVAL there without touching the capture).
 * Every call looks up the array's device address on the current device.
 * All calls share the one array and it keeps the last call's contents; every
 * call rewrites what it needs and resets its counters, but calls whose work
 * overlaps on the GPU (different streams, or a call enqueued before the
 * previous one has finished on another stream) race on it, and so do calls
 * made at the same time from several host threads, even on one stream (one
 * call's upload can land between another's upload and its launch): callers
 * must serialise their calls. */
int stencil_batch_run_noalloc(const stencil_t* grids, const int* T, int n, const stencil_tuning* tuning,
                              void* cuda_stream, int* status_out);

/* Make the handle's later calls enqueue their work on cuda_stream (NULL: the
 * legacy default stream). Ordering against work already enqueued on the
 * previous stream is the caller's (events). */
int stencil_set_stream(stencil_t h, void* cuda_stream);

/* Wait for the handle's stream; returns STENCIL_ECUDA on an asynchronous error
 * and STENCIL_ETIMEOUT when the status word is set (as stencil_status). */
int stencil_sync(stencil_t h);

/* Static description of a status code. */
const char* stencil_strerror(int status);

/* Release the handle (not the caller's arrays). */
int stencil_destroy(stencil_t h);

#ifdef __cplusplus
}
#endif

#endif /* STENCIL_GB300_H */
