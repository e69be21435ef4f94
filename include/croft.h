/*
 * croft.h - C ABI of the GB300 3D complex-to-complex FFT library (libcroft.so).
 *
 * The operation (paper Sec. 2.1):
 *   forward,  Eq. (1): Y(k) = sum_j X(j) exp(-2 pi i (kx jx/Nx + ky jy/Ny + kz jz/Nz))
 *   backward, Eq. (2): the same sum with exponent sign +.  Eq. (2) prints a
 *             1/(Nx Ny Nz) factor; this library does NOT apply it (both
 *             directions unnormalised, so backward(forward(X)) = Nx*Ny*Nz * X).
 * computed as the paper's row-column method (Sec. 4.1, steps 1-9): batched 1D
 * FFTs along each axis with the data rearrangement between axes fused into the
 * FFT passes, and the result returned in the input layout (Sec. 4.2, last
 * sentence).
 *
 * Data layout (every entry point): a grid of shape (nx, ny, nz) in C order, z
 * contiguous (stride 1), y with stride nz, x with stride ny*nz; elements are
 * complex64 stored as interleaved {float re, float im} (8 bytes).
 *
 * Pointers named `in` / `out` are DEVICE pointers (cudaMalloc, torch CUDA
 * tensors, ...) owned by the caller, 16-byte aligned.  `in == out` (in place)
 * is allowed; any other overlap of the two ranges is rejected.  `in` is not
 * modified unless it equals `out`.
 *
 * Streams are passed as `void*` holding a cudaStream_t (NULL = the legacy
 * default stream).  Execution is asynchronous and stream-ordered: no exec call
 * synchronises the device.  Launch failures are returned as CROFT_ERR_CUDA.
 *
 * Thread safety: distinct plans may be used concurrently from any threads and
 * streams.  One plan may have at most one exec in flight at a time.
 *
 * There is no CPU fallback: without a usable sm_103 device plan creation
 * fails with CROFT_ERR_CUDA.
 */
#ifndef CROFT_H_
#define CROFT_H_

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct croft_plan_s* croft_plan; /* opaque, owned by the library */

typedef enum {
    CROFT_C2C_F32 = 0,           /* complex64 in/out, FP32 CUDA-core butterflies */
    CROFT_C2C_F32_TC_BF16X3 = 1, /* complex64 in/out, a radix-16 stage on tensor cores
                                    (split bf16 hi+lo operands, FP32 accumulate) */
    CROFT_C2C_F64 = 2,           /* complex128 in/out (16-byte elements), FP64 butterflies and
                                    twiddles: the paper's double complex (Sec. 5).  Axes: powers of
                                    two up to 1024 and 3, 5, 6, 10, 12, 15, 48, 60, 96, 120; three-pass
                                    schedule; single-grid plans only */
    CROFT_C2C_F32_TC_FP16X3 = 3  /* complex64 in/out, a radix-16 stage on tensor cores with split
                                    fp16 hi+lo operands (~22 significant bits), each butterfly
                                    scaled by a power of two into fp16's range first, FP32
                                    accumulate */
} croft_dtype;
/* Tensor-core dtypes (CROFT_C2C_F32_TC_*): every axis whose length has a factor 16 runs its
 * first stage, a radix-16 one, as a split-operand GEMM on the tensor cores and the rest of its
 * schedule on the CUDA cores (axes of 16 .. 1024 points; a longer one makes plan creation fail
 * with CROFT_ERR_UNSUPPORTED_SIZE rather than fall back to FP32); an axis without a factor 16
 * has no radix-16 stage and runs on the CUDA cores.
 * croft_plan_tc_axes reports which axes run on the tensor cores. */

typedef enum {
    CROFT_OK = 0,
    CROFT_ERR_INVALID_ARG = 1,       /* null/misaligned pointer, partial overlap, bad enum */
    CROFT_ERR_UNSUPPORTED_SIZE = 2,  /* an axis outside 1..4096 or not of the form 2^a 3^b 5^c */
    CROFT_ERR_OOM = 3,               /* a device or host allocation failed */
    CROFT_ERR_CUDA = 4,              /* CUDA runtime error (no device, launch failure, ...) */
    CROFT_ERR_TIMEOUT = 5            /* a bounded device-side wait gave up (batched form) */
} croft_status;

/* Human-readable name of a status code (static string, never NULL). */
const char* croft_status_string(croft_status s);

/*
 * croft_plan_create - plan a single (nx, ny, nz) transform on the current device.
 *
 * Paper: the single reusable 1D plan covering all pencils ("option 4",
 * Sec. 5.1) and the three-axis schedule of Sec. 4.1.  Factorises each axis
 * into radix 16/8/4/2/15/9/5/3 stages (the odd factors in the fewest
 * stages of at most 16 points), builds twiddle tables
 * w = exp(-2 pi i r/n) in float64 with exact integer reduction of r and rounds
 * them to float32, and uploads them.
 *
 *   out   : receives the plan (set to NULL on failure).
 *   nx,ny,nz : axis lengths, each 1..4096 and 2^a 3^b 5^c.  A length-1 axis
 *           is the identity.
 *   dtype : CROFT_C2C_F32, CROFT_C2C_F32_TC_BF16X3, CROFT_C2C_F32_TC_FP16X3 or
 *           CROFT_C2C_F64.
 * Returns CROFT_OK, CROFT_ERR_INVALID_ARG (out NULL, bad dtype),
 * CROFT_ERR_UNSUPPORTED_SIZE, CROFT_ERR_OOM or CROFT_ERR_CUDA.
 * The environment variable CROFT_LOG=1 prints the chosen schedule to stderr.
 */
croft_status croft_plan_create(croft_plan* out, int nx, int ny, int nz, croft_dtype dtype);

/*
 * Pass schedules.
 *   CROFT_SCHEDULE_THREE_PASS : one pass per axis (z, y, x): the paper's three
 *       1D-FFT steps (Sec. 4.1, steps 1, 5, 9) with each rearrangement fused
 *       into the next pass; the grid crosses HBM three times per transform.
 *   CROFT_SCHEDULE_PLANE_FUSED : steps 1-5 as one pass (the 2D FFT of every
 *       yz-plane, one plane per thread-block cluster, the column all-to-all
 *       done through distributed shared memory), then the x pass; the grid
 *       crosses HBM twice.  Available for the plane shapes the library
 *       instantiates (ny x nz in {32x32, 64x64, 128x128, 256x256, 384x384});
 *       other shapes give CROFT_ERR_UNSUPPORTED_SIZE.
 *   CROFT_SCHEDULE_SLAB_L2 : steps 1-5 slab by slab: for each slab of x-planes
 *       (about CROFT_SLAB_MB MiB, default 16) the z pass then the y pass, so the
 *       y pass reads the z pass's output from the L2 cache and the grid crosses
 *       HBM about twice per transform; then the x pass.  The paper's chunking of
 *       the transposes into K pieces (Sec. 5.1), here sized to the cache.
 *   CROFT_SCHEDULE_AUTO : THREE_PASS (measured faster on GB300 so far); with the
 *       environment variable CROFT_SCHEDULE_AUTO_FUSED=1, PLANE_FUSED where available.
 *   CROFT_SCHEDULE_TUNED : measured at plan creation (the paper tunes its options 1-4 and
 *       the chunk count K by hand, Sec. 5.1): for each column pass of a 270..512-point axis
 *       the kernel (16- or 8-column tile, near-equal or radix-16-first power-of-two split,
 *       or the tensor-copy ring kernel), then the schedule (three-pass with those kernels,
 *       slab, fused plane), each timed on the device; the fastest is kept and cached on
 *       disk (CROFT_TUNE_CACHE, default ~/.croft_tune_cache.txt) keyed by shape, dtype, GPU
 *       and CUDA version.  Needs two grid-sized scratch buffers during creation (without
 *       them it plans by the rules); croft_plan_describe reports the choice.  Tensor-core
 *       and complex128 plans have nothing to choose and plan THREE_PASS.
 */
typedef enum {
    CROFT_SCHEDULE_AUTO = 0,
    CROFT_SCHEDULE_THREE_PASS = 1,
    CROFT_SCHEDULE_PLANE_FUSED = 2,
    CROFT_SCHEDULE_SLAB_L2 = 3,
    CROFT_SCHEDULE_TUNED = 4
} croft_schedule;

/*
 * croft_plan_tc_axes - which axes of a single-grid plan run a radix-16 stage on the
 * tensor cores: bit a set for axis a (0 = x, 1 = y, 2 = z).  0 for FP32 / FP64 plans, batched
 * plans and NULL.  The library's own statement of a plan's per-axis arithmetic (the
 * precision of every result of a tensor-core plan follows from it).
 */
int croft_plan_tc_axes(croft_plan plan);

/* croft_plan_create with an explicit schedule (same arguments and errors;
 * CROFT_ERR_INVALID_ARG for an unknown schedule). */
croft_status croft_plan_create_schedule(croft_plan* out, int nx, int ny, int nz, croft_dtype dtype,
                                        croft_schedule schedule);

/*
 * Batched form: `count` independent grids of (possibly) different shapes,
 * e.g. the per-system PME meshes of an ensemble.  Each grid is transformed
 * exactly as by a single-grid plan of its shape (Eq. 1 / Eq. 2 unnormalised,
 * same layout rules); the grids share launches.
 *
 * croft_plan_create_batched_mode:
 *   dims  : host array of 3*count ints, grid g is (dims[3g], dims[3g+1], dims[3g+2]).
 *   mode  : CROFT_BATCH_ONE_LAUNCH - every tile of every pass of every grid in
 *               one persistent kernel launch (work counter, per-grid pass
 *               dependencies as bounded device-side waits); recorded in a CUDA
 *               graph per direction.
 *           CROFT_BATCH_PER_PASS  - the same work in three launches (z, y, x) of
 *               one CTA per tile, ordered by kernel boundaries; CUDA graph per
 *               direction.
 *           CROFT_BATCH_PER_GRID  - one single-grid plan per grid, launched in turn.
 *           CROFT_BATCH_GROUPED   - per pass, one launch per distinct axis length,
 *               covering the tiles of every grid with that length (the
 *               single-grid pass kernel specialised on the length, with a
 *               per-CTA grid lookup); the launches of one pass run concurrently
 *               and the passes are ordered by the edges of a CUDA graph per
 *               direction.
 *           CROFT_BATCH_AUTO      - time the four on scratch buffers at creation
 *               and keep the fastest; the choice is cached in the text file named
 *               by $CROFT_TUNE_CACHE (default $HOME/.croft_tune_cache.txt), keyed by
 *               the sizes, GPU name and CUDA runtime version.  CROFT_TUNE=off skips
 *               the timing and uses GROUPED (the fastest in every measurement so far).
 *   Grids with an axis > 128 always run on their own single-grid plan.
 * croft_plan_create_batched: the same with CROFT_BATCH_AUTO.
 * Paper: many 1D FFTs under one plan ("option 4") and the chunk count K
 * trading call count against chunk size (Sec. 5.1).
 * Returns CROFT_OK, CROFT_ERR_INVALID_ARG (count < 1, NULL dims/out, bad mode
 * or dtype), CROFT_ERR_UNSUPPORTED_SIZE (an axis, or the tensor-core dtype),
 * CROFT_ERR_OOM or CROFT_ERR_CUDA.  The plan owns a small device workspace
 * (work counters, per-grid completion counts, status word) and pinned host
 * memory for the grids' descriptors.
 */
typedef enum {
    CROFT_BATCH_AUTO = 0,
    CROFT_BATCH_ONE_LAUNCH = 1,
    CROFT_BATCH_PER_PASS = 2,
    CROFT_BATCH_PER_GRID = 3,
    CROFT_BATCH_GROUPED = 4
} croft_batch_mode;

croft_status croft_plan_create_batched(croft_plan* out, int count, const int* dims, croft_dtype dtype);
croft_status croft_plan_create_batched_mode(croft_plan* out, int count, const int* dims, croft_dtype dtype,
                                            croft_batch_mode mode);

/*
 * croft_exec_batched_forward / _backward: in and out are HOST arrays of
 * `count` DEVICE pointers (grid g reads in[g], writes out[g]); each pair obeys
 * the single-grid rules (16-byte aligned, in[g] == out[g] or disjoint).
 * Stream-ordered.  The grids' descriptors travel through pinned host memory
 * owned by the plan, so an exec first waits (on the host) until the previous
 * exec of the same plan has started executing on the device.
 * Device-side waits that run out set the plan's device status to
 * CROFT_ERR_TIMEOUT (croft_plan_last_device_status); the exec itself still
 * returns CROFT_OK in that case because it does not synchronise.
 */
croft_status croft_exec_batched_forward(croft_plan plan, void* const* in, void* const* out, void* stream);
croft_status croft_exec_batched_backward(croft_plan plan, void* const* in, void* const* out, void* stream);

/* Budget, in SM clock cycles, of each bounded device-side wait of a batched
 * plan (default 4e9, about two seconds).  No effect on single-grid plans. */
croft_status croft_plan_set_wait_limit(croft_plan plan, long long cycles);

/* Test hook for the failure path: when enabled, the y-pass tiles of grid 0
 * wait for one more finished z tile than grid 0 has, a count nothing ever
 * reaches, so their waits run out after the wait limit and the plan reports
 * CROFT_ERR_TIMEOUT.  ONE_LAUNCH schedule only.  Never hangs the GPU. */
croft_status croft_plan_set_test_unsatisfiable_wait(croft_plan plan, int enable);

/*
 * croft_exec_batched_noalloc - the batched transform for callers that cannot
 * allocate device memory.  The paper has no counterpart; this is a library
 * service.
 *
 * Who needs it: code that runs inside a framework whose caching allocator owns
 * all of the device's memory (so a plan's own cudaMalloc would fail or fight
 * the pool), serving and real-time loops whose policy forbids device
 * allocation on the request path (cudaMalloc may synchronise the device), and
 * plug-ins that are not allowed to keep device memory of their own between
 * calls.  Every other entry point here needs a plan, and plans allocate
 * (twiddle tables, work lists, counters).
 *
 * What it does: exactly what a CROFT_BATCH_ONE_LAUNCH batched plan's exec does
 * (same persistent kernel, same tiles, so the same bits), but the kernel's
 * working memory - work counter, per-grid completion counts, status word, grid
 * descriptors, work list and twiddle tables - lives in one statically sized
 * __device__ array inside libcroft.so (about 1.1 MiB; every GPU that loads the
 * library holds it until the process exits).  The call builds those tables on
 * the host, copies them into the array on `stream`, clears the counters and
 * launches; it calls no cudaMalloc / cudaFree and no allocating library
 * routine.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it for the life of the process; make that
 * first call before any stream capture, and do not use the entry point across
 * a cudaDeviceReset (the kept address would belong to the destroyed context).
 * The tables are copied from host memory that the call owns only while it
 * runs (pageable; cudaMemcpyAsync stages it before returning), so a copy
 * recorded into a graph would read freed memory when replayed: the call
 * returns CROFT_ERR_INVALID_ARG, before any device work, when `stream` is
 * capturing.
 *
 *   count     : number of grids, 1..CROFT_NOALLOC_MAX_GRIDS.
 *   dims      : host array of 3*count axis lengths; each axis 1..128 of the
 *               form 2^a 3^b 5^c.
 *   in, out   : host arrays of `count` device pointers, as for
 *               croft_exec_batched_forward (16-byte aligned, in[g] == out[g]
 *               or disjoint).
 *   direction : -1 forward (Eq. 1), +1 backward (Eq. 2, unnormalised).
 *   stream    : cudaStream_t or NULL.
 * Returns CROFT_OK, CROFT_ERR_INVALID_ARG (NULL or misaligned pointers, a
 * direction other than -1 / +1, partial overlap of in[g] and out[g], or a
 * capturing stream), CROFT_ERR_UNSUPPORTED_SIZE (more
 * than CROFT_NOALLOC_MAX_GRIDS grids, an axis outside the list above, or more
 * than CROFT_NOALLOC_MAX_ITEMS work items - a 128^3 grid has 1536 - i.e. the
 * batch does not fit the static array) or CROFT_ERR_CUDA.
 *
 * All calls share the one array and it keeps the last call's contents, so two
 * calls whose work overlaps on the GPU (different streams, or different host
 * threads without ordering) race and corrupt each other; calls on one stream
 * are ordered and safe.  The bounded device-side waits are those of the
 * batched plans; a wait that runs out leaves the affected grids incomplete and
 * is not reported by this call (use a batched plan when that status matters).
 */
#define CROFT_NOALLOC_MAX_GRIDS 256
#define CROFT_NOALLOC_MAX_ITEMS 65536
croft_status croft_exec_batched_noalloc(int count, const int* dims, void* const* in, void* const* out, int direction,
                                        void* stream);

/*
 * croft_exec_forward - Eq. (1), unnormalised, out = F(in).
 * croft_exec_backward - Eq. (2) with exponent +, WITHOUT the 1/N factor.
 *
 *   plan : from croft_plan_create.
 *   in, out : device pointers to nx*ny*nz complex64 (layout above).
 *   stream : cudaStream_t or NULL.
 * Returns CROFT_OK, CROFT_ERR_INVALID_ARG (NULL plan/pointer, pointer not
 * 16-byte aligned, partial overlap of in/out) or CROFT_ERR_CUDA.
 */
croft_status croft_exec_forward(croft_plan plan, const void* in, void* out, void* stream);
croft_status croft_exec_backward(croft_plan plan, const void* in, void* out, void* stream);

/*
 * croft_exec_axes - the 1D transforms of a subset of the axes only (Eq. 1 / Eq. 2 restricted
 * to those axes; the others untouched): the local steps of a transform whose grid is
 * distributed over several processes or GPUs in slabs (Sec. 2.2.1, and steps 1, 5 and 9 of
 * Sec. 4.1).  A process holding an x-slab runs the z and y axes, an all-to-all regroups the
 * grid into y-slabs, and each process then runs the x axis.
 *
 *   plan      : a single-grid plan with one pass per axis (CROFT_SCHEDULE_THREE_PASS, which
 *               AUTO gives); the fused-plane and slab schedules give CROFT_ERR_INVALID_ARG.
 *   in, out   : device pointers as for croft_exec_forward (in == out allowed).
 *   axes      : bit a set to transform axis a (0 = x, 1 = y, 2 = z); 0 copies in to out.
 *   direction : -1 forward (Eq. 1), +1 backward (Eq. 2, unnormalised).
 *   stream    : cudaStream_t or NULL.
 * Returns CROFT_OK, CROFT_ERR_INVALID_ARG or CROFT_ERR_CUDA.  Asynchronous like exec; with
 * croft_plan_set_timing enabled it records one event per pass it runs (croft_plan_pass_times).
 */
croft_status croft_exec_axes(croft_plan plan, const void* in, void* out, int axes, int direction, void* stream);

/*
 * croft_transpose_blocks - out[j][i] = in[i][j] for an in array of d0 x d1 blocks of
 * block_bytes each (C order): the pack / unpack of the slab exchange (the paper's pack and
 * unpack around the all-to-all, Sec. 4.1 steps 2 and 4), as pitched copy-engine copies on
 * `stream` (min(d0, d1) of them).  No library allocation.
 *
 *   in, out : device pointers, disjoint (overlap gives CROFT_ERR_INVALID_ARG).
 * Returns CROFT_OK, CROFT_ERR_INVALID_ARG or CROFT_ERR_CUDA.
 */
croft_status croft_transpose_blocks(const void* in, void* out, long long d0, long long d1, long long block_bytes,
                                    void* stream);

/*
 * croft_exec_convolve - the reciprocal-space step of particle-mesh Ewald, the
 * application that motivates the paper (Sec. 1):
 *
 *     out = B(G * F(in)),   F = Eq. (1), B = Eq. (2) with exponent + and no 1/N,
 *
 * i.e. the circular convolution of `in` with B(G).  G is a real array indexed
 * like F's output (k = (kx, ky, kz), same layout as the grid); for PME it is
 * the influence function.
 *
 * The forward transform runs its passes up to the last axis; that axis's
 * forward 1D FFT, the multiply by G and its backward 1D FFT run fused in one
 * kernel (one HBM round trip instead of three); then the backward passes of
 * the other axes.  A 3D grid takes 5 launches.  Plans whose last pass cannot
 * take the fusion (a grid of one point, a last pass that is a fused yz-plane
 * or a tensor-core pass) run F, a separate multiply and B instead.  There is
 * no counterpart of this entry point in the paper beyond the application it
 * describes.
 *
 *   plan : a single-grid plan (any dtype and schedule).
 *   in, out : device pointers to nx*ny*nz complex elements of the plan's dtype,
 *       16-byte aligned; in == out is allowed, partial overlap is not.
 *   g : device pointer to nx*ny*nz reals (float for the complex64 dtypes,
 *       double for CROFT_C2C_F64), aligned to its element size; must not
 *       overlap `out`.  Read only.
 *   stream : cudaStream_t or NULL.  Asynchronous, stream-ordered; allocates
 *       nothing.
 * Returns CROFT_OK, CROFT_ERR_INVALID_ARG (NULL plan/pointer, batched plan,
 * misaligned pointer, overlap) or CROFT_ERR_CUDA.  With timing enabled,
 * croft_plan_pass_times reports one time per launch group in execution order.
 */
croft_status croft_exec_convolve(croft_plan plan, const void* in, void* out, const void* g, void* stream);

/*
 * croft_exec_host_pipeline - transform `count` HOST-resident grids, streaming
 * them through the GPU.  For grid i: copy host_in[i] to the device, apply the
 * requested operations in place (CROFT_OP_FORWARD: Eq. 1; CROFT_OP_BACKWARD:
 * Eq. 2 unnormalised; both: forward then backward, e.g. a convolution round
 * trip), copy the result to host_out[i].  The copies and the transform of
 * different grids overlap: grid i+1 uploads and grid i-1 downloads while grid
 * i is transformed, on three internal streams ordered by events (the paper's
 * chunked overlap of communication with computation, Sec. 5.1, applied to the
 * host link).  Stream-ordered with respect to `stream`: the pipeline starts
 * after the work already queued on it and `stream` waits for its end.
 *
 *   host_in, host_out : host arrays of `count` host pointers to nx*ny*nz
 *       complex64 each; page-locked memory (cudaMallocHost / cudaHostRegister)
 *       for the copies to overlap.  host_in[i] == host_out[i] is allowed.
 *   ops : CROFT_OP_FORWARD, CROFT_OP_BACKWARD or both (bitwise or).
 * The first call allocates three device buffers of one grid each plus the
 * streams and events; they stay with the plan (croft_plan_workspace_bytes).
 * Single-grid plans only.  Returns CROFT_OK, CROFT_ERR_INVALID_ARG,
 * CROFT_ERR_OOM or CROFT_ERR_CUDA.
 */
typedef enum { CROFT_OP_FORWARD = 1, CROFT_OP_BACKWARD = 2 } croft_op;
croft_status croft_exec_host_pipeline(croft_plan plan, int count, const void* const* host_in, void* const* host_out,
                                      int ops, void* stream);

/* Device scratch bytes held by the plan (0 when every pass runs in place;
 * batched plans: their counters and status word; after a host pipeline call:
 * its three grid buffers). */
size_t croft_plan_workspace_bytes(croft_plan plan);

/* Number of kernel launches one exec of this plan issues. */
int croft_plan_num_launches(croft_plan plan);

/*
 * croft_plan_describe - write a one-line description of the schedule (axes,
 * radix order, tile shape and launch shape of every pass) into buf (always
 * NUL-terminated when cap > 0).  Returns the length the full text needs.
 */
int croft_plan_describe(croft_plan plan, char* buf, int cap);

/*
 * Per-pass timing (tracing hook).  When enabled, each exec records a CUDA
 * event on the exec stream before the first pass and after every logical pass
 * (the slab schedule's z+y launches count as one pass).
 * croft_plan_pass_times waits for the last exec's events and writes the
 * duration in milliseconds of each pass into ms[0 .. min(cap, passes)-1];
 * it returns the number of passes timed, 0 when timing is off or no exec ran,
 * or -1 on a CUDA error.
 */
croft_status croft_plan_set_timing(croft_plan plan, int enable);
int croft_plan_pass_times(croft_plan plan, float* ms, int cap);

/*
 * Status written by bounded device-side waits during the last exec of this
 * plan (CROFT_OK or CROFT_ERR_TIMEOUT).  Synchronises with the plan's last
 * exec.  Plans without device-side waits always return CROFT_OK.
 */
croft_status croft_plan_last_device_status(croft_plan plan);

/* Release a plan and its device tables.  NULL is a no-op returning CROFT_OK.
 * Synchronises with any exec of the plan still in flight. */
croft_status croft_plan_destroy(croft_plan plan);

/*
 * Host-side planning helpers (no device needed; used by the tests).
 *
 * croft_factorize - the radix schedule the library uses for a length-n axis,
 * in execution order.  Writes up to cap radices and returns how many stages
 * there are, or -1 if n is unsupported.
 *
 * croft_twiddle_table - the float32 twiddle table for a length-n axis and
 * the given radix schedule (as returned by croft_factorize): for the stage
 * with radix R whose input sub-transforms have length p (the product of the
 * earlier radices), entry p-1 + (j-1)*p + k holds exp(-2 pi i j k/(p R)) for
 * j = 1..R-1, k = 0..p-1.  Writes 2*(n-1) floats (re, im interleaved).
 * Returns n-1, or -1 on bad arguments.
 */
int croft_factorize(int n, int* radices, int cap);
int croft_twiddle_table(int n, const int* radices, int nstages, float* out);

/*
 * Testing hooks (host side only; nothing here touches the GPU).
 *
 * croft_debug_fail_allocation(k): the k-th device or pinned-host allocation the
 * library makes from now on fails as if the device were out of memory (k = 0
 * disarms).  Every entry point that allocates must then return CROFT_ERR_OOM
 * (or fall back) and release what it had already allocated.
 * croft_debug_live_allocations(): allocations made by the library and not yet
 * released (a leak check).
 */
void croft_debug_fail_allocation(int k);
long croft_debug_live_allocations(void);

#ifdef __cplusplus
}
#endif

#endif /* CROFT_H_ */
