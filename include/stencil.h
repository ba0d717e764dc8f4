/*
 * GB300 stencil operator library -- C ABI.
 *
 * The library computes the stencil sweep of ForgeStencil Sec. 2.1,
 *     u^{t+1}(p) = sum_{o in S} c_o u^t(p + o)            (constant coefficients), or
 *     u^{t+1}(p) = sum_{o in S} w_o(p) u^t(p + o)         (coefficients that vary in space),
 * for an offset set S of star, box or diamond type and order (radius) r = 1..4 on a 2D or 3D
 * grid, iterated over time steps (Sec. 2.1; several steps may be fused into one launch,
 * Sec. 4.3).  Values are stored as f32, f16 or bf16 and accumulated in f32.
 *
 * Conventions shared by every entry point:
 *  - Return value: STENCIL_OK (0) or a negative STENCIL_ERR_* code.  No C++ exception
 *    crosses this boundary.  stencil_strerror() names a code.
 *  - Grids are dense and row-major: dims[] lists the extents slowest axis first ((nz, ny, nx)
 *    in 3D, (ny, nx) in 2D) and the last axis is contiguous.  No padding.
 *  - Offsets are written slowest axis first and enumerated in the canonical order:
 *    lexicographic over (dz, dy, dx), each component from -r to r, restricted to the shape.
 *    Star: one nonzero component at most; box: max |component| <= r; diamond: sum of
 *    |component| <= r.  Coefficient arrays follow this order (stencil_offsets returns it).
 *  - Boundaries: STENCIL_DIRICHLET0 updates every cell and reads 0 outside the grid;
 *    STENCIL_PERIODIC wraps every read (index mod extent).
 *  - Pointers named `in`, `out`, `coeff_arrays[i]` are DEVICE pointers owned by the caller.
 *    `in` and `out` must not overlap.  Device buffers aligned to 16 bytes whose row length in
 *    bytes is a multiple of 16 take the vectorised path; others take a scalar path (still on
 *    the GPU, slower).
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default stream).  Launches
 *    are asynchronous; argument errors are returned at once, CUDA launch errors as
 *    STENCIL_ERR_CUDA, and errors detected by a kernel (a bounded wait that expired) are
 *    latched in the plan's device status word, read by stencil_sync_status (batches:
 *    stencil_batch_status; wave plans: wave_sync_status).
 *  - A plan is not thread-safe: do not use one handle from two host threads at once.
 */
#ifndef GB300_STENCIL_H
#define GB300_STENCIL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------------------------ */
#define STENCIL_OK 0
#define STENCIL_ERR_BADARG (-1)      /* invalid argument (null pointer, bad size, ...)       */
#define STENCIL_ERR_UNSUPPORTED (-2) /* valid request this build has no kernel for          */
#define STENCIL_ERR_OOM (-3)         /* device or host allocation failed                    */
#define STENCIL_ERR_CUDA (-4)        /* a CUDA runtime call failed                           */
#define STENCIL_ERR_TIMEOUT (-5)     /* a bounded device-side wait expired                   */
#define STENCIL_ERR_BOUNDS (-6)      /* a device-side index check failed                     */

/* ---- enumerations ------------------------------------------------------------------------ */
#define STENCIL_STAR 0
#define STENCIL_BOX 1
#define STENCIL_DIAMOND 2
#define STENCIL_CUSTOM 3   /* any offset set of max-norm <= radius, given by the caller       */

#define STENCIL_F32 0
#define STENCIL_F16 1
#define STENCIL_BF16 2

#define STENCIL_DIRICHLET0 0
#define STENCIL_PERIODIC 1

#define STENCIL_CONST 0    /* one coefficient per offset                                      */
#define STENCIL_VAR 1      /* one coefficient array per offset, read at the output cell       */
#define STENCIL_DIVKGRAD 2 /* div(k grad u), unit spacing, conservative star-1 form (below)   */

typedef struct stencil_plan_s *stencil_handle;
typedef struct stencil_batch_s *stencil_batch;

/* ---- plans ------------------------------------------------------------------------------- */

/* stencil_plan -- validate a stencil request and choose its kernel (Sec. 2.1: offset set,
 * coefficients, grid and precision; Sec. 4.3: the kernel is specialised per stencil type,
 * grid shape and precision).
 *   out      receives the new handle (host memory owned by the library; free with
 *            stencil_destroy).  The call allocates no device memory.
 *   ndim     2 or 3; dims[ndim] extents, slowest first, each >= 1.
 *   shape    STENCIL_STAR / BOX / DIAMOND; radius 1..4 (kind DIVKGRAD: star, radius 1).
 *            STENCIL_CUSTOM: the offset set S is any set of ncoeffs distinct offsets (Sec. 2.1
 *            defines the sweep over an arbitrary S) listed in custom_offsets[ncoeffs * ndim]
 *            (int32, slowest component first, host memory, copied), every component within
 *            [-radius, radius]; kind must be STENCIL_CONST (else UNSUPPORTED).  The sweep runs
 *            on the kernel of the smallest compiled star, diamond or box set containing S,
 *            with weight 0 on its other offsets (so the result is the sum over S alone;
 *            terms are added in that set's canonical order).
 *   kind     STENCIL_CONST: coeffs[ncoeffs] holds one weight per offset -- in canonical order,
 *            or in the order of custom_offsets (ncoeffs must equal the offset count); the
 *            values are copied.
 *            STENCIL_VAR / STENCIL_DIVKGRAD: coeffs must be NULL and ncoeffs 0; the arrays are
 *            passed to stencil_apply_var.
 *   custom_offsets  NULL unless shape is STENCIL_CUSTOM.
 *   dtype    storage type of every grid array (STENCIL_F32 / F16 / BF16).
 *   boundary STENCIL_DIRICHLET0 or STENCIL_PERIODIC.
 * Errors: BADARG for out-of-range values, a count mismatch, repeated custom offsets or
 * custom_offsets given for another shape (or missing for STENCIL_CUSTOM); UNSUPPORTED for a
 * combination without a kernel; OOM when 65536 plans are alive.  The kernel choice comes from
 * the dispatch map (stencil_load_dispatch_map) or from built-in defaults. */
int stencil_plan(stencil_handle *out, int ndim, const int64_t *dims, int shape, int radius,
                 int kind, const double *coeffs, int64_t ncoeffs, const int32_t *custom_offsets,
                 int dtype, int boundary);

/* stencil_plan_kernel_set -- the compiled offset set the plan's kernels run: its shape
 * (STENCIL_STAR / BOX / DIAMOND) and radius; for a custom plan, the set chosen to contain it.
 * Either pointer may be NULL. */
int stencil_plan_kernel_set(stencil_handle h, int *shape, int *radius);

/* stencil_offsets -- the plan's offsets in canonical order (a custom plan: in the order the
 * caller gave them, the order of its coefficients).  Writes min(n, capacity) rows of
 * ndim int32 (slowest component first) to offsets_out (may be NULL when capacity is 0) and the
 * full count to *n. */
int stencil_offsets(stencil_handle h, int32_t *offsets_out, int64_t capacity, int64_t *n);

/* stencil_destroy -- free a plan and any device scratch it allocated (synchronises the
 * device before freeing).  NULL is accepted. */
int stencil_destroy(stencil_handle h);

/* ---- sweeps ------------------------------------------------------------------------------ */

/* stencil_apply -- `steps` >= 1 sweeps of a STENCIL_CONST plan: out = A^steps in
 * (Sec. 2.1 update rule iterated over t; fused groups of steps per launch as in Sec. 4.3).
 * Between steps the values are rounded to the storage type (round to nearest even), also
 * inside a fused launch, so the result does not depend on how steps are grouped.
 * `in` is not modified.  steps > 1 ping-pongs through `out` and one grid-sized scratch buffer
 * that the plan allocates on first use (cudaMalloc) and keeps until stencil_destroy. */
int stencil_apply(stencil_handle h, const void *in, void *out, int steps, void *stream);

/* stencil_apply_adjoint -- out = (A^T)^steps in for a STENCIL_CONST plan: the transposed sweep
 * (A^T y)[q] = sum_o c_o y[q - o], i.e. the stencil with every offset flipped. */
int stencil_apply_adjoint(stencil_handle h, const void *in, void *out, int steps, void *stream);

/* stencil_apply_reaction -- `steps` explicit steps of a reaction-diffusion equation whose
 * spatial operator is the plan's sweep A, with the stencil and the pointwise physics fused in
 * one launch per step (Sec. 4.3 fuses a stencil with an application's physics):
 *     u^{t+1} = u^t + dt * ( (A u^t) + c1 u^t + c3 (u^t)^3 )
 * (Allen-Cahn with a Laplacian A: c1 = 1/eps^2, c3 = -1/eps^2; c3 = 0: linear reaction).  In
 * FP32 each cell computes fma(dt, fma(c3, u*u*u, fma(c1, u, L)), u) with L = (A u)[p], and
 * rounds the result to the storage type.  STENCIL_CONST plans whose kernel set is a star of
 * radius 1, 2 or 4 or the radius-1 box, f32 or bf16 storage (else UNSUPPORTED); dt, c1, c3
 * finite (else BADARG); `in`, `out`, `steps`, scratch and errors as stencil_apply. */
int stencil_apply_reaction(stencil_handle h, const void *in, void *out, int steps, double dt,
                           double c1, double c3, void *stream);

/* stencil_apply_var -- sweeps of a STENCIL_VAR or STENCIL_DIVKGRAD plan.
 *   VAR:      coeff_arrays[npts] are device pointers to grid-shaped arrays of the storage
 *             type; out[p] = sum_o coeff_arrays[o][p] * in[p + o]  (Sec. 2.1).
 *   DIVKGRAD: coeff_arrays[0] is k (grid-shaped, storage type, k > 0);
 *             out[p] = sum_axes [ kf+ (u[p+e] - u[p]) - kf- (u[p] - u[p-e]) ],
 *             kf+- = (k[p] + k[p+-e]) / 2; with STENCIL_DIRICHLET0, u reads 0 and k reads
 *             k[p] outside the grid.  This operator is symmetric.
 * `coeff_arrays` itself is a HOST array of device pointers. */
int stencil_apply_var(stencil_handle h, const void *in, const void *const *coeff_arrays,
                      void *out, int steps, void *stream);

/* stencil_apply_adjoint_var -- the transpose of stencil_apply_var:
 *   VAR:      out[q] = sum_o coeff_arrays[o][q - o] * in[q - o]  (offset flipped, coefficient
 *             gathered at the shifted cell);
 *   DIVKGRAD: the operator is symmetric, so this equals stencil_apply_var. */
int stencil_apply_adjoint_var(stencil_handle h, const void *in,
                              const void *const *coeff_arrays, void *out, int steps,
                              void *stream);

/* stencil_apply_host -- stencil_apply on HOST buffers: copies `in_host` to a device staging
 * buffer, sweeps, and copies the result to `out_host`, then synchronises `stream`; the result
 * is bit for bit that of stencil_apply.  3D grids on the streaming kernel are pipelined over
 * z slabs: input slabs are copied in on a stream of the plan's; sweep t of the output planes
 * up to A - t*radius runs as soon as input planes [0, A) have landed (a wavefront over z; on
 * a periodic grid the planes near either end, which read wrapped planes, follow once the
 * input is complete), and the finished planes of the last sweep are copied out on a second
 * stream of the plan's, so both copy directions overlap the sweeps and each other (work
 * queued on `stream` before the call is ordered before the copies).  Pinned host memory gives
 * full copy bandwidth.  The staging buffers, streams and events are created on first use and
 * kept by the plan. */
int stencil_apply_host(stencil_handle h, const void *in_host, void *out_host, int steps,
                       void *stream);

/* stencil_apply_noalloc -- stencil_apply for callers that may not allocate device memory.
 * The paper has no counterpart; this is a library service.  stencil_apply obtains its
 * multi-step scratch grid with cudaMalloc on first use, which some callers cannot allow: code
 * inside a framework whose memory pool already holds the device's memory, and
 * latency-critical loops that cannot absorb cudaMalloc's implicit device synchronisation.
 * This call computes the same sweeps (same kernels, same step grouping, same results) but
 * ping-pongs through a fixed array compiled into the library:
 *   - no cudaMalloc/cudaFree or other allocating call is made;
 *   - grids larger than STENCIL_NOALLOC_SCRATCH_BYTES (in bytes of the storage type) are
 *     rejected with STENCIL_ERR_BADARG before anything is launched;
 *   - the array is reserved on every GPU that loads the library, until the process exits;
 *   - the first call on each device looks up the array's device address with that device
 *     current; make that first call before any stream capture begins;
 *   - all calls share the array, so calls whose kernels may run at the same time on the GPU
 *     (different streams, no ordering) race and must be serialised by the caller.
 * Arguments, plan kinds and errors otherwise as stencil_apply. */
#define STENCIL_NOALLOC_SCRATCH_BYTES ((size_t)16 * 1024 * 1024)
int stencil_apply_noalloc(stencil_handle h, const void *in, void *out, int steps, void *stream);

/* stencil_sync_status -- synchronise `stream` and return the first error latched by a kernel
 * of this plan since the last call (then clear it): STENCIL_ERR_TIMEOUT when a bounded
 * device-side wait of the plane ring (the streaming and div(k grad u) kernels) expired, in
 * which case that launch's output is incomplete.  Each plan owns one status word in a fixed
 * device array of the library (nothing is allocated; at most 65536 plans and wave plans may
 * be alive at once, more give STENCIL_ERR_OOM from stencil_plan); read it with the device that
 * ran the plan current. */
int stencil_sync_status(stencil_handle h, void *stream);

/* stencil_set_wait_limit -- bound on every device-side wait of this plan's ring kernels
 * (default 2 s; 0 < seconds <= 3600), and, for fault-injection tests only, a number of extra
 * arrivals (0 .. 1000; 0 in normal use) that each ring slot's "consumers are done" barrier
 * waits for and that never come.  With phantom_arrivals > 0, a launch whose CTAs walk more
 * planes than the ring holds gives up after about `seconds`: the producer's wait for a free
 * slot expires, every copy it issued still lands before its CTA exits, and the next
 * stencil_sync_status returns STENCIL_ERR_TIMEOUT.  Takes effect at the next launch. */
int stencil_set_wait_limit(stencil_handle h, double seconds, int phantom_arrivals);

/* ---- batched sweeps (many grids, one persistent launch) ---------------------------------- */

typedef struct {
    stencil_handle plan; /* a 2D STENCIL_CONST plan describing this grid                    */
    const void *in;      /* device input, plan's dims and dtype                             */
    void *out;           /* device output                                                    */
} stencil_batch_item;

/* stencil_batch_plan -- build a tile work list over `n` grids (2D, constant coefficients,
 * any mix of star/box/diamond shapes of radius 1-2, dtypes, boundaries and sizes; other
 * plans give UNSUPPORTED) for `steps` sweeps each, allocate the
 * device scratch it needs, and capture one persistent cooperative kernel (plus the reset of
 * its counters) into a CUDA graph.  Every step boundary is a device-wide barrier whose wait
 * is bounded; an expired wait latches STENCIL_ERR_TIMEOUT.  The plans and buffers named by
 * `items` must outlive the batch; the items array is copied. */
int stencil_batch_plan(stencil_batch *out, const stencil_batch_item *items, int n, int steps);

/* stencil_batch_plan_tiles -- stencil_batch_plan with the launch shape chosen by the caller
 * (the autotuner's knob): output tiles of tile_y x tile_x cells, `fuse` steps per group (a
 * group's steps run in a tile grown by radius x fuse cells, with the intermediate levels
 * rounded to the storage type in shared memory, so the result does not depend on fuse; one
 * device-wide barrier per group).  0 selects the default (32 x 120 tiles, one step per
 * group).  UNSUPPORTED when the grown tile does not fit in shared memory. */
int stencil_batch_plan_tiles(stencil_batch *out, const stencil_batch_item *items, int n,
                             int steps, int tile_y, int tile_x, int fuse);

/* stencil_batch_launch -- launch the captured graph on `stream`. */
int stencil_batch_launch(stencil_batch b, void *stream);

/* stencil_batch_status -- synchronise `stream` and return the batch's latched device error. */
int stencil_batch_status(stencil_batch b, void *stream);

/* stencil_batch_destroy -- free the batch, its graph and its scratch. */
int stencil_batch_destroy(stencil_batch b);

/* stencil_batch_set_wait_limit -- set the bound on every device-side barrier wait of the
 * batch (default 2 s) and, for fault-injection tests only, a number of extra arrivals each
 * barrier waits for that never come (0 in normal use).  With phantom_arrivals > 0 a launch of
 * more than one step ends with STENCIL_ERR_TIMEOUT after about `seconds`, without hanging.
 * Synchronises the device. */
int stencil_batch_set_wait_limit(stencil_batch b, double seconds, int phantom_arrivals);

/* stencil_batch_info -- work tiles, persistent blocks and whether the launch was captured in
 * a CUDA graph (1) or is issued directly (0).  Any pointer may be NULL. */
int stencil_batch_info(stencil_batch b, int *ntiles, int *nblocks, int *graph_captured);

/* ---- tuning and dispatch ----------------------------------------------------------------- */

typedef struct {
    int family;  /* kernel family chosen (STENCIL_FAMILY_*)                                     */
    int block_x; /* threads along x (streaming family: 128 cells / one 16-byte vector each)      */
    int block_y; /* threads along y (streaming family: block_x * block_y a multiple of 32, at
                    most 224; 3D stars of radius >= 3: 256 with one row per thread, 448 with
                    two rows per thread in f32 storage)                                       */
    int vec_y;   /* rows per thread (streaming 1, 2 or 4 by stencil; div(k grad u) 1 or 2;
                    general variable-coefficient sweeps 1)                                   */
    int z_chunk; /* planes per CTA (3D); 0 = an equal share per resident CTA (streaming and
                    div(k grad u)) or whole columns (general variable-coefficient sweeps);
                    -1 (streaming and div(k grad u)) = every tile column cut into the same
                    number of near-equal chunks, as many as the resident CTAs allow, so that
                    the CTAs of neighbouring tiles sweep the same planes at the same time     */
    int fuse;    /* time steps fused per launch                                                 */
    int tile_x;  /* output tile width of fused 2D kernels (0 = default)                         */
    int tile_y;  /* output tile height of fused 2D kernels (0 = default)                        */
    int stages;  /* shared-memory ring depth of the streaming loader, 2..16 planes; 0 = as deep
                    as the shared memory left by the CTAs that fit on an SM allows             */
} stencil_variant;

#define STENCIL_FAMILY_STREAM 1 /* one sweep per launch, z-streaming tiles on a plane ring fed
                                   by a producer warp (tensor copies)                        */
#define STENCIL_FAMILY_FUSED2D 2 /* several 2D sweeps per launch in a shared-memory tile      */
#define STENCIL_FAMILY_FUSED3D 3 /* two 3D sweeps per launch on the plane ring (temporal
                                    blocking, Sec. 4.3): the intermediate plane stays in shared
                                    memory; star/diamond radius 1-2 and the radius-1 box; fuse
                                    must be 2, vec_y 2 (f32) or 1 (16-bit storage), block_y
                                    >= 2 * radius; an odd last step runs on the streaming
                                    kernel                                                     */
#define STENCIL_FAMILY_TENSOR 4  /* the radius-2 box (2D and 3D) on the tensor cores, Toeplitz
                                    packing of the x direction (Sec. 6, tensor-core mapping):
                                    f16/bf16 storage, zero Dirichlet, rows a multiple of 8
                                    cells; tile_x = 16, 32 or 64 outputs per CTA, vec_y warps
                                    issue the MMAs, each for every vec_y-th output plane (0 or
                                    1, 2, or 4 with tile_x 64), z_chunk planes per CTA (0 = one
                                    wave), stages plane slots (0 = automatic, else 5..12);
                                    block_y must be 0 or 1, block_x is ignored. Accumulates in
                                    FP32 with the coefficients split into two 16-bit parts, so
                                    results equal the FP32 path to within rounding, not bit
                                    for bit */

/* stencil_plan_get_variant / stencil_plan_set_variant -- read or override the kernel variant
 * a plan uses (the autotuner's knob).  set validates the variant against the plan and returns
 * BADARG or UNSUPPORTED without changing the plan when it cannot run. */
int stencil_plan_get_variant(stencil_handle h, stencil_variant *v);
int stencil_plan_set_variant(stencil_handle h, const stencil_variant *v);

/* stencil_load_dispatch_map -- replace the process-wide dispatch map with the one in the
 * text file at `path` (format: lines "ndim shape radius dtype boundary kind size_class
 * [geometry] : family block_x block_y vec_y z_chunk fuse tile_x tile_y [stages]", '#'
 * comments; a key field of -1 matches anything, a missing geometry field reads as -1 and a
 * missing stages field as 0; the first matching line wins; lines "batch dtype : tile_y
 * tile_x fuse" give stencil_batch_plan its launch shape for batches of that storage type).
 * Plans created
 * afterwards use it.  NULL restores the built-in defaults.  If the environment variable
 * STENCIL_DISPATCH_MAP names a file, it is loaded once before the first stencil_plan. */
int stencil_load_dispatch_map(const char *path);

/* stencil_size_class -- the size class (0 .. 3) a grid of `cells` cells falls in. */
int stencil_size_class(int64_t cells);

/* stencil_geometry_class -- the geometry class of a grid in the dispatch key (Sec. 4.3: the
 * kernel is specialised per grid shape): 1 for a 3D slab thin in z (nz * 8 <= ny and
 * nz * 8 <= nx), 0 otherwise (cube-like 3D grids, every 2D grid).  dims as in stencil_plan. */
int stencil_geometry_class(int ndim, const int64_t *dims);

/* ---- introspection ----------------------------------------------------------------------- */

/* stencil_launch_count -- number of kernels this library has launched in the process. */
uint64_t stencil_launch_count(void);

/* stencil_strerror -- static string naming a status code. */
const char *stencil_strerror(int code);

/* stencil_abi_version -- ABI version of this header (STENCIL_ABI_VERSION). */
#define STENCIL_ABI_VERSION 2
int stencil_abi_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GB300_STENCIL_H */
