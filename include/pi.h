/*
 * pi.h -- C ABI of libpi: cutoff-radius pair interactions on a regular cell
 * grid, on one NVIDIA GB300 (sm_103a).
 *
 * The method is the one of arXiv 2406.16091 (Algis, Bramas, Darles, Aveneau):
 *   Sec. 2  bin the particles -- cell index of each particle from its
 *           position, per-cell count with atomics, exclusive prefix sum over
 *           the counts (Fig. 1: C+1 offsets, the last one N), scatter into
 *           cell-sorted structure-of-arrays copies -- then, for every
 *           particle i, sum a kernel K(r_ij) over all j != i with
 *           r_ij < r_c found in its own cell and the 26 neighbouring cells.
 *   Sec. 3  the cell width is at least r_c; inputs are positions, the
 *           per-cell counts and start offsets; outputs are per-particle
 *           values in SoA form.
 *
 * Conventions for every call:
 *   - Device pointers are plain CUDA device addresses of the device that was
 *     current when the context was created.  Host pointers are marked so.
 *   - Every call is asynchronous on the given stream unless it says it
 *     synchronises; a NULL stream is the legacy default stream.
 *   - Calls return a pi_status.  Argument errors are detected on the host
 *     and returned at once, with nothing enqueued.  Errors found by the GPU
 *     (a position outside the box, a device-side wait that ran out) are kept
 *     in a device error word and returned by pi_sync_status(); after such an
 *     error the outputs of the failed step are undefined, and the library
 *     stays usable (the next pi_bin clears the word).
 *   - Nothing aborts, nothing throws across the ABI, no device wait is
 *     unbounded.
 *   - A context is not thread-safe: one host thread at a time per context.
 */
#ifndef PI_H
#define PI_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque, library-owned.  Holds the grid and every device buffer binning needs. */
typedef struct pi_ctx pi_ctx;

/* A CUDA stream handle (identical to cudaStream_t / CUstream). */
typedef struct CUstream_st* pi_stream;

/* Simulation box: half-open [lo, hi) per axis, not periodic (Alg. 5 clips
 * the neighbour range with Max(0, .) and Min(limit, .)). */
typedef struct {
    float lo[3];
    float hi[3];
} pi_box;

typedef enum {
    PI_OK = 0,
    PI_ERR_INVALID_ARG = 1, /* bad argument, detected on the host */
    PI_ERR_CAPACITY = 2,    /* n > n_max, or an internal size limit */
    PI_ERR_OUT_OF_BOX = 3,  /* some position outside [lo, hi) or NaN (device) */
    PI_ERR_NOT_BINNED = 4,  /* pi_interact before a successful pi_bin */
    PI_ERR_CUDA = 5,        /* a CUDA runtime call failed; see pi_last_error() */
    PI_ERR_TIMEOUT = 6,     /* a bounded device-side wait ran out (device) */
    PI_ERR_NOMEM = 7,       /* device allocation failed */
    PI_ERR_CHECK = 8        /* debug builds (PI_CHECK): an index failed its bounds
                               check and the access was skipped (device); the
                               check's site is in pi_last_error() */
} pi_status;

/* Output order of pi_interact. */
enum {
    PI_ORDER_SORTED = 0,   /* out[k] belongs to the particle in sorted slot k */
    PI_ORDER_ORIGINAL = 1  /* out[i] belongs to input particle i */
};

/* Keys of pi_set_option(). */
enum {
    /* Interaction algorithm.  PI_ALGO_TILED (default): per-target x-windows
     * over the x-sorted neighbour X-rows, in the shape PI_OPT_TILE selects;
     * PI_ALGO_PPNL is Alg. 1 of the paper (Par-Part-NoLoop: one thread per
     * particle, the 27-cell stencil read from global memory), kept as the
     * in-library comparator. */
    PI_OPT_ALGO = 1,
    /* Accumulation: PI_PREC_FP32 (default) plain FP32 sums; PI_PREC_KAHAN
     * compensated FP32 sums per particle and output (a Kahan step per
     * accepted pair; pairs that fail the test are skipped). */
    PI_OPT_PRECISION = 2,
    /* Upper bound, in nanoseconds, of every device-side wait (default 1e9). */
    PI_OPT_WAIT_LIMIT_NS = 3,
    /* Test hook for the failure path: when 1, the first tile of the scan
     * never publishes its prefix, so the other tiles' bounded waits run out
     * and pi_sync_status() returns PI_ERR_TIMEOUT.  Default 0. */
    PI_OPT_TEST_WITHHOLD_SCAN = 4,
    /* Interaction kernel K (PI_KERNEL_*), default PI_KERNEL_GAUSSIAN. */
    PI_OPT_KERNEL = 5,
    /* Tile shape of the tiled interaction (each thread evaluates two
     * targets): 0, 1, 2 for one CTA per chunk with 32, 64, 128 threads and
     * 768, 1280, 2432 staged particles; 3, 4 for the warp-specialised form
     * (one producer warp stages chunks of up to 2432 particles into 2
     * buffers for 4 or 8 consumer warps); 5 for the direct form (no
     * staging: one thread per target pair reads its sources from global
     * memory through L1; every kernel K and both precision modes); 6 for the
     * direct form with four targets per thread (fewer source reads per
     * evaluation, more evaluations: faster at high occupancy).  With a
     * kernel other than the Gaussian, shapes 0 - 4 all run shape 2's
     * one-target form.  Default PI_TILE_AUTO: shape 6 for the plain
     * (PI_PREC_FP32) Gaussian and low-FLOP kernels when the last pi_bin put
     * 8 or more particles per cell on average and enough particles for one
     * full wave of shape 6 (4 x 640 per SM), shape 5 otherwise.
     * pi_autotune sets a shape from measurements.  Results do not depend on
     * it. */
    PI_OPT_TILE = 6,
    /* Binning: PI_BIN_PER_PARTICLE (default) takes one global atomic and
     * one 32-byte provisional record per particle; PI_BIN_BUCKETED counts
     * the particles per bucket of consecutive cells and ranks each bucket's
     * cells in shared memory, when the bucket-by-chunk count matrix fits the
     * context (up to about 8 M cells; the per-particle path otherwise);
     * PI_BIN_RADIX sorts the particles by cell with a stable
     * least-significant-digit radix sort (digits of up to 9 bits, one count,
     * scan and split pass per digit) and then gathers the sorted arrays,
     * when its count matrices fit the context (the per-particle path
     * otherwise).  Results are the same bit for bit. */
    PI_OPT_BINNING = 7,
    /* Diagnostics: 1 makes the direct interaction kernels (PI_OPT_TILE 5 and
     * 6) run a copy that counts their target-source evaluations -- each
     * target against every source slot of its group's windows, the padding
     * of four-source trips included -- into a device counter that
     * pi_eval_count reads; 0 (default) counts nothing.  The copy exists for
     * the Gaussian kernel in PI_PREC_FP32 (the windows, and so the count,
     * depend on the positions and r_c only); other kernels, the Kahan mode,
     * the staged shapes, Alg. 1 and pi_autotune's timed trials count
     * nothing.  The count restarts at every pi_bin.  Results do not depend
     * on it. */
    PI_OPT_COUNT_EVALS = 8
};
enum { PI_TILE_AUTO = -1 };
enum { PI_BIN_PER_PARTICLE = 0, PI_BIN_BUCKETED = 1, PI_BIN_RADIX = 2 };
enum { PI_ALGO_TILED = 0, PI_ALGO_PPNL = 1 };
enum { PI_PREC_FP32 = 0, PI_PREC_KAHAN = 1 };

/* Interaction kernels K(r) (the h argument of pi_interact is their length):
 *   PI_KERNEL_GAUSSIAN  exp(-r^2 / h^2).
 *   PI_KERNEL_LJ        the Lennard-Jones potential of Sec. 7.1 with E0 = 1,
 *                       length sigma = h and a softening of sigma/10:
 *                       4 (s^6 - s^3), s = sigma^2 / (r^2 + sigma^2 / 100).
 *   PI_KERNEL_LOWFLOP   1: the cheap synthetic kernel of Sec. 7.2 (S counts
 *                       the neighbours, V sums their offsets).
 *   PI_KERNEL_HIGHFLOP  the Lennard-Jones value followed by 150 FLOP that
 *                       leave it unchanged: the expensive synthetic kernel of
 *                       Sec. 7.2 (Fig. 7). */
enum { PI_KERNEL_GAUSSIAN = 0, PI_KERNEL_LJ = 1, PI_KERNEL_LOWFLOP = 2, PI_KERNEL_HIGHFLOP = 3 };

/* Creates a context on the current CUDA device for boxes of the given shape.
 *   box   host pointer; lo < hi on every axis, all finite.
 *   r_c   cutoff radius > 0.  Cells per axis n_d = max(1, floor((hi_d -
 *         lo_d) / r_c)) computed in FP64, so every cell is at least r_c wide
 *         (Sec. 3); C = nx*ny*nz must stay below 2^31.
 *   n_max largest particle count a later pi_bin may pass, 0 <= n_max < 2^31 - 64.
 *   out   receives the context; the caller owns it and frees it with pi_destroy.
 * Allocates all device buffers once (about 72 B per particle + 28 B per cell).
 * Errors: PI_ERR_INVALID_ARG, PI_ERR_NOMEM, PI_ERR_CUDA. */
pi_status pi_create(const pi_box* box, float r_c, int64_t n_max, pi_ctx** out);

/* Re-targets a single-system context to another box and cutoff without
 * allocating: the grid of (box, r_c) must have at most as many cells as the
 * grid the context was created with (PI_ERR_CAPACITY otherwise); n_max is
 * unchanged.  The new constants are written by a launch on `stream`, so work
 * enqueued on that stream afterwards sees them; the context must be binned
 * again before pi_interact.  Used to keep device-resident contexts for jobs
 * of varying shape (serving).  The grid follows pi_create's rule (Sec. 3:
 * cells at least r_c wide).  Errors: PI_ERR_INVALID_ARG (also for a batch
 * context), PI_ERR_CAPACITY, PI_ERR_CUDA. */
pi_status pi_reconfigure(pi_ctx* ctx, const pi_box* box, float r_c, pi_stream stream);

/* Frees the context and its device buffers (synchronises the device first).
 * NULL is accepted.  No passage of the paper: library housekeeping. */
pi_status pi_destroy(pi_ctx* ctx);

/* Binning (Sec. 2, Fig. 1).  x, y, z: device arrays of n FP32 positions
 * (SoA, caller-owned, read only).  0 <= n <= n_max; n = 0 is a valid no-op
 * that leaves an empty grid.  Enqueues, on `stream`:
 *   a1/a2  cell index of each particle, cell = cx + nx*(cy + ny*cz) with
 *          c_d = clamp(floor((x_d - lo_d) * inv_w_d), 0, n_d - 1) in FP32,
 *          and an atomic count per cell;
 *   a3     a single-pass exclusive scan (C+1 offsets, offsets[C] = n) that
 *          also records M_C, the largest cell count (Sec. 5.1);
 *   a4     a stable scatter: inside a cell, particles keep input order.
 * Results stay in the context; read them with pi_binned().
 * Errors: PI_ERR_INVALID_ARG, PI_ERR_CAPACITY (n > n_max), PI_ERR_CUDA; a
 * position outside [lo, hi) is reported later as PI_ERR_OUT_OF_BOX. */
pi_status pi_bin(pi_ctx* ctx, const float* x, const float* y, const float* z, int64_t n,
                 pi_stream stream);

/* Interaction (Sec. 2, Sec. 3) over the particles of the last pi_bin: for
 * every particle i, with d_ij = p_j - p_i and the pair test done in FP32 as
 * r2 = fma(dz,dz,fma(dy,dy,dx*dx)) < fl32(r_c*r_c):
 *   nbr[i] = number of j != i passing the test,
 *   S[i]   = sum_j K_ij,  K_ij = exp(-r_ij^2 / h^2),
 *   V[i]   = sum_j d_ij K_ij   (Vx, Vy, Vz).
 * S, Vx, Vy, Vz: device FP32 arrays of n entries (caller-owned, written).
 * nbr: device uint32 array of n entries, or NULL to skip the counts.
 * Every path excludes the self pair by identity (j != i of Sec. 2), so a
 * distinct particle at the same position counts, with K = 1 and a zero
 * vector term.
 * h > 0 and finite, with a finite FP32 kernel scale: -log2(e)/h^2 for the
 * Gaussian (h above about 6.5e-20), h^2 finite and non-zero for the
 * Lennard-Jones kernels; otherwise PI_ERR_INVALID_ARG.  Terms are FP32: a
 * Gaussian term below 2^-126 (the smallest normal FP32 number, reached
 * where (r/h)^2 > 87) is flushed to zero, so each output carries at most
 * that much per neighbour (|d_ij| times that for V) beyond its relative
 * error.  out_order: PI_ORDER_SORTED or PI_ORDER_ORIGINAL.
 * Output arrays must not alias each other or the inputs of pi_bin.
 * Errors: PI_ERR_INVALID_ARG, PI_ERR_NOT_BINNED, PI_ERR_CUDA. */
pi_status pi_interact(pi_ctx* ctx, float h, float* S, float* Vx, float* Vy, float* Vz,
                      uint32_t* nbr, int out_order, pi_stream stream);

/* End-to-end step through host memory (one step of Sec. 2's method: the
 * binning of pi_bin and the interaction of pi_interact): copies n positions
 * from the host arrays hx, hy, hz into context-owned device buffers, runs
 * pi_bin and pi_interact, copies the outputs back into the host arrays hS,
 * hVx, hVy, hVz (and hnbr unless NULL), then synchronises `stream` and
 * returns the step's status (device-side errors included).  Pinned host
 * memory gives asynchronous copies; pageable memory works too.  The device
 * staging buffers are allocated on the first call (n_max entries).  Errors:
 * those of pi_bin, pi_interact and pi_sync_status, PI_ERR_NOMEM.
 */
pi_status pi_run_host(pi_ctx* ctx, const float* hx, const float* hy, const float* hz,
                      int64_t n, float h, float* hS, float* hVx, float* hVy, float* hVz,
                      uint32_t* hnbr, int out_order, pi_stream stream);

/* One job of a request loop (one step of Sec. 2's method on the job's own box
 * and cutoff), enqueued without waiting: re-targets the context to (box, r_c)
 * when they differ from its current ones (as pi_reconfigure: the new grid
 * must fit the context), copies the n host positions into the context's
 * device staging buffers, runs pi_bin and pi_interact, and copies the outputs
 * back into the host arrays -- all on `stream`, in that order, nothing
 * synchronised.  The host arrays must stay valid and untouched until the
 * stream reaches this point (record an event after the call); pinned memory
 * makes the copies asynchronous.  The staging buffers are allocated on the
 * first pi_run_host / pi_submit_host call of a context (a warm-up call keeps
 * that out of a request loop).  Device-side errors surface in pi_sync_status.
 * Errors returned at once: those of pi_reconfigure, pi_bin and pi_interact,
 * PI_ERR_NOMEM.
 */
pi_status pi_submit_host(pi_ctx* ctx, const pi_box* box, float r_c, const float* hx, const float* hy,
                         const float* hz, int64_t n, float h, float* hS, float* hVx, float* hVy,
                         float* hVz, uint32_t* hnbr, int out_order, pi_stream stream);

/* pi_submit_host (Sec. 2's step, as above) with host arrays that may lie in
 * blocks, so that the step makes as few as one host-to-device and one
 * device-to-host copy instead of up to eight.  in_stride = 0: x, y, z are separate
 * arrays (three copies); in_stride > 0: they lie in one block, hy = hx +
 * in_stride and hz = hx + 2*in_stride (checked), and travel as one copy of
 * 2*in_stride + n entries, the gaps included.  out_stride likewise for S, Vx,
 * Vy, Vz and, unless NULL, the counts: hVx = hS + out_stride, ..., hnbr =
 * (uint32_t*)(hS + 4*out_stride).  A block must be one host allocation
 * covering the copied range.  A non-zero stride is a multiple of 4 with n <=
 * stride <= n_max + 4 rounded up to a multiple of 4.  Otherwise as
 * pi_submit_host.  Errors: PI_ERR_INVALID_ARG (a stride outside these limits
 * or arrays not at their stride) and those of pi_submit_host.
 */
pi_status pi_submit_host_strided(pi_ctx* ctx, const pi_box* box, float r_c, const float* hx, const float* hy,
                                 const float* hz, int64_t in_stride, int64_t n, float h, float* hS, float* hVx,
                                 float* hVy, float* hVz, uint32_t* hnbr, int64_t out_stride, int out_order,
                                 pi_stream stream);

/* ---- Batches: many independent systems per context --------------------
 *
 * A batch context holds num_systems independent systems, each with its own
 * box, cutoff and particle capacity; one pi_batch_bin / pi_batch_interact
 * runs every step of the path for all of them in one launch per kernel
 * (the interaction hands out the X-rows of all systems from one work
 * queue).  Particles are concatenated in system order: in a call with
 * counts n[0..S-1], system s owns the input entries and the sorted slots
 * [P_s, P_s + n[s]), P_s = n[0] + ... + n[s-1]; its cells follow those of
 * the systems before it in the counts/offsets arrays.  The single-system
 * calls above are the num_systems = 1 case.
 */

/* Creates a batch context on the current device.  boxes, r_c and n_max are
 * host arrays of num_systems entries (1 <= num_systems <= 2048), each checked
 * as in pi_create (Sec. 3's grid per system); the total of the cells stays
 * below 2^31 and the total of n_max below 2^31 - 64.  Errors:
 * PI_ERR_INVALID_ARG, PI_ERR_NOMEM, PI_ERR_CUDA.
 */
pi_status pi_batch_create(int32_t num_systems, const pi_box* boxes, const float* r_c,
                          const int64_t* n_max, pi_ctx** out);

/* Binning of every system (as pi_bin: Sec. 2, Fig. 1).  x, y, z: device
 * arrays of the concatenated positions; n: host array of num_systems counts,
 * 0 <= n[s] <= n_max[s].  Errors: as pi_bin.
 */
pi_status pi_batch_bin(pi_ctx* ctx, const float* x, const float* y, const float* z,
                       const int64_t* n, pi_stream stream);

/* Interaction of every system (as pi_interact: Sec. 2, Sec. 3).  h: host
 * array of num_systems kernel lengths, each as in pi_interact.  Outputs are
 * device arrays of the concatenated particles.  Errors: as pi_interact.
 */
pi_status pi_batch_interact(pi_ctx* ctx, const float* h, float* S, float* Vx, float* Vy, float* Vz,
                            uint32_t* nbr, int out_order, pi_stream stream);

/* Autotuner of the interaction for the data of the last pi_bin /
 * pi_batch_bin (Sec. 5 sizes its launches from M_C and the shared memory;
 * here the candidates are measured instead): runs the interaction
 * (arguments as pi_batch_interact, h one entry per system) once untimed and
 * `reps` times timed (1 <= reps <= 100) with each tile shape of the tiled
 * algorithm (PI_OPT_TILE 0..6), then with PI_ALGO_PPNL, and -- for a batch
 * context -- with a shape per occupancy regime: the systems are grouped by
 * mean particles per cell (below 4, 4 to 8, 8 and more), each group is
 * timed alone with shapes 5 and 6 and takes the faster, and the resulting
 * per-system plan (pi_batch_set_tiles) is timed as a whole.  The candidate
 * with the smallest median time is kept for later calls (PI_OPT_ALGO,
 * PI_OPT_TILE or the per-system plan); *chosen receives its index (0..6 =
 * tile shape, 7 = PI_ALGO_PPNL, 8 = the per-regime plan) and ms[9] the
 * medians in milliseconds (ms[8] = 0 for a single system); either pointer
 * may be NULL.  The choice changes only the speed: every tile shape sums
 * each target's terms in the same order, so their outputs are identical;
 * PPNL's agree with them within the stated tolerance.  Synchronises
 * `stream`.  The output arrays hold the results of the chosen
 * configuration.  Errors: those of pi_batch_interact, PI_ERR_INVALID_ARG,
 * PI_ERR_CUDA (the previous configuration is then kept). */
pi_status pi_autotune(pi_ctx* ctx, const float* h, float* S, float* Vx, float* Vy, float* Vz,
                      uint32_t* nbr, int out_order, int reps, int32_t* chosen, float* ms,
                      pi_stream stream);

/* Number of systems, total cells and total particle capacity (host outputs,
 * any may be NULL).  No passage of the paper: library housekeeping. */
pi_status pi_batch_info(const pi_ctx* ctx, int32_t* num_systems, int64_t* total_cells,
                        int64_t* total_n_max);

/* Per-system tile shapes of a batch context (a shape per occupancy regime
 * of the systems; Sec. 5 sizes its kernels per problem): tiles is a
 * host array of num_systems entries, each 5 (two targets per thread) or 6
 * (four targets per thread), or NULL to clear the plan.  Under a plan
 * pi_batch_interact (with PI_ALGO_TILED) makes one launch of each shape in
 * use, over the P ranges of its systems; outputs do not depend on the
 * shapes.  The ranges are written into the context by a small launch on the
 * interaction's stream whenever the plan or the particle counts change.
 * pi_autotune may set a plan.  Host-side only.  Errors: PI_ERR_INVALID_ARG. */
pi_status pi_batch_set_tiles(pi_ctx* ctx, const int32_t* tiles);

/* The per-system tile shapes in use into tiles (host array of num_systems):
 * 5 or 6 under a plan, -1 for every system without one.  No passage of the
 * paper: library housekeeping. */
pi_status pi_batch_tiles(const pi_ctx* ctx, int32_t* tiles);

/* Grid dimensions (nx, ny, nz) of one system into dims (host array of 3):
 * n_d = max(1, floor((hi_d - lo_d) / r_c)), the grid of cells at least r_c
 * wide of Sec. 3.  PI_ERR_INVALID_ARG for a system index out of range. */
pi_status pi_batch_grid(const pi_ctx* ctx, int32_t system, int32_t dims[3]);

/* Grid dimensions (nx, ny, nz) of the first system into dims (host array of
 * 3), as pi_batch_grid (Sec. 3's grid of cells at least r_c wide). */
pi_status pi_grid(const pi_ctx* ctx, int32_t dims[3]);

/* Borrowed device pointers to the binning results, valid until the next
 * pi_bin or pi_destroy (any pointer argument may be NULL): the arrays of
 * Fig. 1 and Sec. 2 --
 *   counts[C] particles per cell; offsets[C+1] start of each cell in sorted
 *   order, offsets[C] = n; perm[n] input index of sorted slot k;
 *   sx, sy, sz[n] positions in sorted order (the secondary SoA copy).
 * The library owns them; read them only after the work of the last pi_bin
 * on its stream is complete. */
pi_status pi_binned(const pi_ctx* ctx, const uint32_t** counts, const uint32_t** offsets,
                    const uint32_t** perm, const float** sx, const float** sy,
                    const float** sz);

/* Copies the binning results of the last pi_bin (Fig. 1 and Sec. 2, as in
 * pi_binned) into caller-owned device buffers, asynchronously on `stream`
 * (any pointer may be NULL to skip it):
 * counts[C], offsets[C+1] (uint32), perm[n] (uint32), sx, sy, sz[n] (FP32),
 * with C and n as in pi_binned().  Errors: PI_ERR_INVALID_ARG,
 * PI_ERR_NOT_BINNED, PI_ERR_CUDA. */
pi_status pi_copy_binned(const pi_ctx* ctx, uint32_t* counts, uint32_t* offsets, uint32_t* perm,
                         float* sx, float* sy, float* sz, pi_stream stream);

/* FP64 totals for the invariant check of the interaction's vector sums: each
 * within-cutoff pair appears once from each side with opposite d_ij, so the
 * V outputs of a system total zero up to rounding (Sec. 2's pair set is
 * symmetric).  v: device FP32 array over the particles of the last pi_bin
 * (any of the outputs of pi_interact, in either order); out: device array of
 * num_systems doubles, out[s] = sum of v over system s, accumulated in FP64
 * in a fixed order (the same result on every run).  Asynchronous on stream.
 * Errors: PI_ERR_INVALID_ARG, PI_ERR_NOT_BINNED, PI_ERR_CUDA. */
pi_status pi_total_f64(pi_ctx* ctx, const float* v, double* out, pi_stream stream);

/* Synchronises `stream`, then returns the device-side status of the work
 * enqueued so far (PI_ERR_CHECK in a debug build, PI_ERR_TIMEOUT,
 * PI_ERR_OUT_OF_BOX, PI_ERR_CAPACITY or PI_OK) and, if max_per_cell is not NULL, M_C of the last pi_bin (the
 * largest cell count, which Sec. 5.1 uses to size its shared memory).  The
 * status check itself has no passage in the paper: library housekeeping. */
pi_status pi_sync_status(pi_ctx* ctx, pi_stream stream, uint32_t* max_per_cell);

/* Sets an option (keys PI_OPT_*).  Host-side only; takes effect for work
 * enqueued afterwards.  Errors: PI_ERR_INVALID_ARG for an unknown key or
 * value.  The options select among the paper's kernels (Alg. 1, Sec. 7.1-7.2)
 * and the build's own shapes; the call itself is library housekeeping. */
pi_status pi_set_option(pi_ctx* ctx, int key, int64_t value);

/* Exclusive scan of per-cell counts that allocates nothing.
 *
 * No passage of the paper corresponds to this entry point: it is the scan of
 * pi_bin's step a3 offered on its own to callers that cannot allocate device
 * memory -- code whose device memory is reserved up front by another
 * allocator (a framework's caching allocator, a solver that owns a fixed
 * budget), or a latency-critical loop that must not call cudaMalloc/cudaFree,
 * which can synchronise the whole device.
 *
 *   counts  device array of C uint32 counts (caller-owned, read only),
 *           16-byte aligned (the scan reads four counts at a time).
 *   C       1 <= C <= 16,777,216 (2^24); larger C returns PI_ERR_CAPACITY.
 *   offsets device array of C+1 uint32 (caller-owned, written), 16-byte
 *           aligned: offsets[c] = sum of counts[0..c-1], offsets[C] = the
 *           total.  A pointer that is not 16-byte aligned (a view that
 *           starts at an odd element, say) returns PI_ERR_INVALID_ARG with
 *           nothing enqueued.
 *   result  optional device array of 2 uint32 (caller-owned, written):
 *           result[0] = the largest count (M_C), result[1] = device error
 *           bits (0 = ok; non-zero means a bounded wait ran out and offsets
 *           are undefined).  May be NULL.
 * Asynchronous on `stream`.  Calls no cudaMalloc, cudaFree or allocating
 * routine: the scan's scratch (a 256-byte control block and one 8-byte
 * descriptor per 4096 counts, about 33 KB in all) is one fixed __device__
 * array that every GPU loading the library holds until the process exits.
 * The first call on a device looks up that array's device address (with the
 * device current) and caches it; make that first call before any stream
 * capture.  Every call shares the array and clears what it needs first, so
 * calls that may overlap on the GPU (other streams, other host threads) race
 * and must be serialised by the caller.  If that first look-up fails, the
 * failure is kept for the device and every later call on it returns
 * PI_ERR_CUDA; pi_last_error() names the cause of every error.
 * Errors: PI_ERR_INVALID_ARG, PI_ERR_CAPACITY (also for a device index of
 * 64 or more), PI_ERR_CUDA. */
pi_status pi_scan_counts_noalloc(const uint32_t* counts, int64_t C, uint32_t* offsets,
                                 uint32_t* result, pi_stream stream);

/* ---- Serving: a request loop over device-resident slots ---------------
 *
 * Continuous batching on one GPU, as a native host loop.  A server owns
 * "slots": single-system contexts, each with its own stream, completion
 * event and pinned scratch block.  A job runs on one slot as one
 * pi_submit_host_strided call (re-target to the job's box and cutoff, copy
 * in, bin, interact, copy out) -- the kernels a lone pi_bin + pi_interact
 * would run, so a job's results do not depend on the jobs beside it.  Slots
 * come in capacity buckets; a job waits in the queue of the smallest bucket
 * whose capacity holds both its particles and its grid's cells, and may also
 * take a free slot of a larger bucket.  When every slot that fits a job is
 * busy, the server makes a new one while the bucket's slot limit, the HBM
 * budget and the device's free memory allow (memory-based admission);
 * otherwise the job waits.  Completion is polled with cudaEventQuery.
 */
typedef struct pi_server pi_server;

enum { PI_SERVER_MAX_BUCKETS = 16 };

/* One request (host memory; pinned memory makes the copies asynchronous). */
typedef struct {
    const float* x;      /* positions: n entries each; with in_stride > 0,   */
    const float* y;      /* y and z are x + in_stride and x + 2*in_stride    */
    const float* z;      /* (one block, one copy) and these two are ignored  */
    int64_t in_stride;   /* 0 or a stride as in pi_submit_host_strided       */
    int64_t n;           /* particles, >= 0                                  */
    pi_box box;          /* the job's box and cutoff (any grid that fits a   */
    float r_c;           /* bucket)                                          */
    float h;             /* kernel length, > 0                               */
    float* S;            /* outputs, n entries each, in input order; all    */
    float* Vx;           /* four NULL: the results go to the slot's scratch  */
    float* Vy;           /* block, which the slot's next job overwrites      */
    float* Vz;
    uint32_t* nbr;       /* neighbour counts, or NULL                        */
    int64_t out_stride;  /* 0 or a stride as in pi_submit_host_strided       */
    double arrival;      /* seconds after the start of pi_server_run         */
    double t_start;      /* written: when the job was enqueued on a slot     */
    double t_done;       /* written: when its completion was seen            */
    int64_t slot_capacity; /* written: capacity of the slot that ran it      */
} pi_job;

/* (The serving calls below have no passage in the paper, which runs one
 * system at a time; each job is one step of Sec. 2's method.)
 * Device memory one slot of the given particle capacity is charged against
 * the HBM budget: capacity * 144 bytes + 1 MiB (the context, up to one cell
 * per particle, and its staging buffers). */
int64_t pi_server_slot_bytes(int64_t capacity);

/* Creates a server on the current device (no passage of the paper: the
 * request loop is the build's own).  capacity: num_buckets (1 ..
 * PI_SERVER_MAX_BUCKETS) distinct particle capacities (each also the cell
 * capacity of its slots), 1 .. 2^30; initial_slots: slots made at once per
 * bucket (NULL: none; fewer if the budget runs out); max_slots_per_bucket >=
 * 1; hbm_budget: bytes the slots may be charged (<= 0: half of the device's
 * free memory).  Errors: PI_ERR_INVALID_ARG, PI_ERR_NOMEM, PI_ERR_CUDA.
 */
pi_status pi_server_create(int32_t num_buckets, const int64_t* capacity, const int32_t* initial_slots,
                           int32_t max_slots_per_bucket, int64_t hbm_budget, pi_server** out);

/* Serves num_jobs jobs (each one step of Sec. 2's method), blocking until all
 * are complete: a job is admitted once `arrival` seconds have passed since
 * the call started and a slot that fits it is free (oldest arrival first).
 * Writes each job's t_start, t_done and slot_capacity, and the time from the
 * start to the last completion into *makespan_s (may be NULL).  Every job is
 * checked first: PI_ERR_INVALID_ARG for a bad job, PI_ERR_CAPACITY for one
 * that fits no bucket (nothing runs then).  Afterwards the device status of
 * every slot is collected as in pi_sync_status.  The host arrays of a job
 * must stay valid until the call returns.  The calling thread polls while
 * jobs run (it sleeps only when nothing is running or queued).  Like a
 * context, a server is used by one host thread at a time.
 */
pi_status pi_server_run(pi_server* srv, pi_job* jobs, int64_t num_jobs, double* makespan_s);

/* Buckets (num_buckets; capacity and slots as arrays of that length, any
 * pointer may be NULL) and the bytes charged to the HBM budget.  No passage
 * of the paper: library housekeeping. */
pi_status pi_server_info(const pi_server* srv, int32_t* num_buckets, int64_t* capacity, int32_t* slots,
                         int64_t* hbm_used);

/* Destroys the server and its slots (waits for their streams).  NULL is
 * accepted.  No passage of the paper: library housekeeping. */
pi_status pi_server_destroy(pi_server* srv);

/* Number of kernels this context has launched since pi_create (host
 * counter).  No passage of the paper: library housekeeping. */
pi_status pi_launch_count(const pi_ctx* ctx, uint64_t* count);

/* Synchronises `stream` and reads the target-source evaluations the direct
 * kernels counted since the last pi_bin (PI_OPT_COUNT_EVALS) into
 * *evaluations; divided by the within-cutoff pairs (the sum of the nbr
 * output) it is the evaluations per useful pair.  PI_ERR_INVALID_ARG for a
 * NULL argument, PI_ERR_CUDA if the stream or the copy fails.  No passage of
 * the paper: library diagnostics (Sec. 7.2 counts the candidates of the
 * 27-cell stencil; this counts what the culling leaves). */
pi_status pi_eval_count(pi_ctx* ctx, pi_stream stream, uint64_t* evaluations);

/* Static text for a status code.  No passage of the paper: library
 * housekeeping. */
const char* pi_status_str(pi_status s);

/* Text of the last error seen by this host thread ("" if none): the CUDA
 * error of a failed runtime call, or the reason of some argument errors.
 * No passage of the paper: library housekeeping. */
const char* pi_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PI_H */
