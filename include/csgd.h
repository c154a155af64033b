/*
 * csgd.h - C ABI of the GB300 (sm_103a) block solver for y = Ax + e.
 *
 * Method: Gao & Blumensath, "Distributed computation of linear inverse problems
 * with application to computed tomography reconstruction" (arXiv:1709.00953):
 * coordinate-reduced steepest gradient descent (CSGD, Alg. 1-3) and its grouped
 * variant (GCSGD, Alg. 4).  A is never stored: every entry A_i^j (length of
 * ray i inside voxel j, Sec. II-A) is recomputed on the GPU by Siddon traversal.
 *
 * Conventions shared by every call
 * --------------------------------
 * Status: every function returns an int32_t status, CSGD_OK (0) or a negative
 *   CSGD_ERR_* code; csgd_last_error() returns a message for the calling
 *   thread's last failure.  Nothing throws across this ABI.
 * Handles: created by *_create / csgd_block_partition, released by *_destroy.
 *   Destroy functions accept NULL and return CSGD_OK.  A partition keeps a
 *   reference to nothing the caller owns (it copies what it needs), but it must
 *   outlive the solvers created from it, and a geometry must outlive its
 *   partitions.
 * Vectors: FP32, contiguous, owned by the caller, never retained after the
 *   call returns.  Unless a flag says otherwise they are DEVICE pointers (for
 *   example torch.Tensor.data_ptr() of a CUDA tensor) on the current device.
 *   Volumes are row-major [nz][ny][nx] (x fastest; nz = 1 in 2D); sinograms are
 *   [view][v-bin][u-bin] (u fastest).
 * Streams: a csgd_stream is a cudaStream_t; NULL is the legacy default stream.
 *   Device work is enqueued asynchronously on it unless a function says it
 *   synchronises.  Calls that use the same solver must be issued on one stream
 *   (or be serialised by the caller).
 * Geometry (the paper is silent on these; every part of this project uses
 *   them): the grid is centred on the origin with cubic voxels of edge h; view
 *   angle t gives the central direction d_c = (-cos t, -sin t, 0), the detector
 *   axes e_u = (-sin t, cos t, 0) and e_v = (0, 0, 1); the centre of bin k of n
 *   lies at (k - (n-1)/2) * pitch; flat detectors are perpendicular to d_c at
 *   distance sdd from the source S = sod (cos t, sin t, 0) (Sec. II-D); the
 *   curved detector is an arc centred on the source with angular pitch.
 */
#ifndef CSGD_H
#define CSGD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CSGD_OK 0
#define CSGD_ERR_INVALID_ARG (-1)
#define CSGD_ERR_OOM (-2)
#define CSGD_ERR_CUDA (-3)
#define CSGD_ERR_TIMEOUT (-4)
#define CSGD_ERR_STATE (-5)
#define CSGD_ERR_UNSUPPORTED (-6)

typedef struct csgd_geometry csgd_geometry;
typedef struct csgd_partition csgd_partition;
typedef struct csgd_solver csgd_solver;
typedef void* csgd_stream; /* cudaStream_t */

/* ---------------------------------------------------------------------------
 * Geometry (Sec. II-A model, Sec. II-D / Sec. III scan set-ups)
 * ------------------------------------------------------------------------- */
enum {
    CSGD_PARALLEL_2D = 0,  /* rays along d_c through s_k e_u                   */
    CSGD_FAN_2D_FLAT = 1,  /* point source, flat detector                      */
    CSGD_FAN_2D_CURVED = 2,/* point source, detector arc centred on the source */
    CSGD_CONE_3D = 3,      /* point source on a circle, flat 2D detector       */
    CSGD_CUSTOM_3D = 4     /* arbitrary per-view source / detector poses       */
};

typedef struct {
    int32_t kind;          /* CSGD_PARALLEL_2D .. CSGD_CUSTOM_3D                  */
    int32_t n[3];          /* voxels along x, y, z (n[2] is ignored in 2D)        */
    double h;              /* voxel edge (world units, > 0)                       */
    int32_t n_views;       /* number of views (> 0)                               */
    const double* angles;  /* host, n_views angles in radians (kinds 0..3)        */
    const double* poses;   /* host, n_views x 12: S, C, e_u, e_v (CUSTOM_3D only);
                              e_u, e_v unit, orthogonal, perpendicular to C - S    */
    int32_t nu, nv;        /* detector bins along e_u and e_v (nv = 1 in 2D)      */
    double pu, pv;         /* bin pitch (world units; radians along the arc for
                              CSGD_FAN_2D_CURVED)                                 */
    double sod, sdd;       /* source-origin and source-detector distance (fan and
                              cone kinds); the source must lie outside the grid's
                              circumscribed sphere                                 */
} csgd_geometry_desc;

/* Validates and copies desc (host arrays are copied).  Host only, no GPU work.
 * CSGD_ERR_INVALID_ARG on a malformed description. */
int32_t csgd_geometry_create(const csgd_geometry_desc* desc, csgd_geometry** out);
int32_t csgd_geometry_destroy(csgd_geometry* geom);

/* ---------------------------------------------------------------------------
 * Block partition (Eq. e1; Sec. II-D domain decomposition; Alg. 3 P(I,J))
 * ------------------------------------------------------------------------- */
typedef struct {
    int32_t tiles[3];      /* column blocks: cuboid tiles per axis; along an axis
                              with N voxels and T tiles, tile t covers
                              [floor(tN/T), floor((t+1)N/T)).  Tile index
                              j = (tz*TY + ty)*TX + tx.  tiles[2] ignored in 2D.  */
    int32_t view_blocks;   /* number of view sets (ignored if view_block_of)      */
    const int32_t* view_block_of; /* optional host map view -> view set (values
                              0..B-1, every set non-empty); NULL = contiguous
                              views split at floor(kV/B)                           */
    int32_t det_blocks_u;  /* detector sub-areas along u (bins split at floor(k nu/DU)) */
    int32_t det_blocks_v;  /* ... and along v                                     */
} csgd_partition_desc;

typedef struct {
    int32_t m;             /* row blocks: m = B * DV * DU; row block
                              i = (vb*DV + dv)*DU + du = view set x sub-area      */
    int32_t n;             /* column blocks (tiles)                               */
    int64_t n_rays;        /* rows of A = n_views * nu * nv                        */
    int64_t n_voxels;      /* columns of A                                        */
    int64_t z_floats;      /* floats of the solver's z store (shadow rectangles)  */
} csgd_partition_info;

/* Builds the row and column blocks, the importance table P(I,J) = P_S/P_T of
 * Alg. 3 (exact shadow of each tile, in detector-bin units) and the per
 * (view, tile) ray tables, and uploads the tables to the current device
 * (synchronously).  CSGD_ERR_INVALID_ARG on bad counts, CSGD_ERR_OOM /
 * CSGD_ERR_CUDA on device failures. */
int32_t csgd_block_partition(const csgd_geometry* geom, const csgd_partition_desc* desc,
                             csgd_partition** out);
int32_t csgd_partition_destroy(csgd_partition* part);
int32_t csgd_partition_get_info(const csgd_partition* part, csgd_partition_info* info);

/* P(I,J) of Alg. 3 as an m x n row-major host array P[i*n + j] (FP64). */
int32_t csgd_partition_probabilities(const csgd_partition* part, double* P);

/* ---------------------------------------------------------------------------
 * Block operators (Alg. 1: z_I = A_I^J x_J and g_J = (A_I^J)^T r_I)
 * ------------------------------------------------------------------------- */
/* out[i] = (accumulate ? out[i] : 0) + sum_{j in J} A_ij x_j for every row i of
 * the union of the row blocks row_blocks[0..n_rb) (host array, distinct
 * indices); column block J = tile j.  x: full volume (device); out: full
 * sinogram (device); rows outside the union are not touched.  Lengths are
 * recomputed by Siddon traversal in FP32 with compensated accumulation. */
int32_t csgd_project_block(const csgd_partition* part, const int32_t* row_blocks, int32_t n_rb,
                           int32_t j, const float* x, float* out, int32_t accumulate,
                           csgd_stream stream);

/* g[v] = (accumulate ? g[v] : 0) + sum_{i in I} A_iv r_i for every voxel v of
 * tile j (other voxels untouched); I = union of row_blocks.  r: full sinogram
 * (device); g: full volume (device).  The same Siddon lengths as
 * csgd_project_block (the same plane crossings), gathered per voxel over the
 * rays of its shadow (no atomics), with compensated accumulation over views. */
int32_t csgd_backproject_block(const csgd_partition* part, const int32_t* row_blocks,
                               int32_t n_rb, int32_t j, const float* r, float* g,
                               int32_t accumulate, csgd_stream stream);

/* Backprojection that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory while they
 * run, such as a pre-planned real-time loop that must not call cudaMalloc or an
 * embedding whose memory is all handed out at start-up.  It computes the same g
 * as csgd_backproject_block (same kernels, same arguments and layouts), but its
 * scratch ray table is a fixed array of CSGD_NOALLOC_MAX_RAYS records (32 bytes
 * each, 8 MiB) in the library's global memory, held by every GPU that loads the
 * library until the process exits; it calls no cudaMalloc, cudaFree or other
 * allocating routine, host or device, when it succeeds.
 * Requirements and limits:
 *  - the rays of the call (views of the row blocks x bins of the tile's shadow
 *    in their sub-areas) must number at most CSGD_NOALLOC_MAX_RAYS; otherwise
 *    CSGD_ERR_INVALID_ARG is returned and nothing is launched;
 *  - the partition's tables must already be on the device: make one ordinary
 *    device call with it first (for example csgd_project_block), otherwise
 *    CSGD_ERR_STATE is returned;
 *  - the first call on a device looks up the array's device address with that
 *    device current; make that first call before any stream capture;
 *  - all calls share the array and it keeps the last call's contents: calls
 *    that overlap on the GPU (other streams, other host threads) race on it and
 *    must be serialised by the caller. */
#define CSGD_NOALLOC_MAX_RAYS 262144
int32_t csgd_backproject_block_noalloc(const csgd_partition* part, const int32_t* row_blocks,
                                       int32_t n_rb, int32_t j, const float* r, float* g,
                                       int32_t accumulate, csgd_stream stream);

/* out = A x over all rows and all tiles (device pointers). */
int32_t csgd_project_full(const csgd_partition* part, const float* x, float* out,
                          csgd_stream stream);

/* ---------------------------------------------------------------------------
 * Solver (Alg. 2 / 3 / 4 around the Alg. 1 step)
 * ------------------------------------------------------------------------- */
enum { CSGD_SAMPLE_SEQUENTIAL = 0, CSGD_SAMPLE_UNIFORM = 1, CSGD_SAMPLE_IMPORTANCE = 2,
       CSGD_SAMPLE_MIXED = 3 };
enum { CSGD_SYNC_COLUMN = 0, CSGD_SYNC_EPOCH = 1 };

typedef struct {
    int32_t sampling;      /* CSGD_SAMPLE_*: Alg. 2 order, uniform, Alg. 3
                              importance, Sec. III-D mixed                        */
    int32_t sync;          /* CSGD_SYNC_COLUMN: refresh r after each column block
                              (Alg. 2-4 as printed); CSGD_SYNC_EPOCH: one refresh
                              per epoch (Sec. II-F parameter-server reading)       */
    int32_t group_size;    /* s of Alg. 4 (1 = CSGD)                               */
    int32_t reserved;
    double alpha;          /* fraction of row blocks drawn per column block       */
    double gamma;          /* fraction of column blocks visited per epoch         */
    double b;              /* beta = b * P_S(I_g,J) / P_T(J)                       */
    double theta_step;     /* mixed sampling: theta grows by this per epoch       */
    uint64_t seed;         /* SplitMix64 seed of the block schedule               */
} csgd_solver_params;

/* Random choice of blocks, shared bit-for-bit with any implementation of the
 * same rules: SplitMix64 (Steele, Lea & Flood 2014); per epoch a Fisher-Yates
 * column permutation (first ceil(gamma n) columns), then per column
 * ceil(alpha m / s) groups of s weighted draws without replacement (walk the
 * remaining blocks in index order; the first whose running weight sum exceeds
 * u * total is taken; drawing stops when no positive weight is left).
 * Writes, for n_epochs epochs from the seed, the flat encoding
 *   per epoch: n_cols, then per column: j, n_groups, then per group: size, rows...
 * into out (host, capacity ints); *len receives the length (also when the
 * capacity is too small, in which case CSGD_ERR_INVALID_ARG is returned). */
int32_t csgd_schedule_generate(const csgd_partition* part, const csgd_solver_params* params,
                               int32_t n_epochs, int32_t* out, int64_t capacity, int64_t* len);

/* Device bytes a solver on this partition allocates (admission control). */
int32_t csgd_solver_footprint_bytes(const csgd_partition* part, const csgd_solver_params* params,
                                    int64_t* bytes);

/* Allocates the solver state on the current device and initialises it from y
 * (device sinogram, copied): x = 0, z = 0, r = y (Alg. 2 initialisation).
 * Synchronises the stream.  CSGD_ERR_OOM when the device is full. */
int32_t csgd_solver_create(const csgd_partition* part, const csgd_solver_params* params,
                           const float* y, csgd_stream stream, csgd_solver** out);
int32_t csgd_solver_destroy(csgd_solver* solver);

/* Re-initialises the state from new data y (host pointer if y_on_host != 0,
 * else device) and restarts the schedule from the seed.  Asynchronous. */
int32_t csgd_solver_reset(csgd_solver* solver, const float* y, int32_t y_on_host,
                          csgd_stream stream);

typedef struct {
    int32_t j;             /* column block                                        */
    int32_t n_rows;        /* number of row blocks in the group                   */
    const int32_t* row_blocks; /* host, distinct row block indices                */
} csgd_block_choice;

typedef struct {
    int64_t step;          /* global step index                                   */
    int32_t j;             /* column block (-1 in csgd_solver_history)            */
    int32_t n_rows;        /* row blocks in the group (-1 in csgd_solver_history) */
    double beta, gg, qq, mu; /* beta of Alg. 3; g^T g; ||A g||^2; step length      */
    int64_t nnz;           /* non-zeros of A_{I_g}^J (history only)               */
} csgd_step_info;

/* One Alg. 1 step.  choice == NULL takes the next step of the schedule (and
 * ends the column batch / epoch when the schedule does); otherwise the given
 * block choice is applied as a batch of its own (refresh after it).  If info is
 * non-NULL the stream is synchronised and the step's scalars are returned. */
int32_t csgd_solve_step(csgd_solver* solver, const csgd_block_choice* choice,
                        csgd_step_info* info, csgd_stream stream);

typedef struct {
    int64_t steps;         /* steps executed by this call                         */
    int64_t epochs;        /* epochs closed so far                                */
    int64_t nnz;           /* non-zeros of A visited by the forward passes        */
    double updates;        /* ray-voxel updates = 3 * nnz (one backprojection and
                              two forward products per non-zero)                  */
    double residual_norm;  /* ||y - A x|| (FP64), only if compute_residual       */
    int64_t rays;          /* sum over the steps of the rays of I_g that can meet
                              tile J (the rows a step reads r and writes z on)    */
    int64_t tile_voxels;   /* sum over the steps of the voxels of tile J          */
} csgd_report;

/* Runs n_steps steps of the schedule, then closes the epoch (refresh and
 * averaging, even mid-epoch) and writes x (row-major volume) to x_out (host
 * pointer if x_on_host != 0, else device; may be NULL).  If report is non-NULL
 * the stream is synchronised and the report filled; compute_residual != 0 adds
 * a full forward projection for ||y - A x||. */
int32_t csgd_solve(csgd_solver* solver, int64_t n_steps, float* x_out, int32_t x_on_host,
                   csgd_report* report, int32_t compute_residual, csgd_stream stream);

/* Copies the per-step scalars of the last `capacity` steps since the last reset
 * (oldest first) to out (host); *count receives how many were written. */
int32_t csgd_solver_history(csgd_solver* solver, csgd_step_info* out, int64_t capacity,
                            int64_t* count);

/* Checkpoint and resume (the paper has no counterpart: the paper's runs are
 * short; long or preemptible runs need it).  The state of a solver is its whole
 * iteration state: y, x, x^, the per-tile candidate counts, r, the z store, the
 * pending refresh of epoch sync, the schedule's generator state and the rest of
 * the current epoch's schedule, the counters (epochs, steps, non-zeros) and the
 * per-step history.  It is written to a caller-owned host buffer in a
 * versioned, self-describing layout (little-endian, as the host writes it).
 *   csgd_solver_state_bytes: size of the state of this solver, in bytes.
 *   csgd_solver_get_state: writes the state to buf (capacity bytes, at least
 *     csgd_solver_state_bytes); synchronises the stream.  CSGD_ERR_INVALID_ARG
 *     if the buffer is too small.
 *   csgd_solver_set_state: restores a state written by csgd_solver_get_state of
 *     a solver on an equal partition (same sizes) with equal parameters; the run
 *     then continues exactly as the saved one would have.  Synchronises the
 *     stream.  CSGD_ERR_STATE if the buffer is not such a state (bad magic or
 *     version, other sizes or parameters, truncated); the solver is unchanged
 *     then. */
int32_t csgd_solver_state_bytes(const csgd_solver* solver, int64_t* bytes);
int32_t csgd_solver_get_state(csgd_solver* solver, void* buf, int64_t capacity,
                              csgd_stream stream);
int32_t csgd_solver_set_state(csgd_solver* solver, const void* buf, int64_t size,
                              csgd_stream stream);

/* ---------------------------------------------------------------------------
 * Solves as CUDA graphs, and many solves in one launch
 * (the paper has no counterpart: these serve batched and repeated solves)
 * ------------------------------------------------------------------------- */
typedef struct csgd_graph csgd_graph;

/* Captures a whole solve of this solver into a CUDA graph: reset to x = 0,
 * z = 0, r = y (the solver's current y), then n_steps steps of the schedule
 * from the seed, closing the epoch at the end, then x to x_out (device, or
 * pinned host memory if x_on_host; may be NULL).  The schedule is planned and
 * uploaded once, here; every launch repeats the same solve.  Launching the
 * graph leaves the solver's host-side counters (epochs, steps) untouched, so
 * mixing graph launches with csgd_solve needs a csgd_solver_reset in between.
 * A solver's graph must not run concurrently with other work on that solver. */
int32_t csgd_solver_graph_create(csgd_solver* solver, int64_t n_steps, float* x_out,
                                 int32_t x_on_host, csgd_graph** out);
/* One graph that runs the given solve graphs concurrently (child graphs without
 * dependencies): all block steps of all problems in one launch.  The parts must
 * belong to different solvers and must outlive nothing: the batch copies them. */
int32_t csgd_graph_batch_create(csgd_graph* const* parts, int32_t n, csgd_graph** out);
/* Enqueues the graph on the stream (asynchronous). */
int32_t csgd_graph_launch(csgd_graph* graph, csgd_stream stream);
int32_t csgd_graph_destroy(csgd_graph* graph);

/* Many solves in ONE persistent kernel launch with a device work queue (the
 * paper's parallel block steps, Sec. II-F, taken across problems: the paper
 * has no batching of its own).  For every solver the whole solve is planned as
 * in csgd_solver_graph_create (reset, n_steps[k] steps of the schedule from
 * the seed, the epoch closed at the end, x to the device array x_out[k] if not
 * NULL); each kernel of it becomes a task of thread blocks, and the problems'
 * task lists are interleaved.  One launch of the executor (captured with the
 * solvers' resets in a CUDA graph) runs all of them: each block takes the next
 * block of work from a ticket counter, waits until its problem's earlier
 * kernels have completed, runs it and counts it as done.  Every such wait is
 * bounded by wait_limit_ns of GPU time (0 selects 2 s); a wait that runs out
 * stops the launch and csgd_batch_status returns CSGD_ERR_TIMEOUT.
 * The executor runs every solve with its solver's lanes per ray (1 when the
 * model chooses), 256-thread blocks and, for the gather backprojection, 4 view
 * groups per block (bricks run as the scatter): results equal the solvers' own
 * solves to rounding.  The solvers
 * must stay alive, on one device, all 2D or all 3D, and must not be used
 * otherwise while the batch may run (the batch keeps their planned schedules
 * on the device).
 *   stall_last_task: a test hook: the last task of the first problem waits for
 *   a block of work that never completes, so that the bound on the wait can be
 *   checked; 0 in normal use. */
typedef struct csgd_batch csgd_batch;
typedef struct {
    int64_t wait_limit_ns;
    int32_t stall_last_task;
    int32_t reserved;
} csgd_batch_params;
int32_t csgd_batch_create(csgd_solver* const* solvers, const int64_t* n_steps,
                          float* const* x_out, int32_t n, const csgd_batch_params* params,
                          csgd_batch** out);
/* Enqueues the batch's graph on the stream (asynchronous). */
int32_t csgd_batch_launch(csgd_batch* batch, csgd_stream stream);
/* Waits for the batch's last launch; CSGD_ERR_TIMEOUT if one of its waits ran
 * out (the solvers' states are then undefined), CSGD_OK otherwise. */
int32_t csgd_batch_status(csgd_batch* batch);
/* Tasks, blocks of work and executor blocks of the batch (for reports). */
int32_t csgd_batch_info(csgd_batch* batch, int32_t* n_tasks, int64_t* n_units, int32_t* grid);
int32_t csgd_batch_destroy(csgd_batch* batch);

/* Launch shapes (the paper has no counterpart: these tune the GPU kernels, not
 * the method).  bp_groups = view groups per backprojection CTA (1..8) of the
 * voxel-driven gather, -1 for the ray-driven scatter backprojection (each
 * ray walks the tile and adds len * r to 32-bit fixed-point sums with integer
 * atomics: exact and order-independent, so also deterministic), or -2, -3, -4
 * for the brick backprojection with brick shape 0, 1, 2 (3D bricks of 16 x 16
 * x 16, 8 or 4 voxels, 2D bricks of 32^2, 16^2 or 8^2: a block per brick walks
 * the lines that cross it and sums in shared-memory fixed point); fwd_lanes =
 * lanes per ray of the dual forward and of the scatter (1, 2 or 4); 0 selects
 * the library's model (gather, occupancy-based groups, lanes by ray count).
 * They change only the rounding of the sums, i.e. results at rounding level.
 *   csgd_solver_set_launch: sets them; CSGD_ERR_INVALID_ARG out of range.
 *   csgd_solver_autotune: times the backprojection for every group count, the
 *     scatter and the three brick shapes, then the dual forward (plus the
 *     scatter, if chosen) for every lane count over the first trial_steps
 *     steps of the schedule (kernel time by CUDA events), keeps the fastest
 *     and resets the solver (x = 0, z = 0, r = y, schedule from the seed);
 *     writes the choice to bp_groups / fwd_lanes if non-NULL.  Synchronises. */
int32_t csgd_solver_set_launch(csgd_solver* solver, int32_t bp_groups, int32_t fwd_lanes);
int32_t csgd_solver_autotune(csgd_solver* solver, int64_t trial_steps, int32_t* bp_groups,
                             int32_t* fwd_lanes, csgd_stream stream);

/* Per-kernel timing (the paper has no counterpart; it supports the roofline
 * measurements).  While enabled, every kernel launch of csgd_solve /
 * csgd_solve_step is bracketed by CUDA events on the caller's stream.
 * csgd_solver_profile_read synchronises on the last event and sums the
 * elapsed times per kernel kind: 0 backprojection, 1 dual forward product,
 * 2 epilogue (z, r, x^ updates), 3 epoch close (averaging). */
typedef struct {
    int64_t launches[4];
    double ms[4];
} csgd_kernel_times;
int32_t csgd_solver_profile(csgd_solver* solver, int32_t enable);
int32_t csgd_solver_profile_read(csgd_solver* solver, csgd_kernel_times* out, int32_t reset);

/* Message of the calling thread's last failure ("" if none). */
const char* csgd_last_error(void);

/* Library version string. */
const char* csgd_version(void);

#ifdef __cplusplus
}
#endif

#endif /* CSGD_H */
