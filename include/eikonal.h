/*
 * eikonal.h -- C ABI of libeikonal.so, a B300 (sm_103a) solver for the
 * Eikonal equation ||grad phi|| = 1/F (eq. 3) on uniform 2D/3D grids by the
 * improved fast iterative method (Algorithm 2, Sec. 3): a tile active-list
 * value update without neighbour convergence checks (Step 2), then a remedy
 * pass that finds and recomputes wrongly settled values (Step 3).
 *
 * Discretisation: first-order Godunov upwind scheme, eq. (4) in 2D and eq. (6)
 * in 3D, isotropic spacing h (Alg 1.1 / Alg 1.3); every node's value is the
 * exact root of its eq.-(6) residual given its neighbours.
 *
 * Layout (every entry point): a grid is row-major (nz, ny, nx), x fastest,
 * flat index = (k*ny + j)*nx + i; a 2D grid has nz = 1.  Arrays of the
 * solver's precision are float32 (EIK_FP32, default) or float64 (EIK_FP64,
 * validation mode), both for F, source values, phi and adjoint arrays.
 *
 * Semantics:
 *   - F > 0 is a speed; F == 0 is impassable (eq. 8 barrier): such a node keeps
 *     phi = +inf unless it is a source.  Unreachable nodes get +inf.
 *   - Sources are (flat index, value) pairs held fixed (Dirichlet, Alg 2
 *     Step 1).  A duplicated index keeps the smaller value.
 *
 * Ownership: the caller owns every buffer.  Device pointers (F, phi, source
 * arrays, workspace, adjoint arrays) must be device-accessible memory of the
 * current device; "host" arrays are read during the call only.  The library
 * allocates no device memory: it uses the caller's workspace, of at least
 * eik_*workspace_size() bytes, 256-byte aligned.  All device work is enqueued
 * on `stream` (a cudaStream_t; NULL = legacy default stream).
 *
 * Synchronisation and errors: argument errors are found on the host and
 * returned before anything is enqueued.  Errors found on the device (a
 * source index out of range, the iteration cap, an internal wait that timed
 * out) are written into the workspace; they are returned, and the stream is
 * synchronised, only when `stats` is non-NULL.  With stats == NULL the call
 * returns after enqueuing (EIK_OK) and the result is ready when the stream
 * reaches that point.  Calls that share a workspace must not overlap on the
 * device.  eik_last_error() gives a thread-local message for the last
 * non-zero return.
 */
#ifndef EIKONAL_H_
#define EIKONAL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* return codes */
#define EIK_OK 0
#define EIK_ERR_ARG 1          /* invalid argument (dims, h, pointer, workspace, source index) */
#define EIK_ERR_NOCONVERGE 2   /* iteration cap reached; phi holds valid upper bounds */
#define EIK_ERR_CUDA 3         /* a CUDA launch or runtime call failed */
#define EIK_ERR_DEVICE 4       /* a bounded device-side wait timed out (eik_options.wait_limit_us);
                                  phi holds upper bounds */

/* tile shapes (nodes per tile along x, y, z) */
#define EIK_TILE_AUTO 0
#define EIK_TILE_8x8x8 1
#define EIK_TILE_4x4x4 2
#define EIK_TILE_8x8x4 3
#define EIK_TILE_16x16x1 4     /* 2D grids (nz == 1) only */
#define EIK_TILE_8x4x4 5
#define EIK_TILE_8x8x1 6       /* 2D grids (nz == 1) only */

/* schedules of the iteration loops */
#define EIK_SCHED_AUTO 0
#define EIK_SCHED_PERSISTENT 1 /* one cooperative launch, bounded grid barriers */
#define EIK_SCHED_HOSTLOOP 2   /* one launch per iteration, host reads the list size (synchronising) */
#define EIK_SCHED_ASYNC 3      /* one cooperative launch, device work queue, no per-iteration barrier */

/* Step-2 convergence test of an Active tile (Algorithm 2 moves a point to
 * Source when its recomputation no longer changes it):
 *   CONFIRM  a visit that changes nothing (the tile is visited again after
 *            any visit that changed it, in a later iteration)
 *   SWEEP    the relaxation inside a visit ends with a sweep that changes
 *            nothing (the same test, taken at sweep granularity) */
#define EIK_CONVERGE_AUTO 0
#define EIK_CONVERGE_CONFIRM 1
#define EIK_CONVERGE_SWEEP 2

/* method (the loop structure; both reach the same discrete solution):
 *   IFIM  Algorithm 2 (Sec. 3): Step 2 without neighbour convergence checks,
 *         then the remedy pass (Step 3)
 *   FIM   the fast iterative method of Sec. 2.3 at tile granularity: a
 *         visit relaxes the tile to its local fixed point, and every
 *         neighbour tile across a face whose values dropped is listed again,
 *         whatever its state (the neighbour convergence check, taken by the
 *         neighbour's own next visit); no Step 3.  `converge` and
 *         `skip_remedy` do not apply, and its one loop is reported in the
 *         Step-3 statistics (iters_remedy, tiles_remedy) */
#define EIK_METHOD_IFIM 0
#define EIK_METHOD_FIM 1

/* precision */
#define EIK_FP32 0
#define EIK_FP64 1

/* one grid: nx, ny, nz >= 1 nodes; spacing h > 0 along x, and hy, hz along
 * y and z (0 = h: the square mesh of Alg 1.1 / Alg 1.3).  Unequal spacings
 * solve eq. (5)/(6) as written with dx, dy, dz (Alg 1.2, with the validity
 * thresholds); all grids of one call must have the same ratios hy/h and hz/h
 * (hz is ignored when nz == 1), and the adjoint takes equal spacings only. */
typedef struct {
    int64_t nx, ny, nz;
    double h;
    double hy, hz;
} eik_grid;

/* per-call options; a zero-filled struct (or NULL) selects the defaults */
typedef struct {
    int32_t tile;         /* EIK_TILE_* (0 = auto: 16x16x1 for 2D, else 8x8x8) */
    int32_t schedule;     /* EIK_SCHED_* (0 = auto: persistent when co-residency allows) */
    int64_t max_iters;    /* cap per loop (update, remedy); 0 = automatic */
    int32_t precision;    /* EIK_FP32 / EIK_FP64 */
    int32_t skip_remedy;  /* 1 = stop after Step 2 (ablation; the result may be wrong) */
    float order;          /* list order: 0 = default (the Step-3 and FIM lists bucketed with width
                             4; the Step-2 lists bucketed too on 2D grids, unordered on 3D grids),
                             > 0 = both loops bucketed with this width in tile-crossing times (the
                             mean crossing time, from the mean slowness), < 0 = unordered (every
                             listed tile visited in every iteration, the schedule of Algorithm 2
                             as printed) */
    int32_t converge;     /* Step-2 convergence test of a tile (EIK_CONVERGE_*) */
    int32_t method;       /* EIK_METHOD_* (0 = IFIM) */
    int32_t wait_limit_us; /* bound on every device-side wait of the call (grid barriers, queue
                              slots), microseconds of %globaltimer; 0 = 2 s.  A wait that runs out
                              raises device flag bit 1, every thread block leaves the launch, phi
                              keeps valid upper bounds and the call reports EIK_ERR_DEVICE.  < 0 is
                              EIK_ERR_ARG. */
    float remedy_order;   /* the Step-3 (and FIM) list order alone, where the Step-2 lists are
                             unordered (3D grids with order 0, or order < 0): 0 = as `order` sets
                             it, > 0 = bucketed with this width, < 0 = unordered.  Ignored when the
                             Step-2 lists are bucketed.  Any order gives the same solution; the
                             fastest width depends on the problem (autotune.py tries some).  The
                             adjoint's width comes from `order` alone (0 = its default, 2). */
} eik_options;

/* run statistics (filled when a stats pointer is passed; the call then synchronises) */
typedef struct {
    int64_t iters_update;     /* Step-2 iterations (tile-list passes) */
    int64_t iters_remedy;     /* Step-3 loop iterations */
    int64_t tiles_update;     /* tile visits in Step 2 */
    int64_t tiles_flagged;    /* tiles put into Remedy by the Step-3 recomputation */
    int64_t tiles_remedy;     /* tile visits in the Step-3 loop */
    int64_t sweeps;           /* in-tile relaxation sweeps, summed over visits */
    int64_t tiles_deferred;   /* listed tiles passed over by the ordered schedule */
    int32_t status;           /* EIK_* code of the device-side run */
    int32_t device_flags;     /* bit 0 cap hit, bit 1 wait timeout, bit 2 bad source, bit 3 list overflow;
                                 checked build (libeikonal_debug.so) only: bit 4 a tile id out of range,
                                 bit 5 a NaN written to phi or lambda (both reported as EIK_ERR_DEVICE) */
    double ms_total;          /* device time of the call, first to last kernel (CUDA events on `stream`) */
    double ms_loop;           /* device time of the Step-2/3 loop launch(es) */
} eik_stats;

/*
 * Workspace bytes for one grid / for a batch of B grids (host arrays), for the
 * given options (tile shape and precision matter).  Returns 0 on invalid input.
 */
size_t eik_workspace_size(const eik_grid *grid, const eik_options *opt);
size_t eik_workspace_size_batched(int64_t B, const eik_grid *grids, const eik_options *opt);

/*
 * Solve eq. (6) on one grid by Algorithm 2 (Steps 1-3, Sec. 3.1.2).
 *   grid     host; dims and spacing
 *   F        device [nz][ny][nx]; speeds, F >= 0 (F == 0 impassable)
 *   src_idx  device [n_src] int64 flat indices (checked on the device; an
 *            index out of range is ignored and reported as EIK_ERR_ARG)
 *   src_val  device [n_src] fixed values (precision type)
 *   phi      device [nz][ny][nx] output, written completely
 * Returns EIK_OK or an EIK_ERR_* code (see the synchronisation note above).
 */
int eik_solve(const eik_grid *grid, const void *F, const int64_t *src_idx, const void *src_val,
              int64_t n_src, void *phi, void *workspace, size_t workspace_bytes, void *stream,
              const eik_options *opt, eik_stats *stats);

/*
 * Solve B independent grids in one set of launches (one persistent launch for
 * all of them).  Not in the paper: a batched form of the same method.
 *   grids        host [B]
 *   F_packed     device; instance b reads F_packed + F_offsets[b] (elements),
 *                a [nz][ny][nx] block; instances may share a block
 *   F_offsets    host [B] element offsets
 *   src_idx/val  device; the sources of instance b are entries
 *                src_offsets[b] .. src_offsets[b+1]-1 (flat indices into b's grid)
 *   src_offsets  host [B+1], non-decreasing, src_offsets[0] = 0
 *   phi_packed   device; instance b writes phi_packed + phi_offsets[b]
 *   phi_offsets  host [B] element offsets (output blocks must not overlap)
 * stats (nullable) receives totals over the batch.
 */
int eik_solve_batched(int64_t B, const eik_grid *grids, const void *F_packed, const int64_t *F_offsets,
                      const int64_t *src_idx, const void *src_val, const int64_t *src_offsets,
                      void *phi_packed, const int64_t *phi_offsets, void *workspace,
                      size_t workspace_bytes, void *stream, const eik_options *opt, eik_stats *stats);

/*
 * Adjoint of the discrete solve (not in the paper): the gradient dL/ds of a
 * loss L(phi) with respect to slowness s = 1/F, by the adjoint-state method
 * applied to the eq.-(6) residual G_i = sum_d ((phi_i - m_{i,d})^+)^2 - h^2 s_i^2
 * (m_{i,d}: the selected upwind neighbour on axis d, argmin of the two, the
 * lower flat index on a tie).  lambda solves J^T lambda = r with r = dL/dphi;
 * dL/ds_i = 2 h^2 s_i lambda_i, and 0 at sources, unreachable and impassable
 * nodes.  phi is the forward solution (a checkpoint, typically from
 * eik_solve_batched with the same grids, F and sources).
 *   grids, F_packed, F_offsets, src_idx, src_offsets   as for eik_solve_batched
 *   phi_packed/phi_offsets   device forward solutions, one [nz][ny][nx] block per instance
 *   r_packed                 device dL/dphi, same offsets as phi
 *   g_packed/g_offsets       device output, ACCUMULATED (g += dL/ds); instances may share a
 *                            block (g_offsets equal, equal dims) to sum their gradients, in
 *                            instance order; blocks at different offsets must not overlap
 *                            (EIK_ERR_ARG otherwise)
 * stats (nullable): tiles_remedy = adjoint tile visits, iters_remedy = iterations.
 * Workspace: eik_adjoint_workspace_size_batched (4 arrays of the precision per node).
 * Options: tile and order as for the solve, but with the adjoint's own defaults
 * (tile 8x8x8 in 3D, order 8: its lists are ordered by a static key, -max phi
 * per tile, so lambda flows from late to early arrivals); method, converge and
 * skip_remedy do not apply.  The result does not depend on tile, order or
 * schedule: the sum in each node has a fixed order, and so has the sum over the
 * instances that share a gradient block (no atomics), so repeated calls are
 * bit-identical.
 */
size_t eik_adjoint_workspace_size_batched(int64_t B, const eik_grid *grids, const eik_options *opt);
int eik_adjoint_batched(int64_t B, const eik_grid *grids, const void *F_packed, const int64_t *F_offsets,
                        const void *phi_packed, const int64_t *phi_offsets, const int64_t *src_idx,
                        const int64_t *src_offsets, const void *r_packed, void *g_packed, const int64_t *g_offsets,
                        void *workspace, size_t workspace_bytes, void *stream, const eik_options *opt,
                        eik_stats *stats);
/* one grid: F, phi, r, g device [nz][ny][nx]; src_idx device [n_src]; g accumulated */
int eik_adjoint(const eik_grid *grid, const void *F, const void *phi, const int64_t *src_idx, int64_t n_src,
                const void *r, void *g, void *workspace, size_t workspace_bytes, void *stream,
                const eik_options *opt, eik_stats *stats);

/*
 * Shortest paths by descent on an arrival-time map (the application of
 * Example 4, Sec. 4.1: from a destination back to the source).  The paper
 * names gradient descent on phi without the discrete rule; this is the
 * steepest descent on the grid graph: the next node is the neighbour among
 * the 26 (8 when nz == 1) adjacent nodes with the smallest slope
 * (phi[nb] - phi[cur]) / |x_nb - x_cur| (physical distance with the grid's
 * spacings) among those with phi[nb] < phi[cur], evaluated in double; ties go
 * to the lower flat index.  A path ends at a node without a lower neighbour
 * (a source, for a phi from eik_solve) or when its row is full.
 *   grid       host; dims and spacings (h, hy, hz as for eik_solve)
 *   precision  EIK_FP32 / EIK_FP64: the element type of phi
 *   phi        device [nz][ny][nx] arrival times (e.g. eik_solve's output)
 *   start_idx  device [n_paths] int64 flat start nodes
 *   max_len    nodes per row of `path` (>= 1; n_paths * max_len <= 2^34)
 *   path       device [n_paths][max_len] int64 output: node ids, start first,
 *              -1 past the end of the path
 *   len        device [n_paths] int64 output: nodes on each path; 0 when phi
 *              is +inf at the start (unreachable), -1 when the start index is
 *              outside the grid
 * Asynchronous on `stream`; argument errors are returned before any launch.
 */
int eik_backtrace(const eik_grid *grid, int precision, const void *phi, const int64_t *start_idx, int64_t n_paths,
                  int64_t max_len, int64_t *path, int64_t *len, void *stream);

/*
 * eik_solve without any device allocation and without a workspace argument.
 * The paper has no counterpart: this is for callers that must not allocate
 * device memory at solve time -- e.g. a latency-critical loop that cannot
 * afford the device-wide synchronisation cudaMalloc/cudaFree imply, or a host
 * framework that owns all device memory and cannot lend a workspace.
 * Scratch comes from one static device array of 64 MiB built into the
 * library (held by every GPU that loads it, until the process exits); grids
 * whose eik_workspace_size() exceeds it are rejected with EIK_ERR_ARG.  Every
 * call made outside stream capture looks up the array's device address on the
 * current device (so a cudaDeviceReset() in between is harmless); a call made
 * while `stream` is being captured reuses the address of the last uncaptured
 * call on that device, so make one call on each device before any capture
 * (EIK_ERR_ARG otherwise).  All
 * calls share the one array: calls whose work overlaps on a GPU race and
 * corrupt each other's results, so serialise them (one stream, or events).
 * Arguments, results and errors as for eik_solve.
 */
int eik_solve_noalloc(const eik_grid *grid, const void *F, const int64_t *src_idx, const void *src_val,
                      int64_t n_src, void *phi, void *stream, const eik_options *opt, eik_stats *stats);

/*
 * Diagnostics: per-iteration trace of the persistent schedule on the current
 * device.  While a buffer is set, every solve on that device writes into it:
 * buf[0] = number of records, then records of 4 uint64 = {globaltimer ns,
 * phase (0 start, 1 Step-2 iteration, 2 Step-3 seed pass, 3 remedy iteration,
 * 4 iteration of the FIM loop; plus 256 when the iteration ran in throughput
 * mode, a warp per tile, instead of a thread group per tile), list size,
 * tiles visited}, one after each iteration's barrier, up to
 * `capacity` records (the buffer needs 4*capacity + 1 uint64, device memory,
 * 8-byte aligned).  Pass NULL to stop tracing.  Not synchronised with running
 * solves: set it between them.
 */
int eik_set_trace(void *device_buffer, int64_t capacity);

/* thread-local message describing the last non-zero return (never NULL) */
const char *eik_last_error(void);

/* library version string */
const char *eik_version(void);

#ifdef __cplusplus
}
#endif

#endif /* EIKONAL_H_ */
