/*
 * libtga -- best-improvement VRP local search on one GB300 (sm_103a).
 *
 * One local-search step evaluates the whole neighbourhood of the current
 * solution -- relocate, swap, intra-route 2-opt, inter-route 2-opt* and
 * or-opt (runs of 2 and 3 customers), optionally also the swaps of runs --
 * scores every candidate with an exact integer O(1) delta of distance +
 * w_load * capacity excess + w_tw * time warp, reduces to the best move, and
 * applies it on the device.  The CVRP, the VRPTW and the VRPSPDTW (pickups
 * and deliveries; the capacity excess of the largest load on board) are
 * supported.
 * The method is the node-based tensorised move evaluation of the paper
 * (Section 5.3, "node-based extraction", Eqs. "node_based1"/"node_based2"),
 * built on sequence concatenation (Section 4.3) over an attribute-based
 * solution representation (Section 5.2), with best improvement
 * (Section 5.3.4, Eq. "min_obj") and the descent loop of the appendix
 * algorithm "Feasible and infeasible search".
 *
 * Conventions shared by every call:
 *  - Nodes: depot 0, customers 1..n.  Distances are int32, row-major
 *    (n+1)*(n+1), symmetric with a zero diagonal; travel time equals
 *    distance.
 *  - Solution: a giant tour tour[n] (customers in route order) plus
 *    route_start[m+1]: route r is tour[route_start[r] .. route_start[r+1]-1]
 *    between two depot visits (Section 2, "S = {R_1..R_M}").  Empty routes
 *    are allowed and keep their slot; m never changes.
 *  - Anchors: customers 1..n; the start depot of route r is anchor n+1+r;
 *    W = n+1+m.  A move is (op, a, b) with op ranks
 *      0 relocate  (a customer, b anchor: move a to just after b)
 *      1 swap      (customers a < b)
 *      2 2-opt     (customers of one route, pos(a) < pos(b): reverse a..b)
 *      3 2-opt*    (anchors, route(a) < route(b): exchange the tails after a, b)
 *      4 or-opt 2, 5 or-opt 3 (a = first customer of the run, b anchor
 *        outside the run, b != pred(a): move the run after b)
 *      6 swap of a customer a with the run of two starting at b (optional)
 *      7 swap of the runs of two starting at a < b (optional)
 *    and move index idx = op*W*W + a*W + b (requires 6*W*W < 2^32, or
 *    8*W*W < 2^32 with ranks 6 and 7).
 *  - The best move is the smallest (delta, idx); a move is accepted iff
 *    delta < 0.
 *  - All pointers in tga_instance / tga_solution are DEVICE pointers owned by
 *    the caller; they must stay valid until tga_destroy.  The solution
 *    arrays are updated in place by tga_apply_move / tga_descend.
 *  - Every call is asynchronous on the context's stream unless stated;
 *    errors found on the device are reported by the next synchronising call
 *    (tga_descend, tga_sync, tga_get_stats).
 *  - Integer range: the library rejects (TGA_ERR_RANGE) a state in which a
 *    route built from two current routes plus three moved customers could
 *    cost 2^27 or more, so every delta fits in int32 with room for the
 *    invalid-candidate offset.
 */
#ifndef TGA_H
#define TGA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream handle (cudaStream_t); NULL is the legacy default stream. */
typedef struct CUstream_st *tga_stream_t;

typedef struct tga_ctx tga_ctx;

enum {
    TGA_OK = 0,
    TGA_ERR_INVALID = 1,   /* bad sizes, ids, op mask, non-candidate move, bad solution */
    TGA_ERR_RANGE = 2,     /* int32 headroom or move-index bound violated */
    TGA_ERR_NOMEM = 3,     /* device allocation failed */
    TGA_ERR_CUDA = 4,      /* a CUDA runtime call failed */
    TGA_ERR_TIMEOUT = 5,   /* a bounded device-side wait ran out */
    TGA_ERR_STATE = 6,     /* call not allowed in the context's current state */
    TGA_ERR_CHECK = 7,     /* internal consistency check: an applied move's delta differs from its evaluation */
    TGA_ERR_BOUNDS = 8     /* index-checked build only: a device-side index check failed (tga_get_bounds_report) */
};

/* Problem data (Section 2).  has_tw = 0 is the CVRP: service, tw_early and
 * tw_late may then be NULL.  w_load / w_tw are the penalty weights of the
 * penalised objective; both must be >= 0.
 *
 * pickup = NULL: no pickups (CVRP, VRPTW); the load term penalises the total
 * delivery of a route above the capacity.  pickup != NULL: the VRP with
 * simultaneous pickup and delivery and time windows (VRPSPDTW, Section 2;
 * has_tw must be 1, else TGA_ERR_INVALID -- a VRPSPD without windows is
 * passed with windows [0, horizon] and zero service times).  A vehicle
 * leaves the depot with the deliveries of its whole route, drops demand[x]
 * and collects pickup[x] at each customer, and the load term penalises the
 * largest load on board above the capacity (attributes L_I, L_O, L_M of
 * Section 4.3.2).  pickup[x] >= 0, pickup[0] = 0 (checked on the device by
 * tga_build_attrs: TGA_ERR_INVALID).  Contexts with pickups run the
 * single-instance paths (every descent mode, tga_eval_best_move_noalloc);
 * tga_descend_batch and tga_set_granular refuse them with TGA_ERR_STATE. */
typedef struct {
    int32_t n_customers;       /* n >= 1 */
    int32_t n_routes;          /* m >= 1 */
    int32_t capacity;          /* Q >= 0 */
    int32_t has_tw;            /* 0 CVRP, 1 VRPTW */
    int32_t w_load, w_tw;
    const int32_t *dist;       /* device, (n+1)*(n+1) */
    const int32_t *demand;     /* device, n+1, demand[0] = 0 */
    const int32_t *service;    /* device, n+1 (VRPTW), service[0] = 0 */
    const int32_t *tw_early;   /* device, n+1 (VRPTW), [0] = depot opening */
    const int32_t *tw_late;    /* device, n+1 (VRPTW), [0] = latest return */
    const int32_t *pickup;     /* device, n+1, or NULL (see above) */
} tga_instance;

typedef struct {
    int32_t *tour;             /* device, n */
    int32_t *route_start;      /* device, m+1 */
} tga_solution;

/* A decoded move.  delta is the objective change (negative = improving);
 * valid = 0 means the neighbourhood was empty. */
typedef struct {
    int32_t delta;
    uint32_t move_index;
    int32_t op, a, b;
    int32_t valid;
} tga_move;

typedef struct {
    int64_t steps;             /* applied moves */
    int64_t candidates;        /* candidate moves evaluated, all evaluations */
    int64_t initial_cost;      /* cost when the attributes were (re)built */
    int64_t final_cost;        /* current cost */
    int32_t status;            /* TGA_OK or the first device-side error */
    int32_t local_optimum;     /* 1 if the last evaluation found no delta < 0 */
    int64_t evaluations;       /* neighbourhood evaluations */
} tga_stats;

/* Create a context for one instance + solution.
 *  op_mask: bit k enables op rank k; must be non-zero and < 256.  Ranks:
 *  0 relocate, 1 swap, 2 2-opt, 3 2-opt*, 4 / 5 or-opt of 2 / 3 customers
 *  (0x3F = all of these), 6 a customer exchanged with a run of two
 *  consecutive customers (a = the customer, b = the run's first), 7 two runs
 *  of two exchanged (a < b, the runs' firsts) -- the Swap of Section 5.3.1
 *  with run lengths N1, N2 in {1, 2}; in and across routes, runs keep their
 *  orientation and must not share a customer.  Ranks 6 and 7 run on the
 *  per-step descent paths (graph and host-launched; the persistent mode
 *  refuses them with TGA_ERR_STATE and the automatic mode takes the graph),
 *  need n + m + 1 <= 23170 (8 W^2 < 2^32), have no pickup variant (a
 *  pickup instance with them: TGA_ERR_INVALID) and are refused by the
 *  batched launch and the edge-based extraction (TGA_ERR_STATE).
 *  Validates sizes on the host (TGA_ERR_INVALID / TGA_ERR_RANGE for
 *  W too large), allocates the context's device workspace (about
 *  4*(n+1)*(n+m+257) bytes for the position-ordered distance copy plus
 *  O(n+m)), and returns *out.  Nothing is computed until tga_build_attrs.
 *  Ownership: the caller keeps the instance and solution memory. */
int tga_create(const tga_instance *inst, const tga_solution *sol, uint32_t op_mask,
               tga_stream_t stream, tga_ctx **out);

/* Build the attribute representation from the caller's solution
 * (Section 5.2 "solution tensor", node-based positional index P_r/P_pi of
 * Section 5.3.1): positions, per-anchor forward/backward segment attributes
 * (distance, load, T_D/T_E/T_L/T_V in the form of Section 4.3), route
 * totals, and the position-ordered distance copy.  Also validates the
 * solution (permutation, route bounds), the matrix (symmetry, zero diagonal,
 * non-negative) and the integer headroom; failures are reported by the next
 * synchronising call.  Resets the step counters and the initial cost. */
int tga_build_attrs(tga_ctx *ctx);

/* Evaluate the whole neighbourhood (Section 5.3 Extraction, Concatenation,
 * Differencing, Evaluation) and write the best move to out_dev (DEVICE
 * memory, one tga_move).  Asynchronous. */
int tga_eval_best_move(tga_ctx *ctx, tga_move *out_dev);

/* Apply a move given in DEVICE memory (Section 5.3.5 "Tensor update", done
 * on the device): rewrite tour/route_start in place, update positions and
 * rebuild the attributes of the touched routes only.  A move with
 * valid == 0 or delta >= 0 is a no-op that marks the context as being at a
 * local optimum.  A move that is not a candidate sets TGA_ERR_INVALID. */
int tga_apply_move(tga_ctx *ctx, const tga_move *move_dev);

/* Best-improvement descent (appendix algorithm "Feasible and infeasible
 * search"): repeat evaluate + apply until no move has delta < 0 or max_steps
 * moves were applied in this call.  The loop runs on the device with no host
 * round trip per step, along the path chosen by tga_set_descent_mode.
 * Builds the attributes first if they were never built.  Synchronises the
 * stream at the end and fills *out_host (may be NULL).  Every path gives the
 * same moves, solution and counters bit for bit. */
int tga_descend(tga_ctx *ctx, int64_t max_steps, tga_stats *out_host);

/* Descent paths.
 *  TGA_DESCENT_PERSISTENT  one cooperative launch for the whole descent: all
 *      CTAs stay resident, evaluate their share of the step, meet at a grid
 *      barrier, CTA 0 applies the move while the others permute distance
 *      columns, and meet again (bounded waits: TGA_ERR_TIMEOUT after 5 s).
 *      The launch claims every SM: do not run it concurrently with other
 *      work that needs the GPU's SMs to make progress.
 *  TGA_DESCENT_GRAPH  a CUDA graph whose conditional while node runs the
 *      per-step kernels (evaluation branches, then apply) until the device
 *      clears the condition; other streams' kernels interleave freely.
 *  TGA_DESCENT_HOST  the same per-step kernels launched from the host in
 *      chunks of 64 steps (for profilers that do not trace kernels inside
 *      conditional graph bodies; also selected by the environment variable
 *      TGA_GRAPH=0).
 *  TGA_DESCENT_AUTO (default)  the path tga_set_tile(ctx, 0, 0) measured
 *      fastest; before any measurement, persistent for instances with
 *      n + m + 1 < 4096 positions, else the graph.  Falls back to the graph
 *      when the cooperative launch is refused. */
enum {
    TGA_DESCENT_AUTO = 0,
    TGA_DESCENT_PERSISTENT = 1,
    TGA_DESCENT_GRAPH = 2,
    TGA_DESCENT_HOST = 3
};
int tga_set_descent_mode(tga_ctx *ctx, int32_t mode);

/* The path the context's last descent took (TGA_DESCENT_*; AUTO if it never
 * descended) and, for the persistent path, its grid size (grid_out may be
 * NULL; 0 for the other paths). */
int tga_get_descent_mode(tga_ctx *ctx, int32_t *last_used, int32_t *grid_out);

/* The tile shape the persistent path uses (rows, column warps, row split):
 * the one the autotuner measured fastest (or set below), else the
 * inter-route tile with the row split raised to at least 4 warps per block.
 * row_split 0 is the strip mode: every CTA walks a contiguous share of the
 * strip-major tile order (the per-step strip kernel's evaluation inside the
 * persistent launch). */
int tga_get_persistent_shape(tga_ctx *ctx, int32_t *rows, int32_t *col_warps, int32_t *row_split);

/* Set the persistent path's tile shape (no counterpart in the paper; a
 * tuning control): rows 8, 16, 32 or 64, col_warps 2, 4 or 8, row_split 1, 2
 * or 4 with col_warps * row_split * 32 = 128 or 256 threads; or row_split 0
 * (strip mode) with rows 16 or 32 and col_warps 4 or 8.  rows = 0 clears
 * the setting (the automatic choice applies again).  TGA_ERR_INVALID for
 * any other shape.  The next persistent descent uses it. */
int tga_set_persistent_shape(tga_ctx *ctx, int32_t rows, int32_t col_warps, int32_t row_split);

/* Descend every context to a local optimum (at most max_steps moves each) in
 * ONE persistent launch on ctxs[0]'s stream (all contexts on one device).
 * Each context is (re)built from its caller solution inside the launch.
 * Per step a job is split into chunks (row tiles of its pair triangle, groups
 * of 8 routes); resident CTAs take chunks of any job and the CTA finishing a
 * job's last chunk applies its move, so large jobs spread over many SMs.
 * Idle CTAs poll under a 20 s limit (TGA_ERR_TIMEOUT).  Results per context
 * equal tga_descend's bit for bit.  Waits for completion.
 * out_host: n entries (may be NULL).  Returns the first error.  Contexts with
 * edge-based extraction or with pickups are refused (TGA_ERR_STATE). */
int tga_descend_batch(tga_ctx **ctxs, int n, int64_t max_steps, tga_stats *out_host);

/* Autotune the batched tile rows (16/32/64) per size bucket (n+m+1 below 400,
 * 800, 1400, above): times evaluation-only batched launches of each bucket's
 * median context and keeps the fastest shape for the whole bucket.
 * rows_out: n entries (may be NULL).  Leaves the contexts to be rebuilt.
 * Refuses the same contexts as tga_descend_batch (TGA_ERR_STATE). */
int tga_batch_autotune(tga_ctx **ctxs, int n, int32_t *rows_out);

/* As tga_descend, but only enqueues the work on the context's stream and
 * returns at once (no synchronisation).  Poll with tga_query; read results
 * with tga_get_stats once done. */
int tga_descend_async(tga_ctx *ctx, int64_t max_steps);

/* *done_out = 1 when all work enqueued on the context's stream has
 * finished, 0 while some is pending.  Never blocks. */
int tga_query(tga_ctx *ctx, int32_t *done_out);

/* Device bytes a context for n customers and m routes allocates at most (its
 * workspace only; the caller's instance and solution arrays come on top):
 * the layout with the pickup and swaps-of-runs records, which a context
 * allocates only when it uses them.  Host-only arithmetic, for admission
 * control by memory budget. */
size_t tga_workspace_bytes(int32_t n_customers, int32_t n_routes);

/* Wait for the context's stream and report the device status. */
int tga_sync(tga_ctx *ctx);

/* Synchronise and copy the counters (steps, candidates, costs, status). */
int tga_get_stats(tga_ctx *ctx, tga_stats *out_host);

/* Synchronise and copy the candidate moves evaluated per operator rank
 * (out_host[8]: relocate, swap, 2-opt, 2-opt*, or-opt 2, or-opt 3, customer
 * with a run of two, two runs of two), summed
 * over all evaluations since tga_build_attrs; their sum is
 * tga_stats.candidates.  Used to count the algorithmic work of a descent
 * per operator (the per-operator breakdown of the paper's Section 6.6). */
int tga_get_op_candidates(tga_ctx *ctx, int64_t *out_host);

/* Record one packed key ((uint32)(delta + 2^31) << 32 | idx) per
 * evaluation into a caller-owned DEVICE buffer of `capacity` entries
 * (NULL disables).  Used to compare whole trajectories. */
int tga_set_move_log(tga_ctx *ctx, uint64_t *log_dev, int64_t capacity);

/* Choose the inter-route tile shape: rows per tile (8, 16, 32 or 64) and
 * warps per block (2, 4 or 8; 32 columns each); 0, 0 runs the built-in
 * autotuner (times every shape, including row-split ones, on the current
 * state).  Call after tga_build_attrs.  With the descent mode
 * TGA_DESCENT_AUTO the autotuner then also times 24-step descents from the
 * current solution along the graph path and along the persistent path under
 * each of its block shapes, and the automatic mode keeps the fastest; the
 * caller's solution is restored and the attributes rebuilt (counters reset),
 * so the context is left as a fresh tga_build_attrs would leave it. */
int tga_set_tile(tga_ctx *ctx, int32_t rows, int32_t warps);
int tga_get_tile(tga_ctx *ctx, int32_t *rows, int32_t *warps);

/* Full tile shape: rows per tile (8/16/32/64), column warps (2/4/8: 32
 * columns each) and a row split (1/2/4 warps share one column slice and
 * divide its rows; col_warps * row_split <= 8).  tga_set_tile(ctx, 0, 0)
 * autotunes over these shapes. */
int tga_set_tile_shape(tga_ctx *ctx, int32_t rows, int32_t col_warps, int32_t row_split);
int tga_get_tile_shape(tga_ctx *ctx, int32_t *rows, int32_t *col_warps, int32_t *row_split);

/* Strip-major inter-route evaluation (the same candidates of Section 5.3.1
 * node-based extraction, another schedule): the tiles (rows 16 or 32, 4 or 8
 * column warps) are ordered column strip by column strip and a grid of
 * resident CTAs walks them in contiguous ranges, keeping each strip's
 * column-anchor constants in registers and copying the next tile's
 * distance rows and row records into shared memory (cp.async, double
 * buffered) while it evaluates the current one.  Used by the per-step
 * descent paths and tga_eval_best_move; tga_get_tile_shape then reports
 * row_split = 0.  The autotuner (tga_set_tile(ctx, 0, 0)) times these
 * shapes beside the one-CTA-per-tile ones.  TGA_ERR_INVALID for other
 * shapes. */
int tga_set_tile_strip(tga_ctx *ctx, int32_t rows, int32_t col_warps);

/* Time the inter-route evaluation kernel alone on the current state:
 * `reps` launches bracketed by CUDA events on the context's stream; writes the
 * mean milliseconds per launch.  Leaves no pending move behind.  Used to
 * report the kernel's roofline fraction. */
int tga_profile_inter(tga_ctx *ctx, int32_t reps, float *ms_per_launch);

/* The same for the inter-route kernel of the swaps of runs (op ranks 6, 7);
 * TGA_ERR_STATE when the context's operator mask has neither rank. */
int tga_profile_xswap(tga_ctx *ctx, int32_t reps, float *ms_per_launch);

/* Measured 32-bit integer throughput of the current device: the denominator
 * of the evaluation kernels' roofline fractions.  The paper has no
 * counterpart (it reports speedups, not rooflines); the evaluation path
 * issues integer additions and minima/maxima only (no tensor-core
 * contraction), so its ceiling is the rate at which the SMs retire such
 * operations.  Launches one dependency-free stream kernel sized to fill
 * every SM (the SM count is read from the device): each thread runs eight
 * independent chains of `iters` x 8 links,
 *   kind 0: x = max(x + a, b)   (one add and one max per link: two-input
 *           operations, one per issued lane -- the issue peak),
 *   kind 1: x = x + x' + a      (two adds per link, which may execute as one
 *           three-input add: more source operations than issued lanes),
 * and writes the best of three timed launches (CUDA events on `stream`,
 * after one warm-up launch) as source integer operations per second
 * (*ops_per_s, two per link) and milliseconds (*ms_out, may be NULL).
 * Synchronous.  TGA_ERR_INVALID for another kind, iters < 1 or a NULL
 * ops_per_s; TGA_ERR_CUDA when a launch fails. */
int tga_measure_int_peak(int32_t kind, tga_stream_t stream, int32_t iters, double *ops_per_s, float *ms_out);

/* Best move of one instance + solution WITHOUT allocating any memory.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot allocate device memory (a host framework that owns every device
 * allocation, a plugin handed only a stream and its buffers, a service that
 * forbids cudaMalloc after start-up).  Inputs are as for tga_create (device
 * pointers, caller-owned; the solution is read, never written); out_dev is
 * one tga_move in caller-owned DEVICE memory.
 * Scratch: a file-scope device array inside the library (about 7 MB; every
 * GPU that loads libtga holds it until the process exits).  Sizes with
 * n + m + 1 > 1280 are rejected with TGA_ERR_RANGE.  No cudaMalloc,
 * cudaFree or allocating library routine is called.
 * The first call on a device looks up the array's device address for that
 * device; make that first call before any stream capture.  Every call
 * shares the one array and overwrites it, so calls whose GPU work overlaps
 * (other streams, other threads) race: serialise them.  Synchronous: waits
 * for `stream`, then returns TGA_OK or the device-side error. */
int tga_eval_best_move_noalloc(const tga_instance *inst, const tga_solution *sol, uint32_t op_mask,
                               tga_stream_t stream, tga_move *out_dev);

/* Edge-based extraction (Section 5.3.1, "edge-based extraction", the
 * paper's ETGA): restrict the inter-route candidates of every evaluation to
 * the node pairs of a granular mask M, given as theta > 0 entries per
 * customer: nbr_dev[x*theta + k], k < theta, are the customers y with
 * M[x][y] = 1 (DEVICE memory, (n+1)*theta int32, row 0 ignored, caller-owned
 * and valid until the mask is replaced or the context destroyed).  Intra-route
 * candidates are always evaluated.  An inter-route candidate (op, a, b) is
 * kept when: relocate / or-opt (the run starting at a moves after b): b is a
 * start depot, or M[a][b]; swap: M[a][b] or M[b][a]; 2-opt*: exactly one of
 * a, b is a start depot, or M[a][b] or M[b][a].  Candidate counts
 * (tga_stats.candidates, tga_get_op_candidates) count the kept candidates.
 * theta = 0 restores the full neighbourhood.  Entries that are not another
 * customer, or theta > n-1, give TGA_ERR_INVALID.  The edge-based extraction
 * runs on the graph and host-launched descent paths (the persistent path
 * returns TGA_ERR_STATE and the automatic mode takes the graph);
 * tga_descend_batch refuses such contexts (TGA_ERR_STATE).  Synchronises the
 * context's stream. */
int tga_set_granular(tga_ctx *ctx, const int32_t *nbr_dev, int32_t theta);

/* Diagnostic: synchronise and copy one internal array to host memory.
 * what: 0 control block, 1 positions (int32 anchor per position), 2 anchor
 * positions, 3 base attributes (64 B per anchor), 4 hoisted constants
 * (128 B per anchor), 5 route records (32 B per route), 6 position-ordered
 * distance copy ((n+1) rows of row_pitch int32), 7 tile list (int2).
 * Copies min(bytes, size) bytes; *size_out (may be NULL) gets the size. */
int tga_debug_read(tga_ctx *ctx, int32_t what, void *host_dst, size_t bytes, size_t *size_out);

/* Diagnostic of the index-checked build (a stand-in for a device memory
 * checker; the paper has no counterpart).  libtga_check.so is the same
 * library compiled with -DTGA_BOUNDS_CHECK: every indexed device access of
 * the search state and the instance is checked against its array's extent;
 * the first failed check is recorded and sets TGA_ERR_BOUNDS, and the access
 * reads or writes element 0 instead, so nothing outside an array is touched.
 * Synchronises the context's stream and writes out[0] = 1 if this library
 * was built with the checks (0: release build, out[1..3] = 0), out[1] = the
 * site of the first failure (file id * 100000 + source line: file ids 1
 * tga_internal.cuh, 2 tga_device.cuh, 3 tga_kernels.cu, 4 tga_persist.cu,
 * 5 tga_batch.cu, 6 tga_noalloc.cu; 0 = no failure), out[2] = its index,
 * out[3] = the array's extent.  Returns TGA_ERR_INVALID for a NULL
 * argument, TGA_ERR_CUDA if the copy fails. */
int tga_get_bounds_report(tga_ctx *ctx, int64_t out[4]);

/* Failure detection (the paper has none; the library's device-side waits
 * are its own): set the time limit of every bounded device wait of this
 * context -- the persistent descent's plan publication and grid barrier
 * (default 5 s), the apply launch's plan flag (1 s) and, for batched
 * descents that include this context, the idle chunk polling (20 s; the
 * smallest limit of the batch's contexts applies).  limit_ns < 0 restores
 * the defaults.  A wait that runs out makes the kernel stop its work and
 * return; the descent or batch then reports TGA_ERR_TIMEOUT, the caller's
 * solution keeps its last written-back state, and tga_build_attrs makes the
 * context usable again.  Meant for tests of this failure path (a tiny
 * limit) and for callers that want a tighter bound. */
int tga_set_wait_limit(tga_ctx *ctx, int64_t limit_ns);

/* Release the context's workspace (not the caller's arrays). */
int tga_destroy(tga_ctx *ctx);

const char *tga_strerror(int code);

#ifdef __cplusplus
}
#endif
#endif
