/*
 * lts.h - C ABI of the GB300 library for Localized Topological Simplification
 * (LTS) of scalar fields on Freudenthal-triangulated 2D and 3D regular grids.
 *
 * The method (Lukasczyk, Garth, Maciejewski, Tierny): given a scalar field f
 * and a list of authorized extrema, compute the order field (Sec. 4.1), find
 * the unauthorized extrema, flood a region from each one up to its first
 * saddle, merging floods that collide (Sec. 4.2 step 1, Sec. 4.3, Sec. 4.4),
 * give every region a local order with only authorized extrema (Sec. 4.2
 * step 2, Eq. 3-5), splice the regions into the global order right before
 * their saddle (Sec. 4.2 step 3, Eq. 6) and flatten their values to the
 * saddle's value (Sec. 4.2 step 4 with zeta = 0).  Minima are processed
 * first, then maxima (Sec. 4: minima are handled symmetrically).
 *
 * Conventions for every entry point
 *   - A grid has dims (X, Y, Z) with Z = 1 in 2D; vertex (x, y, z) has id
 *     x + X*(y + Y*z), i.e. x varies fastest.  Every dim must be >= 2
 *     (except Z = 1 in 2D) and X*Y*Z must be < 2^31.
 *   - Neighbours (Freudenthal / Kuhn triangulation): every vertex whose
 *     offset lies in {0,1}^d or -{0,1}^d, 6 in 2D and 14 in 3D; neighbours
 *     outside the grid are dropped.
 *   - Ties in f are broken by vertex id; -0.0 equals +0.0; a NaN is an error.
 *   - Data pointers marked d_ are DEVICE pointers owned by the caller; the
 *     library never frees or keeps them past the call.  A context owns only
 *     its device workspace.
 *   - Work is enqueued on the context's CUDA stream.  Calls on one context
 *     must not run concurrently (the context is not thread-safe); separate
 *     contexts are independent.
 *   - Errors are returned as lts_status codes; nothing aborts or throws
 *     across this boundary.  lts_last_error() gives a message.
 */
#ifndef LTS_H
#define LTS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lts_ctx lts_ctx;

typedef enum {
    LTS_OK = 0,
    LTS_ERR_ARG = 1,            /* bad dims, sizes, pointers, aliasing, ids out of range */
    LTS_ERR_NAN = 2,            /* the field holds a NaN                                */
    LTS_ERR_NO_AUTHORIZED = 3,  /* a pass has unauthorized extrema but no authorized    */
                                /* extremum of its kind: its floods could never stop    */
    LTS_ERR_OOM = 4,            /* workspace allocation failed or a pool was exhausted  */
    LTS_ERR_CUDA = 5,           /* a CUDA runtime call failed                           */
    LTS_ERR_TIMEOUT = 6,        /* a bounded device-side wait expired                   */
    LTS_ERR_INTERNAL = 7        /* an internal consistency check failed                 */
} lts_status;

typedef enum {
    LTS_MODE_MIN = 1,           /* minima pass only                 */
    LTS_MODE_MAX = 2,           /* maxima pass only                 */
    LTS_MODE_BOTH = 3,          /* minima pass, then maxima pass    */
    /* Flag or-ed into one of the above: the optional post-process of Sec. 4.2
     * step 3 that restores authorized extrema of the other kind swallowed by
     * a region (an authorized minimum inside a region of the maxima pass, an
     * authorized maximum inside one of the minima pass).  Each one, in
     * increasing order of the pass, is moved below every other vertex of its
     * region's block (above the region's block in the minima pass), unless a
     * neighbour of it would then have no higher (lower) neighbour, i.e. would
     * become a new, unauthorized extremum; then it stays swallowed.  Values
     * are not changed (members already take the saddle's value). */
    LTS_MODE_RESTORE = 4
} lts_mode;

typedef struct {
    int32_t ndim;               /* 2 or 3                            */
    int64_t dims[3];            /* X, Y, Z (Z = 1 when ndim == 2)    */
} lts_grid;

/* Per-call statistics ([0] = minima pass, [1] = maxima pass). */
typedef struct {
    int64_t n_vertices;
    int64_t removed[2];          /* unauthorized extrema flooded                    */
    int64_t regions[2];          /* regions (one per hill chain)                    */
    int64_t region_vertices[2];  /* vertices moved (region members, saddles apart)  */
    int64_t max_region[2];       /* members of the largest region                   */
    int32_t max_local_floods[2]; /* most propagations one region needed in step 2   */
    int64_t total_local_floods[2];
    int64_t heap_spills[2];      /* floods whose queue outgrew the register frontier */
    float stage_us[8];           /* device time per stage: order field, classify,   */
                                 /* propagation, regions, local order, reorder      */
                                 /* (summed over passes); [6] total; [7] unused.    */
                                 /* Local order includes the reorder's rank prefix, */
                                 /* which runs beside it; persistence-driven calls  */
                                 /* count the selection in classify.                */
    int64_t kernel_launches;     /* CUDA kernels this call launched                 */
    int64_t fallback_regions[2]; /* regions whose step-2 alternation, seeded from   */
                                 /* the current authorized minima as the paper     */
                                 /* says, did not end (a cycle), and which were    */
                                 /* redone with every vertex of R other than s     */
                                 /* that has an outside neighbour as a seed         */
    int64_t restored[2];         /* swallowed authorized extrema restored           */
                                 /* (LTS_MODE_RESTORE)                              */
} lts_stats;

/* Creates a context on CUDA device `device` whose workspace fits grids of up
 * to `max_vertices` vertices.  `cuda_stream` is a cudaStream_t (NULL: the
 * legacy default stream) on which all work of the context is enqueued.
 * On success *out receives the context.
 * Errors: LTS_ERR_ARG (out NULL, max_vertices < 4 or >= 2^31),
 *         LTS_ERR_CUDA (device), LTS_ERR_OOM (workspace allocation). */
lts_status lts_create(lts_ctx** out, int device, int64_t max_vertices, void* cuda_stream);

/* Device workspace bytes a context needs for grid g (0 if g is invalid);
 * for admission control before lts_create. */
size_t lts_workspace_bytes(const lts_grid* g);

/* Simplifies one field.
 *   g              grid (see conventions); N = X*Y*Z <= the context's max_vertices
 *   d_field        device float32[N], the input f (not modified)
 *   d_authorized   device int32[n_authorized]: ids of authorized extrema, minima
 *                  and maxima together; an id that is not an extremum of a
 *                  pass's kind is ignored by that pass; duplicates allowed.
 *                  May be NULL when n_authorized == 0.
 *   mode           LTS_MODE_MIN / MAX / BOTH
 *   d_out_field    device float32[N]: g, the simplified field (step 4, zeta = 0:
 *                  every moved vertex takes its saddle's value bit for bit)
 *   d_out_order    device int32[N]: the new order field (a permutation of 0..N-1)
 *   opt_stats      if non-NULL, filled after the call completes.
 * The outputs must not overlap the input or each other (LTS_ERR_ARG).
 * The call enqueues its kernels and then waits for them (one small read of
 * the status word), so on return the outputs are final and the status holds
 * any device-side error (NaN, no authorized extremum, timeout, pool overflow).
 * When the propagations' queues outgrow a workspace pool (regions covering a
 * large share of the grid), the call doubles that pool (the larger pool is
 * kept for later calls) and runs again, up to 3 times; LTS_ERR_OOM remains
 * when that is not enough or the device has no memory left.
 * Authorized ids outside [0, N) give LTS_ERR_ARG (detected on the device). */
lts_status lts_simplify(lts_ctx* ctx, const lts_grid* g, const float* d_field,
                        const int32_t* d_authorized, int64_t n_authorized, lts_mode mode,
                        float* d_out_field, int32_t* d_out_order, lts_stats* opt_stats);

/* The same as lts_simplify for a float64 field (Sec. 4.1 on float64 values):
 *   d_field        device float64[N], the input f (not modified)
 *   d_out_field    device float64[N]: g, every moved vertex takes its saddle's
 *                  float64 value bit for bit
 * The order field sorts the float64 values (ties by vertex id, -0.0 equal to
 * +0.0, a NaN is LTS_ERR_NAN) with a 64-bit radix sort; every later step
 * works on the order field and is the float32 path's.  The outputs must not
 * overlap the input or each other (8 bytes per vertex for the fields).
 * Waiting, pool growth and errors as in lts_simplify. */
lts_status lts_simplify_f64(lts_ctx* ctx, const lts_grid* g, const double* d_field,
                            const int32_t* d_authorized, int64_t n_authorized, lts_mode mode,
                            double* d_out_field, int32_t* d_out_order, lts_stats* opt_stats);

/* Critical points of an order field (Sec. 3.1), e.g. to check the output of
 * lts_simplify against Eq. 1: for every vertex, the number of connected
 * components of its lower link and of its upper link in the Freudenthal
 * triangulation.  Interior vertices are classified with a table of their
 * lower-neighbour pattern (2^6 or 2^14 entries, built per context); vertices
 * on the grid boundary count components over their present neighbours.
 *   d_order    device int32[N]: an injective order (e.g. d_out_order)
 *   d_lower    device int8[N] or NULL: lower link components per vertex
 *   d_upper    device int8[N] or NULL: upper link components per vertex
 *   counts     host int64[6]: minima (no lower link), maxima (no upper link),
 *              regular vertices (both connected), saddles (the rest), and the
 *              sums over the vertices of (lower components - 1) and of
 *              (upper components - 1) where positive (join and split
 *              saddle multiplicities)
 * Synchronous on the context's stream.  Errors: LTS_ERR_ARG (grid, sizes,
 * NULL or overlapping pointers), LTS_ERR_CUDA. */
lts_status lts_classify(lts_ctx* ctx, const lts_grid* g, const int32_t* d_order, int8_t* d_lower, int8_t* d_upper,
                        int64_t* counts);

/* Persistence-driven simplification (Sec. 4.5): removes every extremum whose
 * persistence is at most epsilon, with no list of authorized extrema.
 * Each pass (minima, then maxima, as `mode` says) first starts a propagation
 * from every extremum of its kind on the field it receives (f for the
 * minima pass; for the maxima pass of LTS_MODE_BOTH, the output of the
 * minima pass).  A propagation tracks the scalar difference between the
 * highest extremum of its class and the vertex it takes next, |f(m) - f(v)|
 * computed in double precision from the float32 values, and ends once that
 * difference exceeds epsilon: its extremum is persistent.  The propagation
 * that covers the whole grid (the global extremum's) is persistent as well.
 * The kept extrema are thus those whose Elder-rule persistence (Sec. 3.3)
 * exceeds epsilon, plus the global one of each kind; the pass then runs as
 * in lts_simplify with them authorized.  The result satisfies
 * |d_out_field - d_field| <= epsilon everywhere.
 *   epsilon   absolute threshold in the units of f, >= 0 (else LTS_ERR_ARG)
 * Other arguments, outputs, waiting and errors as in lts_simplify (there is
 * no LTS_ERR_NO_AUTHORIZED: the global extremum is always kept).  In
 * opt_stats, stage_us[1] (classification) includes the selection's
 * propagations, and removed[] counts the extrema found not persistent. */
lts_status lts_simplify_persistence(lts_ctx* ctx, const lts_grid* g, const float* d_field, double epsilon,
                                    lts_mode mode, float* d_out_field, int32_t* d_out_order,
                                    lts_stats* opt_stats);

/* Simplifies nf independent fields (Sec. 4 on each; the paper runs one field
 * at a time, and batching is this library's addition).  Array arguments
 * hold one entry per field, with the meaning they have in lts_simplify;
 * every field must fit the context's max_vertices.  The fields are spread
 * over the context's workspace and up to 31 more (batch_workspaces of
 * lts_set_tuning bounds the total; allocated on first use while the device
 * keeps 1 GiB free beyond them, each sized for the largest field of the
 * batch, kept for later batches), each on its own stream,
 * largest fields first; LTS_ERR_OOM if not even one more fits.  (Streams
 * beyond the process's CUDA_DEVICE_MAX_CONNECTIONS hardware queues share
 * them.)  The extra streams start
 * after the work already on the context's stream, and the call returns when
 * every field is done.  opt_stats, if non-NULL, is an array of nf entries
 * (stage_us is not filled).  Returns LTS_OK when every field succeeded, else
 * the status of the first failing field, whose index the last-error
 * message names; the other fields are still simplified.  Argument errors
 * (LTS_ERR_ARG, naming the field) are reported before any work starts. */
lts_status lts_simplify_batch(lts_ctx* ctx, int32_t nf, const lts_grid* grids, const float* const* d_fields,
                              const int32_t* const* d_authorized, const int64_t* n_authorized, lts_mode mode,
                              float* const* d_out_fields, int32_t* const* d_out_orders, lts_stats* opt_stats);

/* Serving (continuous batching).  lts_submit enqueues one simplification
 * (arguments as in lts_simplify) and returns at once with a ticket (> 0).
 * Requests run on the context's serving workspaces, each with its own stream
 * and each sized for the context's max_vertices: a request goes to an idle
 * workspace, or to a new one while the serving budget (lts_serve_config) and
 * the device's free memory allow, or else behind the requests of the
 * workspace with the fewest outstanding vertices.  Requests on different
 * workspaces run concurrently on the device; each starts after the work the
 * caller had enqueued on the context's stream when it was submitted.  A
 * request's result is the one lts_simplify gives for the same arguments,
 * whatever runs beside it.  Both outputs are working arrays of the passes
 * until the request is done, so requests in flight at the same time must not
 * share an output buffer (inputs may be shared).  lts_poll sets *done to 1 once the request is
 * finished and then returns its status (LTS_OK or the error it met); while it
 * runs, *done is 0 and the return is LTS_OK.  The result of a ticket stays
 * readable until 1024 newer requests have been submitted (later polls give
 * LTS_ERR_ARG); lts_submit waits for the request 1024 places before it if
 * that one is still running.  A failed request leaves its workspace clean for
 * the requests behind it.  The first lts_submit on a context allocates its
 * pinned request ring.  When no serving workspace can be allocated, requests
 * run one after another on the context's own workspace and stream. */
lts_status lts_submit(lts_ctx* ctx, const lts_grid* g, const float* d_field, const int32_t* d_authorized,
                      int64_t n_authorized, lts_mode mode, float* d_out_field, int32_t* d_out_order,
                      uint64_t* ticket);
lts_status lts_poll(lts_ctx* ctx, uint64_t ticket, int* done);

/* Serving limits: at most max_concurrent serving workspaces (0..15; 0 runs
 * every request on the context's own workspace and stream, in submission
 * order) and at most hbm_budget_bytes of device memory for them together
 * (each takes lts_workspace_bytes of the largest grid).  Defaults: 15
 * workspaces, 120 GiB.  Workspaces already allocated are kept; the limits
 * apply to later allocations and to the choice of workspace.  The CUDA
 * runtime maps streams onto CUDA_DEVICE_MAX_CONNECTIONS hardware queues (8
 * unless the process sets that variable before CUDA starts, at most 32);
 * beyond that, workspaces share queues and their work partly serializes.
 * Errors: LTS_ERR_ARG (max_concurrent outside [0, 15], negative budget). */
lts_status lts_serve_config(lts_ctx* ctx, int32_t max_concurrent, int64_t hbm_budget_bytes);

/* Launch tuning of a context (the paper has no counterpart: these are
 * resource choices of this library, picked per workload by the package's
 * autotuner).  A field of 0 keeps the default.
 *   engine_blocks_per_sm: resident 128-thread blocks per multiprocessor of
 *     the persistent propagation engine (1..8; default 8);
 *   team_blocks_per_sm: blocks per multiprocessor of the 16- and 32-lane
 *     local-order team kernels (1..16; default 12);
 *   batch_workspaces: workspaces lts_simplify_batch spreads a batch over,
 *     the context's own included (1..32; default 32).
 * The tuning changes no result, only the launch shapes, and applies to the
 * calls that start after it.  lts_set_tuning with NULL restores the
 * defaults; LTS_ERR_ARG for a value outside its range (nothing changes).
 * lts_get_tuning writes the values in force (defaults as numbers). */
typedef struct lts_tuning {
    int32_t engine_blocks_per_sm;
    int32_t team_blocks_per_sm;
    int32_t batch_workspaces;
    int32_t reserved[5];          /* must be 0 */
} lts_tuning;

lts_status lts_set_tuning(lts_ctx* ctx, const lts_tuning* tuning);
lts_status lts_get_tuning(const lts_ctx* ctx, lts_tuning* out);

/* Message describing the last error on this context ("" if none). */
const char* lts_last_error(const lts_ctx* ctx);

/* Frees the context and its workspace; NULL is ignored. */
void lts_destroy(lts_ctx* ctx);

/* ---- Order field with no allocation at call time -------------------------
 * The paper has no counterpart to this entry point: it is a service for
 * callers that cannot allocate device memory when they call, e.g. a caller
 * that has handed the device's free memory to its own pool allocator (so a
 * cudaMalloc would fail), or one on a latency-bound path where cudaMalloc and
 * cudaFree (which waits for the whole device) are not acceptable.
 *
 * It computes the order field alone, i.e. O(v) = the rank of vertex v when
 * the vertices are sorted by (f(v), v), with -0.0 == +0.0; the result equals
 * d_out_order of lts_simplify with every vertex authorized.  It runs the same
 * sort kernels as lts_simplify, but its scratch is a static device array
 * inside the library, sized for at most LTS_ORDER_STATIC_MAX_VERTICES
 * vertices (16.5 MiB).  CUDA allocates that array once per device when the
 * library's module is loaded there, and under CUDA's default lazy module
 * loading that happens at the first use of the module on the device (the
 * first call of this entry point or of any lts_* call there), not when the
 * library is opened: a caller that hands the device's free memory to its own
 * pool must make one call on each device before doing so.  The call makes no
 * cudaMalloc/cudaFree and needs no context.
 *
 *   device       CUDA device to run on; made current for the call, and the
 *                previously current device is restored before returning
 *   g            grid (see conventions); N = X*Y*Z <= LTS_ORDER_STATIC_MAX_VERTICES
 *   d_field      device float32[N] on `device`, the input f (not modified)
 *   d_order      device int32[N] on `device`: O, a permutation of 0..N-1;
 *                must not overlap d_field
 *   cuda_stream  a cudaStream_t of `device` (NULL: the legacy default stream)
 *   err, err_len if err is non-NULL, receives a message on error ("" on success)
 *
 * Set-up: the first call on each device looks up the scratch's address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture begins on the device, and before the device's
 * free memory is handed to a pool (see above).
 * The call enqueues its kernels on cuda_stream and waits for them (one small
 * read of the status word), so on return d_order is final.
 * Calls on one device share the scratch: calls that overlap in time (from
 * several host threads, or on several streams) race and corrupt each other's
 * results, so serialize them.
 * Errors: LTS_ERR_ARG (invalid grid, N > LTS_ORDER_STATIC_MAX_VERTICES, NULL
 * or overlapping pointers, device outside [0, 256)), LTS_ERR_NAN, LTS_ERR_CUDA,
 * LTS_ERR_TIMEOUT (a bounded wait of the sort expired). */
#define LTS_ORDER_STATIC_MAX_VERTICES (1LL << 20)

lts_status lts_order_field_static(int device, const lts_grid* g, const float* d_field, int32_t* d_order,
                                  void* cuda_stream, char* err, size_t err_len);

#ifdef __cplusplus
}
#endif

#endif /* LTS_H */
