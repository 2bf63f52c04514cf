/*
 * frnn.h - C ABI of libfrnn, a fixed-radius nearest-neighbour (FRNN) graph
 * builder for NVIDIA B300 (sm_103a).
 *
 * The operation (paper: "Accelerating the Inference of the Exa.TrkX Pipeline",
 * Sec. 2 and Sec. 3.4): given n points embedded in a d-dimensional space and a
 * radius r, join every point i to the other points j whose Euclidean distance
 * is within r.  Each row keeps at most k_max neighbours, the nearest ones
 * (Sec. 3.1: exact k-nearest-neighbour search followed by a radius cut).
 * Precisely, with d2(i,j) the float32 sum over t = 0..d-1, in that order, of
 * (x[i][t] - x[j][t])^2 (each subtraction, product and addition rounded once)
 * and r2 = fl32(r * r):
 *
 *     S_i   = { j != i : d2(i,j) <= r2 }
 *     row i = the min(|S_i|, k_max) members of S_i that are smallest by the
 *             pair (d2(i,j), j), listed in increasing (d2, j) order.
 *
 * The result is a CSR graph with directed edges i -> j.  It is bit-exact and
 * deterministic: it does not depend on the device, the launch shape or the
 * batch an event is built in.
 *
 * Conventions for every function:
 *   - Pointers documented as "device" must be device memory of the plan's
 *     device; "host" pointers are ordinary (or pinned) host memory.
 *   - Streams are passed as void* (a cudaStream_t; NULL = the legacy default
 *     stream).  Build calls are asynchronous on that stream unless stated.
 *   - Every function returns an frnn_status; no C++ exception crosses the ABI.
 *     Argument errors are detected on the host before anything is enqueued.
 *     Errors found by kernels (non-finite input, an exhausted edge buffer, a
 *     bounded wait that ran out) are latched in a device status word and
 *     reported by frnn_get_last_status().
 *   - A plan is not thread-safe: use one plan per host thread or per stream.
 */
#ifndef FRNN_H
#define FRNN_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define FRNN_API __attribute__((visibility("default")))
#else
#define FRNN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FRNN_OK = 0,
    FRNN_ERR_INVALID_ARG = 1,     /* bad pointer, size, radius or cap; see each call   */
    FRNN_ERR_CUDA = 2,            /* a CUDA runtime call failed                         */
    FRNN_ERR_OOM = 3,             /* device allocation failed                           */
    FRNN_ERR_NONFINITE_INPUT = 4, /* an event holds NaN or Inf; its rows are left empty */
    FRNN_ERR_TIMEOUT = 5,         /* a bounded device-side wait ran out                 */
    FRNN_ERR_OVERFLOW = 6,        /* the edges did not fit the plan's edge capacity     */
    FRNN_ERR_CAPACITY = 7,        /* the call exceeds a capacity fixed at plan creation */
    FRNN_ERR_CHECK = 8            /* a debug check of a build's output failed (FRNN_DEBUG,
                                     frnn_check_last_build): a defect of the library    */
} frnn_status;

/* k_max value that keeps every row whole: the paper's own FRNN list (Sec. 3.4,
 * all points within r, unsorted).  Rows of at most 32 neighbours still come
 * sorted by (d2, j); longer rows are in no particular order.  The edges must
 * fit the plan's edge capacity (FRNN_ERR_OVERFLOW otherwise). */
#define FRNN_NO_CAP 0

/* Plan flags. */
#define FRNN_EMIT_D2 0x1u    /* also write the float32 d2 of every edge              */
#define FRNN_USE_GRAPH 0x2u  /* replay the build as a CUDA graph captured on first use */
#define FRNN_AUTOTUNE 0x4u   /* a radius build whose call shape has no autotuned entry
                                yet runs frnn_plan_autotune first (synchronously)      */
#define FRNN_DEBUG 0x8u      /* every build (radius or kNN) is followed on its stream by
                                frnn_check_last_build (slow: a brute-force pass)       */

typedef struct frnn_plan frnn_plan; /* opaque; owns all device scratch and outputs */

typedef struct {
    int device;            /* CUDA device ordinal                                     */
    int d_max;             /* largest embedding dimension a call may use, 1..64       */
    int64_t n_max;         /* largest total point count of one call (sum over events) */
    int events_max;        /* largest number of events in one call, >= 1             */
    int k_max_cap;         /* largest neighbour cap of one call, 1..1024              */
    int64_t edge_capacity; /* col slots; 0 = n_max * k_max_cap (never overflows)      */
    int cells_per_point;   /* cell-table slots per point (plus 4096 per event); 0 = 4 */
    uint32_t flags;        /* FRNN_EMIT_D2 | FRNN_USE_GRAPH | FRNN_AUTOTUNE | FRNN_DEBUG */
    int64_t hit_capacity;  /* 4-byte slots in which the neighbour walk keeps every
                              neighbour of rows longer than 24 (384 per row, taken 32
                              rows at a time), so that their k nearest are sorted from
                              those instead of walking their candidates again (rows of
                              up to 12 dims); 0 = none.  Speed only, never the result. */
    uint64_t mem_budget_bytes; /* device memory the plan may take; 0 = no limit.  A plan
                              whose device bytes (frnn_plan_bytes) exceed it is refused
                              by frnn_plan_create with FRNN_ERR_OOM before any device
                              call or allocation                                         */
} frnn_plan_params;

/*
 * Output of a build: one CSR over all events of the call, in event order.
 * Event b owns points ev_off[b] .. ev_off[b+1]-1 of the call (ev_off from the
 * call) and edges edge_off[b] .. edge_off[b+1]-1.  For point p of the call,
 * its row is col[row_ptr[p] .. row_ptr[p+1]-1]; col holds point indices LOCAL
 * to the event (0 .. n_b - 1).  Every pointer is device memory owned by the
 * plan and stays valid until the next build on the plan or its destruction.
 */
typedef struct {
    const int32_t* row_ptr;  /* device, n_total + 1 entries, row_ptr[0] = 0           */
    const int32_t* col;      /* device, n_edges entries used                           */
    const float* d2;         /* device, n_edges entries, or NULL without FRNN_EMIT_D2  */
    const int32_t* edge_off; /* device, n_events + 1 entries                           */
    const int32_t* n_edges;  /* device scalar: total edges (= edge_off[n_events])      */
    int n_events;
    int64_t n_total;
} frnn_csr;

/*
 * Cell-grid and walk tuning (speed only; the result never depends on it).
 * g_max: most gridded dimensions, 1..6 (0 = 4); a cell has 3^(g-1) runs of
 * neighbouring cells, and a dimension is only gridded while the event's cell
 * table (cells_per_point x n + 4096 slots) has room.  cell_scale: cell edge /
 * r, >= 1 (0 = 1).  The dimensions gridded are always the ones of widest extent.
 * walk: how the neighbour walk maps work to the 32 lanes of a warp:
 *   FRNN_WALK_AUTO (0)       query-major where it exists (d <= 12), else
 *                            candidate-major;
 *   FRNN_WALK_CANDIDATES (1) the lanes hold 32 candidates of a cell's
 *                            neighbourhood at a time, tested against the
 *                            cell's queries two per packed operation;
 *   FRNN_WALK_QUERIES (2)    a lane per query, each streaming the candidates
 *                            of its own cell's neighbourhood through a
 *                            one-byte-per-dim key filter and testing only the
 *                            ones that pass exactly (d <= 12; larger d falls
 *                            back to FRNN_WALK_CANDIDATES).
 */
#define FRNN_WALK_AUTO 0
#define FRNN_WALK_CANDIDATES 1
#define FRNN_WALK_QUERIES 2

typedef struct {
    int g_max;
    float cell_scale;
    int walk;
} frnn_tuning;

/*
 * Create a plan: allocates every device buffer a call within the given
 * capacities needs, so builds never allocate.  *out receives the plan.
 * Errors: INVALID_ARG (out or p NULL, a capacity out of range, or
 * n_max * k_max_cap >= 2^31 with edge_capacity = 0), CUDA, OOM.
 */
FRNN_API int frnn_plan_create(frnn_plan** out, const frnn_plan_params* p);

/*
 * Device bytes frnn_plan_create would allocate for these parameters (the
 * footprint a serving layer budgets for).  Errors: INVALID_ARG as
 * frnn_plan_create.
 */
FRNN_API int frnn_plan_bytes(const frnn_plan_params* p, uint64_t* bytes);

/* Free every buffer of the plan (synchronises its device).  NULL is a no-op. */
FRNN_API int frnn_plan_destroy(frnn_plan* plan);

/*
 * Set / read the plan's tuning, used by builds whose call shape has no
 * autotuned entry.  Setting it also drops every autotuned entry.
 */
FRNN_API int frnn_plan_set_tuning(frnn_plan* plan, const frnn_tuning* t);
FRNN_API int frnn_plan_get_tuning(const frnn_plan* plan, frnn_tuning* t);

/*
 * Autotune for a workload (the choice of gridded dimensions the paper makes by
 * hand, Sec. 3.4, and the form of the walk).  Each of the 20 grids g_max in
 * {6, 5, 4, 3, 2} x cell_scale in {1, 1.25, 1.5, 2} is probed on the given
 * events (the grid stages and an exact count of the candidate tests, non-empty
 * cells and cell slots a build would handle, no edges written); the three
 * cheapest by that count are timed with each walk form (best of three builds
 * after a warm-up).  The fastest tuning becomes the plan's tuning and the
 * entry for the call's shape (mean points per event, number of events, d, r,
 * k_max; a plan keeps the last 16 shapes), and is returned in *best with its
 * time in *best_ms (either may be NULL).  Synchronous.  Results never depend
 * on the tuning, only the speed does.  Arguments and errors as
 * frnn_build_graph_batched; the plan's last build is not kept.
 */
FRNN_API int frnn_plan_autotune(frnn_plan* plan, const float* emb, const int64_t* ev_off, int n_events,
                                int d, float r, int k_max, void* stream, frnn_tuning* best,
                                float* best_ms);

/*
 * The tuning a build with these arguments would use: the autotuned entry for
 * its shape (*cached = 1) or the plan's tuning (*cached = 0; cached may be
 * NULL).  Host only.  Errors: INVALID_ARG.
 */
FRNN_API int frnn_plan_tuning_for(const frnn_plan* plan, const int64_t* ev_off, int n_events, int d, float r,
                                  int k_max, frnn_tuning* out, int* cached);

/*
 * Build the graph of one event (Sec. 2, Sec. 3.4; the cap of Sec. 3.1).
 *   emb    device, float32, row-major [n][d] with row stride d, caller-owned;
 *          it must stay unchanged until the stream reaches the end of the build.
 *   n      points, 0 <= n <= n_max.       d  dimension, 1 <= d <= d_max.
 *   r      radius, finite and > 0.        k_max  cap, 1 <= k_max <= k_max_cap,
 *          or FRNN_NO_CAP.
 *   stream cudaStream_t the work is enqueued on (asynchronous; no host sync).
 *   out    receives the plan-owned device pointers (n_events = 1).
 * Errors: INVALID_ARG (NULL plan/out, NULL emb with n > 0, sizes out of range,
 * n * k_max >= 2^31), CAPACITY (n > n_max, d > d_max, k_max > k_max_cap), CUDA.
 */
FRNN_API int frnn_build_graph(frnn_plan* plan, const float* emb, int64_t n, int d, float r, int k_max,
                     void* stream, frnn_csr* out);

/*
 * Build the graphs of several independent events in one pass of the kernels.
 *   emb      device, float32 [ev_off[n_events]][d]: the events' points concatenated.
 *   ev_off   HOST array of n_events + 1 offsets, ev_off[0] = 0, non-decreasing
 *            (empty events are allowed).  Read before the call returns.
 *   n_events 1 <= n_events <= events_max.  Other arguments as frnn_build_graph.
 * Each event's rows are identical to those a separate frnn_build_graph call
 * would give.  Errors: as frnn_build_graph, plus INVALID_ARG for bad offsets.
 */
FRNN_API int frnn_build_graph_batched(frnn_plan* plan, const float* emb, const int64_t* ev_off, int n_events,
                             int d, float r, int k_max, void* stream, frnn_csr* out);

/*
 * Host-to-host form (the whole call a CPU-side user makes): copies the
 * events' points from host memory to the device (into a buffer of n_max x
 * d_max floats the plan reserves at creation), builds, and copies the CSR
 * back.  Synchronous: returns when the host buffers are filled.
 *   h_emb       host float32 [ev_off[n_events]][d] (pinned memory is faster).
 *   h_row_ptr   host int32 [ev_off[n_events] + 1], receives row_ptr.
 *   h_col       host int32 [col_capacity], receives col.
 *   h_edge_off  host int32 [n_events + 1] or NULL.
 *   h_n_edges   host int64, receives the edge count (also when it exceeds
 *               col_capacity, in which case the call returns OVERFLOW and
 *               h_col is not written).
 * Errors: as frnn_build_graph_batched, plus OVERFLOW, and any status the
 * device latched during this build.
 */
FRNN_API int frnn_build_graph_host(frnn_plan* plan, const float* h_emb, const int64_t* ev_off,
                          int n_events, int d, float r, int k_max, int32_t* h_row_ptr,
                          int32_t* h_col, int64_t col_capacity, int32_t* h_edge_off,
                          int64_t* h_n_edges, void* stream);

/*
 * frnn_build_graph_batched with a CUDA event recorded between the stages,
 * for profiling.  Never replays a CUDA graph.  Synchronous: waits for the
 * build, then writes the device time of each stage in milliseconds to
 * stage_ms[0..6]: bounding box and cell grid, cell ids and histogram, cell
 * scan, scatter into cell order (with the filter keys), collect walk, row
 * scan, emit walk.
 * n_stages must be >= 7.  Errors: as frnn_build_graph_batched.
 */
FRNN_API int frnn_build_graph_profiled(frnn_plan* plan, const float* emb, const int64_t* ev_off,
                                       int n_events, int d, float r, int k_max, void* stream,
                                       frnn_csr* out, float* stage_ms, int n_stages);

/*
 * Track labeling on the plan's last build (the step after graph building,
 * Sec. 2: edges passing a score cut grouped into weakly connected
 * components, each a track candidate; Sec. 3.2 uses cuGraph's WCC).  The
 * score here is the edge's d2: edges with d2 <= d2_max are kept, their
 * direction is ignored, and labels[p] (device int32, one per point of the
 * last call) receives the smallest event-local index of p's component.
 * d2_max >= r*r keeps every edge; a smaller cut needs a plan created with
 * FRNN_EMIT_D2.  Asynchronous on `stream` (enqueue it after the build on the
 * same stream); uses the plan's scratch, so it must run before the next
 * build.  Call it only after a build without OVERFLOW.  Errors: INVALID_ARG
 * (NULL, no build yet, NaN cut, cut below r*r without FRNN_EMIT_D2), CUDA;
 * a bounded retry that ran out latches FRNN_ERR_TIMEOUT.
 */
FRNN_API int frnn_label_components(frnn_plan* plan, float d2_max, void* stream, int32_t* labels);

/*
 * Edge features for the filter stage (Sec. 3: the edge-filter network reads
 * the graph's edges in fixed-size batches, 800k edges in the paper): for the
 * edges e_begin .. e_end-1 of the plan's last build (CSR order, call-wide
 * edge numbers as in frnn_csr), out[(e - e_begin) * (2d + 1) + ...] receives
 * x_i[0..d), x_j[0..d) and d2(i, j) (the same float32 value the build
 * tested).  emb: device float32 [n_total][d], the points of the last build.
 * out: device float32 [(e_end - e_begin) * (2d + 1)].  Asynchronous; call
 * after the build on the same stream, before the next build.  Errors:
 * INVALID_ARG (NULL, no build yet, bad range or e_end beyond the edge
 * capacity), CUDA.
 */
FRNN_API int frnn_edge_features(frnn_plan* plan, const float* emb, int64_t e_begin, int64_t e_end, float* out,
                                void* stream);

/*
 * Exact k-nearest-neighbour graphs of a batch of events, with no radius: the
 * paper's kNN route (Sec. 3.1, Faiss IndexFlat exact kNN) without the radius
 * cut that follows it there.  Row i of event b holds the k_b = min(k, n_b - 1)
 * points j != i smallest by (d2, j), d2 as in frnn_build_graph (float32,
 * dims summed in order, no fused multiply-add), in increasing (d2, j) order;
 * so every row of an event has the same length.  Arguments, layout and
 * ownership as frnn_build_graph_batched (no radius; 1 <= k <= k_max_cap);
 * the total sum_b n_b k_b must fit the plan's edge capacity (else
 * FRNN_ERR_CAPACITY, nothing enqueued).  An event holding NaN or Inf keeps
 * its row lengths, its entries are -1 (d2 +Inf) and FRNN_ERR_NONFINITE_INPUT
 * is latched.  The result is the plan's last build for frnn_label_components
 * (cut d2_max = +Inf keeps every edge; a finite cut needs FRNN_EMIT_D2) and
 * frnn_edge_features.  Asynchronous on `stream`; not captured in a CUDA
 * graph.  Errors: INVALID_ARG, CAPACITY, CUDA; TIMEOUT may be latched.
 */
FRNN_API int frnn_knn_graph_batched(frnn_plan* plan, const float* emb, const int64_t* ev_off, int n_events,
                                   int d, int k, void* stream, frnn_csr* out);

/*
 * Synchronise `stream`, then return and clear the status latched by the
 * plan's kernels since the last call (FRNN_OK if none).  If several errors
 * were latched the most severe is returned, in the order CHECK, TIMEOUT,
 * OVERFLOW, NONFINITE_INPUT.  A CUDA error on the stream returns
 * FRNN_ERR_CUDA.
 *
 * TIMEOUT: one of the scans' waits for a preceding tile (each bounded to
 * 2^22 polls and 1 s) ran out, so cell or row offsets of that build may be
 * wrong.  The bit stays latched until this call reads it; until then every
 * kernel that addresses memory through those offsets (scatter, walks, row
 * copy, labeling, edge features) skips its work, so no access leaves the
 * plan's buffers: a radius build returns empty rows (row_ptr all 0), a kNN
 * build rows of unspecified content, labeling one component per point.  On
 * reporting TIMEOUT this call restores the plan's between-builds device
 * state (the next build is exact again) and forgets the last build
 * (frnn_label_components and frnn_edge_features then return INVALID_ARG
 * until the next build).
 */
FRNN_API int frnn_get_last_status(frnn_plan* plan, void* stream);

/*
 * Debug checks of the plan's last build (radius or kNN), enqueued on `stream`
 * as kernels that only read the build's buffers and the caller's input, which
 * must be unchanged since the build.  Labeling and edge features write nothing
 * they read, so the checks may run at any point before the plan's next build.
 * Each check tests one stage's output
 * against what that stage must produce (Sec. 3.4: cell lists, then per-point
 * neighbour lists), in pipeline order:
 *   FRNN_CHECK_EVENT_OFFSETS  edge_off[b] = row_ptr[first point of b], and
 *                             edge_off[n_events] = row_ptr[n_total]
 *   FRNN_CHECK_CELL_TABLE     an event's cell offsets ascend from its first
 *                             sorted position to one past its last
 *   FRNN_CHECK_SCATTER        the sorted order is a permutation of each
 *                             event's points, each inside its cell's range,
 *                             its sorted row the input row bit for bit
 *   FRNN_CHECK_ROW_PTR        row_ptr[0] = 0, rows do not shrink, no row
 *                             exceeds the cap; rows of an event with NaN/Inf
 *                             are empty (radius) or min(k, n_b - 1) long (kNN)
 *   FRNN_CHECK_COLUMN         each column is an index of the event other than
 *                             the row's own (kNN, NaN/Inf event: -1)
 *   FRNN_CHECK_RADIUS         d2(i, j) <= fl32(r * r) (radius builds)
 *   FRNN_CHECK_D2             the emitted d2 equals d2(i, j) bit for bit
 *                             (plans with FRNN_EMIT_D2)
 *   FRNN_CHECK_ORDER          sorted rows ascend strictly by (d2, j) (every
 *                             row but the unsorted ones of FRNN_NO_CAP)
 *   FRNN_CHECK_COMPLETE       brute force over the event: a row holds
 *                             min(k, |S_i|) entries (kNN: min(k, n_b - 1)),
 *                             no other point of the event is smaller by
 *                             (d2, j) than its last, and the sums of its
 *                             columns and their squares match the points that
 *                             belong in it.  In an event of n_b > 2^17 points
 *                             only every ceil(n_b^2 / 2^34)-th row is checked,
 *                             so that no event costs more than 2^34 distances.
 * d2 is recomputed as defined at the top of this file.  Checks 5-9 are
 * skipped when the edges overflowed the edge capacity, and every check when a
 * bounded wait of the build ran out (its rows are empty by design).  A failed
 * check latches FRNN_ERR_CHECK (reported by frnn_get_last_status ahead of the
 * other statuses) and is recorded for frnn_get_last_check.  Cost: on a B300
 * the brute-force pass makes about 5 x 10^11 distance evaluations a second
 * (d = 8; a 64-event batch of 120k-point events takes about 2 s); on a single
 * event large enough to be sampled it has few rows in flight and makes
 * 1-3 x 10^11 a second.  No check
 * traps or faults: every index read from the build's buffers is range-checked
 * before it addresses memory.  Errors: INVALID_ARG (NULL plan, no build yet),
 * CUDA.
 */
#define FRNN_CHECK_NONE 0
#define FRNN_CHECK_EVENT_OFFSETS 1 /* index: event                          */
#define FRNN_CHECK_CELL_TABLE 2    /* index: cell slot of the call's table  */
#define FRNN_CHECK_SCATTER 3       /* index: sorted position                */
#define FRNN_CHECK_ROW_PTR 4       /* index: point of the call              */
#define FRNN_CHECK_COLUMN 5        /* index: edge of the call               */
#define FRNN_CHECK_RADIUS 6        /* index: edge                           */
#define FRNN_CHECK_D2 7            /* index: edge                           */
#define FRNN_CHECK_ORDER 8         /* index: edge                           */
#define FRNN_CHECK_COMPLETE 9      /* index: point                          */
FRNN_API int frnn_check_last_build(frnn_plan* plan, void* stream);

/*
 * Synchronise `stream`, then return the first failure the debug checks have
 * recorded since the last call, and clear the record: *check receives the
 * FRNN_CHECK_* id of the earliest failing stage (FRNN_CHECK_NONE if none) and
 * *index its smallest failing index of that check (-1 if none).  The status
 * bit FRNN_ERR_CHECK is read and cleared by frnn_get_last_status.  Errors:
 * INVALID_ARG (NULL argument), CUDA.
 */
FRNN_API int frnn_get_last_check(frnn_plan* plan, void* stream, int* check, int64_t* index);

/*
 * Failure-detection test hook.  The next build that launches kernels on
 * `plan` (radius or kNN) runs its cell scan with tile 0 waiting for a
 * predecessor that never publishes, so every tile's bounded wait runs out
 * (after about 1 s) and FRNN_ERR_TIMEOUT is latched as described at
 * frnn_get_last_status().  No GPU fault, trap or unbounded wait is involved:
 * the waits end, the kernels return, the context stays usable.  Not for
 * production use.  Errors: INVALID_ARG (NULL plan).
 */
FRNN_API int frnn_plan_test_stall_next_build(frnn_plan* plan);

/*
 * Build the graph of one event without allocating any device memory.  The
 * paper has no counterpart: this is for callers that may not call cudaMalloc
 * (code running inside a framework that owns all device memory and forbids
 * allocation after start-up, or whose device memory is fixed at
 * initialisation).  The caller passes the points and the outputs; every other
 * buffer lives in one array of about 12.5 MB in device memory that each
 * device loading the library holds until the process exits.
 *   emb          device float32 [n][d], row-major, caller-owned.
 *   n <= 32768, d <= 16, k_max <= 64; larger sizes return FRNN_ERR_CAPACITY
 *                (nothing is enqueued).
 *   row_ptr      device int32 [n + 1], receives the row offsets.
 *   col          device int32 [col_capacity], receives the rows (event-local
 *                indices, in increasing (d2, j) order, as frnn_build_graph).
 *   status       device int32, receives the device-side outcome: FRNN_OK,
 *                FRNN_ERR_NONFINITE_INPUT, FRNN_ERR_OVERFLOW (more edges than
 *                col_capacity) or FRNN_ERR_TIMEOUT.
 *   stream       cudaStream_t; asynchronous, no host synchronisation.
 * Runs on the calling thread's current device.  The first call on a device
 * (and the first with a new d rounded up to 4) looks up the array's device
 * address and the launch shapes, which are not stream-ordered calls: make it
 * before any stream capture.  Such a set-up call on a capturing stream
 * returns FRNN_ERR_INVALID_ARG and enqueues nothing.  All calls on a device share the array:
 * calls whose work overlaps on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.  Each call clears what must
 * start at zero, so results never depend on an earlier call.
 * Returns FRNN_OK, FRNN_ERR_INVALID_ARG, FRNN_ERR_CAPACITY or FRNN_ERR_CUDA.
 */
FRNN_API int frnn_build_graph_noalloc(const float* emb, int64_t n, int d, float r, int k_max,
                                      int32_t* row_ptr, int32_t* col, int64_t col_capacity,
                                      int32_t* status, void* stream);

/*
 * Serving: events arriving over time, built with continuous batching.
 * (The paper runs the pipeline per event inside a multithreaded C++ host,
 * Sec. 4, and names a model server as future work, Sec. 6.)  On each of its
 * devices a server owns `slots` regular slots and one spill slot: a slot is a
 * plan with its own stream, its device memory reserved at creation within the
 * per-device budget.  A dispatcher thread starts a batched build on every free
 * slot with the requests that have arrived and not started, in arrival order,
 * as many as fit the slot: batch_points points, batch_events events, and the
 * slot's edges (a request's edges are estimated from the edges per point of
 * the requests finished so far until a build has counted them exactly).
 * Batches on different slots overlap on the device, and requests arriving
 * meanwhile are admitted as slots free up.  When slots on several devices are
 * free, the device with the fewest points in flight is served first.
 *
 * Edge overflow is per request: a batch whose edges exceed its slot completes
 * the requests whose edges fit and re-queues the others, at the front of the
 * queue and with their exact edge counts, onto a regular slot if they fit one,
 * else alone onto a spill slot (room for batch_points x k edges, or for as
 * many edges as the budget leaves).  Only a request with more edges than the
 * spill slot holds fails, with FRNN_ERR_OVERFLOW.  Each request's rows are
 * identical to a separate frnn_build_graph of the same points.
 */
typedef struct frnn_server frnn_server;

typedef struct {
    int device;                /* device of the slots when n_devices is 0             */
    int d;                     /* embedding dimension of every request, 1..64        */
    float r;                   /* radius (finite, > 0)                                */
    int k;                     /* neighbour cap, 1..1024                              */
    int64_t batch_points;      /* points of one batched launch (also the largest event) */
    int batch_events;          /* events of one batched launch                        */
    int slots;                 /* regular slots per device, 1..64                     */
    int edges_per_point;       /* edge capacity of a regular slot per point (0 = min(32, k)) */
    uint64_t mem_budget_bytes; /* device memory the slots of one device may reserve (0 = no limit) */
    int n_devices;             /* 0: the one device `device`; else devices[0 .. n_devices) */
    const int* devices;        /* host array of device ordinals, read during create;
                                  a device listed twice gets two independent sets of slots */
} frnn_server_params;

/* Counters of a server (frnn_server_get_stats). */
typedef struct {
    uint64_t batches;               /* batched builds finished                          */
    uint64_t spill_batches;         /* ... of them on a spill slot                       */
    uint64_t readmitted;            /* requests re-queued after their batch overflowed   */
    uint64_t requests_done;         /* requests finished (any status)                    */
    uint64_t max_queue;             /* most requests waiting at once                     */
    uint64_t regular_edge_capacity; /* edges a regular slot holds                        */
    uint64_t spill_edge_capacity;   /* edges a spill slot holds                          */
} frnn_server_stats;

/*
 * Create a server and its dispatcher thread.  Device memory of all slots is
 * reserved here: FRNN_ERR_OOM if one device's slots (the regular ones plus a
 * spill slot at least as large) exceed mem_budget_bytes, or the device.
 * Errors: INVALID_ARG (sizes out of range, batch_points * k >= 2^31, a bad
 * device ordinal), OOM, CUDA.
 */
FRNN_API int frnn_server_create(frnn_server** out, const frnn_server_params* p);

/* Device bytes the server reserved for its slots (all devices). */
FRNN_API int frnn_server_reserved_bytes(const frnn_server* srv, uint64_t* bytes);

/* Copy the server's counters to *stats.  Errors: INVALID_ARG. */
FRNN_API int frnn_server_get_stats(frnn_server* srv, frnn_server_stats* stats);

/*
 * Queue one event (host float32 [n][d]; the buffer must stay valid and
 * unchanged until frnn_server_wait returns for this ticket; pinned memory
 * copies faster).  Returns at once.  Errors: INVALID_ARG, CAPACITY
 * (n > batch_points), OOM.
 */
FRNN_API int frnn_server_submit(frnn_server* srv, const float* host_emb, int64_t n, uint64_t* ticket);

/*
 * Non-blocking check: *done = 1 once the event of `ticket` is finished (a
 * following frnn_server_wait returns without waiting), else 0.  Errors:
 * INVALID_ARG (NULL, or a ticket unknown or already waited for).
 */
FRNN_API int frnn_server_poll(frnn_server* srv, uint64_t ticket, int* done);

/*
 * Block until the event of `ticket` is built, then copy its CSR (event-local
 * indices) to host buffers: row_ptr [n + 1], col [col_capacity].  *n_edges
 * and *latency_s (arrival to rows on the host) may be NULL.  Each ticket can
 * be waited for once.  Returns the event's status: OVERFLOW if col_capacity
 * is too small, or if the event's edges exceed even a spill slot (*n_edges
 * then receives the edge count).
 */
FRNN_API int frnn_server_wait(frnn_server* srv, uint64_t ticket, int32_t* row_ptr, int32_t* col,
                              int64_t col_capacity, int64_t* n_edges, double* latency_s);

/*
 * Replay an arrival trace through the server: request i, the points
 * host_emb[ev_start[i] .. ev_start[i] + ev_len[i]) (rows of d floats; requests
 * may share points), is submitted arrival_s[i] seconds (non-decreasing) after
 * the call starts, by the calling thread.  Returns when every request is done;
 * latency_s[i] (arrival to rows on the host), n_edges[i] (may be NULL) and
 * *wall_s (may be NULL) are filled in.  The rows themselves are not kept.
 * Returns the first non-OK request status.
 */
FRNN_API int frnn_server_run_trace(frnn_server* srv, const float* host_emb, const int64_t* ev_start,
                                   const int64_t* ev_len, const double* arrival_s, int n_events,
                                   double* latency_s, int64_t* n_edges, double* wall_s);

/* Finish queued work, stop the dispatcher and free everything.  NULL is a no-op. */
FRNN_API int frnn_server_destroy(frnn_server* srv);

/* Static English description of a status code (never NULL). */
FRNN_API const char* frnn_status_string(int status);

/* Library version as major * 10000 + minor * 100 + patch. */
FRNN_API int frnn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FRNN_H */
