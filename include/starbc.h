/*
 * starbc — Brandes betweenness centrality (BC) on one GB300 GPU (sm_103a).
 *
 * The operation (paper Section 2, Fig. 1, the ComputeBC program, which follows
 * Brandes' algorithm): for a multiset S of source vertices of an unweighted
 * undirected graph G,
 *
 *     BC(v) = sum_{s in S, s != v} delta_s(v),
 *     delta_s(v) = sum over BFS children w of v (dist_s(w) = dist_s(v) + 1) of
 *                  (sigma_s(v) / sigma_s(w)) * (1 + delta_s(w)),
 *
 * where sigma_s(v) counts shortest s-v paths, built in a forward BFS by adding
 * sigma over BFS parents (Fig. 1, the iterateInBFS loop) and delta in a
 * reverse-level sweep (Fig. 1, the iterateInReverse loop).  Ordered (s, t)
 * pairs are counted: no halving.  Duplicated sources count once per
 * occurrence.  Vertices not reached from s receive nothing from s.
 *
 * Graph input: int32 CSR, row_ptr[n+1] and col_idx[nnz], both directions of
 * every undirected edge stored (the paper's CSR offset array and edge list,
 * Section 3.1), or the out-arcs of a directed graph (SP_GRAPH_DIRECTED; the
 * in-arcs are built on the GPU, as the paper's generated code keeps a reverse
 * CSR for pulls over in-neighbours, Section 3.3, the PageRank listing).  Rows need not be sorted; a
 * repeated arc counts as a parallel edge and a self-loop is never on a
 * shortest path.
 *
 * Pointers: every array argument may be host memory or device memory of the
 * current device (device memory of another GPU is refused with
 * SP_ERR_INVALID_ARG); the library tells them apart with
 * cudaPointerGetAttributes.  Work is issued on `stream` (a cudaStream_t; NULL
 * is the legacy default stream).
 *
 * Completion: sp_bc, and sp_bc_ex without statistics, are asynchronous when
 * bc_out is device memory: the work is enqueued on `stream` and the call
 * returns without waiting for the GPU (the level loop runs inside persistent
 * kernels; no host decision is needed between levels).  Device sources are
 * read in place and must stay valid until the stream reaches the work; host
 * sources are checked and copied before return.  Such a call still blocks
 * once per graph for one-time set-up (the eccentricity and landmark BFS, and
 * the timing trials that pick a batch width or a plain-form driver for a new
 * graph shape), and whenever it runs the graph-driven plain form.  All other
 * calls (host output, statistics requested, sp_bfs, sp_sigma, graph creation)
 * return once their result is complete.
 *
 * Device memory: a graph owns its CSR copy until sp_graph_destroy.  Each BC
 * call takes its workspace (per-source state, level stack) from a memory pool
 * of the library's own, stream-ordered on `stream`, and returns it at the end
 * of the call; the pool keeps freed memory for later calls (a failed
 * allocation releases it and retries once).
 *
 * Errors: every entry point returns an sp_status.  Argument errors, allocation
 * failures and CUDA errors are returned by the call that met them, and so are
 * errors the GPU finds during a blocking call.  An asynchronous call's device
 * errors (a path count or dependency out of range, a device-side wait that
 * timed out, a source in a device array that is not a vertex, a workspace
 * limit) are latched in the graph's error word and returned, once, by the
 * next call on that graph (which then does nothing else) or by
 * sp_graph_sync.  Conditions that a wider representation fixes are handled
 * on the GPU without the host: counts past the exact integer range or
 * dependencies past FP32 open a fallback launch of the plain form with FP64
 * counts and dependencies that runs in the same stream only when needed, and
 * later calls on the graph start in the representation that fits.
 * sp_last_error() gives a one-line description of the last failure on the
 * calling thread.  Nothing here ever aborts or traps the GPU.
 */
#ifndef STARBC_H
#define STARBC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SP_API __attribute__((visibility("default")))
#else
#define SP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

struct CUstream_st;
typedef struct CUstream_st* sp_stream; /* same type as cudaStream_t */

typedef enum {
    SP_OK = 0,
    SP_NOT_READY = 1,        /* request still running (sp_bc_poll) */
    SP_ERR_INVALID_ARG = -1, /* bad pointer, size, source id or option */
    SP_ERR_OOM = -2,         /* device or pinned host memory exhausted */
    SP_ERR_CUDA = -3,        /* a CUDA runtime call failed */
    SP_ERR_TOO_LARGE = -4,   /* nnz >= 2^31, or a limit of the chosen form exceeded */
    SP_ERR_RANGE = -5,       /* a path count or dependency left the representable range */
    SP_ERR_TIMEOUT = -6,     /* a device-side wait gave up (the launch stopped cleanly) */
    SP_ERR_CANCELLED = -7,   /* request cancelled */
    SP_ERR_BAD_GRAPH = -8,   /* CSR failed validation (row_ptr not monotone, id out of range, ...) */
    SP_ERR_NO_DEVICE = -9    /* no CUDA device of compute capability 10.3 */
} sp_status;

typedef struct sp_graph_s* sp_graph;
typedef struct sp_server_s* sp_server;
typedef int64_t sp_request;

/* ------------------------------------------------------------------------ */
/* Graphs                                                                    */

/* Flags for sp_graph_create. */
#define SP_GRAPH_CHECK_SYMMETRIC 0x1u /* also verify every arc (u,v) has its reverse (v,u) */
#define SP_GRAPH_SORT_ROWS 0x2u       /* sort every row by neighbour id on the GPU (after the copy) */
#define SP_GRAPH_DIRECTED 0x4u        /* row v lists the out-arcs v -> w of a directed graph (see below) */

typedef struct {
    int32_t n;
    int32_t max_degree;
    int64_t nnz;
    int64_t isolated;       /* vertices of degree 0 */
    int32_t sorted_rows;    /* 1 when every row is strictly increasing */
    int32_t has_self_loops; /* 1 when some arc (v,v) exists */
    int32_t has_duplicates; /* 1 when some arc appears twice in a row (only detected on sorted rows) */
    int32_t symmetric;      /* 1 yes, 0 no, -1 not checked */
    int32_t directed;       /* 1 when created with SP_GRAPH_DIRECTED */
    int32_t reserved;
} sp_graph_info;

/*
 * Copy a CSR graph into device memory and validate it on the GPU: row_ptr[0]
 * == 0, row_ptr non-decreasing, row_ptr[n] == nnz, every col_idx in [0, n).
 * The inputs are copied before return (the caller may free them); the graph
 * owns its device memory until sp_graph_destroy.  Blocks until done.
 * n >= 0; nnz < 2^31.  Returns SP_ERR_BAD_GRAPH on a CSR that fails, with the
 * first offending index in sp_last_error().  With SP_GRAPH_SORT_ROWS the rows
 * of the copy are sorted (deterministically, on the GPU) before the checks.
 *
 * With SP_GRAPH_DIRECTED the CSR holds the arcs of a directed graph (row v:
 * the heads w of the arcs v -> w) and BC counts directed shortest paths: the
 * BFS and the dependencies follow out-arcs, path counts are pulled over
 * in-arcs (BFS parents u -> v).  The library builds each vertex's in-arcs
 * (the transpose) on the GPU and keeps one combined row per vertex, out-arcs
 * then in-arcs, so 2 nnz must stay below 2^31 (else SP_ERR_TOO_LARGE);
 * traversed arcs count out-arcs.  Not with SP_GRAPH_CHECK_SYMMETRIC.
 */
SP_API sp_status sp_graph_create(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t nnz,
                          uint32_t flags, sp_stream stream, sp_graph* out);
/* Frees the graph after the work issued on it has finished. */
SP_API sp_status sp_graph_destroy(sp_graph g);
/* Wait for `stream`, then return (and clear) the error latched by an earlier
   asynchronous call on the graph: SP_OK when there is none. */
SP_API sp_status sp_graph_sync(sp_graph g, sp_stream stream);

/*
 * Build a graph from an undirected edge list on the GPU (the CSR offset array
 * and edge list of Section 3.1): for every edge i with src[i] != dst[i] both
 * arcs are stored, rows are sorted by neighbour id and repeated arcs are kept
 * once; self-loops are dropped.  src, dst: int32 [m], host or device, copied
 * before return.  n >= 0 vertices; 2 m < 2^31.  flags: 0,
 * SP_GRAPH_CHECK_SYMMETRIC, or SP_GRAPH_DIRECTED (each edge i is the single
 * arc src[i] -> dst[i]; the graph is directed as for sp_graph_create).  An
 * endpoint outside [0, n) gives SP_ERR_BAD_GRAPH with the edge index in
 * sp_last_error().  Blocks until done.
 */
SP_API sp_status sp_graph_from_edges(const int32_t* src, const int32_t* dst, int64_t m, int32_t n, uint32_t flags,
                                     sp_stream stream, sp_graph* out);

/*
 * Arc weights (BC over weighted shortest paths; the paper's SSSP program
 * relaxes dist[nbr] through dist[v] + weight, Section 3.5, the Min construct).
 * weights: int32 [nnz] parallel to col_idx (the CSR sp_graph_get_csr
 * returns), each in [1, 2^20], host or device, copied before return.  The
 * graph must be undirected with sorted rows and no repeated arc
 * (SP_GRAPH_SORT_ROWS or sp_graph_from_edges give that), and the two arcs of
 * an edge must carry the same weight: checked on the GPU (SP_ERR_BAD_GRAPH
 * with the arc in sp_last_error(); directed graphs: SP_ERR_INVALID_ARG).  From
 * then on sp_bc / sp_bc_ex compute BC with shortest paths by total weight in
 * the weighted form (SP_FORM_WEIGHTED, one block per source: distances by
 * near-far frontier rounds with atomicMin, path counts and dependencies
 * in FP64 over the weighted shortest-path DAG, level by level in distance
 * order); those calls return when the result is complete, and the precision
 * option does not apply (FP64).  sp_bfs still gives hop distances.
 * Calling it again replaces the weights.
 */
SP_API sp_status sp_graph_set_weights(sp_graph g, const int32_t* weights, sp_stream stream);

/* Shortest distances under the graph's weights: dist_out[i * n + v] =
   dist(sources[i], v), -1 when unreachable.  int32 [nsrc][n], host or device.
   Returns when complete. */
SP_API sp_status sp_sssp(sp_graph g, const int32_t* sources, int32_t nsrc, int32_t* dist_out, sp_stream stream);

/* Copy the graph's CSR out: row_ptr_out int32 [n+1], col_idx_out int32 [nnz],
   host or device.  Returns when the copy is complete. */
SP_API sp_status sp_graph_get_csr(sp_graph g, int32_t* row_ptr_out, int32_t* col_idx_out, sp_stream stream);
SP_API sp_status sp_graph_get_info(sp_graph g, sp_graph_info* out);

/* ------------------------------------------------------------------------ */
/* Betweenness centrality                                                   */

enum { SP_FP64 = 0, SP_FP32_DELTA = 1 };
enum { SP_FORM_AUTO = 0, SP_FORM_PLAIN = 1, SP_FORM_BATCHED = 2, SP_FORM_SMALL = 3, SP_FORM_WEIGHTED = 4 };

typedef struct {
    int32_t precision;          /* SP_FP64 (delta in FP64) or SP_FP32_DELTA (delta stored in FP32) */
    int32_t form;               /* SP_FORM_AUTO, SP_FORM_PLAIN (one source at a time per block group),
                                   SP_FORM_BATCHED (bitmap batches of sources) or SP_FORM_SMALL (one
                                   block per source, state in shared memory; graphs of up to about
                                   14,500 vertices, else SP_ERR_TOO_LARGE) */
    int32_t batch;              /* batched form: sources per batch, 32, 64, 128 or 256; 0 = autotuned */
    int32_t max_ctas;           /* cap on the persistent grid (0 = every co-resident CTA) */
    int64_t barrier_timeout_ns; /* per device-side wait; 0 = 20 s */
    int32_t debug_flags;        /* SP_DEBUG_* (tests only) */
    int32_t flags;              /* SP_BC_* */
    int32_t bottom_up;          /* discover bottom-up on levels holding more than n / bottom_up vertices
                                   (direction-optimising BFS; results do not change).  Plain form: 0 =
                                   chosen by the plain-form trial (or 100 on graphs of 2^20+ vertices),
                                   -1 = never.  Batched form (per-source bitmaps): 0 = 100 on graphs of
                                   2^20 or more vertices, else never; -1 = never. */
    int32_t driver;             /* plain form's level loop: SP_DRIVER_AUTO, _PERSISTENT or _GRAPH */
} sp_bc_opts;

/* driver: how the plain form steps from level to level (both give
   bit-identical results when the persistent kernel runs one block group).
   PERSISTENT: one cooperative kernel per call; blocks meet at timed device
   barriers between levels and may form groups that run sources side by side.
   GRAPH: a CUDA graph whose conditional WHILE node runs one kernel per level
   plus a one-thread step that sets the loop condition on the device; one
   source at a time over the whole GPU, no device-side waits.
   AUTO: PERSISTENT, unless a timing trial on the first eight sources of a
   call with at least 16 sources, run once per graph shape and cached, finds
   GRAPH faster.  With bottom_up = 0 the same trial also picks the bottom-up
   threshold (never, n/100 or n/20). */
enum { SP_DRIVER_AUTO = 0, SP_DRIVER_PERSISTENT = 1, SP_DRIVER_GRAPH = 2 };

/* flags: run the batched form's sources in the caller's order.  By default
   they are regrouped so that sources at similar distance from a maximum-degree
   vertex share batches and adjacent lanes (BC is a sum over sources, so only
   the rounding order changes). */
#define SP_BC_KEEP_ORDER 0x1

/* debug_flags: block 0 leaves at one grid barrier without arriving, so the
   other blocks' waits run out and the call returns SP_ERR_TIMEOUT. */
#define SP_DEBUG_SKIP_BARRIER 0x1
/* debug_flags: the plain form keeps each vertex's per-source state in one
   32-byte record (RECORDS) or in separate arrays (ARRAYS) whatever the size of
   the groups' state; by default records are used when there are several
   groups and their state is more than twice the size of L2.  Results are the same bit for bit. */
#define SP_DEBUG_PLAIN_RECORDS 0x2
#define SP_DEBUG_PLAIN_ARRAYS 0x4

typedef struct {
    int64_t traversed_arcs; /* sum over sources s of A_s = sum of degrees of vertices reached from s */
    int64_t reached;        /* sum over sources of |R_s| (including s) */
    int64_t entries;        /* (vertex, level) work entries over all batches (batched form) */
    int64_t scanned_arcs;   /* adjacency entries read, forward + backward */
    int64_t dag_arcs;       /* (arc, source) pairs with the arc on a shortest path from the source */
    double kernel_ms;       /* device time of the BC kernel launches (CUDA events), summed */
    int32_t max_levels;     /* max over sources of L = 1 + eccentricity of s */
    int32_t batches;        /* batches (plain form: one per source) */
    int32_t batch;          /* sources per batch used (1 for the plain form) */
    int32_t form;           /* SP_FORM_PLAIN, SP_FORM_BATCHED, SP_FORM_SMALL or SP_FORM_WEIGHTED */
    int32_t promoted;       /* 1 when FP32 dependencies left the FP32 range and the call reran with FP64 */
    int32_t sigma_float;    /* 1 when path counts needed FP64 with per-level rescaling (a count above
                               2^32 in the batched form, above 2^64 in the plain form, any carry in the
                               small form) */
    int32_t launches;       /* kernel launches of the call, including reruns and autotuning trials */
    int32_t tuned;          /* 1 when this call ran an autotuner (batch width, or the plain form's driver) */
    int32_t driver;         /* plain form: SP_DRIVER_PERSISTENT or SP_DRIVER_GRAPH; 0 for the other forms */
    int32_t bottom_up;      /* plain and batched forms: levels wider than n / bottom_up were discovered
                               bottom-up; 0 = never */
    int32_t shared;         /* serving: requests that shared this request's launch (itself included) */
    int32_t recentred;      /* (level, source) pairs whose FP64 path counts were recentred by a power of
                               two (X6 of the readings; 0 unless sigma_float) */
    int32_t joined;         /* serving: 1 when the request entered a batched launch that was already
                               running, between two of its batches; 0 otherwise */
    int32_t reserved;
} sp_bc_stats;

SP_API void sp_bc_opts_default(sp_bc_opts* o);

/*
 * BC over sources[0..nsrc) into bc_out[n] (FP64, overwritten, not accumulated:
 * the paper's attachNodeProperty(BC = 0) then the per-source sums).
 * sources: int32, host or device; each in [0, n) (host sources are checked
 * before return; a bad source in a device array is a latched error).
 * nsrc == 0 gives all zeros.  bc_out: host or device.  With device bc_out the
 * call is asynchronous on `stream` (see Completion above); with host bc_out
 * it returns when bc_out holds the result.
 */
SP_API sp_status sp_bc(sp_graph g, const int32_t* sources, int32_t nsrc, double* bc_out, sp_stream stream);

/* As sp_bc with options.  `stats` (host, may be NULL) receives the call's
   statistics; a call that asks for them returns when the result is complete. */
SP_API sp_status sp_bc_ex(sp_graph g, const int32_t* sources, int32_t nsrc, const sp_bc_opts* opts, double* bc_out,
                   sp_bc_stats* stats, sp_stream stream);

/*
 * Hop distances of the forward BFS (Fig. 1, iterateInBFS; Section 3.4 BFS
 * traversal): dist_out[i * n + v] = dist(sources[i], v), -1 when unreachable.
 * dist_out: int32 [nsrc][n], host or device.
 */
SP_API sp_status sp_bfs(sp_graph g, const int32_t* sources, int32_t nsrc, int32_t* dist_out, sp_stream stream);

/*
 * Shortest-path counts from one source (Fig. 1, the sigma sums of the forward
 * pass) as mant_out[v] * 2^exp2_out[v], mant in [1, 2), 0 when unreachable.
 * mant_out: double[n]; exp2_out: int64[n]; host or device.
 */
SP_API sp_status sp_sigma(sp_graph g, int32_t src, double* mant_out, int64_t* exp2_out, sp_stream stream);

/*
 * Approximate BC by source sampling (the paper's BC runs a few sources; the
 * paper has no estimator or bound: Section 2 and the BC comparison of Section
 * 5.1).  Sources are drawn uniformly with replacement on the GPU:
 * s_i = floor(x_i * n / 2^64), x_i = SplitMix64(seed, i) (state
 * seed + (i + 1) * 0x9E3779B97F4A7C15, then the published finaliser), i = 0,
 * 1, ...; bc_out[v] = (n / k) * sum_i delta_{s_i}(v) estimates BC over all n
 * sources (unbiased).  Rounds of sources (k_min first, then at most doubling
 * k) run until the empirical Bernstein half-width (Maurer and Pontil 2009,
 * Theorem 4, both sides, union over the n vertices) of every normalised
 * value BC(v) / ((n - 1)(n - 2)) is at most eps with probability at least
 * 1 - alpha, or k reaches k_max:
 *     half = sqrt(2 V L / k) + 7 R L / (3 (k - 1)),  L = ln(4 n / alpha),  R = n / (n - 1),
 * V the largest sample variance of n delta_s(v) / ((n - 1)(n - 2)).  The
 * bound is the fixed-sample bound at each round's k: no correction is made
 * for checking it after several rounds (a union over r rounds would replace
 * alpha by alpha / r).
 *   eps > 0, 0 < alpha < 1, 2 <= k_min <= k_max < 2^31.
 *   opts: precision and form as for sp_bc_ex (the small form is not used).
 *   bc_out: double[n], host or device.  stats (host, may be NULL).
 * Returns when bc_out holds the estimate.
 */
typedef struct {
    int64_t sources;  /* k, sources drawn */
    int32_t rounds;
    int32_t converged; /* 1 when the bound met eps, 0 when k_max stopped the loop */
    double bound;      /* the half-width reached (normalised units) */
    double kernel_ms;  /* device time of the BC launches */
} sp_approx_stats;

SP_API sp_status sp_bc_approx(sp_graph g, uint64_t seed, double eps, double alpha, int64_t k_min, int64_t k_max,
                              const sp_bc_opts* opts, double* bc_out, sp_approx_stats* stats, sp_stream stream);

/*
 * PageRank of a resident graph: the pull form of the paper's generated
 * reduction code for PageRank (Section 3.3, the listing over the reverse
 * CSR).  PR starts at 1/N; every iteration sets, for each vertex v,
 *     PR'(v) = (1 - damping) / N + damping * sum over in-neighbours u of PR(u) / outdeg(u)
 * (an undirected graph's in-neighbours are its neighbours; a vertex without
 * out-arcs passes nothing on) and measures the change sum_v |PR'(v) - PR(v)|.
 * The loop stops after the first iteration whose change is at most `tol`
 * (never when tol < 0) or after max_iter iterations.  FP64 throughout.
 *   damping in [0, 1]; max_iter >= 0.
 *   pr_out: double[n], host or device, overwritten.
 *   iterations_out, change_out: host, may be NULL; the iterations run and the
 *   last change.
 * With device pr_out and both NULL the call is asynchronous on `stream`
 * (device errors latched as for sp_bc); otherwise it returns when pr_out
 * holds the result.
 */
SP_API sp_status sp_pagerank(sp_graph g, double damping, double tol, int32_t max_iter, double* pr_out,
                             int32_t* iterations_out, double* change_out, sp_stream stream);

/*
 * BC for callers that cannot allocate device memory (the paper has no
 * counterpart: this entry point exists for callers such as threads of a
 * framework that owns all device memory, real-time or serving loops that
 * must not call an allocator mid-run, and runtimes with a fixed memory plan).
 * It runs the plain form with all of its scratch in one static device array
 * of about 18 MB, reserved on every GPU that loads the library until the
 * process exits, and calls no allocator.
 *   row_ptr[n+1], col_idx[nnz], sources[nsrc], bc_out[n]: device memory of
 *   the current device; the same CSR rules as sp_graph_create, checked on
 *   the GPU.  n <= 262144 and nnz <= 16777216, else SP_ERR_TOO_LARGE.
 *   bc_out is overwritten.  The call is synchronous: it returns after its
 *   kernels have finished and the result is complete.
 * The first call on a device looks up the array's device address (once per
 * device).  Every call uses
 * the same array, so calls that overlap on the GPU (other streams or host
 * threads) race and must be serialised by the caller.
 */
SP_API sp_status sp_bc_noalloc(const int32_t* row_ptr, const int32_t* col_idx, int32_t n, int64_t nnz,
                               const int32_t* sources, int32_t nsrc, double* bc_out, sp_stream stream);

/* ------------------------------------------------------------------------ */
/* Serving: continuous batching of BC requests over resident graphs          */

/*
 * A server owns `max_slots` scheduler threads, each with its own CUDA stream.
 * Graphs added to it stay resident (the paper keeps the graph on the device
 * across kernels, Section 4.1).  A request is admitted, in arrival order, when
 * its device footprint fits in what is left of `hbm_budget_bytes`; a free slot
 * takes the oldest admitted request and runs it in one persistent launch;
 * when the batched form serves it, every other admitted request on the same
 * graph with the same options joins that launch (continuous batching, up to
 * 1,024 sources at the start), each in 32-source words of its own.  The
 * launch is live: between two of its batches it takes the words of requests
 * on the same graph with the same options admitted since it started (while
 * no other admitted request has waited more than 10 ms), and each request
 * completes as soon as its own words are done, not when the launch ends.
 * With several slots, launches of different slots are sized for the whole
 * GPU and overlap on the device as SMs free up.  A request's result does not
 * depend on what else runs: its words and the order in which their BC is
 * added are fixed by the request alone.  sp_server_add_graph computes the
 * graph's source ordering keys once (a BFS per landmark if not yet done) and
 * keeps a host copy (8 bytes a vertex).
 */
SP_API sp_status sp_server_create(size_t hbm_budget_bytes, int32_t max_slots, sp_server* out);
/* Live launches on (on != 0, the default) or off: off, a batched launch runs
   the requests it started with and later ones wait for the next launch. */
SP_API sp_status sp_server_set_live(sp_server s, int32_t on);
SP_API sp_status sp_server_add_graph(sp_server s, sp_graph g, int32_t* graph_id);
/* bc_out: device double[n] (n of the graph) on the graph's GPU, else SP_ERR_INVALID_ARG;
   sources (host or device) copied before return. */
SP_API sp_status sp_bc_submit(sp_server s, int32_t graph_id, const int32_t* sources, int32_t nsrc,
                       const sp_bc_opts* opts, double* bc_out, sp_request* req);
/*
 * PageRank request (NEXT to BC on the same resident graphs: the paper's
 * PageRank, Section 3.3; the computation of sp_pagerank, run alone in one
 * launch on a free slot).  damping in [0, 1], max_iter >= 0, tol as for
 * sp_pagerank; pr_out: device double[n] on the graph's GPU, else
 * SP_ERR_INVALID_ARG.  The request shares the queue and the memory budget
 * (footprint about 32 bytes a vertex) with BC requests; sp_bc_poll,
 * sp_bc_wait, sp_bc_cancel and sp_request_times serve every kind of request.
 * sp_request_stats of a PageRank request gives kernel_ms, launches and
 * traversed_arcs = arcs x iterations.
 */
SP_API sp_status sp_pagerank_submit(sp_server s, int32_t graph_id, double damping, double tol, int32_t max_iter,
                                    double* pr_out, sp_request* req);
/* Iterations run and last L1 change of a finished PageRank request; SP_NOT_READY while it runs, its
   error if it failed, SP_ERR_INVALID_ARG for a BC request. */
SP_API sp_status sp_request_pagerank(sp_server s, sp_request req, int32_t* iterations, double* change);
/* Requests of either kind: */
SP_API sp_status sp_bc_poll(sp_server s, sp_request req);                     /* SP_OK, SP_NOT_READY or the error */
SP_API sp_status sp_bc_wait(sp_server s, sp_request req, int64_t timeout_ns); /* SP_NOT_READY on timeout */
SP_API sp_status sp_bc_cancel(sp_server s, sp_request req);
/* Host steady-clock times in ns: submission, first batch start, completion (0 if not yet). */
SP_API sp_status sp_request_times(sp_server s, sp_request req, int64_t* submit_ns, int64_t* start_ns, int64_t* done_ns);
/* Statistics of a request (valid once it is done).  traversed_arcs and reached
   are the request's own; when requests shared a launch (shared > 1), entries,
   scanned_arcs and dag_arcs are the launch's, split in proportion to
   traversed_arcs, and kernel_ms is the launch's time.  A request finished by
   a live launch has shared = requests the launch had taken by then, joined =
   1 if it entered the launch while it ran, kernel_ms = time from its entry
   into the launch to its completion, and entries, scanned_arcs, dag_arcs and
   max_levels = 0 (kept per launch, not per request). */
SP_API sp_status sp_request_stats(sp_server s, sp_request req, sp_bc_stats* out);
SP_API sp_status sp_server_destroy(sp_server s); /* waits for running requests */

/* ------------------------------------------------------------------------ */
SP_API const char* sp_status_string(sp_status st);
SP_API const char* sp_last_error(void); /* thread-local; "" when none */

#ifdef __cplusplus
}
#endif
#endif /* STARBC_H */
