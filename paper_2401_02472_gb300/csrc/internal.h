// Host-side declarations shared by the starbc translation units.
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "starbc.h"

namespace sp {

struct Ctl;
struct HubRec;
struct FeedCtl;
struct FeedReq;

// Per-graph words that the device writes and the host reads without a CUDA
// call (mapped pinned host memory): the first error of an asynchronous call,
// returned by the next call on the graph or by sp_graph_sync, and the
// representation hints its launches found (kHint* bits).
struct DevFlags {
    int err;
    int hints;
};
constexpr int kHintSigmaFloat = 1;  // path counts needed FP64 with per-level exponents
constexpr int kHintThetaF64 = 2;    // FP32 dependencies left the FP32 range
constexpr int kHintEntries = 4;     // the batched level stack was too small
constexpr int kHintHubs = 8;        // the batched hub records were too few

// Hooks of an asynchronous call; all null for a synchronous one.  The launch
// is only enqueued and nothing is read back: its kernels skip all work when
// *pre_err holds an error (bad sources found on the device) or when `gate` is
// set and *gate == 0; after the launch a finish kernel moves the launch's
// error word on: a condition that the FP64 fallback launch fixes opens
// *fallback and records a hint, any other error is latched in flags->err.
struct AsyncHooks {
    const int* pre_err = nullptr;
    const int* gate = nullptr;
    DevFlags* flags = nullptr;  // device view of the graph's flags; non-null = asynchronous launch
    int* fallback = nullptr;    // null: no fallback follows, every error is latched
};

// Enqueue the finish step of an asynchronous launch whose control block is d_ctl.
sp_status enqueue_finish(const Ctl* d_ctl, const AsyncHooks& h, cudaStream_t st);

struct Graph {
    int device = 0;
    int32_t n = 0;
    int64_t nnz = 0;
    int32_t* d_rp = nullptr;  // [n+1]
    int32_t* d_ci = nullptr;  // [max(nnz,1)]
    // d_rp / d_ci come from the library's memory pool (sp_graph_create: a
    // destroyed graph's arrays stay mapped for the next one) rather than cudaMalloc
    bool pooled_csr = false;
    sp_graph_info info{};
    // Directed graphs: the kernels read combined rows (out-arcs, then in-arcs
    // tagged with the top bit) and count traversed arcs by out-degree.  For an
    // undirected graph the kernels read d_rp / d_ci themselves.
    bool directed = false;
    int32_t* d_crp = nullptr;   // [n+1]
    int32_t* d_cci = nullptr;   // [2 nnz]
    int32_t* d_odeg = nullptr;  // [n]
    const int32_t* krp() const { return directed ? d_crp : d_rp; }
    const int32_t* kci() const { return directed ? d_cci : d_ci; }
    int64_t knnz() const { return directed ? 2 * nnz : nnz; }
    std::vector<unsigned long long> h_keys;  // source ordering key per vertex (graph_host_keys), or empty
    int32_t* d_w = nullptr;     // arc weights [nnz] (sp_graph_set_weights): BC under these weights
    int32_t w_delta = 1;        // near-far step of the weighted form (sp_graph_set_weights)
    DevFlags* flags_host = nullptr;  // mapped pinned: errors and hints of asynchronous calls
    DevFlags* flags_dev = nullptr;   // the same words, as the device addresses them
    int ecap_mult = 1, hcap_mult = 1;  // batched capacities learnt from asynchronous calls
    std::mutex mu;
    bool sigma_float = false;  // path counts of this graph overflowed 64-bit integers before
    int32_t top_vertex = 0;     // a vertex of maximum degree
    int32_t* d_top_dist = nullptr;  // BFS distances from top_vertex (computed on first use)
    int32_t top_levels = 0;     // 1 + eccentricity of top_vertex (0 until computed)
    int32_t* d_land_dist = nullptr;  // [2][n] BFS distances from the 2nd and 3rd largest-degree vertices
    bool theta_f64 = false;     // FP32 dependencies of this graph left the FP32 range before
    void* step_cache = nullptr; // graph-driven plain form: device state block and instantiated CUDA graphs
    void* pr_plan = nullptr;    // PageRank: the hub rows split into segments (found on first use)
};

// Thread-local error text.
void set_last_error(const std::string& s);
sp_status fail(sp_status st, const std::string& what);
sp_status cuda_fail(cudaError_t e, const char* what);

#define SP_CUDA(call)                                           \
    do {                                                        \
        cudaError_t e_ = (call);                                \
        if (e_ != cudaSuccess) return ::sp::cuda_fail(e_, #call); \
    } while (0)

// Kernel tiers (entries of the level stack by degree).
struct Tiers {
    int t_thread;  // degree <= t_thread: one lane walks the row
    int t_hub;     // degree > t_hub: the row is split into segments of `seg` arcs
    int seg;
};

enum class PlainMode : int { BC = 0, BFS = 1, SIGMA = 2 };

// Exponent bound beyond which a level of FP64 path counts is recentred (X6
// of the readings: the shift is the mean of the level's largest and smallest
// exponents).  512 leaves the widest within-level spread to FP64; when
// dependencies are stored in FP32, theta-hat = (1 + delta) / sigma-hat must
// stay in FP32 normals, so BC calls with FP32 theta recentre at 64.  Every
// form and driver takes the bound from here.
inline int sigma_centre_bound(bool sigma_float, bool theta_f32, PlainMode mode) {
    return sigma_float && theta_f32 && mode == PlainMode::BC ? 64 : 512;
}

struct PlainLaunch {
    const Graph* g;
    const int32_t* d_sources;
    int32_t nsrc;
    double* d_bc;           // BC mode
    int32_t* d_dist;        // BFS mode: [nsrc][n]
    double* d_mant;         // SIGMA mode
    long long* d_exp;       // SIGMA mode
    PlainMode mode;
    bool sigma_float;       // double path counts with per-level rescaling
    bool theta_f32;         // 1/sigma-scaled dependencies stored in FP32
    int max_ctas;
    uint64_t timeout_ns;
    int debug_flags;
    cudaStream_t stream;
    int group_blocks;       // blocks per group (0 = one group of every block)
    int64_t level_cap;      // BFS levels per group; 0 = default
    int bottom_up_den;      // bottom-up discovery on levels wider than n / this (0 = top-down only)
    double* d_sq = nullptr; // BC mode, optional: sum over the sources of delta^2 per vertex
    AsyncHooks async;
};

struct LaunchResult {
    int err = 0;             // device error code (0, sp_status or internal)
    int levels = 0;
    unsigned long long traversed_arcs = 0, reached = 0, entries = 0, scanned_arcs = 0;
    int64_t ecap = 0, hcap = 0, lcap = 0;  // capacities used (batched form)
    unsigned long long dag_arcs = 0;
    double kernel_ms = 0.0;                // CUDA-event time of the launch
    int launches = 0;
    unsigned long long recentred = 0;      // (level, source) pairs recentred
    int grid = 0;
    int groups = 1;
    std::string diag;                      // barrier state when a wait timed out
};

// Summary of where the blocks of a launch stood when a barrier wait timed out.
std::string barrier_diagnostic(const Ctl& h, int grid);

// Run the plain form on L.stream and wait for it; `result` receives the
// device-side error code and statistics.
sp_status run_plain(const PlainLaunch& L, LaunchResult* result);
// The same computation (BC mode, one group) with the level loop driven by a
// CUDA graph: a conditional WHILE node over one kernel per phase.
sp_status run_plain_graph(const PlainLaunch& L, LaunchResult* result);
void destroy_step_cache(Graph* g);

struct SmallLaunch {
    const Graph* g;
    const int32_t* d_sources;
    int32_t nsrc;
    double* d_bc;
    bool theta_f32;
    int max_ctas;
    cudaStream_t stream;
    AsyncHooks async;
};

// Small-graph form: one block per source, per-source state in shared memory.
sp_status run_small(const SmallLaunch& L, LaunchResult* result);
int64_t small_form_max_n(int device);  // largest n whose state fits one block's shared memory

struct BatchedLaunch {
    const Graph* g;
    const int32_t* d_sources;
    int32_t nsrc;
    double* d_bc;
    int width;              // sources per batch: 32, 64, 128 or 256
    bool sigma_float;
    bool theta_f32;
    int max_ctas;
    uint64_t timeout_ns;
    int debug_flags;
    cudaStream_t stream;
    int64_t entry_cap;      // level-stack capacity (entries); 0 = default estimate
    int64_t hub_cap;        // hub records; 0 = default estimate
    int64_t level_cap;      // BFS levels per batch; 0 = default (16384)
    int bottom_up_den;                 // bottom-up discovery on levels with more than n / this entries (0 = never)
    double* d_word_bc;                 // request mode: [nsrc/32][n] per-word partial BC (else null)
    unsigned long long* d_word_stats;  // request mode: [nsrc/32][2]
    double* d_sq = nullptr;            // optional: sum over the sources of delta^2 per vertex
    AsyncHooks async;
    // live feed (serving): d_sources are the feed's lanes (word slots), nsrc is
    // unused, d_word_bc / d_word_stats have word_cap slots
    FeedCtl* feed = nullptr;
    FeedReq* feed_req = nullptr;
    const int32_t* feed_lanes = nullptr;  // live feed: its lanes in host memory (d_sources: device copy)
    FeedReq* req_dev = nullptr;           // live feed: device copy of its request records
    int32_t word_cap = 0;              // request mode: word slots (word index modulo this)
    int32_t req_cap = 0;               // live feed: request slots
    // enqueue only (live feeds): the launch's control block is copied to
    // ctl_out (pinned host) and done_ev recorded after it; the call returns
    // without waiting and `result` gets only the launch shape
    Ctl* ctl_out = nullptr;
    cudaEvent_t done_ev = nullptr;
    cudaHostFn_t on_done = nullptr;    // host function enqueued before done_ev (no CUDA calls in it)
    void* on_done_arg = nullptr;
};

// Serving: several requests on one graph in one batched launch, each
// request's sources in 32-lane words of its own; results and traversal
// counts are assembled per request from its words.
struct RequestPart {
    const int32_t* h_sources;  // host, nsrc entries
    int32_t nsrc;
    double* d_out;             // device [n]
    sp_bc_stats stats;         // filled on return
};
sp_status bc_requests(Graph* g, RequestPart* parts, int nparts, const sp_bc_opts& o, cudaStream_t st);
// Whether a request of nsrc sources with these options runs in the batched form.
bool request_is_batched(Graph* g, int32_t nsrc, const sp_bc_opts& o, cudaStream_t st);

// Serving: one batched launch that keeps taking requests on its graph (with
// the same options) between batches.  open sets the feed up for a launch
// (allocating on first use, reusing the buffers of earlier launches after);
// append adds a request (host sources, regrouped by the graph's source keys)
// unless the feed is full or closed; start enqueues the launch and returns,
// the caller then polls done, appends, and polls ended; scrub clears the per-word vectors after a launch that stopped on
// an error (a finished launch leaves them zero); close frees.
struct LiveFeed {
    Graph* g = nullptr;
    FeedCtl* ctl = nullptr;     // mapped pinned host memory: host addresses
    FeedReq* req = nullptr;     // [req_cap]
    int32_t* lanes = nullptr;   // [word_cap * 32]
    FeedCtl* ctl_d = nullptr;   // the same memory as the device addresses it
    FeedReq* req_d = nullptr;
    int32_t* lanes_d = nullptr;
    int32_t word_cap = 0, req_cap = 0;
    double* d_wbc = nullptr;                 // [word_cap][n], all zero between launches
    size_t wbc_bytes = 0;                    // its allocated size
    unsigned long long* d_wst = nullptr;     // [word_cap][2], all zero between launches
    int32_t* d_lanes = nullptr;              // device copies the launch makes of the lanes and records
    FeedReq* d_req = nullptr;
    int width = 0, bottom_up = 0;
    bool sigma_float = false, theta_f32 = false;
    Ctl* h_ctl = nullptr;                    // pinned host: the last launch's control block
    cudaEvent_t ev = nullptr;                // recorded after it
    int64_t words = 0, nreq = 0;             // appended so far
    int64_t pub_words = 0, pub_nreq = 0;     // of which published to the launch (live_publish)
    int64_t first_open_word = 0, first_open_req = 0;  // oldest request not yet seen done
};
// nsrc: the sources the launch starts with (they pick the batch width when no tuned width is known)
sp_status live_open(Graph* g, const sp_bc_opts& o, int64_t nsrc, LiveFeed* lf, cudaStream_t st);
// Returns the request's index in the feed (>= 0), or -1 when it does not fit
// now (slots of unfinished requests), a source is out of range, or the launch
// has closed.
int64_t live_append(LiveFeed* lf, const int32_t* h_sources, int32_t nsrc, double* d_out);
// Whether request r is finished (its done flag, read with acquire ordering).
bool live_done(const LiveFeed* lf, int64_t r);
// Publish the appended requests to the launch (release): until then it does not see them.
void live_publish(LiveFeed* lf);
void live_retire(LiveFeed* lf);  // advance past the finished requests at the front
int64_t live_ran_words(const LiveFeed* lf);  // words of the batches the launch finished
// Enqueue the live launch on st and return; live_ended polls its end and then
// fills `result` from its control block.
sp_status live_start(LiveFeed* lf, const sp_bc_opts& o, cudaStream_t st, cudaHostFn_t on_done = nullptr,
                     void* on_done_arg = nullptr);
bool live_ended(LiveFeed* lf, LaunchResult* result);
void live_scrub(LiveFeed* lf, cudaStream_t st);
void live_close(LiveFeed* lf, cudaStream_t st);
// Host copy of the per-vertex source ordering keys (live feeds order a
// request's sources with it while the GPU is busy).
sp_status graph_host_keys(Graph* g, cudaStream_t st);

sp_status run_batched(const BatchedLaunch& L, LaunchResult* result);
template <int W>
sp_status launch_batched_w(const BatchedLaunch& L, LaunchResult* result);

// Weighted form (bc_weighted.cu): BC under positive integer arc weights, one
// block per source; or, with d_dist, the shortest distances only.
constexpr int32_t kMaxWeight = 1 << 20;
struct WeightedLaunch {
    const Graph* g;
    const int32_t* d_sources;
    int32_t nsrc;
    double* d_bc;        // BC mode
    int32_t* d_dist;     // distance mode: [nsrc][n], -1 when unreachable
    int64_t dist_cap;    // distances must stay below this (a larger one reruns)
    int max_ctas;
    cudaStream_t stream;
};
sp_status run_weighted(const WeightedLaunch& L, LaunchResult* result);
sp_status set_weights(Graph* g, const int32_t* weights, bool device_src, cudaStream_t st);

// PageRank (pagerank.cu): the pull form over in-arcs, one persistent launch.
struct PrLaunch {
    Graph* g;
    double damping;
    double tol;          // stop after the first iteration whose L1 change is at most tol (< 0: never)
    int32_t max_iter;
    double* d_pr;        // device [n]: the ranks
    int max_ctas;
    uint64_t timeout_ns;
    cudaStream_t stream;
    AsyncHooks async;
};
struct PrResult {
    int err = 0;
    int32_t iterations = 0;
    double change = 0.0;
    double kernel_ms = 0.0;
    int launches = 0;
    int grid = 0;
    std::string diag;
};
sp_status run_pagerank(const PrLaunch& L, PrResult* result);
void destroy_pr_plan(Graph* g);

// CSR construction (graph_build.cu): sort every row in place; build a
// symmetric, deduplicated CSR from an edge list (device arrays).
sp_status sort_rows_device(const int32_t* d_rp, int32_t* d_ci, int32_t n, int64_t nnz, cudaStream_t st);
sp_status csr_from_edges(const int32_t* d_src, const int32_t* d_dst, int64_t m, int32_t n, bool directed,
                         cudaStream_t st, int32_t** d_rp_out, int32_t** d_ci_out, int64_t* nnz_out,
                         std::string* detail);
sp_status combined_rows(const int32_t* d_rp, const int32_t* d_ci, int32_t n, int64_t nnz, cudaStream_t st,
                        int32_t** d_crp, int32_t** d_cci, int32_t** d_odeg);

// Graph validation kernels.
sp_status validate_graph(Graph* g, uint32_t flags, cudaStream_t stream, std::string* detail);

int device_sm_count(int device);
// Stream-ordered allocation of a launch workspace from the library's pool
// (freed with cudaFreeAsync like any stream-ordered allocation).
cudaError_t workspace_alloc(void** p, size_t bytes, cudaStream_t st);
int default_batch_width(int32_t nsrc);
size_t batched_workspace_bytes(const Graph* g, int width, bool theta_f32);

}  // namespace sp
